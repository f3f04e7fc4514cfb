"""Python binding of libkq (include/kq.h): argument marshalling only.

Every function here has the name of the C entry point it calls and passes
device pointers of torch CUDA tensors plus the current CUDA stream.  No step of
the quantizer runs in Python or on the CPU: if libkq.so cannot be loaded, every
call raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np
import torch

from . import build as _build

KQ_OK, KQ_EINVAL, KQ_ECAPACITY, KQ_ECUDA, KQ_ETIMEOUT, KQ_ENOMEM = 0, -1, -2, -3, -4, -5
INIT = {"FGY": 0, "LBG": 1, "MMX": 2, "DEN": 3, "VAR": 4, "SFF": 5, "KPP": 6, "USER": 7, "WU": 8}
LLOYD_LABELS_IN = 1
LLOYD_DENSE = 2
MAX_K = 256

# kq_lloyd_stats, field for field
STATS_DTYPE = np.dtype([("iters", "<i4"), ("converged", "<i4"), ("k_eff", "<i4"), ("status", "<i4"),
                        ("ndc", "<i8"), ("sse", "<f8"), ("sse_prev", "<f8")])
STATS_BYTES = STATS_DTYPE.itemsize  # 40


# kq_batch_item / kq_batch_result, field for field (LP64 layout)
BATCH_ITEM_DTYPE = np.dtype([
    ("rgb", "<u8"), ("idx", "<u8"), ("keys", "<u8"), ("weights", "<u8"), ("labels", "<u8"), ("scratch", "<u8"),
    ("centers", "<u8"), ("palette", "<u8"), ("result", "<u8"), ("n_pixels", "<i8"), ("seed", "<u8"),
    ("eps", "<f8"), ("lbg_eps", "<f8"), ("lbg_conv_eps", "<f8"), ("lbg_max_iter", "<i4"), ("K", "<i4"),
    ("scheme", "<i4"), ("max_iter", "<i4"), ("capacity", "<i4"), ("reserved", "<i4")], align=True)
BATCH_RESULT_DTYPE = np.dtype([("status", "<i4"), ("n_unique", "<i4"), ("lloyd", STATS_DTYPE),
                               ("sse_num", "<i8"), ("t_ns", "<i8", (5,))], align=True)


class BatchConfig(C.Structure):
    _fields_ = [("cluster", C.c_int32), ("reserved", C.c_int32), ("split_pixels", C.c_int64)]


class KqError(RuntimeError):
    def __init__(self, fn: str, status: int):
        super().__init__("%s failed: %s (%d)" % (fn, strerror(status), status))
        self.status = status


class SeedParams(C.Structure):
    _fields_ = [("lbg_eps", C.c_double), ("conv_eps", C.c_double), ("max_iter", C.c_int32),
                ("reserved", C.c_int32)]


_lib: Optional[C.CDLL] = None
_vp = C.c_void_p
_SIGS = {
    "kq_workspace_size": (C.c_size_t, [C.c_int64, C.c_int32]),
    "kq_workspace_init": (C.c_int, [_vp, C.c_size_t, _vp]),
    "kq_histogram": (C.c_int, [_vp, C.c_int64, _vp, _vp, C.c_int32, _vp, _vp, C.c_size_t, _vp]),
    "kq_seed": (C.c_int, [_vp, _vp, _vp, C.c_int32, C.c_int32, C.c_uint64, C.POINTER(SeedParams), _vp, _vp,
                          C.c_size_t, _vp]),
    "kq_lloyd": (C.c_int, [_vp, _vp, _vp, C.c_int32, _vp, C.c_double, C.c_int32, C.c_uint32, _vp, _vp, _vp, _vp,
                           _vp, C.c_size_t, _vp]),
    "kq_map": (C.c_int, [_vp, C.c_int64, _vp, C.c_int32, _vp, _vp, _vp, C.c_size_t, _vp]),
    "kq_lloyd_noalloc": (C.c_int, [_vp, _vp, _vp, C.c_int32, _vp, C.c_double, C.c_int32, C.c_uint32, _vp, _vp,
                                   _vp, _vp, _vp]),
    "kq_pixel_keys": (C.c_int, [_vp, C.c_int64, _vp, _vp, _vp, _vp]),
    "kq_histogram_strided": (C.c_int, [_vp, C.c_int32, C.c_int32, C.c_int64, C.c_int32, _vp, _vp, C.c_int32, _vp,
                                       _vp, C.c_size_t, _vp]),
    "kq_status_read": (C.c_int, [_vp, C.POINTER(C.c_int32), _vp]),
    "kq_status_clear": (C.c_int, [_vp, _vp]),
    "kq_set_wait_limit": (C.c_int, [_vp, C.c_size_t, C.c_uint32, C.c_uint32, _vp]),
    "kq_map_ndc_read": (C.c_int, [_vp, C.POINTER(C.c_int64), _vp]),
    "kq_lab_points": (C.c_int, [_vp, _vp, _vp, _vp]),
    "kq_seed_points": (C.c_int, [_vp, _vp, C.c_int32, C.c_int32, C.c_uint64, _vp, _vp]),
    "kq_lloyd_points": (C.c_int, [_vp, _vp, _vp, C.c_int32, _vp, C.c_double, C.c_int32, C.c_uint32, _vp, _vp, _vp,
                                  _vp, C.c_size_t, _vp]),
    "kq_lab_palette": (C.c_int, [_vp, C.c_int32, _vp, _vp]),
    "kq_map_labels": (C.c_int, [_vp, C.c_int64, _vp, _vp, _vp, _vp, _vp, C.c_size_t, _vp]),
    "kq_strerror": (C.c_char_p, [C.c_int]),
    "kq_batch_scratch_bytes": (C.c_size_t, [C.c_int32]),
    "kq_batch_workspace_size": (C.c_size_t, []),
    "kq_batch_max_cluster": (C.c_int32, []),
    "kq_batch_plan": (C.c_int, [_vp, C.c_int32, _vp, _vp, C.POINTER(C.c_int32)]),
    "kq_batch_run": (C.c_int, [_vp, C.c_int32, _vp, C.c_int32, _vp, _vp, C.c_size_t, _vp]),
    "kq_batch_tune": (C.c_int, [_vp, _vp, C.c_int32, _vp, _vp, C.POINTER(C.c_int32), C.POINTER(C.c_float), _vp,
                                C.c_size_t, _vp]),
    "kq_live_bytes": (C.c_size_t, [C.c_int32]),
    "kq_live_init": (C.c_int, [_vp, C.c_int32]),
    "kq_live_reset": (C.c_int, [_vp, C.c_size_t, _vp]),
    "kq_live_publish": (C.c_int, [_vp, C.c_int32, _vp, C.POINTER(C.c_int64)]),
    "kq_live_done": (C.c_int, [_vp, C.c_int32, C.c_int64]),
    "kq_live_close": (C.c_int, [_vp]),
    "kq_live_run": (C.c_int, [_vp, _vp, C.c_uint32, _vp, C.c_size_t, _vp]),
}


def library_path() -> str:
    return _build.LIB


def lib() -> C.CDLL:
    """Loads libkq.so (building it in-tree if it is missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def strerror(status: int) -> str:
    return lib().kq_strerror(int(status)).decode()


def _ptr(t: Optional[torch.Tensor]) -> Optional[int]:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("libkq takes CUDA tensors (device pointers)")
    if not t.is_contiguous():
        raise ValueError("libkq takes contiguous tensors")
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _check(fn: str, st: int) -> int:
    if st != KQ_OK:
        raise KqError(fn, st)
    return st


def kq_workspace_size(max_pixels: int, max_K: int = MAX_K) -> int:
    return int(lib().kq_workspace_size(int(max_pixels), int(max_K)))


def kq_workspace_init(ws: torch.Tensor, stream=None) -> None:
    _check("kq_workspace_init", lib().kq_workspace_init(_ptr(ws), ws.numel() * ws.element_size(), _stream(stream)))


def kq_histogram(rgb: torch.Tensor, keys: torch.Tensor, weights: torch.Tensor, n_unique: torch.Tensor,
                 ws: torch.Tensor, n_pixels: Optional[int] = None, stream=None) -> None:
    n = rgb.numel() // 3 if n_pixels is None else int(n_pixels)
    cap = min(keys.numel(), weights.numel())
    _check("kq_histogram", lib().kq_histogram(_ptr(rgb) if n else None, n, _ptr(keys), _ptr(weights), cap,
                                              _ptr(n_unique), _ptr(ws), ws.numel() * ws.element_size(),
                                              _stream(stream)))


def kq_seed(keys: torch.Tensor, weights: torch.Tensor, n_unique: torch.Tensor, K: int, scheme, seed: int,
            centers: torch.Tensor, ws: torch.Tensor, lbg_eps: float = 1.0, conv_eps: float = 1e-4,
            max_iter: int = 100, stream=None) -> None:
    sch = INIT[scheme] if isinstance(scheme, str) else int(scheme)
    p = SeedParams(float(lbg_eps), float(conv_eps), int(max_iter), 0)
    _check("kq_seed", lib().kq_seed(_ptr(keys), _ptr(weights), _ptr(n_unique), int(K), sch,
                                    int(seed) & (2**64 - 1), C.byref(p), _ptr(centers), _ptr(ws),
                                    ws.numel() * ws.element_size(), _stream(stream)))


def kq_lloyd(keys: torch.Tensor, weights: torch.Tensor, n_unique: torch.Tensor, K: int, centers: torch.Tensor,
             eps: float, max_iter: int, labels: torch.Tensor, palette: torch.Tensor, ws: torch.Tensor,
             stats: Optional[torch.Tensor] = None, sse_hist: Optional[torch.Tensor] = None, flags: int = 0,
             stream=None) -> None:
    _check("kq_lloyd", lib().kq_lloyd(_ptr(keys), _ptr(weights), _ptr(n_unique), int(K), _ptr(centers), float(eps),
                                      int(max_iter), int(flags), _ptr(labels), _ptr(palette), _ptr(stats),
                                      _ptr(sse_hist), _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)))


def kq_lloyd_noalloc(keys: torch.Tensor, weights: torch.Tensor, n_unique: torch.Tensor, K: int,
                     centers: torch.Tensor, eps: float, max_iter: int, labels: torch.Tensor, palette: torch.Tensor,
                     stats: Optional[torch.Tensor] = None, sse_hist: Optional[torch.Tensor] = None, flags: int = 0,
                     stream=None) -> None:
    """kq_lloyd with its scratch in the library's static device array (no workspace)."""
    _check("kq_lloyd_noalloc", lib().kq_lloyd_noalloc(_ptr(keys), _ptr(weights), _ptr(n_unique), int(K),
                                                      _ptr(centers), float(eps), int(max_iter), int(flags),
                                                      _ptr(labels), _ptr(palette), _ptr(stats), _ptr(sse_hist),
                                                      _stream(stream)))


def kq_map(rgb: torch.Tensor, palette: torch.Tensor, K: int, idx: torch.Tensor, ws: torch.Tensor,
           sse_num: Optional[torch.Tensor] = None, n_pixels: Optional[int] = None, stream=None) -> None:
    n = rgb.numel() // 3 if n_pixels is None else int(n_pixels)
    _check("kq_map", lib().kq_map(_ptr(rgb) if n else None, n, _ptr(palette), int(K), _ptr(idx) if n else None,
                                  _ptr(sse_num), _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)))


def kq_status_read(ws: torch.Tensor, stream=None) -> int:
    v = C.c_int32(0)
    _check("kq_status_read", lib().kq_status_read(_ptr(ws), C.byref(v), _stream(stream)))
    return int(v.value)


def kq_lab_points(keys: torch.Tensor, n_unique: torch.Tensor, points: torch.Tensor, stream=None) -> None:
    _check("kq_lab_points", lib().kq_lab_points(_ptr(keys), _ptr(n_unique), _ptr(points), _stream(stream)))


def kq_seed_points(points: torch.Tensor, n_unique: torch.Tensor, K: int, scheme, seed: int, centers: torch.Tensor,
                   stream=None) -> None:
    sch = INIT[scheme] if isinstance(scheme, str) else int(scheme)
    _check("kq_seed_points", lib().kq_seed_points(_ptr(points), _ptr(n_unique), int(K), sch,
                                                  int(seed) & ((1 << 64) - 1), _ptr(centers), _stream(stream)))


def kq_lloyd_points(points: torch.Tensor, weights: torch.Tensor, n_unique: torch.Tensor, K: int,
                    centers: torch.Tensor, eps: float, max_iter: int, labels: torch.Tensor, ws: torch.Tensor,
                    stats: Optional[torch.Tensor] = None, sse_hist: Optional[torch.Tensor] = None, flags: int = 0,
                    stream=None) -> None:
    _check("kq_lloyd_points", lib().kq_lloyd_points(_ptr(points), _ptr(weights), _ptr(n_unique), int(K),
                                                    _ptr(centers), float(eps), int(max_iter), int(flags),
                                                    _ptr(labels), _ptr(stats), _ptr(sse_hist), _ptr(ws),
                                                    ws.numel() * ws.element_size(), _stream(stream)))


def kq_lab_palette(centers: torch.Tensor, K: int, palette: torch.Tensor, stream=None) -> None:
    _check("kq_lab_palette", lib().kq_lab_palette(_ptr(centers), int(K), _ptr(palette), _stream(stream)))


def kq_map_labels(rgb: torch.Tensor, keys: torch.Tensor, n_unique: torch.Tensor, labels: torch.Tensor,
                  idx: torch.Tensor, ws: torch.Tensor, n_pixels: Optional[int] = None, stream=None) -> None:
    n = rgb.numel() // 3 if n_pixels is None else int(n_pixels)
    _check("kq_map_labels", lib().kq_map_labels(_ptr(rgb) if n else None, n, _ptr(keys), _ptr(n_unique),
                                                _ptr(labels), _ptr(idx) if n else None, _ptr(ws),
                                                ws.numel() * ws.element_size(), _stream(stream)))


def kq_map_ndc_read(ws: torch.Tensor, stream=None) -> int:
    v = C.c_int64(0)
    _check("kq_map_ndc_read", lib().kq_map_ndc_read(_ptr(ws), C.byref(v), _stream(stream)))
    return int(v.value)


def kq_set_wait_limit(ws: torch.Tensor, wait_limit_us: int, missing_arrivals: int = 0, stream=None) -> None:
    _check("kq_set_wait_limit", lib().kq_set_wait_limit(_ptr(ws), ws.numel() * ws.element_size(), int(wait_limit_us),
                                                        int(missing_arrivals), _stream(stream)))


def kq_status_clear(ws: torch.Tensor, stream=None) -> None:
    _check("kq_status_clear", lib().kq_status_clear(_ptr(ws), _stream(stream)))


def parse_stats(stats: torch.Tensor) -> dict:
    raw = stats.detach().cpu().numpy().view(np.uint8)[:STATS_BYTES].tobytes()
    rec = np.frombuffer(raw, dtype=STATS_DTYPE)[0]
    return {k: rec[k].item() for k in STATS_DTYPE.names}


def launches(call: str, n_pixels: int = 1, scheme: str = "KPP", K: int = 1) -> int:
    """Kernels one call enqueues (the library's own kernels, not memsets)."""
    if call == "kq_histogram":
        return 4 if n_pixels > 0 else 3
    if call == "kq_lloyd":
        return 1
    if call == "kq_map":
        return 2 if n_pixels > 0 else 1
    if call == "kq_seed":
        if scheme == "LBG":
            count, m = 3, 1
            while m < K:
                split = m if 2 * m <= K else K - m
                count += 2 + (1 if split < m else 0)
                m += split
            return count
        return {"FGY": 2, "MMX": 3, "KPP": 3, "SFF": 2, "VAR": 3, "DEN": 4, "WU": 7}[scheme]
    raise ValueError(call)


@dataclass
class Result:
    idx: torch.Tensor          # palette index per pixel (uint8, device)
    palette: torch.Tensor      # K x 3 uint8 (device)
    centers: torch.Tensor      # K x 3 float64 (device)
    n_unique: torch.Tensor     # device int32 scalar
    sse_num: torch.Tensor      # device int64 scalar
    stats: torch.Tensor        # raw kq_lloyd_stats bytes (device)


class Quantizer:
    """Device-resident buffers plus the four calls, for images up to `max_pixels`.

    ``quantize(rgb, K, scheme, seed, eps, max_iter)`` runs histogram, seeding,
    Weighted Sort-Means and mapping on the current stream with no host
    synchronisation; read results from the returned device tensors.
    """

    def __init__(self, max_pixels: int, device=None):
        dev = torch.device("cuda") if device is None else torch.device(device)
        self.device = dev
        self.max_pixels = int(max_pixels)
        cap = max(1, min(self.max_pixels, 1 << 24))
        self.capacity = cap
        nbytes = kq_workspace_size(self.max_pixels, MAX_K)
        # zero-filled workspace: the library keeps its tables zeroed from here on
        self.ws = torch.zeros(nbytes, dtype=torch.uint8, device=dev)
        self.keys = torch.empty(cap, dtype=torch.int32, device=dev)
        self.weights = torch.empty(cap, dtype=torch.int32, device=dev)
        self.n_unique = torch.zeros(1, dtype=torch.int32, device=dev)
        self.labels = torch.zeros(cap, dtype=torch.uint8, device=dev)
        self.centers = torch.zeros(MAX_K * 3, dtype=torch.float64, device=dev)
        self.palette = torch.zeros(MAX_K * 3, dtype=torch.uint8, device=dev)
        self.stats = torch.zeros(64, dtype=torch.uint8, device=dev)
        self.sse_num = torch.zeros(1, dtype=torch.int64, device=dev)
        self.idx = torch.empty(max(1, self.max_pixels), dtype=torch.uint8, device=dev)
        self.launches = 0  # library kernels enqueued so far

    def quantize(self, rgb: torch.Tensor, K: int, scheme: str = "KPP", seed: int = 0, eps: float = 1e-4,
                 max_iter: int = 100, flags: int = 0, stream=None) -> Result:
        n = rgb.numel() // 3
        if n > self.max_pixels:
            raise ValueError("image larger than this Quantizer's max_pixels")
        kq_histogram(rgb, self.keys, self.weights, self.n_unique, self.ws, stream=stream)
        c = self.centers[:3 * K]
        kq_seed(self.keys, self.weights, self.n_unique, K, scheme, seed, c, self.ws, conv_eps=eps,
                max_iter=max_iter, stream=stream)
        pal = self.palette[:3 * K]
        kq_lloyd(self.keys, self.weights, self.n_unique, K, c, eps, max_iter, self.labels, pal, self.ws,
                 stats=self.stats, flags=flags, stream=stream)
        idx = self.idx[:n]
        kq_map(rgb, pal, K, idx, self.ws, sse_num=self.sse_num,
               stream=stream)
        self.launches += (launches("kq_histogram", n) + launches("kq_seed", n, scheme, K) + launches("kq_lloyd")
                          + launches("kq_map", n))
        return Result(idx=idx, palette=pal.view(K, 3), centers=c.view(K, 3), n_unique=self.n_unique,
                      sse_num=self.sse_num, stats=self.stats)


class LabQuantizer(Quantizer):
    """k-means in the CIE L*a*b* colour space (Section 2.1): the unique colours'
    L*a*b* points, Forgy seeds among them, Weighted Sort-Means on the points, the
    centres' sRGB palette, and each pixel mapped to its colour's label.  Same
    buffers as Quantizer plus the points; ``centers`` hold L*a*b* x 256 and
    ``stats`` the Lloyd run in those units."""

    def __init__(self, max_pixels: int, device=None):
        super().__init__(max_pixels, device=device)
        self.points = torch.zeros(self.capacity, dtype=torch.int64, device=self.device)

    def quantize(self, rgb: torch.Tensor, K: int, scheme: str = "FGY", seed: int = 0, eps: float = 1e-4,
                 max_iter: int = 100, flags: int = 0, stream=None) -> Result:
        n = rgb.numel() // 3
        if n > self.max_pixels:
            raise ValueError("image larger than this LabQuantizer's max_pixels")
        kq_histogram(rgb, self.keys, self.weights, self.n_unique, self.ws, stream=stream)
        kq_lab_points(self.keys, self.n_unique, self.points, stream=stream)
        c = self.centers[:3 * K]
        kq_seed_points(self.points, self.n_unique, K, scheme, seed, c, stream=stream)
        kq_lloyd_points(self.points, self.weights, self.n_unique, K, c, eps, max_iter, self.labels, self.ws,
                        stats=self.stats, flags=flags, stream=stream)
        pal = self.palette[:3 * K]
        kq_lab_palette(c, K, pal, stream=stream)
        idx = self.idx[:n]
        kq_map_labels(rgb, self.keys, self.n_unique, self.labels, idx, self.ws, stream=stream)
        return Result(idx=idx, palette=pal.view(K, 3), centers=c.view(K, 3), n_unique=self.n_unique,
                      sse_num=self.sse_num, stats=self.stats)


def kq_histogram_strided(rgb: torch.Tensor, height: int, width: int, stride: int, keys: torch.Tensor,
                         weights: torch.Tensor, n_unique: torch.Tensor, ws: torch.Tensor, pitch: Optional[int] = None,
                         stream=None) -> None:
    """Histogram of the pixels (x, y) with x, y multiples of `stride` (Section 2.2)."""
    pitch = 3 * width if pitch is None else pitch
    _check("kq_histogram_strided", lib().kq_histogram_strided(
        _ptr(rgb) if height * width else None, height, width, pitch, stride, _ptr(keys), _ptr(weights),
        keys.numel(), _ptr(n_unique), _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)))


def kq_pixel_keys(rgb: torch.Tensor, keys: torch.Tensor, weights: Optional[torch.Tensor] = None,
                  n_out: Optional[torch.Tensor] = None, stream=None) -> None:
    """Every pixel as its own point (the k-means baseline of Table 1)."""
    n = rgb.numel() // 3
    _check("kq_pixel_keys", lib().kq_pixel_keys(_ptr(rgb) if n else None, n, _ptr(keys), _ptr(weights), _ptr(n_out),
                                                _stream(stream)))


def kq_batch_scratch_bytes(capacity: int) -> int:
    return int(lib().kq_batch_scratch_bytes(int(capacity)))


def kq_batch_workspace_size() -> int:
    return int(lib().kq_batch_workspace_size())


def kq_batch_max_cluster() -> int:
    return int(lib().kq_batch_max_cluster())


def kq_batch_plan(h_items: np.ndarray, cfg: BatchConfig):
    """Host planner: (order as int32 numpy array, n_big)."""
    h_items = np.ascontiguousarray(h_items, dtype=BATCH_ITEM_DTYPE)
    n = h_items.shape[0]
    order = np.zeros(max(n, 1), dtype=np.int32)
    nb = C.c_int32(0)
    _check("kq_batch_plan", lib().kq_batch_plan(h_items.ctypes.data, n, C.byref(cfg), order.ctypes.data,
                                                C.byref(nb)))
    return order[:n], int(nb.value)


def kq_batch_run(items: torch.Tensor, n_items: int, order: torch.Tensor, n_big: int, cfg: BatchConfig,
                 ws: torch.Tensor, stream=None) -> None:
    _check("kq_batch_run", lib().kq_batch_run(_ptr(items), int(n_items), _ptr(order), int(n_big), C.byref(cfg),
                                              _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)))


def kq_batch_tune(h_items: np.ndarray, items: torch.Tensor, order: torch.Tensor, ws: torch.Tensor, stream=None):
    """Autotuner: (best BatchConfig, n_big, ms); `order` receives the best order."""
    h_items = np.ascontiguousarray(h_items, dtype=BATCH_ITEM_DTYPE)
    cfg = BatchConfig()
    nb = C.c_int32(0)
    ms = C.c_float(0.0)
    _check("kq_batch_tune", lib().kq_batch_tune(h_items.ctypes.data, _ptr(items), h_items.shape[0], _ptr(order),
                                                C.byref(cfg), C.byref(nb), C.byref(ms), _ptr(ws),
                                                ws.numel() * ws.element_size(), _stream(stream)))
    return cfg, int(nb.value), float(ms.value)


class LiveQueue:
    """The queue of a live batch launch (kq_live_* in include/kq.h): a page-locked
    host buffer that the host publishes items into and the running kernel claims
    them from.  `capacity` ring slots per class; class 0 goes to thread-block
    clusters, class 1 to single CTAs."""

    def __init__(self, capacity: int):
        self.capacity = int(capacity)
        nbytes = int(lib().kq_live_bytes(self.capacity))
        if nbytes == 0:
            raise ValueError("capacity must be >= 1")
        self.buf = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
        self.ptr = self.buf.data_ptr()
        _check("kq_live_init", lib().kq_live_init(self.ptr, self.capacity))

    def publish(self, cls: int, item: np.ndarray) -> Optional[int]:
        """Publishes one item (a BATCH_ITEM_DTYPE record); its sequence number, or
        None while the ring slot it needs still holds an unfinished item."""
        rec = np.ascontiguousarray(np.asarray(item, dtype=BATCH_ITEM_DTYPE).reshape(1))
        seq = C.c_int64(-1)
        st = lib().kq_live_publish(self.ptr, int(cls), rec.ctypes.data, C.byref(seq))
        if st == KQ_ECAPACITY:
            return None
        _check("kq_live_publish", st)
        return int(seq.value)

    def done(self, cls: int, seq: int) -> bool:
        return lib().kq_live_done(self.ptr, int(cls), int(seq)) == 1

    def close(self) -> None:
        _check("kq_live_close", lib().kq_live_close(self.ptr))

    def tails(self):
        return tuple(int(v) for v in self.buf[:8].numpy().view(np.uint32))


def kq_live_reset(ws: torch.Tensor, stream=None) -> None:
    _check("kq_live_reset", lib().kq_live_reset(_ptr(ws), ws.numel() * ws.element_size(), _stream(stream)))


def kq_live_run(q: LiveQueue, cfg: BatchConfig, idle_us: int, ws: torch.Tensor, stream=None) -> None:
    _check("kq_live_run", lib().kq_live_run(q.ptr, C.byref(cfg), int(idle_us), _ptr(ws),
                                            ws.numel() * ws.element_size(), _stream(stream)))


def _align(v: int, a: int = 256) -> int:
    return (v + a - 1) // a * a


class BatchQuantizer:
    """A batch of images quantized by one persistent launch (kq_batch_run).

    All per-image buffers live in one device arena; ``rgb(i)`` is where image i's
    pixels go, ``run()`` enqueues the batch on the current stream (no host
    synchronisation) and ``capture()`` records it as a CUDA graph that ``replay()``
    launches.
    """

    def __init__(self, n_pixels, Ks, schemes="KPP", seeds=0, eps: float = 1e-4, max_iter: int = 100,
                 lbg_eps: float = 1.0, capacities=None, device=None):
        dev = torch.device("cuda") if device is None else torch.device(device)
        self.device = dev
        n = len(n_pixels)
        self.n_items = n
        Ks = list(Ks) if not isinstance(Ks, int) else [Ks] * n
        schemes = [schemes] * n if isinstance(schemes, str) else list(schemes)
        seeds = [seeds] * n if isinstance(seeds, int) else list(seeds)
        caps = [max(0, min(int(p), 1 << 24)) for p in n_pixels] if capacities is None else list(capacities)
        self.n_pixels = [int(p) for p in n_pixels]
        self.Ks = [int(k) for k in Ks]
        self.capacity = caps
        lay = []
        off = 0
        for i in range(n):
            d = {}
            for name, size in (("rgb", 3 * self.n_pixels[i]), ("idx", self.n_pixels[i]), ("keys", 4 * caps[i]),
                               ("weights", 4 * caps[i]), ("labels", caps[i]),
                               ("scratch", kq_batch_scratch_bytes(caps[i])), ("centers", 24 * self.Ks[i]),
                               ("palette", 3 * self.Ks[i]), ("result", BATCH_RESULT_DTYPE.itemsize)):
                d[name] = (off, size)
                off = _align(off + max(size, 1))
            lay.append(d)
        self.layout = lay
        self.arena = torch.zeros(max(off, 256), dtype=torch.uint8, device=dev)
        base = self.arena.data_ptr()
        items = np.zeros(n, dtype=BATCH_ITEM_DTYPE)
        for i in range(n):
            for name in ("rgb", "idx", "keys", "weights", "labels", "scratch", "centers", "palette", "result"):
                items[i][name] = base + lay[i][name][0]
            items[i]["n_pixels"] = self.n_pixels[i]
            items[i]["seed"] = int(seeds[i]) & ((1 << 64) - 1)
            items[i]["eps"] = eps
            items[i]["lbg_eps"] = lbg_eps
            items[i]["lbg_conv_eps"] = eps
            items[i]["lbg_max_iter"] = max_iter
            items[i]["K"] = self.Ks[i]
            items[i]["scheme"] = INIT[schemes[i]] if isinstance(schemes[i], str) else int(schemes[i])
            items[i]["max_iter"] = max_iter
            items[i]["capacity"] = caps[i]
        self.h_items = items
        self.items = torch.from_numpy(items.view(np.uint8).copy()).to(dev)
        self.order = torch.zeros(max(n, 1), dtype=torch.int32, device=dev)
        self.ws = torch.zeros(kq_batch_workspace_size(), dtype=torch.uint8, device=dev)
        self.cfg = BatchConfig(1, 0, 0)
        self.n_big = 0
        self.plan(self.cfg)
        self.graph = None

    def _view(self, i: int, name: str) -> torch.Tensor:
        off, size = self.layout[i][name]
        return self.arena[off:off + size]

    def rgb(self, i: int) -> torch.Tensor:
        return self._view(i, "rgb")

    def idx(self, i: int) -> torch.Tensor:
        return self._view(i, "idx")

    def keys(self, i: int) -> torch.Tensor:
        return self._view(i, "keys").view(torch.int32)

    def weights(self, i: int) -> torch.Tensor:
        return self._view(i, "weights").view(torch.int32)

    def labels(self, i: int) -> torch.Tensor:
        return self._view(i, "labels")

    def centers(self, i: int) -> torch.Tensor:
        return self._view(i, "centers").view(torch.float64).view(-1, 3)

    def palette(self, i: int) -> torch.Tensor:
        return self._view(i, "palette").view(-1, 3)

    def results(self) -> np.ndarray:
        """Every item's kq_batch_result (synchronizes)."""
        if self.n_items == 0:
            return np.zeros(0, dtype=BATCH_RESULT_DTYPE)
        sz = BATCH_RESULT_DTYPE.itemsize
        offs = torch.tensor([self.layout[i]["result"][0] for i in range(self.n_items)], dtype=torch.int64,
                            device=self.arena.device)
        raw = self.arena[offs[:, None] + torch.arange(sz, device=self.arena.device)[None, :]]
        return np.frombuffer(raw.cpu().numpy().tobytes(), dtype=BATCH_RESULT_DTYPE).copy()

    def plan(self, cfg: BatchConfig) -> None:
        order, nb = kq_batch_plan(self.h_items, cfg)
        if self.n_items:
            self.order[:self.n_items].copy_(torch.from_numpy(order))
        self.cfg, self.n_big = cfg, nb
        self.graph = None

    def tune(self, stream=None) -> float:
        cfg, nb, ms = kq_batch_tune(self.h_items, self.items, self.order, self.ws, stream=stream)
        self.cfg, self.n_big = cfg, nb
        self.graph = None
        return ms

    def run(self, stream=None) -> None:
        kq_batch_run(self.items, self.n_items, self.order, self.n_big, self.cfg, self.ws, stream=stream)

    def capture(self) -> None:
        """Records run() in a CUDA graph (one memset node and one kernel node)."""
        s = torch.cuda.Stream(device=self.device)
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.run()
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.run()
        self.graph = g

    def replay(self) -> None:
        if self.graph is None:
            self.capture()
        self.graph.replay()


def exported_symbols() -> list:
    """Names the header declares (parsed from include/kq.h)."""
    import re

    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "kq.h")
    with open(hdr) as f:
        text = f.read()
    return re.findall(r"^KQ_API\s+[\w\s\*]+?\b(kq_\w+)\s*\(", text, flags=re.M)
