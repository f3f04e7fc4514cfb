"""FP64 CPU oracle for exact k-means colour quantization (Celebi 2011).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline are the only callers.  The product path never imports this package.

This module only marshals numpy arrays into the plain C reference in
``kq_oracle.c``; every step of the arithmetic lives there, with the passage of
the paper it follows.

Functions and the passage each follows:
  histogram   -- Section 2.2 items 1-2 (unique colours with frequency weights)
  assign      -- Algorithm 1 / Algorithm 2 assignment (argmin, lowest index)
  update      -- Algorithm 2 weighted mean, exact integer sums
  lloyd       -- Algorithm 2 loop with the Section 3.3 convergence test
  palette     -- rounding of the final centres to 8-bit colours
  map_pixels  -- Section 1 / 2.1 pixel mapping by full palette search
  mse, psnr   -- Section 3.1, Eqs. 2 and 3
  seed        -- Section 2.3 generic initialization schemes, and WU (Section 3.3)
  wu          -- Wu's greedy orthogonal bipartitioning (Section 3.3, WSM-WU)
  lab, lab_points, lab_palette -- the CIE L*a*b* space of Section 2.1 (sRGB,
                 D65; fixed-point points) and its inverse to an sRGB palette
  assign_points, update_points, lloyd_points, seed_points_fgy -- Algorithm 2
                 and Forgy seeding on fixed-point 3-D points (L*a*b*)

Parity status: every function above is pinned by ``tests/test_oracle_pins.py``
(closed forms, brute force on tiny inputs, invariants, library routines).
"""
from __future__ import annotations

import contextlib
import ctypes as C
import math
import os
from typing import Dict, Optional, Tuple

import numpy as np

from . import build as _build

SCHEMES = {"FGY": 0, "LBG": 1, "MMX": 2, "DEN": 3, "VAR": 4, "SFF": 5, "KPP": 6, "WU": 8}

_libs: Dict[str, C.CDLL] = {}
_variant = "serial"

_u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def _opt(ptr_type):
    """ndpointer that also accepts None (a NULL pointer)."""

    class _Opt(ptr_type):  # type: ignore[misc, valid-type]
        @classmethod
        def from_param(cls, obj):
            if obj is None:
                return None
            return ptr_type.from_param(obj)

    return _Opt


@contextlib.contextmanager
def openmp():
    """Within this block every call runs the OpenMP build of the same C source
    (the assignment's colours split over the host cores).  For timing only: its
    FP64 SSE sums depend on the thread count."""
    global _variant
    old = _variant
    _variant = "openmp"
    try:
        yield
    finally:
        _variant = old


def lib() -> C.CDLL:
    if _variant not in _libs:
        path = _build.build()
        if _variant == "openmp":
            path = _build.LIB_OMP
        L = C.CDLL(path)
        L.or_rand.restype = C.c_uint64
        L.or_rand.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32]
        L.or_below.restype = C.c_uint64
        L.or_below.argtypes = [C.c_uint64, C.c_uint64]
        L.or_histogram.restype = C.c_int64
        L.or_histogram.argtypes = [_u8p, C.c_int64, _opt(_u32p), _opt(_u32p), C.c_int64]
        L.or_assign.restype = C.c_double
        L.or_assign.argtypes = [_u32p, _u32p, C.c_int64, C.c_int, _f64p, _u8p, _opt(_f64p), _opt(_f64p)]
        L.or_update.restype = None
        L.or_update.argtypes = [_u32p, _u32p, C.c_int64, C.c_int, _u8p, _f64p, _f64p, _opt(_i64p)]
        L.or_lloyd.restype = C.c_int
        L.or_lloyd.argtypes = [_u32p, _u32p, C.c_int64, C.c_int, _f64p, C.c_double, C.c_int, _u8p,
                               _opt(_f64p), C.POINTER(C.c_int), _opt(_i64p)]
        L.or_palette.restype = None
        L.or_palette.argtypes = [_opt(_i64p), _f64p, C.c_int, _u8p]
        L.or_map.restype = None
        L.or_map.argtypes = [_u8p, C.c_int64, _u8p, C.c_int, _u8p, C.POINTER(C.c_int64)]
        L.or_seed.restype = C.c_int
        L.or_seed.argtypes = [_u32p, _u32p, C.c_int64, C.c_int, C.c_int, C.c_uint64, C.c_double, C.c_double,
                              C.c_int, _f64p]
        L.or_sff_size.restype = C.c_int64
        L.or_sff_size.argtypes = [C.c_int64, C.c_int]
        L.or_var_channel.restype = C.c_int
        L.or_var_channel.argtypes = [_u32p, _u32p, C.c_int64]
        L.or_wu.restype = C.c_int
        L.or_wu.argtypes = [_u32p, _u32p, C.c_int64, C.c_int, _f64p]
        _i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
        L.or_lab.restype = None
        L.or_lab.argtypes = [C.c_uint32, _f64p]
        L.or_lab_points.restype = None
        L.or_lab_points.argtypes = [_u32p, C.c_int64, _i32p]
        L.or_lab_palette.restype = None
        L.or_lab_palette.argtypes = [_f64p, C.c_int, _u8p]
        L.or_assign_points.restype = C.c_double
        L.or_assign_points.argtypes = [_i32p, _u32p, C.c_int64, C.c_int, _f64p, _u8p, _opt(_f64p), _opt(_f64p)]
        L.or_update_points.restype = None
        L.or_update_points.argtypes = [_i32p, _u32p, C.c_int64, C.c_int, _u8p, _f64p, _f64p, _opt(_i64p)]
        L.or_lloyd_points.restype = C.c_int
        L.or_lloyd_points.argtypes = [_i32p, _u32p, C.c_int64, C.c_int, _f64p, C.c_double, C.c_int, _u8p,
                                      _opt(_f64p), C.POINTER(C.c_int), _opt(_i64p)]
        L.or_seed_points_fgy.restype = None
        L.or_seed_points_fgy.argtypes = [_i32p, C.c_int64, C.c_int, C.c_uint64, _f64p]
        L.or_den_quota.restype = None
        L.or_den_quota.argtypes = [_i64p, _i64p, C.c_int, _i64p]
        _libs[_variant] = L
    return _libs[_variant]


def _pixels(rgb: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(rgb, dtype=np.uint8).reshape(-1)
    if a.size % 3:
        raise ValueError("packed RGB8 input must hold a multiple of 3 bytes")
    return a


def rand(seed: int, stream: int, ctr: int) -> int:
    """Output ``ctr`` of SplitMix64 stream ``stream`` (see kq_oracle.c)."""
    return int(lib().or_rand(seed & (2**64 - 1), stream, ctr))


def below(u: int, m: int) -> int:
    return int(lib().or_below(u, m))


def histogram(rgb: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Unique colours (ascending 24-bit keys) and their pixel counts."""
    a = _pixels(rgb)
    n = a.size // 3
    nu = lib().or_histogram(a, n, None, None, 0)
    keys = np.empty(max(nu, 1), dtype=np.uint32)
    w = np.empty(max(nu, 1), dtype=np.uint32)
    got = lib().or_histogram(a, n, keys, w, nu)
    assert got == nu
    return keys[:nu], w[:nu]


def key_to_rgb(keys: np.ndarray) -> np.ndarray:
    k = np.asarray(keys, dtype=np.uint32)
    return np.stack([(k >> 16) & 255, (k >> 8) & 255, k & 255], axis=1).astype(np.int64)


def assign(keys: np.ndarray, w: np.ndarray, centers: np.ndarray):
    """Labels, best and second-best FP64 distances, and the weighted SSE."""
    keys = np.ascontiguousarray(keys, dtype=np.uint32)
    w = np.ascontiguousarray(w, dtype=np.uint32)
    c = np.ascontiguousarray(centers, dtype=np.float64).reshape(-1)
    K = c.size // 3
    n = keys.size
    lab = np.empty(n, dtype=np.uint8)
    d1 = np.empty(n, dtype=np.float64)
    d2 = np.empty(n, dtype=np.float64)
    sse = lib().or_assign(keys, w, n, K, c, lab, d1, d2)
    return lab, d1, d2, sse


def update(keys: np.ndarray, w: np.ndarray, labels: np.ndarray, centers: np.ndarray):
    """New centres (FP64) and the exact sums K x (S_r, S_g, S_b, W)."""
    keys = np.ascontiguousarray(keys, dtype=np.uint32)
    w = np.ascontiguousarray(w, dtype=np.uint32)
    c = np.ascontiguousarray(centers, dtype=np.float64).reshape(-1)
    K = c.size // 3
    out = np.empty_like(c)
    sums = np.empty(K * 4, dtype=np.int64)
    lib().or_update(keys, w, keys.size, K, np.ascontiguousarray(labels, dtype=np.uint8), c, out, sums)
    return out.reshape(K, 3), sums.reshape(K, 4)


def lloyd(keys: np.ndarray, w: np.ndarray, centers: np.ndarray, eps: float, max_iter: int) -> Dict:
    keys = np.ascontiguousarray(keys, dtype=np.uint32)
    w = np.ascontiguousarray(w, dtype=np.uint32)
    c = np.array(centers, dtype=np.float64).reshape(-1).copy()
    K = c.size // 3
    lab = np.zeros(keys.size, dtype=np.uint8)
    hist = np.zeros(max(1, max_iter), dtype=np.float64)
    conv = C.c_int(0)
    sums = np.zeros(K * 4, dtype=np.int64)
    it = lib().or_lloyd(keys, w, keys.size, K, c, float(eps), int(max_iter), lab, hist, C.byref(conv), sums)
    return {"centers": c.reshape(K, 3), "labels": lab, "sse_hist": hist[:it], "iters": it,
            "converged": bool(conv.value), "sums": sums.reshape(K, 4)}


def palette(sums: Optional[np.ndarray], centers: np.ndarray) -> np.ndarray:
    c = np.ascontiguousarray(centers, dtype=np.float64).reshape(-1)
    K = c.size // 3
    s = None if sums is None else np.ascontiguousarray(sums, dtype=np.int64).reshape(-1)
    pal = np.empty(K * 3, dtype=np.uint8)
    lib().or_palette(s, c, K, pal)
    return pal.reshape(K, 3)


def map_pixels(rgb: np.ndarray, pal: np.ndarray) -> Tuple[np.ndarray, int]:
    """Palette index per pixel and the integer squared-error sum."""
    a = _pixels(rgb)
    p = np.ascontiguousarray(pal, dtype=np.uint8).reshape(-1)
    n = a.size // 3
    idx = np.empty(n, dtype=np.uint8)
    sse = C.c_int64(0)
    lib().or_map(a, n, p, p.size // 3, idx, C.byref(sse))
    return idx, int(sse.value)


def mse(sse_num: int, n_pixels: int) -> float:
    """Section 3.1, Eq. 2: mean squared error over the H x W pixels."""
    return sse_num / n_pixels


def psnr(mse_value: float) -> float:
    """Section 3.1, Eq. 3."""
    return 20.0 * math.log10(255.0 / math.sqrt(mse_value)) if mse_value > 0 else math.inf


def seed(keys: np.ndarray, w: np.ndarray, K: int, scheme: str, seed_value: int,
         lbg_eps: float = 1.0, conv_eps: float = 1e-4, max_iter: int = 100) -> Tuple[np.ndarray, int]:
    keys = np.ascontiguousarray(keys, dtype=np.uint32)
    w = np.ascontiguousarray(w, dtype=np.uint32)
    c = np.zeros(K * 3, dtype=np.float64)
    k_eff = lib().or_seed(keys, w, keys.size, int(K), SCHEMES[scheme], seed_value & (2**64 - 1),
                          float(lbg_eps), float(conv_eps), int(max_iter), c)
    if k_eff < 0:
        raise ValueError("oracle seed failed")
    return c.reshape(K, 3), int(k_eff)


def sff_size(n: int, K: int) -> int:
    return int(lib().or_sff_size(n, K))


def var_channel(keys: np.ndarray, w: np.ndarray) -> int:
    keys = np.ascontiguousarray(keys, dtype=np.uint32)
    return int(lib().or_var_channel(keys, np.ascontiguousarray(w, dtype=np.uint32), keys.size))


def wu(keys: np.ndarray, w: np.ndarray, K: int) -> Tuple[np.ndarray, int]:
    """Wu's greedy orthogonal bipartitioning: (K x 3 box means, boxes made)."""
    keys = np.ascontiguousarray(keys, dtype=np.uint32)
    c = np.zeros(K * 3, dtype=np.float64)
    nb = lib().or_wu(keys, np.ascontiguousarray(w, dtype=np.uint32), keys.size, int(K), c)
    if nb < 0:
        raise ValueError("oracle wu failed")
    return c.reshape(K, 3), int(nb)


LAB_SCALE = 256  # fixed-point units per L*a*b* unit


def lab(keys: np.ndarray) -> np.ndarray:
    """CIE 1976 L*a*b* (D65) of 24-bit sRGB colours, FP64, (n, 3)."""
    keys = np.ascontiguousarray(keys, dtype=np.uint32).reshape(-1)
    out = np.empty((keys.size, 3), dtype=np.float64)
    v = np.empty(3, dtype=np.float64)
    for i, k in enumerate(keys):
        lib().or_lab(int(k), v)
        out[i] = v
    return out


def lab_points(keys: np.ndarray) -> np.ndarray:
    """Fixed-point L*a*b* points (n, 4) int32: round(L*, a*, b* x 256), 0."""
    keys = np.ascontiguousarray(keys, dtype=np.uint32).reshape(-1)
    pts = np.empty((max(keys.size, 1), 4), dtype=np.int32)
    lib().or_lab_points(keys, keys.size, pts)
    return pts[:keys.size]


def lab_palette(centers: np.ndarray) -> np.ndarray:
    """sRGB palette (K, 3) uint8 of centres given in fixed-point L*a*b* units."""
    c = np.ascontiguousarray(centers, dtype=np.float64).reshape(-1)
    pal = np.empty(c.size, dtype=np.uint8)
    lib().or_lab_palette(c, c.size // 3, pal)
    return pal.reshape(-1, 3)


def assign_points(pts: np.ndarray, w: np.ndarray, centers: np.ndarray):
    pts = np.ascontiguousarray(pts, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.uint32)
    c = np.ascontiguousarray(centers, dtype=np.float64).reshape(-1)
    n = pts.shape[0]
    lab_ = np.empty(max(n, 1), dtype=np.uint8)
    d1 = np.empty(max(n, 1), dtype=np.float64)
    d2 = np.empty(max(n, 1), dtype=np.float64)
    sse = lib().or_assign_points(pts, w, n, c.size // 3, c, lab_, d1, d2)
    return lab_[:n], d1[:n], d2[:n], sse


def update_points(pts: np.ndarray, w: np.ndarray, labels: np.ndarray, centers: np.ndarray):
    pts = np.ascontiguousarray(pts, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.uint32)
    c = np.ascontiguousarray(centers, dtype=np.float64).reshape(-1)
    K = c.size // 3
    out = np.empty_like(c)
    sums = np.empty(K * 4, dtype=np.int64)
    lib().or_update_points(pts, w, pts.shape[0], K, np.ascontiguousarray(labels, dtype=np.uint8), c, out, sums)
    return out.reshape(K, 3), sums.reshape(K, 4)


def lloyd_points(pts: np.ndarray, w: np.ndarray, centers: np.ndarray, eps: float, max_iter: int) -> Dict:
    pts = np.ascontiguousarray(pts, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.uint32)
    c = np.array(centers, dtype=np.float64).reshape(-1).copy()
    K = c.size // 3
    lab_ = np.zeros(max(pts.shape[0], 1), dtype=np.uint8)
    hist = np.zeros(max(1, max_iter), dtype=np.float64)
    conv = C.c_int(0)
    sums = np.zeros(K * 4, dtype=np.int64)
    it = lib().or_lloyd_points(pts, w, pts.shape[0], K, c, float(eps), int(max_iter), lab_, hist, C.byref(conv),
                               sums)
    return {"centers": c.reshape(K, 3), "labels": lab_[:pts.shape[0]], "sse_hist": hist[:it], "iters": it,
            "converged": bool(conv.value), "sums": sums.reshape(K, 4)}


def seed_points_fgy(pts: np.ndarray, K: int, seed_value: int) -> np.ndarray:
    pts = np.ascontiguousarray(pts, dtype=np.int32)
    c = np.zeros(K * 3, dtype=np.float64)
    lib().or_seed_points_fgy(pts, pts.shape[0], int(K), seed_value & (2**64 - 1), c)
    return c.reshape(K, 3)


def den_quota(cellw: np.ndarray, celln: np.ndarray, K: int) -> np.ndarray:
    q = np.zeros(64, dtype=np.int64)
    lib().or_den_quota(np.ascontiguousarray(cellw, dtype=np.int64), np.ascontiguousarray(celln, dtype=np.int64),
                       int(K), q)
    return q


def quantize(rgb: np.ndarray, K: int, scheme: str, seed_value: int, eps: float, max_iter: int) -> Dict:
    """The whole method on one image: histogram, seed, Lloyd, palette, mapping."""
    keys, w = histogram(rgb)
    c0, k_eff = seed(keys, w, K, scheme, seed_value, conv_eps=eps, max_iter=max_iter)
    run = lloyd(keys, w, c0, eps, max_iter)
    pal = palette(run["sums"], run["centers"])
    idx, sse = map_pixels(rgb, pal)
    n = _pixels(rgb).size // 3
    return {"keys": keys, "weights": w, "seeds": c0, "k_eff": k_eff, "palette": pal, "idx": idx,
            "sse_num": sse, "mse": mse(sse, n), **run}


def main() -> None:  # pragma: no cover - manual smoke run
    here = os.path.dirname(os.path.abspath(__file__))
    print("oracle library:", _build.build())
    print("location:", here)


if __name__ == "__main__":  # pragma: no cover
    main()
