"""Helpers for the GPU parity tests: run the CUDA path through the C ABI on
seeded inputs and bring results back as numpy arrays."""
import numpy as np
import torch

import oracle
from paper_1101_0395_gb300 import kq

# Match rules (stated in the task contract and derived in the design notes):
NEAR_TIE_REL = 1e-5     # a label may differ only where the oracle's best-vs-second gap is below this
CENTER_ABS = 1e-3       # centres, 0-255 units
MSE_REL = 1e-5          # final MSE / SSE


def require_cuda():
    if not torch.cuda.is_available():
        raise RuntimeError("GPU test run without a CUDA device")
    return torch.device("cuda")


def to_dev(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def u32(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy().view(np.uint32)


def new_ws(max_pixels: int) -> torch.Tensor:
    n = kq.kq_workspace_size(max_pixels, 256)
    return torch.zeros(n, dtype=torch.uint8, device="cuda")


class Run:
    """Device buffers for one image on one workspace."""

    def __init__(self, img: np.ndarray, ws: torch.Tensor = None, capacity: int = None):
        self.img = np.ascontiguousarray(img, dtype=np.uint8)
        self.n = self.img.size // 3
        self.rgb = to_dev(self.img.reshape(-1))
        self.ws = new_ws(max(self.n, 1)) if ws is None else ws
        cap = max(1, min(self.n, 1 << 24)) if capacity is None else capacity
        self.keys = torch.zeros(cap, dtype=torch.int32, device="cuda")
        self.weights = torch.zeros(cap, dtype=torch.int32, device="cuda")
        self.n_unique = torch.zeros(1, dtype=torch.int32, device="cuda")
        self.labels = torch.zeros(cap, dtype=torch.uint8, device="cuda")

    def histogram(self):
        kq.kq_histogram(self.rgb, self.keys, self.weights, self.n_unique, self.ws, n_pixels=self.n)
        torch.cuda.synchronize()
        nu = int(self.n_unique.item())
        return u32(self.keys[:nu]), u32(self.weights[:nu])

    def seed(self, K, scheme, seed, **kw):
        c = torch.zeros(3 * K, dtype=torch.float64, device="cuda")
        kq.kq_seed(self.keys, self.weights, self.n_unique, K, scheme, seed, c, self.ws, **kw)
        torch.cuda.synchronize()
        return c.cpu().numpy().reshape(K, 3)

    def lloyd(self, centers, eps, max_iter, flags=0, labels_in=None):
        K = centers.shape[0]
        c = to_dev(np.asarray(centers, dtype=np.float64).reshape(-1))
        pal = torch.zeros(3 * K, dtype=torch.uint8, device="cuda")
        stats = torch.zeros(64, dtype=torch.uint8, device="cuda")
        hist = torch.zeros(max_iter, dtype=torch.float64, device="cuda")
        if labels_in is not None:
            self.labels[:labels_in.size].copy_(to_dev(labels_in.astype(np.uint8)))
        kq.kq_lloyd(self.keys, self.weights, self.n_unique, K, c, eps, max_iter, self.labels, pal, self.ws,
                    stats=stats, sse_hist=hist, flags=flags)
        torch.cuda.synchronize()
        st = kq.parse_stats(stats)
        nu = int(self.n_unique.item())
        return {"centers": c.cpu().numpy().reshape(K, 3), "palette": pal.cpu().numpy().reshape(K, 3),
                "labels": self.labels[:nu].cpu().numpy().copy(), "stats": st,
                "sse_hist": hist.cpu().numpy()[:st["iters"]]}

    def map(self, palette, rgb=None, idx_offset=0):
        K = palette.shape[0]
        pal = to_dev(np.ascontiguousarray(palette, dtype=np.uint8).reshape(-1))
        out = torch.zeros(self.n + 64, dtype=torch.uint8, device="cuda")
        idx = out[idx_offset:idx_offset + self.n]
        sse = torch.zeros(1, dtype=torch.int64, device="cuda")
        kq.kq_map(self.rgb if rgb is None else rgb, pal, K, idx, self.ws,
                  sse_num=sse, n_pixels=self.n)
        torch.cuda.synchronize()
        return idx.cpu().numpy(), int(sse.item())

    def status(self):
        return kq.kq_status_read(self.ws)


def check_labels(keys, centers, gpu_labels, ora_labels, d1, d2):
    """Labels agree except at oracle near-ties, where the GPU label must be one
    of the near-tied centres.  Returns the number of tolerated flips."""
    diff = np.nonzero(gpu_labels != ora_labels)[0]
    if diff.size == 0:
        return 0
    x = np.stack([(keys[diff] >> 16) & 255, (keys[diff] >> 8) & 255, keys[diff] & 255], axis=1).astype(np.float64)
    tol = NEAR_TIE_REL * np.maximum(d1[diff], 1.0)
    gap = d2[diff] - d1[diff]
    assert np.all(gap <= tol), "label mismatch away from a near-tie at %s" % diff[gap > tol][:10]
    dg = ((x - centers[gpu_labels[diff]]) ** 2).sum(axis=1)
    assert np.all(dg - d1[diff] <= tol), "GPU label is not one of the near-tied centres"
    return int(diff.size)


def lockstep(r, keys, w, c0, passes, dense=False):
    """Lloyd in lockstep with the oracle: every pass starts from the oracle's
    centres (and, for the pruned search, its previous labels).  Labels agree
    except at oracle near-ties; centres are the oracle's update of the GPU labels
    (bit for bit); SSE within MSE_REL.  Returns the number of tolerated near-tie
    flips and the last SSEs."""
    c = np.array(c0, dtype=np.float64)
    prev = None
    flips = 0
    sse_g = sse_o = None
    for i in range(passes):
        lab_o, d1, d2, sse_o = oracle.assign(keys, w, c)
        c_next, sums = oracle.update(keys, w, lab_o, c)
        if dense:
            g = r.lloyd(c, eps=-1.0, max_iter=1, flags=kq.LLOYD_DENSE)
        else:
            g = r.lloyd(c, eps=-1.0, max_iter=1, flags=0 if prev is None else kq.LLOYD_LABELS_IN, labels_in=prev)
        f = check_labels(keys, c, g["labels"], lab_o, d1, d2)
        flips += f
        sse_g = g["stats"]["sse"]
        assert abs(sse_g - sse_o) <= MSE_REL * max(sse_o, 1.0), (i, sse_g, sse_o)
        if f == 0:
            assert np.array_equal(g["centers"], c_next), i
            assert np.array_equal(g["palette"], oracle.palette(sums, c_next)), i
        else:
            c_on_gpu, _ = oracle.update(keys, w, g["labels"], c)
            assert np.array_equal(g["centers"], c_on_gpu), i
        assert np.max(np.abs(g["centers"] - c_next)) <= CENTER_ABS or f > 0
        assert g["stats"]["iters"] == 1
        prev, c = lab_o, c_next
    return flips, sse_g, sse_o
