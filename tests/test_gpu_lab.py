"""k-means in CIE L*a*b* (Section 2.1) against the oracle.

* points: bit-exact fixed point for the test images' colours and for all 2^24
  colours (both sides FP64 with the same operations in the same order);
* seeds: Forgy among the points, bit-exact;
* Lloyd on the points: lockstep with the near-tie rule (labels equal except where
  the oracle's best and second distances are within 1e-5 relative; centres the
  oracle's update of the GPU labels, bit for bit; SSE within 1e-5), pruned ==
  full search bit for bit, K = 1 gives the exact weighted mean;
* palette: the inverse transform, bit-exact 8-bit values;
* mapping: each pixel gets its colour's label; foreign colours are reported.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1101_0395_gb300 import kq, synth
from tests.gpu_helpers import CENTER_ABS, MSE_REL, Run, require_cuda, to_dev, u32

pytestmark = pytest.mark.gpu


def unpack(points: np.ndarray) -> np.ndarray:
    """uint64 points -> (n, 4) int32 as the oracle writes them."""
    p = points.view(np.uint64)
    out = np.zeros((p.size, 4), dtype=np.int32)
    for c in range(3):
        out[:, c] = ((p >> np.uint64(16 * c)) & np.uint64(0xFFFF)).astype(np.uint16).view(np.int16)
    return out


class LabRun:
    def __init__(self, img):
        self.r = Run(img)
        self.keys, self.w = self.r.histogram()
        self.n = self.keys.size
        self.points = torch.zeros(max(self.n, 1), dtype=torch.int64, device="cuda")
        kq.kq_lab_points(self.r.keys, self.r.n_unique, self.points)
        torch.cuda.synchronize()
        self.pts = unpack(self.points[:self.n].cpu().numpy())

    def lloyd(self, c0, eps, max_iter, flags=0, labels_in=None):
        K = c0.shape[0]
        c = to_dev(np.ascontiguousarray(c0, dtype=np.float64).reshape(-1))
        st = torch.zeros(64, dtype=torch.uint8, device="cuda")
        hist = torch.zeros(max_iter, dtype=torch.float64, device="cuda")
        if labels_in is not None:
            self.r.labels[:self.n].copy_(to_dev(labels_in.astype(np.uint8)))
        kq.kq_lloyd_points(self.points, self.r.weights, self.r.n_unique, K, c, eps, max_iter, self.r.labels,
                           self.r.ws, stats=st, sse_hist=hist, flags=flags)
        torch.cuda.synchronize()
        s = kq.parse_stats(st)
        return {"centers": c.cpu().numpy().reshape(K, 3), "labels": self.r.labels[:self.n].cpu().numpy().copy(),
                "stats": s, "sse_hist": hist.cpu().numpy()[:s["iters"]]}


@pytest.fixture(scope="module")
def paper():
    require_cuda()
    return LabRun(synth.WORKLOADS["paper_512"].make(3))


@pytest.fixture(scope="module")
def plain():
    require_cuda()
    return LabRun(synth.WORKLOADS["plain_256"].make(1))


def test_points_match_the_oracle(paper, plain):
    for lr in (paper, plain):
        assert np.array_equal(lr.pts, oracle.lab_points(lr.keys))


def test_points_of_every_colour_match_the_oracle():
    # all 2^24 colours, in slices of 2^22
    require_cuda()
    step = 1 << 22
    keys = torch.arange(0, 1 << 24, dtype=torch.int32, device="cuda")
    pts = torch.zeros(1 << 24, dtype=torch.int64, device="cuda")
    n = torch.tensor([1 << 24], dtype=torch.int32, device="cuda")
    kq.kq_lab_points(keys, n, pts)
    torch.cuda.synchronize()
    got = pts.cpu().numpy()
    for lo in range(0, 1 << 24, step):
        want = oracle.lab_points(np.arange(lo, lo + step, dtype=np.uint32))
        assert np.array_equal(unpack(got[lo:lo + step]), want), lo


@pytest.mark.parametrize("K", [1, 16, 256])
def test_forgy_seeds_among_points(paper, K):
    c = torch.zeros(3 * K, dtype=torch.float64, device="cuda")
    kq.kq_seed_points(paper.points, paper.r.n_unique, K, "FGY", 41 + K, c)
    torch.cuda.synchronize()
    assert np.array_equal(c.cpu().numpy().reshape(K, 3), oracle.seed_points_fgy(paper.pts, K, 41 + K))


def test_forgy_seeds_when_k_exceeds_the_points():
    require_cuda()
    img = np.array([[10, 20, 30], [40, 50, 60], [10, 20, 30]], dtype=np.uint8)
    lr = LabRun(img)
    c = torch.zeros(3 * 5, dtype=torch.float64, device="cuda")
    kq.kq_seed_points(lr.points, lr.r.n_unique, 5, "FGY", 3, c)
    torch.cuda.synchronize()
    assert np.array_equal(c.cpu().numpy().reshape(5, 3), oracle.seed_points_fgy(lr.pts, 5, 3))


def lockstep_points(lr, c0, passes):
    c = np.array(c0, dtype=np.float64)
    prev = None
    flips = 0
    for i in range(passes):
        lab_o, d1, d2, sse_o = oracle.assign_points(lr.pts, lr.w, c)
        c_next, _ = oracle.update_points(lr.pts, lr.w, lab_o, c)
        g = lr.lloyd(c, -1.0, 1, flags=0 if prev is None else kq.LLOYD_LABELS_IN, labels_in=prev)
        x = lr.pts[:, :3].astype(np.float64)
        diff = np.nonzero(g["labels"] != lab_o)[0]
        if diff.size:
            tol = 1e-5 * np.maximum(d1[diff], 1.0)
            assert np.all(d2[diff] - d1[diff] <= tol), i
            dg = ((x[diff] - c[g["labels"][diff]]) ** 2).sum(axis=1)
            assert np.all(dg - d1[diff] <= tol), i
            flips += diff.size
        c_on_gpu, _ = oracle.update_points(lr.pts, lr.w, g["labels"], c)
        assert np.array_equal(g["centers"], c_on_gpu), i
        assert abs(g["stats"]["sse"] - sse_o) <= MSE_REL * max(sse_o, 1.0), (i, g["stats"]["sse"], sse_o)
        assert np.max(np.abs(g["centers"] - c_next)) <= CENTER_ABS * oracle.LAB_SCALE or diff.size
        prev, c = lab_o, c_next
    return flips


@pytest.mark.parametrize("K", [16, 64, 256])
def test_lloyd_points_lockstep(paper, K):
    c0 = oracle.seed_points_fgy(paper.pts, K, 7 + K)
    lockstep_points(paper, c0, 5)


def test_lloyd_points_free_run_pruned_equals_dense_and_oracle(paper, plain):
    for lr, K in ((plain, 16), (paper, 128)):
        c0 = oracle.seed_points_fgy(lr.pts, K, 5)
        a = lr.lloyd(c0, 1e-4, 100)
        b = lr.lloyd(c0, 1e-4, 100, flags=kq.LLOYD_DENSE)
        assert np.array_equal(a["labels"], b["labels"]) and np.array_equal(a["centers"], b["centers"])
        assert np.array_equal(a["sse_hist"], b["sse_hist"])
        assert a["stats"]["ndc"] < b["stats"]["ndc"]
        o = oracle.lloyd_points(lr.pts, lr.w, c0, 1e-4, 100)
        print("\n[L*a*b* K=%d] passes gpu=%d oracle=%d, final SSE rel. diff %.2e"
              % (K, a["stats"]["iters"], o["iters"], abs(a["stats"]["sse"] - o["sse_hist"][-1]) / o["sse_hist"][-1]))
        if o["iters"] == a["stats"]["iters"] and np.array_equal(o["labels"], a["labels"]):
            assert np.array_equal(o["centers"], a["centers"])
            assert abs(a["stats"]["sse"] - o["sse_hist"][-1]) <= MSE_REL * o["sse_hist"][-1]


def test_lloyd_points_k1_is_the_weighted_mean(plain):
    g = plain.lloyd(np.array([[5000.0, 100.0, -100.0]]), 1e-4, 10)
    W = int(plain.w.astype(np.int64).sum())
    for ch in range(3):
        S = int((plain.w.astype(np.int64) * plain.pts[:, ch].astype(np.int64)).sum())
        assert g["centers"][0, ch] == S / W


def test_lab_palette_matches_the_oracle(paper):
    rng = np.random.default_rng(5)
    # final centres of a run, the points themselves and random points of the gamut
    c0 = oracle.seed_points_fgy(paper.pts, 64, 9)
    run = paper.lloyd(c0, 1e-4, 50)
    cents = np.concatenate([run["centers"], paper.pts[:2000, :3].astype(np.float64),
                            rng.uniform([0, -80, -100], [100, 90, 90], size=(3000, 3)) * oracle.LAB_SCALE])
    for lo in range(0, cents.shape[0], 256):
        c = cents[lo:lo + 256]
        K = c.shape[0]
        pal = torch.zeros(3 * K, dtype=torch.uint8, device="cuda")
        kq.kq_lab_palette(to_dev(np.ascontiguousarray(c.reshape(-1))), K, pal)
        torch.cuda.synchronize()
        assert np.array_equal(pal.cpu().numpy().reshape(K, 3), oracle.lab_palette(c)), lo


def test_map_labels(paper):
    lr = paper
    c0 = oracle.seed_points_fgy(lr.pts, 32, 2)
    run = lr.lloyd(c0, 1e-4, 30)
    img = synth.WORKLOADS["paper_512"].make(3)
    n = img.size // 3
    idx = torch.zeros(n, dtype=torch.uint8, device="cuda")
    kq.kq_map_labels(lr.r.rgb, lr.r.keys, lr.r.n_unique, lr.r.labels, idx, lr.r.ws)
    torch.cuda.synchronize()
    px = img.reshape(-1, 3).astype(np.uint32)
    pk = (px[:, 0] << 16) | (px[:, 1] << 8) | px[:, 2]
    assert np.array_equal(idx.cpu().numpy(), run["labels"][np.searchsorted(lr.keys, pk)])
    assert lr.r.status() == kq.KQ_OK
    # another image's pixels: colours missing from these keys are reported
    other = to_dev(synth.WORKLOADS["paper_512"].make(4).reshape(-1))
    kq.kq_map_labels(other, lr.r.keys, lr.r.n_unique, lr.r.labels, idx, lr.r.ws)
    assert kq.kq_status_read(lr.r.ws) == kq.KQ_EINVAL
    kq.kq_status_clear(lr.r.ws)
    # the table is zero again: the first mapping repeats exactly
    kq.kq_map_labels(lr.r.rgb, lr.r.keys, lr.r.n_unique, lr.r.labels, idx, lr.r.ws)
    torch.cuda.synchronize()
    assert lr.r.status() == kq.KQ_OK
    assert np.array_equal(idx.cpu().numpy(), run["labels"][np.searchsorted(lr.keys, pk)])


def test_lab_quantizer_pipeline_against_the_oracle():
    require_cuda()
    img = synth.WORKLOADS["plain_256"].make(6)
    n = img.size // 3
    q = kq.LabQuantizer(n)
    rgb = to_dev(img.reshape(-1))
    res = q.quantize(rgb, 24, "FGY", 77, 1e-4, 100)
    torch.cuda.synchronize()
    keys, w = oracle.histogram(img)
    pts = oracle.lab_points(keys)
    c0 = oracle.seed_points_fgy(pts, 24, 77)
    o = oracle.lloyd_points(pts, w, c0, 1e-4, 100)
    st = kq.parse_stats(res.stats)
    assert st["status"] == kq.KQ_OK and st["k_eff"] == 24
    assert abs(st["sse"] - o["sse_hist"][-1]) <= 1e-4 * o["sse_hist"][-1]
    if st["iters"] == o["iters"]:
        assert np.max(np.abs(res.centers.cpu().numpy() - o["centers"])) <= CENTER_ABS * oracle.LAB_SCALE
        assert np.array_equal(res.palette.cpu().numpy(), oracle.lab_palette(o["centers"]))
    px = img.reshape(-1, 3).astype(np.uint32)
    pk = (px[:, 0] << 16) | (px[:, 1] << 8) | px[:, 2]
    lab = q.labels[:keys.size].cpu().numpy()
    assert np.array_equal(res.idx.cpu().numpy(), lab[np.searchsorted(keys, pk)])
    assert np.array_equal(u32(q.keys[:keys.size]), keys)
