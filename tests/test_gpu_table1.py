"""The k-means baseline of Table 1: k-means on all N pixels (every pixel its own
point, full search) and Weighted Sort-Means on the unique colours, from the same
centres for 20 passes, reach the same centres bit for bit: the exact integer sums
of a cluster do not depend on whether a colour is counted once per pixel or once
with its pixel count, and both searches take the same FP32 argmin.  The k-means
path is also checked against the oracle's plain Lloyd on the N pixels, in
lockstep and as a free run."""
import numpy as np
import pytest
import torch

import oracle
from paper_1101_0395_gb300 import kq, synth
from tests.gpu_helpers import CENTER_ABS, MSE_REL, Run, lockstep, require_cuda, to_dev, u32

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("K", [16, 64])
def test_kmeans_on_all_pixels_equals_wsm(K):
    require_cuda()
    img = synth.WORKLOADS["plain_256"].make(3)
    n = img.size // 3
    rgb = to_dev(img.reshape(-1))
    q = kq.Quantizer(n)
    kq.kq_histogram(rgb, q.keys, q.weights, q.n_unique, q.ws)
    c0 = torch.zeros(3 * K, dtype=torch.float64, device="cuda")
    kq.kq_seed(q.keys, q.weights, q.n_unique, K, "FGY", 5, c0, q.ws)
    c_wsm = c0.clone()
    pal_wsm = torch.zeros(3 * K, dtype=torch.uint8, device="cuda")
    st_wsm = torch.zeros(64, dtype=torch.uint8, device="cuda")
    kq.kq_lloyd(q.keys, q.weights, q.n_unique, K, c_wsm, -1.0, 20, q.labels, pal_wsm, q.ws, stats=st_wsm)
    pk = torch.zeros(n, dtype=torch.int32, device="cuda")
    pw = torch.zeros(n, dtype=torch.int32, device="cuda")
    pn = torch.zeros(1, dtype=torch.int32, device="cuda")
    kq.kq_pixel_keys(rgb, pk, pw, pn)
    ws2 = torch.zeros(kq.kq_workspace_size(n, 256), dtype=torch.uint8, device="cuda")
    c_km = c0.clone()
    pal_km = torch.zeros(3 * K, dtype=torch.uint8, device="cuda")
    st_km = torch.zeros(64, dtype=torch.uint8, device="cuda")
    lab_km = torch.zeros(n, dtype=torch.uint8, device="cuda")
    kq.kq_lloyd(pk, pw, pn, K, c_km, -1.0, 20, lab_km, pal_km, ws2, stats=st_km, flags=kq.LLOYD_DENSE)
    torch.cuda.synchronize()
    assert int(pn.item()) == n and np.all(u32(pw) == 1)
    px = img.reshape(-1, 3).astype(np.uint32)
    assert np.array_equal(u32(pk), (px[:, 0] << 16) | (px[:, 1] << 8) | px[:, 2])
    s_wsm, s_km = kq.parse_stats(st_wsm), kq.parse_stats(st_km)
    assert s_wsm["iters"] == s_km["iters"] == 20
    assert torch.equal(c_wsm, c_km) and torch.equal(pal_wsm, pal_km)
    assert abs(s_wsm["sse"] - s_km["sse"]) <= MSE_REL * s_km["sse"]
    nu = int(q.n_unique.item())
    keys = u32(q.keys[:nu])
    lab_of_colour = q.labels[:nu].cpu().numpy()
    pos = np.searchsorted(keys, u32(pk))
    assert np.array_equal(lab_km.cpu().numpy(), lab_of_colour[pos])
    assert s_km["ndc"] == n * K * 20
    assert s_wsm["ndc"] < nu * K * 20


def _pixel_points(img):
    """k-means on all N pixels: every pixel its own point of weight 1, in pixel order."""
    px = img.reshape(-1, 3).astype(np.uint32)
    keys = (px[:, 0] << 16) | (px[:, 1] << 8) | px[:, 2]
    return keys, np.ones(keys.size, dtype=np.uint32)


@pytest.mark.parametrize("K", [16, 64])
def test_kmeans_on_all_pixels_against_the_oracle(K):
    """The k-means baseline (Section 3.2, Table 1: 20 passes from the same random
    centres) against the oracle's plain Lloyd on the same N points: lockstep for
    20 passes, then the free run of 20 fixed passes."""
    require_cuda()
    img = synth.WORKLOADS["plain_256"].make(3)
    r = Run(img)
    kq.kq_pixel_keys(r.rgb, r.keys, r.weights, r.n_unique)
    torch.cuda.synchronize()
    pkeys, ones = _pixel_points(img)
    assert int(r.n_unique.item()) == pkeys.size
    assert np.array_equal(u32(r.keys), pkeys) and np.all(u32(r.weights) == 1)
    ukeys, uw = oracle.histogram(img)
    c0, _ = oracle.seed(ukeys, uw, K, "FGY", 5)  # Forgy centres, as in Table 1
    flips, _, _ = lockstep(r, pkeys, ones, c0, 20, dense=True)
    g = r.lloyd(c0, eps=-1.0, max_iter=20, flags=kq.LLOYD_DENSE)
    o = oracle.lloyd(pkeys, ones, c0, -1.0, 20)
    assert g["stats"]["iters"] == o["iters"] == 20
    assert g["stats"]["ndc"] == pkeys.size * K * 20
    assert abs(g["stats"]["sse"] - o["sse_hist"][-1]) <= MSE_REL * o["sse_hist"][-1]
    assert np.allclose(g["sse_hist"], o["sse_hist"], rtol=MSE_REL, atol=0.0)
    if flips == 0:
        assert np.array_equal(g["labels"], o["labels"])
        assert np.array_equal(g["centers"], o["centers"])
        assert np.array_equal(g["palette"], oracle.palette(o["sums"], o["centers"]))
    else:
        assert np.max(np.abs(g["centers"] - o["centers"])) <= CENTER_ABS
