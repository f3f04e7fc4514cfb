"""The k-means baseline of Table 1: k-means on all N pixels (every pixel its own
point, full search) and Weighted Sort-Means on the unique colours, from the same
centres for 20 passes, reach the same centres bit for bit: the exact integer sums
of a cluster do not depend on whether a colour is counted once per pixel or once
with its pixel count, and both searches take the same FP32 argmin."""
import numpy as np
import pytest
import torch

from paper_1101_0395_gb300 import kq, synth
from tests.gpu_helpers import MSE_REL, require_cuda, to_dev, u32

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
