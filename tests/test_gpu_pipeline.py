"""The whole path through the public API (Quantizer -> the four C calls) on the
workload bench.py times: 512 x 512, K = 256, k-means++ seeds, eps 1e-4, at most
100 passes.  Every step is checked against the oracle: histogram and seeds
bit-exact, every Lloyd pass from the GPU's own state, mapping bit-exact."""
import numpy as np
import pytest
import torch

import oracle
from paper_1101_0395_gb300 import kq, synth
from tests.gpu_helpers import Run, require_cuda, to_dev, u32
from tests.test_gpu_lloyd import gpu_trajectory

pytestmark = pytest.mark.gpu

BENCH_SEED = 1101


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    require_cuda()


@pytest.mark.parametrize("name,K", [("paper_512", 256), ("plain_256", 16)])
def test_quantizer_end_to_end(name, K):
    wl = synth.WORKLOADS[name]
    img = wl.make(0)
    q = kq.Quantizer(img.size // 3)
    res = q.quantize(to_dev(img.reshape(-1)), K, "KPP", BENCH_SEED, wl.eps, wl.max_iter)
    torch.cuda.synchronize()
    nu = int(res.n_unique.item())
    keys, w = u32(q.keys[:nu]), u32(q.weights[:nu])
    ok, ow = oracle.histogram(img)
    assert np.array_equal(keys, ok) and np.array_equal(w, ow)
    c0, _ = oracle.seed(keys, w, K, "KPP", BENCH_SEED)
    r = Run(img)
    r.histogram()
    c, labels, hist, _, _ = gpu_trajectory(r, keys, w, c0, wl.eps, wl.max_iter)
    st = kq.parse_stats(res.stats)
    assert st["iters"] == hist.size and st["sse"] == hist[-1]
    assert np.array_equal(res.centers.cpu().numpy(), c)
    assert np.array_equal(q.labels[:nu].cpu().numpy(), labels)
    _, sums = oracle.update(keys, w, labels, c)
    pal = res.palette.cpu().numpy()
    assert np.array_equal(pal, oracle.palette(sums, c))
    oidx, osse = oracle.map_pixels(img, pal)
    assert np.array_equal(res.idx.cpu().numpy(), oidx)
    assert int(res.sse_num.item()) == osse
    assert kq.kq_status_read(q.ws) == kq.KQ_OK


def test_quantizer_reuse_across_images():
    q = kq.Quantizer(512 * 512)
    for i, name in enumerate(["paper_512", "plain_256", "paper_512"]):
        img = synth.WORKLOADS[name].make(i + 5)
        res = q.quantize(to_dev(img.reshape(-1)), 32, "VAR", 0, 1e-4, 100)
        torch.cuda.synchronize()
        pal = res.palette.cpu().numpy()
        oidx, osse = oracle.map_pixels(img, pal)
        assert np.array_equal(res.idx.cpu().numpy(), oidx) and int(res.sse_num.item()) == osse
        nu = int(res.n_unique.item())
        ok, ow = oracle.histogram(img)
        assert nu == ok.size and np.array_equal(u32(q.keys[:nu]), ok)
