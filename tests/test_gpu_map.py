"""kq_map vs the oracle: indices and squared-error sums bit-exact."""
import numpy as np
import pytest
import torch

import oracle
from paper_1101_0395_gb300 import synth
from tests.gpu_helpers import Run, require_cuda, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    require_cuda()


def palette_for(keys, K, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 256, size=(K, 3)).astype(np.uint8)


@pytest.mark.parametrize("name,K", [("plain_256", 16), ("paper_512", 32), ("paper_512", 256)])
def test_map_workloads(name, K):
    img = synth.WORKLOADS[name].make(1)
    r = Run(img)
    keys, w = r.histogram()
    pal = palette_for(keys, K, K)
    idx, sse = r.map(pal)
    oidx, osse = oracle.map_pixels(img, pal)
    assert np.array_equal(idx, oidx) and sse == osse


@pytest.mark.parametrize("n", [1, 7, 16, 17, 100, 4099])
@pytest.mark.parametrize("offset", [0, 1, 5])
def test_map_ragged_and_misaligned(n, offset):
    rng = np.random.default_rng(n * 31 + offset)
    img = rng.integers(0, 256, size=(n, 3), dtype=np.uint8)
    img[n // 3:] = img[n // 3:] // 16 * 16
    r = Run(img)
    keys, w = r.histogram()
    pal = palette_for(keys, 40, n)
    buf = torch.zeros(img.size + 64, dtype=torch.uint8, device="cuda")
    buf[offset:offset + img.size] = to_dev(img.reshape(-1))
    idx, sse = r.map(pal, rgb=buf[offset:offset + img.size], idx_offset=(offset * 7) % 16)
    oidx, osse = oracle.map_pixels(img, pal)
    assert np.array_equal(idx, oidx) and sse == osse


def test_map_ties_go_to_lowest_index():
    img = np.array([[10, 10, 10], [20, 20, 20], [15, 15, 15], [0, 0, 0]] * 10, dtype=np.uint8)
    pal = np.array([[20, 20, 20], [10, 10, 10], [10, 10, 10], [20, 20, 20]], dtype=np.uint8)
    r = Run(img)
    r.histogram()
    idx, sse = r.map(pal)
    oidx, osse = oracle.map_pixels(img, pal)
    assert np.array_equal(idx, oidx) and sse == osse
    assert idx[:4].tolist() == [1, 0, 0, 1]


def test_map_k1_and_k256():
    img = synth.WORKLOADS["plain_256"].make(3)
    r = Run(img)
    keys, w = r.histogram()
    for K in (1, 256):
        pal = palette_for(keys, K, 99 + K)
        idx, sse = r.map(pal)
        oidx, osse = oracle.map_pixels(img, pal)
        assert np.array_equal(idx, oidx) and sse == osse


def test_map_large_sampled():
    # 4096 x 4096: every pixel's index checked on a 200k-pixel sample, the error
    # sum checked exactly through the unique colours
    img = synth.WORKLOADS["large_4096"].make(0)
    r = Run(img)
    keys, w = r.histogram()
    pal = palette_for(keys, 256, 7)
    idx, sse = r.map(pal)
    px = img.reshape(-1, 3)
    sel = np.random.default_rng(0).choice(px.shape[0], 200_000, replace=False)
    oidx, _ = oracle.map_pixels(px[sel], pal)
    assert np.array_equal(idx[sel], oidx)
    uimg = oracle.key_to_rgb(keys).astype(np.uint8)
    uidx, _ = oracle.map_pixels(uimg, pal)
    d = ((oracle.key_to_rgb(keys) - pal[uidx].astype(np.int64)) ** 2).sum(axis=1)
    assert sse == int((d * w.astype(np.int64)).sum())


def test_map_needs_no_histogram_and_keeps_no_state():
    # kq_map depends on the pixels and the palette only: two images mapped in turn on
    # one workspace, with no histogram computed, each equal to the oracle's mapping
    from paper_1101_0395_gb300 import kq

    a = synth.WORKLOADS["plain_256"].make(0)
    b = synth.WORKLOADS["paper_512"].make(1)
    ws = torch.zeros(kq.kq_workspace_size(b.size // 3, 256), dtype=torch.uint8, device="cuda")
    for K, seed in ((64, 5), (200, 6)):
        pal = palette_for(None, K, seed)
        for img in (a, b, a):
            r = Run(img, ws=ws)
            idx, sse = r.map(pal)
            oidx, osse = oracle.map_pixels(img, pal)
            assert np.array_equal(idx, oidx) and sse == osse
    assert kq.kq_status_read(ws) == kq.KQ_OK


@pytest.mark.parametrize("K", [1, 2, 16, 256])
def test_map_pruned_search_counts(K):
    # the palette search is exact and prunes: N <= NDC <= N K
    from paper_1101_0395_gb300 import kq

    img = synth.WORKLOADS["paper_512"].make(2)
    r = Run(img)
    keys, w = r.histogram()
    pal = palette_for(keys, K, 3 * K)
    idx, sse = r.map(pal)
    oidx, osse = oracle.map_pixels(img, pal)
    assert np.array_equal(idx, oidx) and sse == osse
    ndc = kq.kq_map_ndc_read(r.ws)
    n = img.size // 3
    assert n <= ndc <= n * K
    if K == 256:
        assert ndc < n * K // 16


def test_map_duplicate_and_clustered_palettes():
    # palettes with repeated entries and entries closer together than the colours
    img = synth.WORKLOADS["plain_256"].make(2)
    r = Run(img)
    keys, w = r.histogram()
    rng = np.random.default_rng(77)
    base = rng.integers(0, 256, size=(8, 3))
    pal = np.concatenate([base, base, base + rng.integers(-2, 3, size=(8, 3))]).clip(0, 255).astype(np.uint8)
    rng.shuffle(pal)
    idx, sse = r.map(pal)
    oidx, osse = oracle.map_pixels(img, pal)
    assert np.array_equal(idx, oidx) and sse == osse
