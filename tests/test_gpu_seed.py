"""kq_seed vs the oracle: every integer scheme and WU (integer moments, FP64 in one
fixed order) bit-exact; LBG within tolerance."""
import numpy as np
import pytest

import oracle
from paper_1101_0395_gb300 import synth
from tests.gpu_helpers import CENTER_ABS, Run, require_cuda

pytestmark = pytest.mark.gpu

EXACT = ["FGY", "MMX", "DEN", "VAR", "SFF", "KPP", "WU"]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    require_cuda()


@pytest.fixture(scope="module")
def plain():
    img = synth.WORKLOADS["plain_256"].make(0)
    r = Run(img)
    keys, w = r.histogram()
    return r, keys, w


@pytest.fixture(scope="module")
def paper():
    img = synth.WORKLOADS["paper_512"].make(0)
    r = Run(img)
    keys, w = r.histogram()
    return r, keys, w


@pytest.mark.parametrize("scheme", EXACT)
@pytest.mark.parametrize("K,seed", [(1, 3), (16, 11), (37, 12)])
def test_seed_exact_plain(plain, scheme, K, seed):
    r, keys, w = plain
    got = r.seed(K, scheme, seed)
    want, _ = oracle.seed(keys, w, K, scheme, seed)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("scheme", EXACT)
@pytest.mark.parametrize("K", [32, 256])
def test_seed_exact_paper_scale(paper, scheme, K):
    r, keys, w = paper
    got = r.seed(K, scheme, 2024 + K)
    want, _ = oracle.seed(keys, w, K, scheme, 2024 + K)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("scheme", EXACT + ["LBG"])
def test_seed_k_at_least_unique(scheme):
    img = np.array([[1, 2, 3], [4, 5, 6], [1, 2, 3], [200, 100, 50]], dtype=np.uint8)
    r = Run(img)
    keys, w = r.histogram()
    got = r.seed(5, scheme, 9)
    want, k_eff = oracle.seed(keys, w, 5, scheme, 9)
    assert k_eff == 3 and np.array_equal(got, want)


@pytest.mark.parametrize("K", [1, 2, 3, 8, 13])
def test_seed_lbg(plain, K):
    r, keys, w = plain
    got = r.seed(K, "LBG", 0, lbg_eps=1.0, conv_eps=1e-4, max_iter=100)
    want, _ = oracle.seed(keys, w, K, "LBG", 0, lbg_eps=1.0, conv_eps=1e-4, max_iter=100)
    if K == 1:
        assert np.array_equal(got, want)  # the centroid: exact sums, one FP64 division
    assert np.max(np.abs(got - want)) <= CENTER_ABS


@pytest.fixture(scope="module")
def large():
    img = synth.WORKLOADS["large_4096"].make(0)
    r = Run(img)
    keys, w = r.histogram()
    return r, keys, w


@pytest.mark.parametrize("scheme,K,seed", [("KPP", 256, 1), ("MMX", 256, 2), ("KPP", 7, 3), ("MMX", 2, 4)])
def test_seed_exact_grid(large, scheme, K, seed):
    """N' = 1.28 M, beyond one thread-block cluster: the whole-grid kernel, each
    block holding its slice in shared memory."""
    r, keys, w = large
    assert len(keys) > 1_000_000
    got = r.seed(K, scheme, seed)
    want, _ = oracle.seed(keys, w, K, scheme, seed)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("scheme", ["KPP", "MMX"])
def test_seed_exact_grid_slices_in_global_memory(scheme):
    """Uniform random 2048 x 2048 image, ~3.7 M unique colours: slices larger than a
    block keeps in shared memory, so D^2 stays in global memory."""
    img = np.random.default_rng(77).integers(0, 256, size=(2048, 2048, 3), dtype=np.uint8)
    r = Run(img)
    keys, w = r.histogram()
    assert len(keys) > 3_000_000
    got = r.seed(16, scheme, 5)
    want, _ = oracle.seed(keys, w, 16, scheme, 5)
    assert np.array_equal(got, want)


def test_seed_wu_single_cell_and_large(large):
    """All colours in one 8x8x8 cell: one box, every centre its mean.  And the
    4096 x 4096 image (1.28 M colours) at K = 256."""
    img = np.array([[8, 16, 0], [9, 16, 7], [8, 20, 3], [9, 20, 0]] * 5, dtype=np.uint8)
    r = Run(img)
    keys, w = r.histogram()
    got = r.seed(3, "WU", 0)
    want, _ = oracle.seed(keys, w, 3, "WU", 0)
    assert np.array_equal(got, want) and np.all(got == got[0])
    rb, kb, wb = large
    got = rb.seed(256, "WU", 0)
    want, _ = oracle.seed(kb, wb, 256, "WU", 0)
    assert np.array_equal(got, want)
