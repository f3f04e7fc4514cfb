"""Failure detection on the device without a GPU fault.

kq_set_wait_limit gives the bounded waits of the kernels (the grid barriers of
the whole-grid Lloyd and k-means++ launches, the mbarrier exchanges of the
cluster k-means++) a 1 ms limit and makes them expect one arrival that never
comes (no block is missing in fact: the
count is raised on the host).  Every wait then runs out: the kernel writes
KQ_ETIMEOUT to the workspace's status word (and to kq_lloyd's statistics),
the other waiters give up in turn, and the launch returns.  After
kq_status_clear the same workspace gives the normal results.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1101_0395_gb300 import kq, synth
from tests.gpu_helpers import Run, require_cuda

pytestmark = pytest.mark.gpu

LIMIT_US = 1000


@pytest.fixture(scope="module")
def paper():
    require_cuda()
    r = Run(synth.WORKLOADS["paper_512"].make(2))
    keys, w = r.histogram()
    return r, keys, w


@pytest.fixture(scope="module")
def many():
    # ~377k unique colours: Lloyd and k-means++ run on the whole grid (grid barriers)
    require_cuda()
    rng = np.random.default_rng(20110)
    img = rng.integers(0, 256, size=(600, 640, 3), dtype=np.uint8)
    r = Run(img)
    keys, w = r.histogram()
    assert keys.size > (1 << 17)
    return r, keys, w


def test_lloyd_grid_barrier_times_out_and_recovers(many):
    r, keys, w = many
    c0, _ = oracle.seed(keys, w, 64, "KPP", 3)
    want = r.lloyd(c0, eps=1e-4, max_iter=100)
    kq.kq_set_wait_limit(r.ws, LIMIT_US, missing_arrivals=1)
    got = r.lloyd(c0, eps=1e-4, max_iter=100)  # synchronizes: every block has returned
    assert r.status() == kq.KQ_ETIMEOUT
    assert got["stats"]["status"] == kq.KQ_ETIMEOUT
    assert got["stats"]["converged"] == 0
    kq.kq_status_clear(r.ws)
    assert r.status() == kq.KQ_OK
    again = r.lloyd(c0, eps=1e-4, max_iter=100)
    assert again["stats"]["status"] == kq.KQ_OK
    assert again["stats"]["iters"] == want["stats"]["iters"]
    assert np.array_equal(again["centers"], want["centers"]) and np.array_equal(again["labels"], want["labels"])


@pytest.mark.parametrize("scheme", ["KPP", "MMX"])
def test_cluster_seeding_exchange_times_out_and_recovers(paper, scheme):
    # N' ~ 100k: k-means++ / minmax run in one thread-block cluster, whose per-round
    # exchange waits on an mbarrier for every warp's value (plus the missing one)
    r, keys, w = paper
    want, _ = oracle.seed(keys, w, 32, scheme, 11)
    kq.kq_set_wait_limit(r.ws, LIMIT_US, missing_arrivals=1)
    r.seed(32, scheme, 11)
    assert r.status() == kq.KQ_ETIMEOUT
    kq.kq_status_clear(r.ws)
    got = r.seed(32, scheme, 11)
    assert r.status() == kq.KQ_OK
    assert np.array_equal(got, want)


def test_grid_seeding_barrier_times_out_and_recovers(many):
    # above one cluster's capacity, k-means++ runs on the whole grid
    r, keys, w = many
    assert keys.size > 16 * 11264
    want, _ = oracle.seed(keys, w, 16, "KPP", 5)
    kq.kq_set_wait_limit(r.ws, LIMIT_US, missing_arrivals=1)
    r.seed(16, "KPP", 5)
    assert r.status() == kq.KQ_ETIMEOUT
    kq.kq_status_clear(r.ws)
    got = r.seed(16, "KPP", 5)
    assert r.status() == kq.KQ_OK
    assert np.array_equal(got, want)


def test_limit_alone_changes_nothing(many):
    # a limit far above the run time, no missing arrival: normal results
    r, keys, w = many
    c0, _ = oracle.seed(keys, w, 16, "FGY", 1)
    want = r.lloyd(c0, eps=1e-4, max_iter=50)
    kq.kq_set_wait_limit(r.ws, 2_000_000, missing_arrivals=0)
    got = r.lloyd(c0, eps=1e-4, max_iter=50)
    assert r.status() == kq.KQ_OK and got["stats"]["status"] == kq.KQ_OK
    assert np.array_equal(got["centers"], want["centers"])
    kq.kq_status_clear(r.ws)
    torch.cuda.synchronize()
