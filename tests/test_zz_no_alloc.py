"""kq_lloyd_noalloc: the Lloyd entry point for callers that cannot allocate
device memory (the library keeps its scratch in a static device array).

Called twice in a row through the C ABI, it must give what kq_lloyd with a
caller-allocated workspace gives on the same inputs: the same labels and
palette, centres within 1e-3 and SSE within 1e-5.  This file is collected last
so that a run stopping at the first failure has run every other test first.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1101_0395_gb300 import kq, synth
from tests.gpu_helpers import CENTER_ABS, MSE_REL, Run, require_cuda, to_dev

pytestmark = pytest.mark.gpu


def _noalloc(r, c0, eps, max_iter, flags=0, labels_in=None, with_stats=True):
    K = c0.shape[0]
    nu = int(r.n_unique.item())
    c = to_dev(np.ascontiguousarray(c0, dtype=np.float64).reshape(-1))
    labels = torch.zeros(max(nu, 1), dtype=torch.uint8, device="cuda")
    if labels_in is not None:
        labels[:nu].copy_(to_dev(np.asarray(labels_in, dtype=np.uint8)))
    pal = torch.zeros(3 * K, dtype=torch.uint8, device="cuda")
    stats = torch.zeros(64, dtype=torch.uint8, device="cuda")
    hist = torch.zeros(max_iter, dtype=torch.float64, device="cuda")
    kq.kq_lloyd_noalloc(r.keys, r.weights, r.n_unique, K, c, eps, max_iter, labels, pal,
                        stats=stats if with_stats else None, sse_hist=hist, flags=flags)
    torch.cuda.synchronize()
    if not with_stats:
        return {"centers": c.cpu().numpy().reshape(K, 3), "labels": labels[:nu].cpu().numpy()}
    st = kq.parse_stats(stats)
    return {"centers": c.cpu().numpy().reshape(K, 3), "palette": pal.cpu().numpy().reshape(K, 3),
            "labels": labels[:nu].cpu().numpy(), "stats": st, "sse_hist": hist.cpu().numpy()[:st["iters"]]}


@pytest.mark.parametrize("name,K,flags", [("plain_256", 16, 0), ("paper_512", 256, 0),
                                          ("paper_512", 64, kq.LLOYD_DENSE), ("paper_512", 64, kq.LLOYD_LABELS_IN)])
def test_noalloc_matches_workspace_entry_point_twice(name, K, flags):
    require_cuda()
    img = synth.WORKLOADS[name].make(4)
    r = Run(img)
    keys, w = r.histogram()
    c0, _ = oracle.seed(keys, w, K, "KPP", 17)
    labels_in = None
    if flags & kq.LLOYD_LABELS_IN:
        labels_in, _, _, _ = oracle.assign(keys, w, c0)
    want = r.lloyd(c0, eps=1e-4, max_iter=100, flags=flags, labels_in=labels_in)
    for _ in range(2):
        got = _noalloc(r, c0, 1e-4, 100, flags=flags, labels_in=labels_in)
        assert got["stats"]["status"] == kq.KQ_OK
        assert got["stats"]["iters"] == want["stats"]["iters"]
        assert np.array_equal(got["labels"], want["labels"])
        assert np.array_equal(got["palette"], want["palette"])
        assert np.max(np.abs(got["centers"] - want["centers"])) <= CENTER_ABS
        assert abs(got["stats"]["sse"] - want["stats"]["sse"]) <= MSE_REL * max(want["stats"]["sse"], 1.0)
        assert np.allclose(got["sse_hist"], want["sse_hist"], rtol=MSE_REL, atol=0.0)


def test_noalloc_without_stats_then_with_stats():
    # a call that writes no statistics leaves nothing behind in the shared scratch
    # array that the next call could see: it clears the control block itself
    require_cuda()
    img = synth.WORKLOADS["plain_256"].make(5)
    r = Run(img)
    keys, w = r.histogram()
    c0, _ = oracle.seed(keys, w, 32, "FGY", 2)
    want = r.lloyd(c0, eps=1e-4, max_iter=60)
    first = _noalloc(r, c0, 1e-4, 60, with_stats=False)
    assert np.array_equal(first["labels"], want["labels"])
    got = _noalloc(r, c0, 1e-4, 60)
    assert got["stats"]["status"] == kq.KQ_OK and got["stats"]["iters"] == want["stats"]["iters"]
    assert got["stats"]["ndc"] == want["stats"]["ndc"]
    assert np.array_equal(got["labels"], want["labels"])
    assert np.max(np.abs(got["centers"] - want["centers"])) <= CENTER_ABS


def test_noalloc_rejects_too_many_colours():
    require_cuda()
    r = Run(synth.image(16, 16, 2, 12.0, 4.0, 5))
    r.histogram()
    with pytest.raises(kq.KqError) as e:
        _noalloc(r, np.zeros((257, 3)), 1e-4, 10)
    assert e.value.status == kq.KQ_EINVAL
