"""Batched quantization (kq_batch_run): many images of uneven size and K in one
persistent launch, each image taken whole by one CTA or one thread-block cluster.

Every image of the batch is checked against the oracle the way the single-image
path is: histogram bit-exact; for the integer seeding schemes the centres equal
a pass-by-pass GPU replay from the oracle's own seeds (each pass of which is
checked against the oracle's assignment and update); palette and mapping
bit-exact against the oracle given the final sums.  LBG (floating-point seeds)
is compared with the single-image calls on the same image.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1101_0395_gb300 import kq, synth
from tests.gpu_helpers import MSE_REL, Run, require_cuda, to_dev, u32
from tests.test_gpu_lloyd import gpu_trajectory

pytestmark = pytest.mark.gpu

EPS, MAX_ITER = 1e-4, 100

# (height, width, K, scheme): uneven sizes, every scheme, the degenerate cases
CASES = [
    (96, 80, 16, "KPP"), (130, 70, 64, "MMX"), (40, 50, 8, "FGY"), (200, 150, 32, "VAR"),
    (120, 100, 24, "DEN"), (90, 90, 40, "SFF"), (64, 72, 12, "LBG"), (150, 220, 256, "KPP"),
    (70, 64, 1, "KPP"), (5, 4, 64, "KPP"), (0, 0, 8, "MMX"), (33, 17, 20, "USER"),
    (260, 240, 128, "MMX"), (31, 29, 5, "VAR"), (48, 48, 200, "DEN"), (180, 200, 64, "WU"),
]


def _images():
    out = []
    for i, (h, w, K, s) in enumerate(CASES):
        if h * w == 0:
            out.append(np.zeros((0, 3), dtype=np.uint8))
        else:
            out.append(synth.batch_image(h, w, 7000 + i))
    return out


@pytest.fixture(scope="module")
def batch_inputs():
    require_cuda()
    return _images()


def _make(imgs, capacities=None):
    n = [im.size // 3 for im in imgs]
    Ks = [c[2] for c in CASES]
    schemes = [c[3] for c in CASES]
    seeds = [11 + 3 * i for i in range(len(CASES))]
    bq = kq.BatchQuantizer(n, Ks, schemes, seeds, EPS, MAX_ITER, capacities=capacities)
    for i, im in enumerate(imgs):
        if n[i]:
            bq.rgb(i).copy_(to_dev(im.reshape(-1)))
        if schemes[i] == "USER":
            keys, w = oracle.histogram(im)
            c0, _ = oracle.seed(keys, w, Ks[i], "FGY", 99)
            bq.centers(i).copy_(to_dev(c0))
    return bq, seeds


def _check_item(bq, i, im, seed, res):
    h, w_, K, scheme = CASES[i]
    assert res["status"] == kq.KQ_OK, (i, res["status"])
    keys, w = oracle.histogram(im) if im.size else (np.zeros(0, np.uint32), np.zeros(0, np.uint32))
    nu = keys.size
    assert res["n_unique"] == nu
    assert np.array_equal(u32(bq.keys(i)[:nu]), keys) and np.array_equal(u32(bq.weights(i)[:nu]), w)
    cen = bq.centers(i).cpu().numpy()
    pal = bq.palette(i).cpu().numpy()
    st = res["lloyd"]
    if scheme == "LBG":
        q = kq.Quantizer(max(1, im.size // 3))
        r = q.quantize(to_dev(im.reshape(-1)), K, "LBG", seed, EPS, MAX_ITER)
        torch.cuda.synchronize()
        assert np.array_equal(r.palette.cpu().numpy(), pal)
        assert np.max(np.abs(r.centers.cpu().numpy() - cen)) <= 1e-9
    elif nu > 0:
        if scheme == "USER":
            c0, _ = oracle.seed(keys, w, K, "FGY", 99)
        else:
            c0, _ = oracle.seed(keys, w, K, scheme, seed)
        r = Run(im)
        r.histogram()
        c, labels, hist, _, _ = gpu_trajectory(r, keys, w, c0, EPS, MAX_ITER)
        assert st["iters"] == hist.size, (i, st["iters"], hist.size)
        assert np.array_equal(cen, c)
        assert np.array_equal(bq.labels(i)[:nu].cpu().numpy(), labels)
        assert abs(st["sse"] - hist[-1]) <= 1e-6 * max(hist[-1], 1.0)
        _, sums = oracle.update(keys, w, labels, c)
        assert np.array_equal(pal, oracle.palette(sums, c))
    if im.size:
        oidx, osse = oracle.map_pixels(im, pal)
        assert np.array_equal(bq.idx(i).cpu().numpy(), oidx)
        assert res["sse_num"] == osse
    else:
        assert res["sse_num"] == 0


def _configs():
    require_cuda()
    cfgs = [(1, 0)]
    mc = kq.kq_batch_max_cluster()
    if mc >= 2:
        cfgs.append((2, 6000))
    if mc >= 4:
        cfgs.append((mc, 6000))
    return cfgs


@pytest.mark.parametrize("which", [0, 1, 2])
def test_batch_matches_oracle(batch_inputs, which):
    cfgs = _configs()
    if which >= len(cfgs):
        pytest.skip("cluster size not available")
    C, split = cfgs[which]
    bq, seeds = _make(batch_inputs)
    bq.plan(kq.BatchConfig(C, 0, split))
    if C > 1:
        assert bq.n_big >= 3
    bq.run()
    torch.cuda.synchronize()
    res = bq.results()
    for i, im in enumerate(batch_inputs):
        _check_item(bq, i, im, seeds[i], res[i])


def test_batch_graph_replay_is_repeatable(batch_inputs):
    bq, _ = _make(batch_inputs)
    C = kq.kq_batch_max_cluster()
    bq.plan(kq.BatchConfig(C, 0, 6000) if C > 1 else kq.BatchConfig(1, 0, 0))
    bq.capture()
    outs = []
    for _ in range(2):
        bq.replay()
        torch.cuda.synchronize()
        outs.append((bq.arena.clone(), bq.results()))
    # the USER centres are overwritten by the first run: compare everything else
    res0, res1 = outs[0][1], outs[1][1]
    for i, c in enumerate(CASES):
        if c[3] == "USER":
            continue
        for f in ("status", "n_unique", "lloyd", "sse_num"):
            assert res0[i][f].tobytes() == res1[i][f].tobytes(), (i, f)
        t = res1[i]["t_ns"]
        assert np.all(np.diff(t) >= 0) and t[0] > 0
        for name in ("idx", "keys", "weights", "labels", "centers", "palette"):
            off, size = bq.layout[i][name]
            assert torch.equal(outs[0][0][off:off + size], outs[1][0][off:off + size]), (i, name)


def test_batch_capacity_and_invalid_items(batch_inputs):
    caps = [max(0, min(im.size // 3, 1 << 24)) for im in batch_inputs]
    caps[0] = 10  # far fewer than this image's unique colours
    bq, _ = _make(batch_inputs, capacities=caps)
    bq.run()
    torch.cuda.synchronize()
    res = bq.results()
    keys, _ = oracle.histogram(batch_inputs[0])
    assert res[0]["status"] == kq.KQ_ECAPACITY and res[0]["n_unique"] == keys.size
    # the workspace tables were left clean: the next image on it is exact
    for i in (1, 7):
        keys, w = oracle.histogram(batch_inputs[i])
        assert res[i]["status"] == kq.KQ_OK and res[i]["n_unique"] == keys.size
        assert np.array_equal(u32(bq.keys(i)[:keys.size]), keys)
    # an invalid item is reported on the device and skipped
    bad = bq.h_items.copy()
    bad[2]["K"] = 0
    items = torch.from_numpy(bad.view(np.uint8).copy()).cuda()
    kq.kq_batch_run(items, bq.n_items, bq.order, 0, kq.BatchConfig(1, 0, 0), bq.ws)
    torch.cuda.synchronize()
    assert bq.results()[2]["status"] == kq.KQ_EINVAL
    with pytest.raises(kq.KqError):
        kq.kq_batch_plan(bad, kq.BatchConfig(1, 0, 0))


def test_batch_autotuner(batch_inputs):
    bq, seeds = _make(batch_inputs)
    ms = bq.tune()
    assert ms > 0 and bq.cfg.cluster in (1, 2, 4, 8, 16)
    bq.run()
    torch.cuda.synchronize()
    res = bq.results()
    for i in (0, 3, 7):
        _check_item(bq, i, batch_inputs[i], seeds[i], res[i])


def test_batch_large_member_on_a_cluster():
    """A 1024 x 768 image with K = 256 beside small ones, on the largest cluster."""
    require_cuda()
    C = kq.kq_batch_max_cluster()
    if C < 2:
        pytest.skip("no thread-block clusters")
    imgs = [synth.batch_image(768, 1024, 8101), synth.batch_image(64, 80, 8102), synth.batch_image(100, 90, 8103)]
    Ks, seeds = [256, 16, 32], [5, 6, 7]
    bq = kq.BatchQuantizer([im.size // 3 for im in imgs], Ks, "KPP", seeds, EPS, MAX_ITER)
    for i, im in enumerate(imgs):
        bq.rgb(i).copy_(to_dev(im.reshape(-1)))
    bq.plan(kq.BatchConfig(C, 0, 100000))
    assert bq.n_big == 1
    bq.run()
    torch.cuda.synchronize()
    res = bq.results()
    im = imgs[0]
    keys, w = oracle.histogram(im)
    assert res[0]["status"] == kq.KQ_OK and res[0]["n_unique"] == keys.size
    assert np.array_equal(u32(bq.keys(0)[:keys.size]), keys)
    c0, _ = oracle.seed(keys, w, 256, "KPP", 5)
    q = Run(im)
    q.histogram()
    g = q.lloyd(c0, eps=EPS, max_iter=MAX_ITER)
    st = res[0]["lloyd"]
    assert st["iters"] == g["stats"]["iters"]
    assert np.array_equal(bq.centers(0).cpu().numpy(), g["centers"])
    assert abs(st["sse"] - g["stats"]["sse"]) <= MSE_REL * g["stats"]["sse"]
    pal = bq.palette(0).cpu().numpy()
    assert np.array_equal(pal, g["palette"])
    oidx, osse = oracle.map_pixels(im, pal)
    assert np.array_equal(bq.idx(0).cpu().numpy(), oidx) and res[0]["sse_num"] == osse
