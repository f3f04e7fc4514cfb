"""Pins the FP64 oracle to facts fixed outside itself: published generator
vectors, a hand-worked example, closed forms, library routines, invariants of
Lloyd's method and brute force on tiny inputs.  CPU only."""
import itertools
import math
from collections import Counter
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1101_0395_gb300 import synth
from tests.conftest import read_golden


def rgb_of(keys):
    return oracle.key_to_rgb(keys)


def keys_of(points):
    p = np.asarray(points, dtype=np.uint32)
    return ((p[:, 0] << 16) | (p[:, 1] << 8) | p[:, 2]).astype(np.uint32)


# --------------------------------------------------------------------------- RNG
def test_splitmix64_published_vectors():
    for seed, idx, out in read_golden("splitmix64_vectors.txt"):
        assert oracle.rand(int(seed), 0, int(idx)) == int(out, 0)


def test_rand_streams_match_independent_numpy_generator():
    # synth.py implements the same published generator separately (numpy, vectorised)
    for seed, stream in [(0, 0), (7, 3), (2**63 + 5, 16 + 63)]:
        ref = synth.splitmix_stream(seed, stream, 50)
        got = [oracle.rand(seed, stream, i) for i in range(50)]
        assert got == [int(x) for x in ref]


def test_below_is_high_half_of_product():
    rng = np.random.default_rng(0)
    for _ in range(200):
        u = int(rng.integers(0, 2**63)) * 2 + int(rng.integers(0, 2))
        m = int(rng.integers(1, 2**40))
        b = oracle.below(u, m)
        assert b == (u * m) >> 64 and 0 <= b < m
    assert oracle.below(2**64 - 1, 1000) == 999
    assert oracle.below(0, 1000) == 0


# --------------------------------------------------------------------- histogram
def test_histogram_matches_numpy_unique():
    img = synth.WORKLOADS["plain_256"].make(0)
    keys, w = oracle.histogram(img)
    p = img.reshape(-1, 3).astype(np.uint32)
    uk, cnt = np.unique((p[:, 0] << 16) | (p[:, 1] << 8) | p[:, 2], return_counts=True)
    assert np.array_equal(keys, uk) and np.array_equal(w, cnt)
    assert int(w.sum()) == img.shape[0] * img.shape[1]
    assert np.all(np.diff(keys.astype(np.int64)) > 0)


def test_histogram_brute_force_tiny():
    rng = np.random.default_rng(1)
    img = rng.integers(0, 4, size=(7, 5, 3)).astype(np.uint8) * 85
    counts = Counter()
    for px in img.reshape(-1, 3):
        counts[(int(px[0]) << 16) | (int(px[1]) << 8) | int(px[2])] += 1
    keys, w = oracle.histogram(img)
    assert list(keys) == sorted(counts)
    assert list(w) == [counts[k] for k in sorted(counts)]


def test_histogram_every_colour_once():
    # a 4096 x 4096 image holding each 24-bit colour exactly once: N' = 2^24, all w = 1
    k = np.arange(1 << 24, dtype=np.uint32)
    rng = np.random.default_rng(2)
    rng.shuffle(k)
    img = np.stack([(k >> 16) & 255, (k >> 8) & 255, k & 255], axis=1).astype(np.uint8)
    keys, w = oracle.histogram(img)
    assert keys.size == 1 << 24
    assert np.array_equal(keys, np.arange(1 << 24, dtype=np.uint32))
    assert np.all(w == 1)


def test_histogram_degenerate():
    keys, w = oracle.histogram(np.full((3, 3, 3), 200, dtype=np.uint8))
    assert list(keys) == [(200 << 16) | (200 << 8) | 200] and list(w) == [9]
    keys, w = oracle.histogram(np.zeros((0, 3), dtype=np.uint8))
    assert keys.size == 0 and w.size == 0


# ---------------------------------------------------------------- assign/update
def brute_assign(points, centers):
    labels, best = [], []
    for x in points:
        ds = [sum((float(x[j]) - float(c[j])) ** 2 for j in range(3)) for c in centers]
        m = min(ds)
        labels.append(ds.index(m))  # first (lowest) index of the minimum
        best.append(m)
    return labels, best


def test_assign_brute_force_and_ties():
    pts = [(0, 0, 0), (10, 0, 0), (5, 0, 0), (3, 4, 0), (255, 255, 255), (7, 7, 7)]
    cents = np.array([[5, 0, 0], [0, 0, 0], [10, 0, 0], [0, 0, 0], [250.5, 255, 255]], dtype=np.float64)
    keys = keys_of(pts)
    w = np.array([1, 2, 3, 4, 5, 6], dtype=np.uint32)
    lab, d1, d2, sse = oracle.assign(keys, w, cents)
    bl, bd = brute_assign(pts, cents)
    assert list(lab) == bl
    assert lab[0] == 1  # (0,0,0) equals centres 1 and 3: lowest index wins
    assert np.allclose(d1, bd)
    assert d2[0] == 0.0  # a tie has a zero gap to the second-best distance
    assert sse == pytest.approx(float(np.dot(w, bd)), rel=1e-15)


def test_update_is_exact_weighted_mean():
    rng = np.random.default_rng(3)
    pts = rng.integers(0, 256, size=(40, 3))
    keys = keys_of(pts)
    w = rng.integers(1, 1000, size=40).astype(np.uint32)
    labels = (np.arange(40) % 3).astype(np.uint8)
    c_in = np.array([[1.0, 2.0, 3.0], [4.0, 5.0, 6.0], [7.0, 8.0, 9.0], [-1.0, 300.0, 0.5]])
    c_out, sums = oracle.update(keys, w, labels, c_in)
    for k in range(3):
        m = labels == k
        W = int(w[m].sum())
        for ch in range(3):
            S = int((w[m].astype(np.int64) * pts[m, ch]).sum())
            assert sums[k, ch] == S
            assert c_out[k, ch] == float(Fraction(S, W))  # correctly rounded quotient
        assert sums[k, 3] == W
    assert np.array_equal(c_out[3], c_in[3])  # empty cluster keeps its centre
    assert np.all(sums[3] == 0)


# -------------------------------------------------------------------- Lloyd
def test_worked_example():
    rows = read_golden("wsm_worked_example.txt")
    g = {r[0]: r[1:] for r in rows}
    pts = [tuple(int(v) for v in s.split(",")[:3]) for s in g["points"]]
    w = np.array([int(s.split(",")[3]) for s in g["points"]], dtype=np.uint32)
    seeds = np.array([[float(v) for v in s.split(",")] for s in g["seeds"]])
    run = oracle.lloyd(keys_of(pts), w, seeds, float(g["eps"][0]), 100)
    assert run["iters"] == int(g["iters"][0])
    assert np.allclose(run["sse_hist"], [float(v) for v in g["sse"]], rtol=1e-12)
    assert np.allclose(run["centers"], [[float(v) for v in s.split(",")] for s in g["centers"]], rtol=1e-12)
    assert list(run["labels"]) == [int(v) for v in g["labels"]]
    pal = oracle.palette(run["sums"], run["centers"])
    assert pal.tolist() == [[int(v) for v in s.split(",")] for s in g["palette"]]
    # expand to pixels: each point repeated by its weight
    img = np.repeat(np.array(pts, dtype=np.uint8), w.astype(np.int64), axis=0)
    idx, sse_num = oracle.map_pixels(img, pal)
    assert oracle.mse(sse_num, img.shape[0]) == float(g["mse"][0])
    assert oracle.psnr(oracle.mse(sse_num, img.shape[0])) == pytest.approx(float(g["psnr"][0]), rel=1e-15)
    for _, eps, iters in (r for r in rows if r[0] == "stop"):
        assert oracle.lloyd(keys_of(pts), w, seeds, float(eps), 100)["iters"] == int(iters)


@pytest.fixture(scope="module")
def small_image():
    img = synth.image(48, 40, 6, 12.0, 4.0, 77)
    keys, w = oracle.histogram(img)
    return img, keys, w


def test_k1_gives_weighted_mean(small_image):
    img, keys, w = small_image
    seeds, _ = oracle.seed(keys, w, 1, "FGY", 5)
    run = oracle.lloyd(keys, w, seeds, 1e-4, 10)
    px = img.reshape(-1, 3).astype(np.int64)
    n = px.shape[0]
    for ch in range(3):
        assert run["centers"][0, ch] == float(Fraction(int(px[:, ch].sum()), n))
    assert run["sums"][0, 3] == n


def test_k_equals_unique_count_gives_zero_sse(small_image):
    _, keys, w = small_image
    K = min(keys.size, 256)
    sub_k, sub_w = keys[:K], w[:K]
    seeds = rgb_of(sub_k).astype(np.float64)
    run = oracle.lloyd(sub_k, sub_w, seeds, 1e-4, 10)
    assert run["sse_hist"][0] == 0.0 and run["iters"] == 1 and run["converged"]
    assert np.array_equal(run["centers"], seeds)


def test_lloyd_invariants(small_image):
    _, keys, w = small_image
    for K in (2, 5, 16):
        seeds, _ = oracle.seed(keys, w, K, "FGY", 11 + K)
        run = oracle.lloyd(keys, w, seeds, -1.0, 25)  # fixed 25 iterations
        assert run["iters"] == 25
        h = run["sse_hist"]
        assert np.all(h[1:] <= h[:-1] * (1 + 1e-12))  # SSE never increases
        # re-run one assignment against the centres that produced the last labels
        x = rgb_of(keys).astype(np.float64)
        prev = oracle.lloyd(keys, w, seeds, -1.0, 24)["centers"]
        d = ((x[:, None, :] - prev[None, :, :]) ** 2).sum(axis=2)
        assert np.array_equal(run["labels"], np.argmin(d, axis=1))  # every label is an argmin
        # centres equal the weighted means of the final labels
        for k in range(K):
            m = run["labels"] == k
            if m.any():
                W = int(w[m].sum())
                for ch in range(3):
                    S = int((w[m].astype(np.int64) * x[m, ch].astype(np.int64)).sum())
                    assert run["centers"][k, ch] == float(Fraction(S, W))


def test_stopping_rule_follows_history(small_image):
    _, keys, w = small_image
    seeds, _ = oracle.seed(keys, w, 8, "KPP", 3)
    eps = 1e-3
    run = oracle.lloyd(keys, w, seeds, eps, 200)
    h = run["sse_hist"]
    stop = [i for i in range(1, len(h)) if (h[i - 1] - h[i]) / h[i] <= eps]
    assert run["converged"] and run["iters"] == stop[0] + 1
    assert all((h[i - 1] - h[i]) / h[i] > eps for i in range(1, len(h) - 1))


def test_weighted_unique_equals_unweighted_pixels(small_image):
    img, keys, w = small_image
    px = img.reshape(-1, 3).astype(np.uint32)
    pkeys = ((px[:, 0] << 16) | (px[:, 1] << 8) | px[:, 2]).astype(np.uint32)
    ones = np.ones(pkeys.size, dtype=np.uint32)
    seeds, _ = oracle.seed(keys, w, 6, "MMX", 9)
    a = oracle.lloyd(keys, w, seeds, -1.0, 12)
    b = oracle.lloyd(pkeys, ones, seeds, -1.0, 12)
    pos = np.searchsorted(keys, pkeys)
    assert np.array_equal(a["labels"][pos], b["labels"])
    assert np.max(np.abs(a["centers"] - b["centers"])) <= 1e-9
    assert np.array_equal(a["sums"], b["sums"])
    assert np.allclose(a["sse_hist"], b["sse_hist"], rtol=1e-12)


def partition_sse(points, weights, labels, K):
    total = Fraction(0)
    for k in range(K):
        mem = [i for i in range(len(points)) if labels[i] == k]
        if not mem:
            continue
        W = sum(weights[i] for i in mem)
        for ch in range(3):
            S = sum(weights[i] * points[i][ch] for i in mem)
            Q = sum(weights[i] * points[i][ch] ** 2 for i in mem)
            total += Fraction(Q) - Fraction(S * S, W)
    return total


@pytest.mark.parametrize("case", range(6))
def test_brute_force_tiny_partitions(case):
    rng = np.random.default_rng(100 + case)
    n = int(rng.integers(4, 9))
    K = int(rng.integers(2, 4))
    pts = [tuple(int(v) for v in rng.integers(0, 40, size=3)) for _ in range(n)]
    pts = list(dict.fromkeys(pts))
    n = len(pts)
    keys = keys_of(pts)
    order = np.argsort(keys)
    keys = keys[order]
    pts = [pts[i] for i in order]
    wts = [int(v) for v in rng.integers(1, 6, size=n)]
    w = np.array(wts, dtype=np.uint32)
    best, best_lab = None, None
    for lab in itertools.product(range(K), repeat=n):
        if len(set(lab)) < K:
            continue
        s = partition_sse(pts, wts, lab, K)
        if best is None or s < best:
            best, best_lab = s, lab
    seeds, _ = oracle.seed(keys, w, K, "FGY", case)
    run = oracle.lloyd(keys, w, seeds, 0.0, 100)
    lab = [int(v) for v in run["labels"]]
    s_run = partition_sse(pts, wts, lab, K)
    assert s_run >= best
    # fixed point: one more assignment keeps the labels
    lab2, _, _, _ = oracle.assign(keys, w, run["centers"])
    assert list(lab2) == lab
    # no single-point move lowers the SSE
    for i in range(n):
        for k in range(K):
            if k != lab[i]:
                moved = list(lab)
                moved[i] = k
                if len(set(moved)) == len(set(lab)):
                    assert partition_sse(pts, wts, moved, K) >= s_run
    # started from the optimal partition's means, Lloyd stays at the optimum
    opt_c = np.zeros((K, 3))
    for k in range(K):
        mem = [i for i in range(n) if best_lab[i] == k]
        W = sum(wts[i] for i in mem)
        for ch in range(3):
            opt_c[k, ch] = float(Fraction(sum(wts[i] * pts[i][ch] for i in mem), W))
    run2 = oracle.lloyd(keys, w, opt_c, 0.0, 100)
    assert partition_sse(pts, wts, [int(v) for v in run2["labels"]], K) == best


# ------------------------------------------------------------ palette / mapping
def test_palette_round_half_up_and_clamp():
    sums = np.array([[3, 5, 7, 2],      # 1.5, 2.5, 3.5 -> 2, 3, 4
                     [10, 11, 0, 4],    # 2.5, 2.75, 0 -> 3, 3, 0
                     [0, 0, 0, 0]], dtype=np.int64)
    c = np.array([[1.5, 2.5, 3.5], [2.5, 2.75, 0.0], [-3.2, 254.5, 300.0]])
    pal = oracle.palette(sums, c)
    assert pal.tolist() == [[2, 3, 4], [3, 3, 0], [0, 255, 255]]
    rng = np.random.default_rng(4)
    for _ in range(200):
        W = int(rng.integers(1, 10**9))
        S = int(rng.integers(0, 255 * W + 1))
        p = oracle.palette(np.array([[S, S, S, W]], dtype=np.int64), np.zeros((1, 3)))
        assert int(p[0, 0]) == math.floor(Fraction(S, W) + Fraction(1, 2))


def test_map_brute_force_and_ties():
    rng = np.random.default_rng(5)
    img = rng.integers(0, 256, size=(9, 7, 3)).astype(np.uint8)
    pal = rng.integers(0, 256, size=(12, 3)).astype(np.uint8)
    pal[7] = pal[2]  # duplicate entry: index 2 must win
    idx, sse = oracle.map_pixels(img, pal)
    tot = 0
    for i, x in enumerate(img.reshape(-1, 3).astype(int)):
        ds = [int(((x - p.astype(int)) ** 2).sum()) for p in pal]
        assert idx[i] == ds.index(min(ds))
        tot += min(ds)
    assert sse == tot
    assert 7 not in set(idx.tolist())


def test_mse_psnr_closed_forms():
    assert oracle.psnr(1.0) == pytest.approx(20 * math.log10(255), rel=1e-15)
    assert oracle.psnr(255.0 ** 2) == pytest.approx(0.0, abs=1e-12)
    assert oracle.mse(300, 100) == 3.0


# --------------------------------------------------------------------- seeding
def test_sff_subset_sizes():
    for K, s in read_golden("sff_subset_sizes.txt"):
        assert oracle.sff_size(10**6, int(K)) == int(s)
    # ceil(2 K ln K) is never within 1e-6 of an integer for K <= 256, so the
    # rounding of log() on any machine cannot change it
    for K in range(2, 257):
        v = 2 * K * math.log(K)
        assert abs(v - round(v)) > 1e-6
    assert oracle.sff_size(50, 256) == 50


def test_fgy_distinct_and_uniform():
    keys = keys_of([(i, 0, 0) for i in range(6)])
    w = np.ones(6, dtype=np.uint32)
    firsts = Counter()
    for s in range(3000):
        c, _ = oracle.seed(keys, w, 3, "FGY", s)
        r = [int(v) for v in c[:, 0]]
        assert len(set(r)) == 3
        firsts[r[0]] += 1
    chi2 = sum((firsts[i] - 500) ** 2 / 500 for i in range(6))
    assert chi2 < 30  # 5 d.o.f.; p ~ 1.5e-5


def brute_maxmin(x, first, K, candidates):
    chosen = [first]
    for _ in range(1, K):
        best, arg = -1, None
        for i in candidates:
            m = min(int(((x[i] - x[j]) ** 2).sum()) for j in chosen)
            if m > best:
                best, arg = m, i
        chosen.append(arg)
    return chosen


def test_mmx_brute_force(small_image):
    _, keys, w = small_image
    x = rgb_of(keys)
    n = keys.size
    for s, K in [(1, 4), (2, 9), (3, 17)]:
        c, _ = oracle.seed(keys, w, K, "MMX", s)
        first = int(synth.splitmix_stream(s, 3, 1)[0]) * n >> 64
        chosen = brute_maxmin(x, first, K, range(n))
        assert np.array_equal(c, x[chosen].astype(np.float64))


def test_sff_brute_force(small_image):
    _, keys, w = small_image
    x = rgb_of(keys)
    n = keys.size
    for s, K in [(4, 5), (6, 12)]:
        size = oracle.sff_size(n, K)
        # independent partial Fisher-Yates on the numpy generator
        a = list(range(n))
        u = synth.splitmix_stream(s, 4, size)
        for j in range(size):
            r = j + ((int(u[j]) * (n - j)) >> 64)
            a[j], a[r] = a[r], a[j]
        sub = sorted(a[:size])
        first = sub[(int(synth.splitmix_stream(s, 5, 1)[0]) * size) >> 64]
        chosen = brute_maxmin(x, first, K, sub)
        c, _ = oracle.seed(keys, w, K, "SFF", s)
        assert np.array_equal(c, x[chosen].astype(np.float64))


def test_kpp_sampling_frequencies():
    pts = [(0, 0, 0), (1, 0, 0), (3, 0, 0), (10, 0, 0), (10, 2, 0)]
    keys = keys_of(pts)
    w = np.array([3, 1, 2, 1, 4], dtype=np.uint32)
    x = np.array(pts)
    trials = 6000
    first = Counter()
    second_given0 = Counter()
    for s in range(trials):
        c, _ = oracle.seed(keys, w, 2, "KPP", s)
        i0 = [tuple(r) for r in x].index(tuple(int(v) for v in c[0]))
        i1 = [tuple(r) for r in x].index(tuple(int(v) for v in c[1]))
        first[i0] += 1
        if i0 == 0:
            second_given0[i1] += 1
    p = w / w.sum()
    chi2 = sum((first[i] - trials * p[i]) ** 2 / (trials * p[i]) for i in range(5))
    assert chi2 < 25
    d2 = ((x - x[0]) ** 2).sum(axis=1) * w
    q = d2 / d2.sum()
    m = sum(second_given0.values())
    assert second_given0[0] == 0  # a chosen point has D = 0 and is never drawn again
    chi2 = sum((second_given0[i] - m * q[i]) ** 2 / (m * q[i]) for i in range(1, 5))
    assert chi2 < 25


def test_kpp_first_centre_follows_inverse_cdf():
    keys = keys_of([(0, 0, 0), (1, 0, 0), (2, 0, 0)])
    w = np.array([5, 1, 2], dtype=np.uint32)
    for s in range(50):
        c, _ = oracle.seed(keys, w, 1 + 1, "KPP", s)
        t = (int(synth.splitmix_stream(s, 2, 1)[0]) * 8) >> 64
        want = 0 if t < 5 else (1 if t < 6 else 2)
        assert int(c[0, 0]) == want


def test_var_hand_example():
    # R spans 0..200, G and B nearly constant -> channel R; sorted by R with key ties
    pts = [(200, 0, 0), (0, 1, 0), (50, 0, 0), (100, 0, 1), (100, 0, 0), (150, 1, 1), (10, 0, 0), (60, 0, 0)]
    keys = keys_of(pts)
    order = np.argsort(keys)
    keys = keys[order]
    w = np.ones(len(pts), dtype=np.uint32)
    assert oracle.var_channel(keys, w) == 0
    c, _ = oracle.seed(keys, w, 3, "VAR", 0)
    # sorted by R (ties by key): R = 0,10,50,60,100(0,0),100(0,1),150,200
    # groups [0,2) [2,5) [5,8): middles 0, 3, 6 -> R = 0, 60, 150
    assert c.tolist() == [[0, 1, 0], [60, 0, 0], [150, 1, 1]]


def test_var_weighted_channel_and_brute_force(small_image):
    _, keys, w = small_image
    x = rgb_of(keys)
    wf = w.astype(object)
    var = []
    for ch in range(3):
        W = int(w.sum())
        s1 = sum(int(a) * int(b) for a, b in zip(wf, x[:, ch]))
        s2 = sum(int(a) * int(b) ** 2 for a, b in zip(wf, x[:, ch]))
        var.append(W * s2 - s1 * s1)
    ch = int(np.argmax(var))
    assert oracle.var_channel(keys, w) == ch
    n = keys.size
    order = sorted(range(n), key=lambda i: (int(x[i, ch]), int(keys[i])))
    for K in (3, 10):
        c, _ = oracle.seed(keys, w, K, "VAR", 0)
        want = [x[order[(g * n // K + (g + 1) * n // K - 1) // 2]] for g in range(K)]
        assert np.array_equal(c, np.array(want, dtype=np.float64))


def largest_remainder(weights, seats):
    tot = sum(weights)
    quotas = [Fraction(seats * wv, tot) for wv in weights]
    base = [int(q) for q in quotas]
    left = seats - sum(base)
    order = sorted(range(len(weights)), key=lambda i: (-(quotas[i] - base[i]), i))
    for i in order[:left]:
        base[i] += 1
    return base


def test_den_quota_hand_example():
    cellw = np.zeros(64, dtype=np.int64)
    celln = np.zeros(64, dtype=np.int64)
    cellw[[0, 5, 9]] = [600, 300, 100]
    celln[[0, 5, 9]] = [2, 10, 10]
    q = oracle.den_quota(cellw, celln, 10)
    # first pass: 6, 3, 1 -> cell 0 capped at 2; the other 8 seats split 300:100 -> 6, 2
    assert q[0] == 2 and q[5] == 6 and q[9] == 2 and q.sum() == 10


def test_den_quota_properties():
    rng = np.random.default_rng(6)
    for _ in range(100):
        celln = np.where(rng.random(64) < 0.4, rng.integers(1, 30, 64), 0).astype(np.int64)
        if celln.sum() == 0:
            continue
        cellw = celln * rng.integers(1, 50, 64)
        K = int(rng.integers(1, min(256, int(celln.sum())) + 1))
        q = oracle.den_quota(cellw, celln, K)
        assert q.sum() == K and np.all(q <= celln) and np.all(q >= 0)
        if np.all(largest_remainder(list(cellw), K) <= celln):
            assert q.tolist() == largest_remainder(list(cellw), K)


def test_den_centres_come_from_their_cells(small_image):
    _, keys, w = small_image
    x = rgb_of(keys)
    cell = (x[:, 0] >> 6) * 16 + (x[:, 1] >> 6) * 4 + (x[:, 2] >> 6)
    cellw = np.bincount(cell, weights=w, minlength=64).astype(np.int64)
    celln = np.bincount(cell, minlength=64).astype(np.int64)
    for K in (4, 13):
        c, _ = oracle.seed(keys, w, K, "DEN", 8)
        q = oracle.den_quota(cellw, celln, K)
        cc = (c[:, 0].astype(int) >> 6) * 16 + (c[:, 1].astype(int) >> 6) * 4 + (c[:, 2].astype(int) >> 6)
        assert np.bincount(cc, minlength=64).tolist() == q.tolist()
        assert np.all(np.diff(cc) >= 0)  # cells in ascending order
        assert len({tuple(r) for r in c}) == K


def test_lbg_structure(small_image):
    _, keys, w = small_image
    x = rgb_of(keys).astype(np.float64)
    c1, _ = oracle.seed(keys, w, 1, "LBG", 0)
    W = int(w.sum())
    for ch in range(3):
        S = int((w.astype(np.int64) * x[:, ch].astype(np.int64)).sum())
        assert c1[0, ch] == float(Fraction(S, W))
    c2, _ = oracle.seed(keys, w, 2, "LBG", 0, lbg_eps=1.0, conv_eps=1e-4, max_iter=100)
    ref = oracle.lloyd(keys, w, np.stack([c1[0] - 1.0, c1[0] + 1.0]), 1e-4, 100)["centers"]
    assert np.array_equal(c2, ref)
    # K = 3: the third centre comes from splitting the 2-means cluster of larger SSE
    run2 = oracle.lloyd(keys, w, np.stack([c1[0] - 1.0, c1[0] + 1.0]), 1e-4, 100)
    lab = run2["labels"]
    sse = []
    for k in range(2):
        m = lab == k
        mu = (w[m, None] * x[m]).sum(axis=0) / w[m].sum()
        sse.append(float((w[m] * ((x[m] - mu) ** 2).sum(axis=1)).sum()))
    j = int(np.argmax(sse))
    start = run2["centers"].copy()
    third = start[j] + 1.0
    start[j] = start[j] - 1.0
    ref3 = oracle.lloyd(keys, w, np.vstack([start, third]), 1e-4, 100)["centers"]
    c3, _ = oracle.seed(keys, w, 3, "LBG", 0)
    assert np.array_equal(c3, ref3)


def test_k_at_least_unique_count():
    keys = keys_of([(1, 2, 3), (4, 5, 6), (7, 8, 9)])
    w = np.array([1, 1, 1], dtype=np.uint32)
    for scheme in oracle.SCHEMES:
        c, k_eff = oracle.seed(keys, w, 5, scheme, 1)
        assert k_eff == 3
        assert c.tolist() == [[1, 2, 3], [4, 5, 6], [7, 8, 9], [7, 8, 9], [7, 8, 9]]


def test_seeds_are_data_points(small_image):
    _, keys, w = small_image
    kset = set(int(k) for k in keys)
    for scheme in ("FGY", "MMX", "DEN", "VAR", "SFF", "KPP"):
        c, _ = oracle.seed(keys, w, 16, scheme, 42)
        ck = keys_of(c.astype(np.int64))
        assert all(int(k) in kset for k in ck)
        if scheme != "VAR":
            assert len(set(int(k) for k in ck)) == 16


# ---------------------------------------------------------------- WU (Section 3.3)
def _wu_cells(keys, w):
    cells = {}
    for k, wt in zip(keys.tolist(), w.tolist()):
        r, g, b = k >> 16, (k >> 8) & 255, k & 255
        c = (r >> 3, g >> 3, b >> 3)
        m = cells.setdefault(c, [0, 0, 0, 0, 0])
        m[0] += wt
        m[1] += wt * r
        m[2] += wt * g
        m[3] += wt * b
        m[4] += wt * (r * r + g * g + b * b)
    return cells


def _wu_box_mom(cells, lo, hi):
    m = [0, 0, 0, 0, 0]
    for c, v in cells.items():
        if all(lo[a] <= c[a] < hi[a] for a in range(3)):
            for j in range(5):
                m[j] += v[j]
    return m


def _wu_exact(keys, w, K):
    """Wu's greedy bipartitioning in exact rational arithmetic, written from the
    method's statement: split the box of largest weighted variance by the cut
    that minimizes the sum of the two halves' variances."""
    from fractions import Fraction as F

    cells = _wu_cells(keys, w)

    def var(lo, hi):
        vol = (hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2])
        m = _wu_box_mom(cells, lo, hi)
        if vol <= 1 or m[0] == 0:
            return F(0)
        return F(m[4]) - F(m[1] ** 2 + m[2] ** 2 + m[3] ** 2, m[0])

    boxes = [([0, 0, 0], [32, 32, 32])]
    vv = [var(*boxes[0])]
    nxt = 0
    while len(boxes) < K and vv[nxt] > 0:
        lo, hi = boxes[nxt]
        best, cut = None, None
        for ax in range(3):
            for p in range(lo[ax] + 1, hi[ax]):
                h_hi = list(hi)
                h_hi[ax] = p
                r_lo = list(lo)
                r_lo[ax] = p
                ma, mb = _wu_box_mom(cells, lo, h_hi), _wu_box_mom(cells, r_lo, hi)
                if ma[0] == 0 or mb[0] == 0:
                    continue
                tot = (F(ma[4]) - F(ma[1] ** 2 + ma[2] ** 2 + ma[3] ** 2, ma[0])) + \
                      (F(mb[4]) - F(mb[1] ** 2 + mb[2] ** 2 + mb[3] ** 2, mb[0]))
                if best is None or tot < best:
                    best, cut = tot, (ax, p)
        if cut is None:
            vv[nxt] = F(0)
        else:
            ax, p = cut
            h_hi = list(hi)
            h_hi[ax] = p
            r_lo = list(lo)
            r_lo[ax] = p
            boxes[nxt] = (lo, h_hi)
            boxes.append((r_lo, hi))
            vv[nxt] = var(lo, h_hi)
            vv.append(var(r_lo, hi))
        nxt = max(range(len(boxes)), key=lambda k: (vv[k], -k))
    cen = []
    for lo, hi in boxes:
        m = _wu_box_mom(cells, lo, hi)
        cen.append([m[1] / m[0], m[2] / m[0], m[3] / m[0]])
    return np.array(cen), len(boxes)


def test_wu_k1_is_the_weighted_mean():
    rng = np.random.default_rng(41)
    keys = np.unique(rng.integers(0, 1 << 24, 500, dtype=np.uint32))
    w = rng.integers(1, 1000, keys.size).astype(np.uint32)
    c, nb = oracle.wu(keys, w, 1)
    assert nb == 1
    W = int(w.astype(np.int64).sum())
    for ch, sh in enumerate((16, 8, 0)):
        s = int(((keys.astype(np.int64) >> sh) & 255).dot(w.astype(np.int64)))
        assert c[0, ch] == s / W


@pytest.mark.parametrize("seed", [3, 4, 5])
def test_wu_matches_an_exact_rational_greedy(seed):
    """Clustered random colours (a few cells), K = 2..7: the same boxes as exact
    rational arithmetic, hence the same means."""
    rng = np.random.default_rng(seed)
    base = rng.integers(0, 256, (6, 3))
    pts = (base[rng.integers(0, 6, 300)] + rng.integers(-20, 21, (300, 3))).clip(0, 255)
    keys = np.unique(((pts[:, 0] << 16) | (pts[:, 1] << 8) | pts[:, 2]).astype(np.uint32))
    w = rng.integers(1, 50, keys.size).astype(np.uint32)
    for K in range(2, 8):
        c, nb = oracle.wu(keys, w, K)
        ce, nbe = _wu_exact(keys, w, K)
        assert nb == nbe
        assert np.array_equal(c[:nb], ce)


def test_wu_cannot_split_a_single_cell():
    # every colour in one 8 x 8 x 8 cell: one box, all centres its mean
    keys = np.array([(r << 16) | (g << 8) | b for r in (8, 9) for g in (16, 20) for b in (0, 7)], dtype=np.uint32)
    w = np.arange(1, keys.size + 1, dtype=np.uint32)
    c, nb = oracle.wu(keys, w, 5)
    assert nb == 1 and np.all(c == c[0])
    c2, k_eff = oracle.seed(keys, w, 5, "WU", 0)
    assert k_eff == 5 and np.array_equal(c, c2)


# --------------------------------------------------------------------------- CIE L*a*b*
def test_lab_reference_values():
    # the sRGB primaries and secondaries and the mid grey, as tabulated for the
    # standard definitions (tests/golden/lab_reference.txt)
    for row in read_golden("lab_reference.txt"):
        r, g, b = (int(v) for v in row[:3])
        want = np.array([float(v) for v in row[3:]])
        got = oracle.lab(np.array([(r << 16) | (g << 8) | b]))[0]
        assert np.all(np.abs(got - want) <= 6e-5 + 1e-9), (row, got)


def test_lab_closed_forms():
    # black is the origin; white is L* = 100 with a* = b* = 0 (the matrix rows sum to
    # the white point to 1e-7); every neutral grey has a* = b* = 0 and L* grows with
    # the grey level; below the linear segment's end (8-bit 10: 10/255 < 0.04045) L*
    # follows the closed form 116 (t / (3 (6/29)^2) + 4/29) - 16 = 903.3 t for Y = t
    greys = np.arange(256, dtype=np.uint32) * 0x010101
    lab = oracle.lab(greys)
    assert np.array_equal(lab[0], [0.0, 0.0, 0.0])
    assert abs(lab[255, 0] - 100.0) < 1e-4 and np.all(np.abs(lab[255, 1:]) < 1e-4)
    assert np.all(np.abs(lab[:, 1:]) < 1e-4)
    assert np.all(np.diff(lab[:, 0]) > 0)
    for v in range(1, 11):
        y = (v / 255.0) / 12.92 * (0.2126729 + 0.7151522 + 0.0721750)
        L = 116.0 * (y / (3.0 * (6.0 / 29.0) ** 2) + 4.0 / 29.0) - 16.0
        assert abs(lab[v, 0] - L) < 1e-9
    # a* > 0 towards red, b* > 0 towards yellow, b* < 0 towards blue
    red, yellow, blue = oracle.lab(np.array([0xFF0000, 0xFFFF00, 0x0000FF], dtype=np.uint32))
    assert red[1] > 0 and yellow[2] > 0 and blue[2] < 0


def test_lab_points_and_palette_round_trip():
    # fixed point is round(value * 256); the inverse transform of an 8-bit colour's
    # point rounds back to that colour (the quantisation error, 1/512 L*a*b* unit, is
    # far below one 8-bit step); all 256 greys, the corners of the cube, 20000 colours
    rng = np.random.default_rng(1976)
    keys = np.concatenate([np.arange(256, dtype=np.uint32) * 0x010101,
                           np.array([0, 0xFF0000, 0x00FF00, 0x0000FF, 0xFFFF00, 0xFF00FF, 0x00FFFF, 0xFFFFFF],
                                    dtype=np.uint32),
                           rng.integers(0, 1 << 24, size=20000).astype(np.uint32)])
    pts = oracle.lab_points(keys)
    lab = oracle.lab(keys[:300])
    assert np.array_equal(pts[:300, :3], np.rint(lab * oracle.LAB_SCALE).astype(np.int32))
    assert np.all(pts[:, 3] == 0)
    pal = oracle.lab_palette(pts[:, :3].astype(np.float64))
    assert np.array_equal(keys_of(pal), keys)
    # out-of-gamut centres clamp: a very saturated L*a*b* point maps inside the cube
    far = oracle.lab_palette(np.array([[60.0, 200.0, -200.0]]) * oracle.LAB_SCALE)
    assert far.dtype == np.uint8 and far.shape == (1, 3)


def test_points_lloyd_equals_rgb_lloyd_on_rgb_points(small_image):
    # with each colour's three bytes as the point, the points path is exactly the
    # RGB path: same labels, centres, SSE history and sums (pins assign/update/loop)
    _, keys, w = small_image
    pts = np.zeros((keys.size, 4), dtype=np.int32)
    pts[:, :3] = rgb_of(keys)
    for K, scheme in ((1, "FGY"), (7, "FGY"), (16, "KPP")):
        seeds, _ = oracle.seed(keys, w, K, scheme, 31 + K)
        a = oracle.lloyd(keys, w, seeds, 1e-4, 40)
        b = oracle.lloyd_points(pts, w, seeds, 1e-4, 40)
        assert a["iters"] == b["iters"] and np.array_equal(a["labels"], b["labels"])
        assert np.array_equal(a["centers"], b["centers"]) and np.array_equal(a["sums"], b["sums"])
        assert np.array_equal(a["sse_hist"], b["sse_hist"])
    # Forgy among points draws the same indices as Forgy among colours
    for K in (1, 5, 64):
        want, _ = oracle.seed(keys, w, K, "FGY", 99)
        assert np.array_equal(oracle.seed_points_fgy(pts, K, 99), want)


def test_points_lloyd_invariants_in_lab(small_image):
    # L*a*b* points: K = 1 gives the exact weighted mean, SSE never increases, every
    # label is an argmin, centres are the exact weighted means of their labels, and
    # the weighted run on unique colours equals the unweighted run on all pixels
    img, keys, w = small_image
    pts = oracle.lab_points(keys)
    one = oracle.lloyd_points(pts, w, oracle.seed_points_fgy(pts, 1, 3), 1e-4, 10)
    W = int(w.astype(np.int64).sum())
    for ch in range(3):
        S = int((w.astype(np.int64) * pts[:, ch].astype(np.int64)).sum())
        assert one["centers"][0, ch] == S / W
    seeds = oracle.seed_points_fgy(pts, 12, 8)
    run = oracle.lloyd_points(pts, w, seeds, -1.0, 20)
    h = run["sse_hist"]
    assert np.all(h[1:] <= h[:-1] * (1 + 1e-12))
    prev = oracle.lloyd_points(pts, w, seeds, -1.0, 19)["centers"]
    d = ((pts[:, None, :3].astype(np.float64) - prev[None, :, :]) ** 2).sum(axis=2)
    assert np.array_equal(run["labels"], np.argmin(d, axis=1))
    for k in np.unique(run["labels"]):
        m = run["labels"] == k
        Wk = int(w[m].astype(np.int64).sum())
        for ch in range(3):
            Sk = int((w[m].astype(np.int64) * pts[m, ch].astype(np.int64)).sum())
            assert run["centers"][k, ch] == Sk / Wk
    px = img.reshape(-1, 3).astype(np.uint32)
    pkeys = (px[:, 0] << 16) | (px[:, 1] << 8) | px[:, 2]
    ppts = oracle.lab_points(pkeys)
    full = oracle.lloyd_points(ppts, np.ones(pkeys.size, dtype=np.uint32), seeds, -1.0, 20)
    assert np.allclose(full["centers"], run["centers"], rtol=0, atol=1e-9)
    pos = np.searchsorted(keys, pkeys)
    assert np.array_equal(full["labels"], run["labels"][pos])
