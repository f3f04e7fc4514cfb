"""Live batches (kq_live_*): images published into a batch launch that is
already running.

Every image's results must be those of kq_batch_run on the same item with the
same group shape (a cluster for class 0, a single CTA for class 1), bit for
bit: the palette indices, palette, centres, N', the Lloyd statistics and the
squared-error sum.  kq_batch_run itself is checked against the oracle in
test_gpu_batch.py.  The inputs and outputs of the live items sit in page-locked
host memory, which the running kernel reads and writes directly.
"""
import time

import numpy as np
import pytest
import torch

from paper_1101_0395_gb300 import kq, synth
from tests.gpu_helpers import require_cuda

pytestmark = pytest.mark.gpu

EPS, MAX_ITER = 1e-4, 100
SPLIT = 1 << 15
SCHEMES = ["KPP", "MMX", "FGY", "VAR", "DEN", "SFF", "WU", "KPP", "LBG"]


def _cases():
    rng = np.random.default_rng(77)
    out = []
    for i in range(22):
        h = int(2 ** rng.uniform(4, 9))
        w = max(1, int(h * rng.uniform(0.5, 2.0)))
        K = int(rng.choice([1, 8, 16, 32, 64, 128, 256]))
        out.append((h, w, K, SCHEMES[i % len(SCHEMES)], 500 + 7 * i))
    out.append((0, 0, 8, "KPP", 9))  # an empty image
    out.append((3, 2, 64, "MMX", 10))  # K above N'
    return out


CASES = _cases()


def _images():
    return [synth.batch_image(h, w, s) if h * w else np.zeros((0, 3), np.uint8) for (h, w, _, _, s) in CASES]


def _align(v):
    return (v + 255) // 256 * 256


def _cluster():
    c = min(4, kq.kq_batch_max_cluster())
    return c if c >= 2 else 1


@pytest.fixture(scope="module")
def reference():
    """kq_batch_run results for both launch shapes."""
    require_cuda()
    imgs = _images()
    n = [im.size // 3 for im in imgs]
    out = {}
    for C in sorted({1, _cluster()}):
        bq = kq.BatchQuantizer(n, [c[2] for c in CASES], [c[3] for c in CASES], [c[4] for c in CASES], EPS,
                               MAX_ITER)
        for i, im in enumerate(imgs):
            if n[i]:
                bq.rgb(i).copy_(torch.from_numpy(im.reshape(-1)).cuda())
        bq.plan(kq.BatchConfig(C, 0, SPLIT))
        bq.run()
        torch.cuda.synchronize()
        res = bq.results()
        out[C] = [dict(idx=bq.idx(i).cpu().numpy(), palette=bq.palette(i).cpu().numpy(),
                       centers=bq.centers(i).cpu().numpy(), result=res[i]) for i in range(len(imgs))]
    return imgs, out


class LiveItems:
    """Items whose pixels and outputs are in page-locked host memory and whose
    colour lists and scratch are in device memory."""

    HOST = ("rgb", "idx", "centers", "palette", "result")
    DEV = ("keys", "weights", "labels", "scratch")

    def __init__(self, imgs, C):
        self.n = [im.size // 3 for im in imgs]
        hl, dl, ho, do = [], [], 0, 0
        for i, (h, w, K, scheme, seed) in enumerate(CASES):
            cap = max(0, min(self.n[i], 1 << 24))
            sizes = {"rgb": 3 * self.n[i], "idx": self.n[i], "centers": 24 * K, "palette": 3 * K,
                     "result": kq.BATCH_RESULT_DTYPE.itemsize, "keys": 4 * cap, "weights": 4 * cap, "labels": cap,
                     "scratch": kq.kq_batch_scratch_bytes(cap)}
            h_, d_ = {}, {}
            for name in self.HOST:
                h_[name] = (ho, sizes[name])
                ho = _align(ho + max(sizes[name], 1))
            for name in self.DEV:
                d_[name] = (do, sizes[name])
                do = _align(do + max(sizes[name], 1))
            hl.append(h_)
            dl.append(d_)
        self.host = torch.zeros(max(ho, 256), dtype=torch.uint8).pin_memory()
        self.dev = torch.zeros(max(do, 256), dtype=torch.uint8, device="cuda")
        self.hl, self.dl = hl, dl
        hb, db = self.host.data_ptr(), self.dev.data_ptr()
        self.items = np.zeros(len(imgs), dtype=kq.BATCH_ITEM_DTYPE)
        self.cls = []
        for i, (h, w, K, scheme, seed) in enumerate(CASES):
            it = self.items[i]
            for name in self.HOST:
                it[name] = hb + hl[i][name][0]
            for name in self.DEV:
                it[name] = db + dl[i][name][0]
            it["n_pixels"], it["seed"], it["eps"] = self.n[i], seed, EPS
            it["lbg_eps"], it["lbg_conv_eps"], it["lbg_max_iter"] = 1.0, EPS, MAX_ITER
            it["K"], it["scheme"], it["max_iter"] = K, kq.INIT[scheme], MAX_ITER
            it["capacity"] = max(0, min(self.n[i], 1 << 24))
            self.cls.append(0 if C > 1 and self.n[i] > SPLIT else 1)
            if self.n[i]:
                self.view(i, "rgb")[:] = torch.from_numpy(imgs[i].reshape(-1))

    def view(self, i, name):
        off, size = self.hl[i][name]
        return self.host[off:off + size]

    def out(self, i):
        K = CASES[i][2]
        return dict(idx=self.view(i, "idx").numpy().copy(), palette=self.view(i, "palette").numpy().reshape(K, 3),
                    centers=self.view(i, "centers").numpy().view(np.float64).reshape(K, 3),
                    result=np.frombuffer(self.view(i, "result").numpy().tobytes(), dtype=kq.BATCH_RESULT_DTYPE)[0])


def _same(got, want, i):
    assert np.array_equal(got["idx"], want["idx"]), i
    assert np.array_equal(got["palette"], want["palette"]), i
    assert np.array_equal(got["centers"], want["centers"]), i
    g, w = got["result"], want["result"]
    assert g["status"] == w["status"] and g["n_unique"] == w["n_unique"] and g["sse_num"] == w["sse_num"], i
    for f in ("iters", "converged", "k_eff", "status", "ndc", "sse", "sse_prev"):
        assert g["lloyd"][f] == w["lloyd"][f], (i, f)


def _wait_done(q, pending, limit_s=60.0):
    t0 = time.time()
    while pending:
        pending = [p for p in pending if not q.done(*p)]
        if pending and time.time() - t0 > limit_s:
            raise AssertionError("live items not done: %s" % pending[:4])
        time.sleep(0.0002)


@pytest.mark.parametrize("shape", ["single", "cluster"])
def test_live_items_join_the_running_launch(reference, shape):
    imgs, ref = reference
    C = 1 if shape == "single" else _cluster()
    if shape == "cluster" and C == 1:
        pytest.skip("no thread-block clusters on this device")
    li = LiveItems(imgs, C)
    q = kq.LiveQueue(64)
    ws = torch.zeros(kq.kq_batch_workspace_size(), dtype=torch.uint8, device="cuda")
    kq.kq_live_reset(ws)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    kq.kq_live_run(q, kq.BatchConfig(C, 0, SPLIT), 500_000, ws, stream=s)
    ev = torch.cuda.Event()
    ev.record(s)
    pending = []
    for i in range(len(CASES)):
        seq = q.publish(li.cls[i], li.items[i])
        assert seq is not None
        pending.append((li.cls[i], seq, i))
        if i % 5 == 4:
            time.sleep(0.002)  # later items arrive while the launch runs the first ones
    _wait_done(q, [(c, sq) for c, sq, _ in pending])
    assert not ev.query()  # still the same launch: every item joined it
    q.close()
    s.synchronize()
    for c, sq, i in pending:
        _same(li.out(i), ref[C][i], i)


@pytest.mark.parametrize("shape", ["single", "cluster"])
def test_live_ring_reuse_idle_exit_and_relaunch(reference, shape):
    imgs, ref = reference
    C = 1 if shape == "single" else _cluster()
    if shape == "cluster" and C == 1:
        pytest.skip("no thread-block clusters on this device")
    li = LiveItems(imgs, C)
    q = kq.LiveQueue(3)  # fewer slots than items: slots are reused once their items are done
    ws = torch.zeros(kq.kq_batch_workspace_size(), dtype=torch.uint8, device="cuda")
    kq.kq_live_reset(ws)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    cfg = kq.BatchConfig(C, 0, SPLIT)
    ev = None
    launches = 0

    def ensure_running():
        nonlocal ev, launches
        if ev is None or ev.query():
            kq.kq_live_run(q, cfg, 2000, ws, stream=s)  # 2 ms idle limit
            ev = torch.cuda.Event()
            ev.record(s)
            launches += 1

    order = list(range(len(CASES)))
    half = len(order) // 2
    done_items = []
    for phase in (order[:half], order[half:]):
        pending = []
        for i in phase:
            t0 = time.time()
            while True:
                seq = q.publish(li.cls[i], li.items[i])
                if seq is not None:
                    break
                ensure_running()
                pending = [p for p in pending if not q.done(p[0], p[1])]
                assert time.time() - t0 < 60.0, "ring slot never freed"
                time.sleep(0.0002)
            # the slot now holds this item: the one it held before was done (the
            # publication checks that), and its done mark is gone
            pending = [p for p in pending if not (p[0] == li.cls[i] and p[1] == seq - q.capacity)]
            pending.append((li.cls[i], seq, i))
            done_items.append((li.cls[i], seq, i))
            ensure_running()
        t0 = time.time()
        while pending:
            ensure_running()
            pending = [p for p in pending if not q.done(p[0], p[1])]
            assert time.time() - t0 < 60.0, ("live items not done", pending, q.tails(), launches, ev.query())
            time.sleep(0.0002)
        # nothing more to take: the launch leaves after its idle limit
        s.synchronize()
        assert ev.query()
    assert launches >= 2
    q.close()
    for c, sq, i in done_items:
        _same(li.out(i), ref[C][i], i)


def test_live_close_ends_an_idle_launch():
    require_cuda()
    q = kq.LiveQueue(4)
    ws = torch.zeros(kq.kq_batch_workspace_size(), dtype=torch.uint8, device="cuda")
    kq.kq_live_reset(ws)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    kq.kq_live_run(q, kq.BatchConfig(1, 0, 0), 10_000_000, ws, stream=s)  # a 10 s idle limit
    ev = torch.cuda.Event()
    ev.record(s)
    time.sleep(0.01)
    assert not ev.query()
    t0 = time.time()
    q.close()
    s.synchronize()
    assert time.time() - t0 < 2.0
