"""Host logic of the serving loop (no GPU): the first-fit arena, memory
admission in arrival order, continuous batching over several waves in flight,
and the Poisson arrival trace."""
import numpy as np

from paper_1101_0395_gb300 import serve


class FakeBackend:
    """Stands in for the device: a wave completes after `delay` polls."""

    def __init__(self, delay=2):
        self.delay = delay
        self.launched = []      # (slot, [rid...], arena bytes in use at launch)
        self.server = None

    def scratch_bytes(self, cap):
        return 8 * cap + 256

    def setup(self, pool_bytes, streams, max_wave):
        self.pool_bytes, self.n_streams, self.max_wave = pool_bytes, streams, max_wave

    def launch(self, slot, batch):
        self.launched.append((slot, [r.rid for r in batch], self.server.arena.in_use))
        return {"polls": 0, "slot": slot}

    def done(self, h):
        h["polls"] += 1
        return h["polls"] > self.delay

    def collect(self, h, batch):
        for r in batch:
            r.result = {"slot": h["slot"]}


def _req(rid, npx, K=16, arrival=0.0):
    return serve.Request(rid=rid, rgb=np.zeros((npx, 3), dtype=np.uint8), K=K, arrival=arrival)


def _server(pool, streams=2, max_wave=8, delay=2):
    be = FakeBackend(delay)
    srv = serve.Server(be, pool, streams=streams, max_wave=max_wave)
    be.server = srv
    return srv, be


def test_arena_first_fit_coalesces_and_never_overlaps():
    rng = np.random.default_rng(3)
    a = serve.Arena(1 << 20)
    live = {}
    for _ in range(2000):
        if live and rng.random() < 0.45:
            off = list(live)[rng.integers(len(live))]
            a.release(off)
            del live[off]
        else:
            n = int(rng.integers(1, 40000))
            off = a.alloc(n)
            if off is not None:
                assert off % 256 == 0
                live[off] = serve._align(n)
        spans = sorted(live.items())
        for (o1, n1), (o2, _) in zip(spans, spans[1:]):
            assert o1 + n1 <= o2
        assert a.in_use == sum(live.values()) <= a.size
    for off in list(live):
        a.release(off)
    assert a.free == [(0, 1 << 20)] and a.in_use == 0


def test_memory_admission_in_arrival_order():
    one = serve.request_layout(10000, 16, FakeBackend().scratch_bytes)[1]
    srv, be = _server(pool=2 * one + 1000, streams=4, max_wave=8)
    for i in range(6):
        srv.submit(_req(i, 10000))
    peak = 0
    for _ in range(100):
        srv.step()
        peak = max(peak, srv.arena.in_use)
        if srv.idle():
            break
    assert srv.idle() and len(srv.finished) == 6
    assert peak <= srv.arena.size and srv.arena.peak <= 2 * one
    admitted = [r.rid for r in sorted(srv.finished, key=lambda r: (r.admitted, r.rid))]
    assert admitted == list(range(6))
    assert all(len(rids) <= 2 for _, rids, _ in be.launched)


def test_a_large_request_is_not_overtaken():
    small = serve.request_layout(1000, 16, FakeBackend().scratch_bytes)[1]
    big = serve.request_layout(50000, 16, FakeBackend().scratch_bytes)[1]
    srv, be = _server(pool=big + small, streams=2, max_wave=8)
    srv.submit(_req(0, 1000))
    srv.submit(_req(1, 1000))
    srv.submit(_req(2, 50000))
    srv.submit(_req(3, 1000))
    srv.step()
    assert be.launched[0][1] == [0, 1]          # the big one does not fit beside them
    srv.drain()
    order = [rids for _, rids, _ in be.launched]
    assert order[1] == [2, 3]


def test_waves_overlap_and_late_arrivals_join_the_next_wave():
    srv, be = _server(pool=1 << 30, streams=2, max_wave=4, delay=3)
    for i in range(3):
        srv.submit(_req(i, 500))
    srv.step()                       # wave 0 launches with the three waiting requests
    srv.submit(_req(3, 500))
    srv.submit(_req(4, 500))
    srv.step()                       # wave 1 launches while wave 0 is still running
    assert len(srv.running) == 2
    assert be.launched[0][1] == [0, 1, 2] and be.launched[1][1] == [3, 4]
    assert be.launched[0][0] != be.launched[1][0]
    srv.submit(_req(5, 500))
    srv.step()                       # both workspaces busy: request 5 waits
    assert [r.rid for r in srv.waiting] == [5]
    srv.drain()
    assert sorted(r.rid for r in srv.finished) == list(range(6))
    assert srv.waves == 3


def test_run_trace_and_summary():
    srv, _ = _server(pool=1 << 30, streams=2, max_wave=16, delay=1)
    reqs = [_req(i, 100 + i, arrival=0.0005 * i) for i in range(20)]
    out = serve.run_trace(srv, reqs, poll_s=0.0001)
    assert out["requests"] == 20 and out["p99_ms"] >= out["p50_ms"] >= 0.0
    assert all(r.done >= r.arrival for r in reqs)


def test_poisson_arrivals():
    t = serve.poisson_arrivals(200.0, 30.0, 7)
    assert np.all(np.diff(t) > 0) and t[-1] < 30.0
    assert abs(t.size - 6000) < 4 * np.sqrt(6000)
    assert np.array_equal(t, serve.poisson_arrivals(200.0, 30.0, 7))


class FakeSoloBackend(FakeBackend):
    has_solo = True
    solo_slots = 1

    def __init__(self, delay=2):
        super().__init__(delay)
        self.solo = []

    def launch_solo(self, r):
        self.solo.append(r.rid)
        return {"polls": 0, "slot": -1}


def test_short_queues_use_the_whole_gpu_lane_and_long_ones_batch():
    be = FakeSoloBackend(delay=2)
    srv = serve.Server(be, 1 << 30, streams=2, max_wave=8, solo_queue=2)
    be.server = srv
    srv.submit(_req(0, 500))
    srv.step()
    assert be.solo == [0] and not be.launched          # one waiting, device idle: solo
    srv.submit(_req(1, 500))
    srv.step()
    assert be.solo == [0] and not be.launched          # solo lane busy, short queue: wait for it
    for i in range(2, 6):
        srv.submit(_req(i, 500))
    srv.step()
    assert be.launched and be.launched[0][1] == [1, 2, 3, 4, 5]  # long queue: a batch wave
    srv.submit(_req(6, 500))
    srv.step()
    assert 6 not in be.solo                            # a batch wave runs: short queues join batch lanes
    assert be.launched[-1][1] == [6]
    srv.drain()
    assert sorted(r.rid for r in srv.finished) == list(range(7))
    assert srv.solo_inflight == 0


def test_whole_gpu_lane_keeps_solo_slots_requests_in_flight():
    be = FakeSoloBackend(delay=3)
    be.solo_slots = 2
    srv = serve.Server(be, 1 << 30, streams=2, max_wave=8, solo_queue=4)
    be.server = srv
    for i in range(3):
        srv.submit(_req(i, 500))
    srv.step()
    srv.step()
    assert be.solo == [0, 1] and not be.launched       # two in flight, the third waits for a slot
    assert srv.solo_inflight == 2
    srv.drain()
    assert be.solo == [0, 1, 2] and srv.solo_inflight == 0
    assert sorted(r.rid for r in srv.finished) == [0, 1, 2]


class FakeLiveBackend:
    """A live launch on the host: items publish into a ring of `capacity` slots
    per class and finish `work` steps after they were published; the launch
    'runs' until `idle` steps pass without items in flight."""

    def __init__(self, capacity=4, work=2, idle=3, split=1000):
        self.capacity, self.work, self.idle, self.split = capacity, work, idle, split
        self.launches = 0
        self.running_for = 0

    def scratch_bytes(self, cap):
        return 0

    def pixels_in_place(self, r):
        return False

    def setup(self, pool_bytes, host_bytes):
        self.tail = [0, 0]
        self.slot = [[None] * self.capacity, [None] * self.capacity]  # (seq, steps left)
        self.collected = []

    def tick(self):
        for c in (0, 1):
            for j, v in enumerate(self.slot[c]):
                if v is not None and v[1] > 0:
                    self.slot[c][j] = (v[0], v[1] - 1)
        self.running_for = max(0, self.running_for - 1)

    def ensure_running(self):
        if self.running_for == 0:
            self.launches += 1
        self.running_for = self.idle

    def publish(self, r):
        c = 0 if r.n_pixels > self.split else 1
        t = self.tail[c]
        j = t % self.capacity
        old = self.slot[c][j]
        if old is not None and old[1] > 0:
            return None  # the slot's item is not done
        self.slot[c][j] = (t, self.work)
        self.tail[c] += 1
        return (c, t)

    def done(self, c, seq):
        v = self.slot[c][seq % self.capacity]
        return v is not None and v[0] == seq and v[1] == 0

    def collect(self, r):
        self.collected.append(r.rid)


def _live_reqs(sizes):
    return [serve.Request(rid=i, rgb=np.zeros(3 * n, np.uint8), K=8) for i, n in enumerate(sizes)]


def test_live_server_admits_in_order_by_memory_and_ring():
    be = FakeLiveBackend(capacity=2, work=2)
    host_one = serve.live_layout(100, 8, be.scratch_bytes, False)[1]
    srv = serve.LiveServer(be, pool_bytes=1 << 20, host_bytes=3 * host_one)
    for r in _live_reqs([100] * 5):
        srv.submit(r)
    srv.step()
    # the ring of class 1 has two slots: two items published, the rest wait
    assert sorted(srv.inflight) == [(1, 0), (1, 1)] and len(srv.waiting) == 3 and be.launches == 1
    for _ in range(3):
        be.tick()
        srv.step()
    assert [r.rid for r in srv.finished][:2] == [0, 1]
    while not srv.idle():
        be.tick()
        srv.step()
    assert [r.rid for r in srv.finished] == [0, 1, 2, 3, 4]
    assert be.collected == [0, 1, 2, 3, 4]
    assert srv.host_arena.in_use == 0 and srv.dev_arena.in_use == 0
    assert srv.max_inflight <= 2


def test_live_server_blocks_on_memory_without_overtaking():
    be = FakeLiveBackend(capacity=8, work=3)
    big = serve.live_layout(1000, 8, be.scratch_bytes, False)[1]
    small = serve.live_layout(10, 8, be.scratch_bytes, False)[1]
    srv = serve.LiveServer(be, pool_bytes=1 << 20, host_bytes=big + 256)  # < big + small
    for r in _live_reqs([10, 1000, 10]):
        srv.submit(r)
    srv.step()
    # the large request does not fit beside the first small one; the second small
    # one, behind it, is not admitted first
    assert list(srv.inflight.values())[0].rid == 0 and len(srv.inflight) == 1
    assert [r.rid for r in srv.waiting] == [1, 2]
    while not srv.idle():
        be.tick()
        srv.step()
    assert [r.rid for r in srv.finished] == [0, 1, 2]


def test_live_server_retires_an_item_whose_slot_was_reused():
    # an item finishes, but the server has not seen its mark when the next
    # publication takes its slot: it is retired at that moment
    be = FakeLiveBackend(capacity=1, work=1)
    real_done = be.done
    be.done = lambda c, seq: False  # the marks stay unseen
    srv = serve.LiveServer(be, pool_bytes=1 << 20, host_bytes=1 << 20)
    reqs = _live_reqs([50, 50])
    srv.submit(reqs[0])
    srv.step()
    be.tick()  # item 0 is done
    srv.submit(reqs[1])
    srv.step()  # publishing item 1 reuses item 0's slot
    assert [r.rid for r in srv.finished] == [0] and list(srv.inflight) == [(1, 1)]
    be.done = real_done
    while not srv.idle():
        be.tick()
        srv.step()
    assert [r.rid for r in srv.finished] == [0, 1]


def test_live_server_relaunches_after_idle_exit():
    be = FakeLiveBackend(capacity=4, work=1, idle=2)
    srv = serve.LiveServer(be, pool_bytes=1 << 20, host_bytes=1 << 20)
    srv.submit(_live_reqs([20])[0])
    while not srv.idle():
        be.tick()
        srv.step()
    for _ in range(4):
        be.tick()  # the launch leaves after its idle limit
    r = _live_reqs([20])[0]
    r.rid = 7
    srv.submit(r)
    while not srv.idle():
        be.tick()
        srv.step()
    assert be.launches == 2 and [x.rid for x in srv.finished] == [0, 7]
