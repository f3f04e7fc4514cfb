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
