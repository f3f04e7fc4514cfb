"""Serving: a request loop with memory admission and continuous batching.

Requests (one image each, with its own K, scheme and seed) arrive over time.
The server keeps on the device

* a pool of device memory from which each admitted request gets one block
  (its pixels, its unique colours and weights, labels, seeding scratch, centres,
  palette, result and output indices: ``request_bytes``), and
* ``streams`` batch workspaces (kq_batch_workspace_size each), whose colour
  tables stay resident and zero between requests.

``step()`` is the scheduler.  It retires every wave whose completion event has
fired (freeing its requests' blocks and its workspace).  While few requests wait
(``solo_queue``) and no batch wave runs, a backend with a whole-GPU lane serves
them one at a time through the four single-image calls, the lowest latency
under light load.  Otherwise, while a workspace is free and requests are
waiting, it forms a wave: requests are taken in arrival
order as long as their blocks fit in the pool (memory admission; the first that
does not fit waits, so no request is overtaken), their pixels are copied in,
and the wave runs as one kq_batch_run on its own stream, followed by the copies
of the results to the host.  A wave started while another is still running
overlaps with it on the device: the running launch's persistent blocks leave
as its queue empties and the new launch's blocks take their SMs.  Each image is
computed by one block group with no data shared with other images, so a
request's result does not depend on what else is in the batch.

``LiveServer`` admits requests into a launch that is already running
(kq_live_*): each admitted request is published into the launch's queue at
once, a group of the persistent kernel takes it as soon as one is free, and the
host retires it when its done mark appears.  Nothing waits for a wave to drain.
Its pixels and outputs stay in page-locked host memory, which the kernel reads
and writes directly; the colour lists and scratch come from a device pool.

The device side sits behind a small backend interface so that the scheduling
logic can be exercised without a GPU.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field
from typing import Deque, Dict, List, Optional, Tuple

import numpy as np

ALIGN = 256


def _align(v: int, a: int = ALIGN) -> int:
    return (v + a - 1) // a * a


class Arena:
    """First-fit allocator over [0, size) with 256-byte alignment (offsets only)."""

    def __init__(self, size: int):
        self.size = int(size)
        self.free: List[Tuple[int, int]] = [(0, self.size)]  # (offset, length), sorted, coalesced
        self.used: Dict[int, int] = {}
        self.in_use = 0
        self.peak = 0

    def alloc(self, nbytes: int) -> Optional[int]:
        n = _align(max(int(nbytes), 1))
        for j, (off, ln) in enumerate(self.free):
            if ln >= n:
                if ln == n:
                    self.free.pop(j)
                else:
                    self.free[j] = (off + n, ln - n)
                self.used[off] = n
                self.in_use += n
                self.peak = max(self.peak, self.in_use)
                return off
        return None

    def release(self, off: int) -> None:
        n = self.used.pop(off)
        self.in_use -= n
        self.free.append((off, n))
        self.free.sort()
        merged: List[Tuple[int, int]] = []
        for o, ln in self.free:
            if merged and merged[-1][0] + merged[-1][1] == o:
                merged[-1] = (merged[-1][0], merged[-1][1] + ln)
            else:
                merged.append((o, ln))
        self.free = merged


RESULT_BYTES = 96  # sizeof(kq_batch_result)


def request_layout(n_pixels: int, K: int, scratch_bytes) -> Tuple[Dict[str, Tuple[int, int]], int]:
    """Offsets (relative to a request's block) and sizes of its device buffers."""
    cap = max(0, min(int(n_pixels), 1 << 24))
    lay: Dict[str, Tuple[int, int]] = {}
    off = 0
    for name, size in (("rgb", 3 * n_pixels), ("idx", n_pixels), ("keys", 4 * cap), ("weights", 4 * cap),
                       ("labels", cap), ("scratch", scratch_bytes(cap)), ("centers", 24 * K),
                       ("palette", 3 * K), ("result", RESULT_BYTES)):
        lay[name] = (off, size)
        off = _align(off + max(size, 1))
    return lay, off


@dataclass
class Request:
    rid: int
    rgb: object                # host pixels, n_pixels x 3 uint8: numpy array or (pinned) torch CPU tensor
    K: int
    scheme: str = "KPP"
    seed: int = 0
    eps: float = 1e-4
    max_iter: int = 100
    arrival: float = 0.0       # seconds on the server's clock
    # filled in by the server
    n_pixels: int = 0
    block: int = -1
    layout: Dict[str, Tuple[int, int]] = field(default_factory=dict)
    nbytes: int = 0
    dev_block: int = -1                                   # LiveServer: device pool block
    dev_layout: Dict[str, Tuple[int, int]] = field(default_factory=dict)
    dev_bytes: int = 0
    admitted: float = -1.0
    done: float = -1.0
    idx: Optional[np.ndarray] = None
    palette: Optional[np.ndarray] = None
    centers: Optional[np.ndarray] = None
    result: Optional[np.ndarray] = None


@dataclass
class Wave:
    slot: int
    requests: List[Request]
    handle: object = None


class Server:
    """Continuous-batching quantization server (see the module docstring)."""

    def __init__(self, backend, pool_bytes: int, streams: int = 2, max_wave: int = 64, clock=time.perf_counter,
                 solo_queue: int = 2):
        """solo_queue: with a backend that has a whole-GPU lane (launch_solo), requests
        are served one at a time on it while at most this many wait and no batch wave
        runs (the lowest latency under light load); longer queues form batch waves."""
        self.backend = backend
        self.solo_queue = int(solo_queue)
        self.solo_inflight = 0
        self.arena = Arena(pool_bytes)
        self.streams = int(streams)
        self.max_wave = int(max_wave)
        self.clock = clock
        self.t0 = clock()
        backend.setup(pool_bytes, self.streams, self.max_wave)
        self.free_slots: Deque[int] = deque(range(self.streams))
        self.waiting: Deque[Request] = deque()
        self.running: List[Wave] = []
        self.finished: List[Request] = []
        self.waves = 0
        self.max_running = 0

    def now(self) -> float:
        return self.clock() - self.t0

    def submit(self, req: Request) -> None:
        npx = req.rgb.numel() if hasattr(req.rgb, "numel") else req.rgb.size
        req.n_pixels = int(npx // 3)
        req.layout, req.nbytes = request_layout(req.n_pixels, req.K, self.backend.scratch_bytes)
        if req.nbytes > self.arena.size:
            raise ValueError("request %d needs %d bytes, more than the whole pool" % (req.rid, req.nbytes))
        self.waiting.append(req)

    def step(self) -> int:
        """Retires finished waves and launches new ones; returns requests completed."""
        done = 0
        still: List[Wave] = []
        for wv in self.running:
            if self.backend.done(wv.handle):
                t = self.now()
                self.backend.collect(wv.handle, wv.requests)
                for r in wv.requests:
                    r.done = t
                    self.arena.release(r.block)
                    self.finished.append(r)
                done += len(wv.requests)
                if wv.slot < 0:
                    self.solo_inflight -= 1
                else:
                    self.free_slots.append(wv.slot)
            else:
                still.append(wv)
        self.running = still
        solo_lane = getattr(self.backend, "has_solo", False)
        batch_running = any(wv.slot >= 0 for wv in self.running)
        if solo_lane and self.waiting and len(self.waiting) <= self.solo_queue and not batch_running:
            # short queue on a device without batch waves: the whole-GPU lane, up to
            # the backend's solo_slots requests in flight (so that one request's
            # copies overlap another's kernels); a full lane is waited for
            if self.solo_inflight >= getattr(self.backend, "solo_slots", 1):
                return done
            r = self.waiting[0]
            off = self.arena.alloc(r.nbytes)
            if off is None:
                return done
            self.waiting.popleft()
            r.block = off
            r.admitted = self.now()
            self.running.append(Wave(-1, [r], self.backend.launch_solo(r)))
            self.solo_inflight += 1
            self.waves += 1
            self.max_running = max(self.max_running, len(self.running))
            return done
        while self.free_slots and self.waiting:
            batch: List[Request] = []
            while self.waiting and len(batch) < self.max_wave:
                r = self.waiting[0]
                off = self.arena.alloc(r.nbytes)
                if off is None:
                    break  # waits for memory; nothing behind it is admitted first
                self.waiting.popleft()
                r.block = off
                r.admitted = self.now()
                batch.append(r)
            if not batch:
                break
            slot = self.free_slots.popleft()
            handle = self.backend.launch(slot, batch)
            self.running.append(Wave(slot, batch, handle))
            self.waves += 1
            self.max_running = max(self.max_running, len(self.running))
        return done

    def idle(self) -> bool:
        return not self.waiting and not self.running

    def drain(self, poll_s: float = 0.0) -> None:
        while not self.idle():
            if self.step() == 0 and poll_s > 0:
                time.sleep(poll_s)


LIVE_HOST = ("rgb", "idx", "centers", "palette", "result")
LIVE_DEV = ("keys", "weights", "labels", "scratch")


def live_layout(n_pixels: int, K: int, scratch_bytes, pixels_in_place: bool):
    """Offsets and sizes of a live request's buffers: (host block, device block).
    With pixels_in_place the request's own page-locked pixels are used as they are."""
    cap = max(0, min(int(n_pixels), 1 << 24))
    sizes = {"rgb": 0 if pixels_in_place else 3 * n_pixels, "idx": n_pixels, "centers": 24 * K, "palette": 3 * K,
             "result": RESULT_BYTES, "keys": 4 * cap, "weights": 4 * cap, "labels": cap,
             "scratch": scratch_bytes(cap)}
    host, dev, ho, do = {}, {}, 0, 0
    for name in LIVE_HOST:
        host[name] = (ho, sizes[name])
        ho = _align(ho + max(sizes[name], 1))
    for name in LIVE_DEV:
        dev[name] = (do, sizes[name])
        do = _align(do + max(sizes[name], 1))
    return host, ho, dev, do


class LiveServer:
    """Continuous admission into a running launch (see the module docstring).

    step() retires every request whose done mark is set, then admits waiting
    requests in arrival order while their host and device blocks fit and the
    queue has a free slot (the first that does not fit waits; nobody overtakes
    it), publishing each at once, and keeps a launch running while requests are
    in flight (the launch leaves by itself after an idle limit)."""

    def __init__(self, backend, pool_bytes: int, host_bytes: int, clock=time.perf_counter):
        self.backend = backend
        self.dev_arena = Arena(pool_bytes)
        self.host_arena = Arena(host_bytes)
        self.clock = clock
        self.t0 = clock()
        backend.setup(pool_bytes, host_bytes)
        self.waiting: Deque[Request] = deque()
        self.inflight: Dict[Tuple[int, int], Request] = {}
        self.finished: List[Request] = []
        self.max_inflight = 0

    def now(self) -> float:
        return self.clock() - self.t0

    def submit(self, req: Request) -> None:
        npx = req.rgb.numel() if hasattr(req.rgb, "numel") else req.rgb.size
        req.n_pixels = int(npx // 3)
        in_place = self.backend.pixels_in_place(req)
        req.layout, req.nbytes, req.dev_layout, req.dev_bytes = live_layout(req.n_pixels, req.K,
                                                                              self.backend.scratch_bytes, in_place)
        if req.nbytes > self.host_arena.size or req.dev_bytes > self.dev_arena.size:
            raise ValueError("request %d does not fit the pools" % req.rid)
        self.waiting.append(req)

    def _retire(self, key, t) -> None:
        r = self.inflight.pop(key)
        self.backend.collect(r)
        r.done = t
        self.host_arena.release(r.block)
        self.dev_arena.release(r.dev_block)
        self.finished.append(r)

    def step(self) -> int:
        """Retires finished requests and admits new ones; returns requests completed."""
        t = self.now()
        done_keys = [k for k in self.inflight if self.backend.done(*k)]
        for k in done_keys:
            self._retire(k, t)
        while self.waiting:
            r = self.waiting[0]
            hb = self.host_arena.alloc(r.nbytes)
            if hb is None:
                break
            db = self.dev_arena.alloc(r.dev_bytes)
            if db is None:
                self.host_arena.release(hb)
                break
            r.block, r.dev_block = hb, db
            key = self.backend.publish(r)
            if key is None:  # no free queue slot
                self.host_arena.release(hb)
                self.dev_arena.release(db)
                break
            self.waiting.popleft()
            r.admitted = self.now()
            # the slot's previous item was done (publication checks that) and its
            # mark is gone with it: retire it now if it is still listed
            prev = (key[0], key[1] - self.backend.capacity)
            if prev in self.inflight:
                self._retire(prev, self.now())
                done_keys.append(prev)
            self.inflight[key] = r
            self.max_inflight = max(self.max_inflight, len(self.inflight))
        if self.inflight:
            self.backend.ensure_running()
        return len(done_keys)

    def idle(self) -> bool:
        return not self.waiting and not self.inflight

    def drain(self, poll_s: float = 0.0) -> None:
        while not self.idle():
            if self.step() == 0 and poll_s > 0:
                time.sleep(poll_s)


def run_trace(server: Server, requests: List[Request], poll_s: float = 0.0002) -> Dict:
    """Submits each request at its arrival time (server clock), runs the
    scheduler until all are done, and summarises latency and throughput."""
    reqs = sorted(requests, key=lambda r: r.arrival)
    server.t0 = server.clock()
    i = 0
    while i < len(reqs) or not server.idle():
        t = server.now()
        while i < len(reqs) and reqs[i].arrival <= t:
            server.submit(reqs[i])
            i += 1
        if server.step() == 0:
            nxt = reqs[i].arrival - server.now() if i < len(reqs) else poll_s
            if nxt > 0:
                time.sleep(min(poll_s, nxt))
    return summarize(reqs)


def summarize(reqs: List[Request]) -> Dict:
    lat = np.array([r.done - r.arrival for r in reqs], dtype=np.float64)
    span = max(r.done for r in reqs) - min(r.arrival for r in reqs) if reqs else 0.0
    px = sum(r.n_pixels for r in reqs)
    return {"requests": len(reqs), "p50_ms": float(np.percentile(lat, 50) * 1e3) if reqs else 0.0,
            "p99_ms": float(np.percentile(lat, 99) * 1e3) if reqs else 0.0,
            "mean_ms": float(lat.mean() * 1e3) if reqs else 0.0,
            "img_per_s": len(reqs) / span if span > 0 else 0.0, "mpix_per_s": px / span / 1e6 if span > 0 else 0.0,
            "span_s": span}


def poisson_arrivals(rate: float, duration: float, seed: int) -> np.ndarray:
    """Arrival times of a Poisson process (exponential gaps from SplitMix64 uniforms)."""
    from . import synth

    n_max = int(rate * duration * 1.5 + 64)
    u = synth.uniform(seed, 30, n_max)
    t = np.cumsum(-np.log1p(-u) / rate)
    return t[t < duration]


class CudaBackend:
    """The device side of the server: one pool tensor, `streams` workspaces, item
    buffers and pinned staging buffers, and one kq_batch_run per wave."""

    OUT = ("idx", "palette", "centers", "result")

    def __init__(self, cluster: int = 1, split_pixels: int = 1 << 62, device=None, solo_max_pixels: int = 0):
        """solo_max_pixels > 0 gives the server a whole-GPU lane (launch_solo) for
        requests up to that many pixels: the four single-image calls on the whole
        GPU, the lowest latency when few requests wait."""
        import torch

        from . import kq

        self.torch, self.kq = torch, kq
        self.device = torch.device("cuda") if device is None else torch.device(device)
        self.cfg = kq.BatchConfig(int(cluster), 0, int(split_pixels))
        self.solo_max_pixels = int(solo_max_pixels)
        self.solo_waves = 0
        self.solo_slots = 2

    def scratch_bytes(self, cap: int) -> int:
        return self.kq.kq_batch_scratch_bytes(cap)

    def setup(self, pool_bytes: int, streams: int, max_wave: int) -> None:
        torch, kq = self.torch, self.kq
        self.pool = torch.empty(pool_bytes, dtype=torch.uint8, device=self.device)
        wsb = kq.kq_batch_workspace_size()
        self.ws = [torch.zeros(wsb, dtype=torch.uint8, device=self.device) for _ in range(streams)]
        isz = kq.BATCH_ITEM_DTYPE.itemsize
        self.items = [torch.empty(max_wave * isz, dtype=torch.uint8, device=self.device) for _ in range(streams)]
        self.order = [torch.empty(max_wave, dtype=torch.int32, device=self.device) for _ in range(streams)]
        self.h_items = [torch.empty(max_wave * isz, dtype=torch.uint8).pin_memory() for _ in range(streams)]
        self.h_order = [torch.empty(max_wave, dtype=torch.int32).pin_memory() for _ in range(streams)]
        self.h_out = [torch.empty(1 << 20, dtype=torch.uint8).pin_memory() for _ in range(streams)]
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(streams)]
        self.events = [torch.cuda.Event() for _ in range(streams)]
        self.h2d_bytes = 0
        self.d2h_bytes = 0
        self.solo = None
        if self.solo_max_pixels > 0:
            self.solo = PlainBackend(self.solo_max_pixels, device=self.device)
            self.solo.setup(0, self.solo_slots, 1)
            self.solo_free = deque(range(self.solo_slots))
        # the workspaces were zero-filled on the current stream; the waves run on
        # their own streams
        torch.cuda.current_stream(self.device).synchronize()

    def _pinned(self, r: "Request"):
        t = r.rgb
        if isinstance(t, np.ndarray):
            t = self.torch.from_numpy(np.ascontiguousarray(t).reshape(-1))
        return t.reshape(-1)

    @property
    def has_solo(self) -> bool:
        return self.solo is not None

    def launch_solo(self, r: Request):
        """One request on the whole GPU through the four single-image calls."""
        if r.n_pixels > self.solo_max_pixels:
            raise ValueError("request larger than the whole-GPU lane's buffers")
        self.solo_waves += 1
        self.h2d_bytes += 3 * r.n_pixels
        self.d2h_bytes += r.n_pixels + 3 * r.K
        return ("solo", self.solo.launch(self.solo_free.popleft(), [r]))

    def launch(self, slot: int, batch: List[Request]):
        torch, kq = self.torch, self.kq
        s = self.streams[slot]
        base = self.pool.data_ptr()
        items = np.zeros(len(batch), dtype=kq.BATCH_ITEM_DTYPE)
        need = sum(_align(r.layout[n][1]) for r in batch for n in self.OUT)
        if need > self.h_out[slot].numel():
            self.h_out[slot] = torch.empty(_align(need * 2, 1 << 20), dtype=torch.uint8).pin_memory()
        stage = self.h_out[slot]
        outs = []
        with torch.cuda.stream(s):
            for j, r in enumerate(batch):
                b = r.block
                for name in ("rgb", "idx", "keys", "weights", "labels", "scratch", "centers", "palette", "result"):
                    items[j][name] = base + b + r.layout[name][0]
                cap = max(0, min(r.n_pixels, 1 << 24))
                items[j]["n_pixels"], items[j]["seed"], items[j]["eps"] = r.n_pixels, r.seed, r.eps
                items[j]["lbg_eps"], items[j]["lbg_conv_eps"], items[j]["lbg_max_iter"] = 1.0, r.eps, r.max_iter
                items[j]["K"], items[j]["scheme"] = r.K, kq.INIT[r.scheme]
                items[j]["max_iter"], items[j]["capacity"] = r.max_iter, cap
                off, size = r.layout["rgb"]
                if size:
                    self.pool[b + off:b + off + size].copy_(self._pinned(r), non_blocking=True)
                    self.h2d_bytes += size
            order, nb = kq.kq_batch_plan(items, self.cfg)
            hi = self.h_items[slot][:items.nbytes]
            hi.numpy()[:] = items.view(np.uint8)
            self.items[slot][:items.nbytes].copy_(hi, non_blocking=True)
            ho = self.h_order[slot][:len(batch)]
            ho.numpy()[:] = order
            self.order[slot][:len(batch)].copy_(ho, non_blocking=True)
            kq.kq_batch_run(self.items[slot], len(batch), self.order[slot], nb, self.cfg, self.ws[slot], stream=s)
            so = 0
            for r in batch:
                b = r.block
                o = {}
                for name in self.OUT:
                    off, size = r.layout[name]
                    if size:
                        stage[so:so + size].copy_(self.pool[b + off:b + off + size], non_blocking=True)
                        self.d2h_bytes += size
                    o[name] = (so, size)
                    so += _align(size)
                outs.append(o)
            ev = self.events[slot]
            ev.record(s)
        return (slot, ev, outs)

    def done(self, handle) -> bool:
        if handle[0] == "solo":
            return self.solo.done(handle[1])
        return handle[1].query()

    def collect(self, handle, batch: List[Request]) -> None:
        kq = self.kq
        if handle[0] == "solo":
            self.solo.collect(handle[1], batch)
            self.solo_free.append(handle[1][0])
            return
        stage = self.h_out[handle[0]].numpy()
        for r, o in zip(batch, handle[2]):
            def get(name):
                so, size = o[name]
                return stage[so:so + size].copy()
            r.idx = get("idx")
            r.palette = get("palette").reshape(-1, 3)
            r.centers = get("centers").view(np.float64).reshape(-1, 3)
            r.result = np.frombuffer(get("result").tobytes(), dtype=kq.BATCH_RESULT_DTYPE)[0]


class PlainBackend:
    """The plain per-image path behind the same scheduler, for comparison: each
    request runs alone through the four single-image calls (kq.Quantizer) on
    the whole GPU, one after another."""

    def __init__(self, max_pixels: int, device=None):
        import torch

        from . import kq

        self.torch, self.kq = torch, kq
        self.device = torch.device("cuda") if device is None else torch.device(device)
        self.max_pixels = int(max_pixels)

    def scratch_bytes(self, cap: int) -> int:
        return self.kq.kq_batch_scratch_bytes(cap)

    def setup(self, pool_bytes: int, streams: int, max_wave: int) -> None:
        torch, kq = self.torch, self.kq
        self.q = [kq.Quantizer(self.max_pixels, device=self.device) for _ in range(streams)]
        self.rgb = [torch.empty(3 * self.max_pixels, dtype=torch.uint8, device=self.device) for _ in range(streams)]
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(streams)]
        self.events = [torch.cuda.Event() for _ in range(streams)]
        self.h_idx = [torch.empty(self.max_pixels, dtype=torch.uint8).pin_memory() for _ in range(streams)]
        self.h_small = [torch.empty(8192, dtype=torch.uint8).pin_memory() for _ in range(streams)]
        # the Quantizers' workspaces were zero-filled on the current stream
        torch.cuda.current_stream(self.device).synchronize()

    def launch(self, slot: int, batch: List[Request]):
        torch = self.torch
        s = self.streams[slot]
        q = self.q[slot]
        outs = []
        with torch.cuda.stream(s):
            for r in batch:
                n = r.n_pixels
                src = r.rgb if not isinstance(r.rgb, np.ndarray) else torch.from_numpy(np.ascontiguousarray(r.rgb))
                d = self.rgb[slot][:3 * n]
                d.copy_(src.reshape(-1), non_blocking=True)
                res = q.quantize(d, r.K, r.scheme, r.seed, r.eps, r.max_iter, stream=s)
                self.h_idx[slot][:n].copy_(res.idx, non_blocking=True)
                hs = self.h_small[slot]
                hs[:3 * r.K].copy_(res.palette.reshape(-1), non_blocking=True)
                hs[1024:1024 + 24 * r.K].copy_(res.centers.reshape(-1).view(torch.uint8), non_blocking=True)
                hs[7168:7208].copy_(res.stats[:40], non_blocking=True)
                hs[7232:7240].copy_(res.sse_num.view(torch.uint8), non_blocking=True)
                hs[7296:7300].copy_(res.n_unique.view(torch.uint8), non_blocking=True)
                outs.append(n)
            self.events[slot].record(s)
        return (slot, self.events[slot], outs)

    def done(self, handle) -> bool:
        return handle[1].query()

    def collect(self, handle, batch: List[Request]) -> None:
        kq = self.kq
        slot = handle[0]
        hs = self.h_small[slot].numpy()
        for r in batch:
            r.idx = self.h_idx[slot][:r.n_pixels].numpy().copy()
            r.palette = hs[:3 * r.K].copy().reshape(-1, 3)
            r.centers = hs[1024:1024 + 24 * r.K].copy().view(np.float64).reshape(-1, 3)
            res = np.zeros(1, dtype=kq.BATCH_RESULT_DTYPE)[0]
            res["lloyd"] = np.frombuffer(hs[7168:7208].tobytes(), dtype=kq.STATS_DTYPE)[0]
            res["sse_num"] = int(hs[7232:7240].view(np.int64)[0])
            res["n_unique"] = int(hs[7296:7300].view(np.int32)[0])
            res["status"] = res["lloyd"]["status"]
            r.result = res


class LiveBackend:
    """The device side of LiveServer: a page-locked host pool (pixels unless the
    request's own are page-locked, indices, centres, palette, result), a device
    pool (colour lists, scratch), one batch workspace and the queue of one live
    launch (kq_live_run), relaunched whenever requests are in flight and the last
    launch has left after its idle limit."""

    def __init__(self, cluster: int = 1, split_pixels: int = 1 << 62, device=None, idle_us: int = 20000,
                 capacity: int = 1024):
        import torch

        from . import kq

        self.torch, self.kq = torch, kq
        self.device = torch.device("cuda") if device is None else torch.device(device)
        self.cfg = kq.BatchConfig(int(cluster), 0, int(split_pixels))
        self.split = int(split_pixels) if int(cluster) > 1 else 1 << 62
        self.idle_us = int(idle_us)
        self.capacity = int(capacity)
        self.launches = 0

    def scratch_bytes(self, cap: int) -> int:
        return self.kq.kq_batch_scratch_bytes(cap)

    def pixels_in_place(self, r: Request) -> bool:
        t = r.rgb
        return hasattr(t, "is_pinned") and t.is_pinned() and t.is_contiguous()

    def setup(self, pool_bytes: int, host_bytes: int) -> None:
        torch, kq = self.torch, self.kq
        self.pool = torch.empty(pool_bytes, dtype=torch.uint8, device=self.device)
        self.host = torch.empty(host_bytes, dtype=torch.uint8).pin_memory()
        self.ws = torch.zeros(kq.kq_batch_workspace_size(), dtype=torch.uint8, device=self.device)
        self.q = kq.LiveQueue(self.capacity)
        kq.kq_live_reset(self.ws)
        self.stream = torch.cuda.Stream(device=self.device)
        self.ev = None
        torch.cuda.synchronize(self.device)

    def ensure_running(self) -> None:
        if self.ev is None or self.ev.query():
            self.kq.kq_live_run(self.q, self.cfg, self.idle_us, self.ws, stream=self.stream)
            self.ev = self.torch.cuda.Event()
            self.ev.record(self.stream)
            self.launches += 1

    def publish(self, r: Request):
        kq = self.kq
        hb, db = self.host.data_ptr() + r.block, self.pool.data_ptr() + r.dev_block
        it = np.zeros(1, dtype=kq.BATCH_ITEM_DTYPE)
        for name in LIVE_HOST:
            it[0][name] = hb + r.layout[name][0]
        for name in LIVE_DEV:
            it[0][name] = db + r.dev_layout[name][0]
        if self.pixels_in_place(r):
            it[0]["rgb"] = r.rgb.data_ptr()
        elif r.n_pixels:
            off, size = r.layout["rgb"]
            src = r.rgb if not isinstance(r.rgb, np.ndarray) else self.torch.from_numpy(np.ascontiguousarray(r.rgb))
            self.host[r.block + off:r.block + off + size].copy_(src.reshape(-1))
        cap = max(0, min(r.n_pixels, 1 << 24))
        it[0]["n_pixels"], it[0]["seed"], it[0]["eps"] = r.n_pixels, r.seed, r.eps
        it[0]["lbg_eps"], it[0]["lbg_conv_eps"], it[0]["lbg_max_iter"] = 1.0, r.eps, r.max_iter
        it[0]["K"], it[0]["scheme"] = r.K, kq.INIT[r.scheme]
        it[0]["max_iter"], it[0]["capacity"] = r.max_iter, cap
        cls = 0 if r.n_pixels > self.split else 1
        seq = self.q.publish(cls, it[0])
        return None if seq is None else (cls, seq)

    def done(self, cls: int, seq: int) -> bool:
        return self.q.done(cls, seq)

    def collect(self, r: Request) -> None:
        kq = self.kq
        h = self.host.numpy()

        def get(name):
            off, size = r.layout[name]
            return h[r.block + off:r.block + off + size].copy()
        r.idx = get("idx")
        r.palette = get("palette").reshape(-1, 3)
        r.centers = get("centers").view(np.float64).reshape(-1, 3)
        r.result = np.frombuffer(get("result").tobytes(), dtype=kq.BATCH_RESULT_DTYPE)[0]

    def close(self) -> None:
        self.q.close()
        self.stream.synchronize()
