#!/usr/bin/env python
"""Benchmark: exact k-means colour quantization (Weighted Sort-Means) on GB300.

One step = the whole hot path on one synthetic 512 x 512 RGB8 image already in
HBM: kq_histogram -> kq_seed (k-means++) -> kq_lloyd (K = 256, eps 1e-4, at most
100 passes) -> kq_map.  Every step is timed with CUDA events on the launching
stream; between steps a 256 MiB buffer is written to flush the 129 MB L2 (not
timed).  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
  python bench.py --workload batched [--count 512]     # img/s, one launch per batch
  python bench.py --workload serving [--rate 200]      # p50/p99 latency under Poisson arrivals
  python bench.py --workload table1                    # k-means on all pixels vs WSM (Table 1, Fig. 2)

Under torchrun (N > 1) every rank quantizes its own image (independent
replicas, no data exchange); value = pixels of all ranks / max step time.
--impl reference times the FP64 CPU oracle on the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "paper_512"
K_DEFAULT = 256
SOLO_QUEUE = 8   # serving: waiting requests up to which the whole-GPU lane serves them one at a time
SCHEME = "KPP"
SEED = 1101
FLOP_PER_DIST = 8          # 3 subtractions, 1 multiply, 2 fused multiply-adds
FP32_LANES_PER_SM = 128
METRIC = "Mpix/s end-to-end"


def parse_args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=300)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="kq", choices=["kq", "reference"])
    p.add_argument("--workload", default=WORKLOAD)
    p.add_argument("--K", type=int, default=K_DEFAULT)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--count", type=int, default=512, help="batched: images per batch")
    p.add_argument("--rate", type=float, default=200.0, help="serving: Poisson arrival rate (req/s)")
    p.add_argument("--duration", type=float, default=10.0, help="serving: arrival trace length (s)")
    p.add_argument("--no-extras", action="store_true",
                   help="default workload: skip the 4096x4096, batched and serving measurements")
    return p.parse_args(argv)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(value: float, world: int) -> float:
    """Max over ranks (host timing plumbing; no data-path collective)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int) -> None:
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def aggregate(pixels_per_rank: int, world: int, ms_per_step_max: float) -> float:
    """Whole-job Mpix/s: pixels processed by all ranks per step / slowest rank's step time."""
    return pixels_per_rank * world / (ms_per_step_max * 1e-3) / 1e6


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms while running."""

    FIELDS = ["clocks.sm", "clocks.max.sm", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) != len(self.FIELDS):
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[2:]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def profile_traffic(name: str):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from the
    committed ncu summary `profiles/<name>`, while the kernel's source still has the
    SHA-256 recorded there; None once the source has changed or the summary is absent."""
    import hashlib

    try:
        with open(os.path.join(ROOT, "profiles", name)) as f:
            lines = f.read().splitlines()
    except OSError:
        return None, "profiles/%s absent" % name
    sha = src = traffic = None
    for ln in lines:
        if ln.startswith("source_sha256:"):
            parts = ln.split()
            sha, src = parts[1], parts[2].strip("()")
        elif ln.startswith("traffic_bytes_per_launch:"):
            traffic = int(ln.split()[1])
    if sha is None or traffic is None:
        return None, "profiles/%s has no traffic line" % name
    try:
        with open(os.path.join(ROOT, src), "rb") as f:
            now = hashlib.sha256(f.read()).hexdigest()
    except OSError:
        return None, "%s absent" % src
    if now != sha:
        return None, "%s changed since profiles/%s was captured" % (src, name)
    return traffic, "profiles/%s (one ncu capture; %s unchanged since)" % (name, src)


def cpu_baseline(img, K: int, eps: float, max_iter: int, budget_s: float = 12.0) -> dict:
    """The FP64 oracle, as it stands, on the host cores: whole quantizations of
    the same image until `budget_s` of CPU work (at least one)."""
    import oracle

    n = img.size // 3
    times = []
    t_total = 0.0
    while not times or t_total < budget_s:
        t0 = time.perf_counter()
        oracle.quantize(img, K, SCHEME, SEED, eps, max_iter)
        dt = time.perf_counter() - t0
        times.append(dt)
        t_total += dt
        if len(times) >= 20:
            break
    mean = sum(times) / len(times)
    out = {"value": n / mean / 1e6, "unit": "Mpix/s", "cores": 1, "kind": "oracle",
           "sample": "%d whole quantization(s) of the %dx%d image (K=%d, %s, eps=%g, <=%d passes), %.1f s"
                     % (len(times), img.shape[0], img.shape[1], K, SCHEME, eps, max_iter, t_total),
           "cpu": cpu_model(), "nproc": os.cpu_count()}
    # the same oracle built with OpenMP over the assignment's colours, all host cores
    times = []
    t_total = 0.0
    with oracle.openmp():
        while not times or t_total < budget_s / 2:
            t0 = time.perf_counter()
            oracle.quantize(img, K, SCHEME, SEED, eps, max_iter)
            dt = time.perf_counter() - t0
            times.append(dt)
            t_total += dt
            if len(times) >= 20:
                break
    mean = sum(times) / len(times)
    out["openmp"] = {"value": n / mean / 1e6, "unit": "Mpix/s", "cores": os.cpu_count(), "kind": "oracle (OpenMP)",
                     "sample": "%d whole quantization(s), %.1f s; only the assignment is parallel" % (len(times), t_total)}
    return out


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                low = line.lower()
                if low.startswith("model name") or low.startswith("cpu part") or low.startswith("hardware"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def workload_config(wl, img, K, n_unique=None, iters=None) -> dict:
    cfg = {"workload": "%s: one %dx%d synthetic RGB8 image (%d regions, noise %g), K=%d, %s seeds, eps=%g, "
                       "<=%d passes" % (wl.name, wl.height, wl.width, wl.regions, wl.sigma_n, K, SCHEME, wl.eps,
                                        wl.max_iter),
           "n_pixels": int(img.size // 3), "K": K, "l2": "flushed between steps (256 MiB write, untimed)",
           "parallelism": "replicas (one image per GPU)"}
    if n_unique is not None:
        cfg["n_unique"] = int(n_unique)
    if iters is not None:
        cfg["lloyd_passes"] = int(iters)
    return cfg


def _gen_batch_image(args):
    from paper_1101_0395_gb300 import synth

    h, w, seed = args
    return synth.batch_image(h, w, seed)


def batch_images(spec, workers=None):
    """The batch's images, generated on all host cores (spawned workers, so no
    CUDA state is ever forked)."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor

    jobs = [(h, w, s) for (h, w), s in zip(spec.sizes, spec.seeds)]
    with ProcessPoolExecutor(max_workers=workers or os.cpu_count(), mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_gen_batch_image, jobs, chunksize=1))


def batched_config(spec, n_px, tuned=None) -> dict:
    cfg = {"workload": "batched: %d synthetic RGB8 images, side log-uniform 64-2048, aspect 0.5-2, K from "
                       "{16,32,64,128,256}, %s seeds, eps=1e-4, <=100 passes; one persistent launch per batch "
                       "(CUDA graph)" % (len(spec.sizes), SCHEME),
           "images": len(spec.sizes), "n_pixels": int(sum(n_px)), "l2": "inputs larger than L2 (no flush)",
           "parallelism": "replicas (one batch per GPU)"}
    if tuned is not None:
        cfg["launch_shape"] = tuned
    return cfg


def run_batched(args, rank, world, local) -> None:
    import numpy as np

    from paper_1101_0395_gb300 import synth

    spec = synth.batch_spec(args.count, seed=3101 + 7 * rank)
    imgs = batch_images(spec)
    import torch

    from paper_1101_0395_gb300 import kq

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n_px = [im.size // 3 for im in imgs]
    bq = kq.BatchQuantizer(n_px, spec.ks, SCHEME, spec.seeds, 1e-4, 100, device=dev)
    h_rgb = [torch.from_numpy(im.reshape(-1)).pin_memory() for im in imgs]
    for i in range(len(imgs)):
        bq.rgb(i).copy_(h_rgb[i], non_blocking=True)
    torch.cuda.synchronize()
    tune_ms = bq.tune()
    shape = {"cluster": bq.cfg.cluster, "split_pixels": bq.cfg.split_pixels, "images_on_clusters": bq.n_big,
             "autotuned_ms": tune_ms}
    bq.capture()
    stream = torch.cuda.current_stream()
    for _ in range(max(3, args.warmup)):
        bq.replay()
    torch.cuda.synchronize()
    res = bq.results()
    if np.any(res["status"] != kq.KQ_OK):
        raise RuntimeError("batch item errors: %s" % np.unique(res["status"]))
    steps = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    props = torch.cuda.get_device_properties(dev)
    clocks = ClockSampler("GPU-%s" % props.uuid if getattr(props, "uuid", None) else str(local))
    clocks.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    for s in range(steps):
        ev[s][0].record(stream)
        bq.replay()
        ev[s][1].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms = reduce_max(sum(a.elapsed_time(b) for a, b in ev) / steps, world)
    n_img = len(imgs)
    value = n_img * world / (ms * 1e-3)
    res = bq.results()
    t = res["t_ns"].astype(np.float64)
    stage = np.diff(t, axis=1) / 1e6
    big = np.zeros(n_img, bool)
    big[bq.order[:bq.n_big].cpu().numpy()] = True
    wgt = np.where(big, bq.cfg.cluster, 1)
    cta_ms = {nm: float((stage[:, j] * wgt).sum()) for j, nm in enumerate(["histogram", "seed", "lloyd", "map"])}
    # end to end: pixels in from pinned host memory, indices and results back
    h_idx = [torch.empty(n, dtype=torch.uint8).pin_memory() for n in n_px]
    e2e_steps = max(3, min(steps, 10))
    e2e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(e2e_steps)]
    for s in range(e2e_steps):
        e2e_ev[s][0].record(stream)
        for i in range(n_img):
            bq.rgb(i).copy_(h_rgb[i], non_blocking=True)
        bq.replay()
        for i in range(n_img):
            h_idx[i].copy_(bq.idx(i), non_blocking=True)
        e2e_ev[s][1].record(stream)
    torch.cuda.synchronize()
    e2e_ms = reduce_max(sum(a.elapsed_time(b) for a, b in e2e_ev) / e2e_steps, world)
    # the plain per-image path on the same GPU and images
    q = kq.Quantizer(max(n_px), device=dev)
    sse_loop = []
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for rep in range(2):
        sse_loop.clear()
        a0.record(stream)
        for i in range(n_img):
            r = q.quantize(bq.rgb(i), spec.ks[i], SCHEME, spec.seeds[i], 1e-4, 100)
            sse_loop.append(r.sse_num.clone())
        a1.record(stream)
        torch.cuda.synchronize()
    loop_ms = a0.elapsed_time(a1)
    sse_b = res["sse_num"].astype(np.int64)
    sse_l = np.array([int(x.item()) for x in sse_loop], dtype=np.int64)
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz") or 2070.0)
    fp32_peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    ndc = float(res["lloyd"]["ndc"].sum())
    achieved = ndc * FLOP_PER_DIST / (ms * 1e-3) / 1e12
    line = {"metric": "batched img/s", "value": value, "unit": "img/s", "n_gpus": world, "steps": steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": batched_config(spec, n_px, shape),
            "clocks": {k: clk[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
            "e2e": {"value": n_img * world / (e2e_ms * 1e-3), "unit": "img/s",
                    "h2d_bytes_per_step": int(3 * sum(n_px)), "d2h_bytes_per_step": int(sum(n_px))},
            "gpu_launches": steps,
            "mpix_per_s": sum(n_px) * world / (ms * 1e-3) / 1e6,
            "roofline": {"kernel": "batch_kernel (kq_batch_run)", "bound": "alu", "achieved": achieved,
                         "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak, "traffic": None,
                         "algorithmic": "%d FLOP per distance x NDC summed over the batch (%.3g)"
                                        % (FLOP_PER_DIST, ndc),
                         "peak_source": "derived: SMs x 128 FP32 lanes x 2 FLOP x max SM clock"},
            "stage_cta_ms": cta_ms,
            "per_image_path": {"value": n_img / (loop_ms * 1e-3), "unit": "img/s", "ms": loop_ms,
                               "same_sse_images": int((sse_b == sse_l).sum()),
                               "mse_batched": float(sse_b.sum() / sum(n_px)),
                               "mse_per_image": float(sse_l.sum() / sum(n_px))}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = batched_cpu_baseline(imgs, spec)
    if rank == 0:
        print(json.dumps(line), flush=True)


def batched_cpu_baseline(imgs, spec, budget_s: float = 15.0) -> dict:
    """The oracle on a size-stratified sample of the batch (every 64th image by
    size), as img/s at the batch's mean image size."""
    import oracle

    order = sorted(range(len(imgs)), key=lambda i: imgs[i].size)
    sample = order[::max(1, len(order) // 8)]
    px, t_total, done = 0, 0.0, 0
    for i in sample:
        t0 = time.perf_counter()
        oracle.quantize(imgs[i], spec.ks[i], SCHEME, spec.seeds[i], 1e-4, 100)
        t_total += time.perf_counter() - t0
        px += imgs[i].size // 3
        done += 1
        if t_total > budget_s:
            break
    mean_px = sum(im.size // 3 for im in imgs) / len(imgs)
    mpix = px / t_total / 1e6
    return {"value": mpix * 1e6 / mean_px, "unit": "img/s", "cores": 1, "kind": "oracle",
            "sample": "%d of %d images (stratified by size), %.1f Mpx in %.1f s = %.3f Mpix/s, at the batch's mean "
                      "of %.0f px per image" % (done, len(imgs), px / 1e6, t_total, mpix, mean_px),
            "cpu": cpu_model(), "nproc": os.cpu_count()}


def serving_trace(args, seed=4101):
    """Arrivals and request shapes: side log-uniform 256-4096 (aspect 0.5-2),
    K uniform in 8..256; images come from a pool of 48 generated images."""
    import numpy as np

    from paper_1101_0395_gb300 import serve, synth

    arrivals = serve.poisson_arrivals(args.rate, args.duration, seed)
    pool = synth.batch_spec(48, side_lo=256, side_hi=4096, seed=seed, k_uniform_range=(8, 256))
    u = synth.uniform(seed, 40, 2 * max(1, arrivals.size))
    picks = (u[0::2] * len(pool.sizes)).astype(int)
    ks = 8 + np.minimum(248, (u[1::2] * 249).astype(int))
    return arrivals, pool, picks, ks


def run_serving(args, rank, world, local) -> None:

    arrivals, pool, picks, ks = serving_trace(args)
    imgs = batch_images(pool)
    import torch

    from paper_1101_0395_gb300 import kq, serve

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    h_imgs = [torch.from_numpy(im.reshape(-1)).pin_memory() for im in imgs]
    max_px = max(im.size // 3 for im in imgs)

    def requests(count=None):
        out = []
        for i in range(arrivals.size if count is None else count):
            j = int(picks[i])
            out.append(serve.Request(rid=i, rgb=h_imgs[j], K=int(ks[i]), scheme=SCHEME, seed=1000 + i,
                                     arrival=float(arrivals[i]) if count is None else 0.0))
        return out

    # launch shape: the autotuner on one wave-sized batch of the pool
    n_px = [im.size // 3 for im in imgs]
    bq = kq.BatchQuantizer(n_px, [int(k) for k in ks[:len(imgs)]], SCHEME, list(range(len(imgs))), device=dev)
    for i in range(len(imgs)):
        bq.rgb(i).copy_(h_imgs[i])
    bq.tune()
    cluster, split = bq.cfg.cluster, bq.cfg.split_pixels
    del bq
    torch.cuda.empty_cache()
    pool_bytes = 48 << 30
    props = torch.cuda.get_device_properties(dev)
    clocks = ClockSampler("GPU-%s" % props.uuid if getattr(props, "uuid", None) else str(local))
    srv = serve.Server(serve.CudaBackend(cluster, split, device=dev, solo_max_pixels=max_px), pool_bytes, streams=2,
                       max_wave=64, solo_queue=SOLO_QUEUE)
    srv.drain()
    for r in requests(8):
        srv.submit(r)
    srv.drain()  # warm-up
    srv.finished.clear()
    clocks.start()
    reqs = requests()
    h2d0, d2h0 = srv.backend.h2d_bytes, srv.backend.d2h_bytes
    out = serve.run_trace(srv, reqs)
    clk = clocks.stop()
    h2d, d2h = srv.backend.h2d_bytes - h2d0, srv.backend.d2h_bytes - d2h0
    waves, solo_waves = srv.waves, srv.backend.solo_waves
    del srv
    torch.cuda.empty_cache()
    # admission into a running launch (live queue), on the same trace
    lbe = serve.LiveBackend(cluster, split, device=dev, idle_us=20000, capacity=4096)
    lsrv = serve.LiveServer(lbe, pool_bytes, 4 << 30)
    for r in requests(8):
        lsrv.submit(r)
    lsrv.drain()
    lsrv.finished.clear()
    lreqs = requests()
    lout = serve.run_trace(lsrv, lreqs)
    lsame = sum(int(a.result["sse_num"]) == int(b.result["sse_num"]) for a, b in zip(reqs, lreqs))
    llaunches = lbe.launches
    lbe.close()
    del lsrv, lbe
    torch.cuda.empty_cache()
    # the plain per-image path behind the same scheduler, on the same trace
    plain = serve.Server(serve.PlainBackend(max_px, device=dev), 1 << 30, streams=1, max_wave=1)
    preqs = requests()
    pout = serve.run_trace(plain, preqs)
    same = sum(int(a.result["sse_num"]) == int(b.result["sse_num"]) for a, b in zip(reqs, preqs))
    line = {"metric": "serve p99 ms", "value": out["p99_ms"], "unit": "ms", "n_gpus": world, "steps": len(reqs),
            "warmup": 8, "ms_per_step": out["mean_ms"], "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "serving: Poisson arrivals at %g req/s for %g s; image side log-uniform 256-4096 "
                                   "(aspect 0.5-2, pool of 48 images), K uniform 8..256, %s seeds, eps=1e-4, "
                                   "<=100 passes; memory-admitted continuous batching on 2 streams; while at most %d requests "
                                   "wait and no batch wave runs, requests go one at a time through the whole-GPU lane"
                                   % (args.rate, args.duration, SCHEME, SOLO_QUEUE),
                       "requests": len(reqs), "launch_shape": {"cluster": cluster, "split_pixels": split},
                       "pool_bytes": pool_bytes, "l2": "inputs larger than L2 (no flush)"},
            "clocks": {k: clk[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
            "e2e": {"value": out["p99_ms"], "unit": "ms", "h2d_bytes_per_step": int(h2d / max(1, len(reqs))),
                    "d2h_bytes_per_step": int(d2h / max(1, len(reqs)))},
            "gpu_launches": None,
            "p50_ms": out["p50_ms"], "img_per_s": out["img_per_s"], "mpix_per_s": out["mpix_per_s"],
            "waves": waves, "solo_waves": solo_waves,
            "live_server": {"p50_ms": lout["p50_ms"], "p99_ms": lout["p99_ms"], "img_per_s": lout["img_per_s"],
                            "mpix_per_s": lout["mpix_per_s"], "launches": llaunches, "same_sse_requests": lsame,
                            "note": "requests admitted into one running launch (kq_live_*); no whole-GPU lane"},
            "per_image_path": {"p50_ms": pout["p50_ms"], "p99_ms": pout["p99_ms"], "img_per_s": pout["img_per_s"],
                               "same_sse_requests": same}}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_table1(args, rank, world, local) -> None:
    """The Table 1 analogue (Section 3.2): k-means on all N pixels against Weighted
    Sort-Means on the unique colours, both from the same Forgy centres for 20 fixed
    passes; the NDC per pixel per pass and the GPU times (palette + mapping), then a
    Fig. 2-style sweep of the WSM time over K."""
    import numpy as np
    import torch

    from paper_1101_0395_gb300 import kq, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = synth.WORKLOADS["paper_512"]
    img = wl.make(rank)
    n = img.size // 3
    rgb = torch.from_numpy(img.reshape(-1)).to(dev)
    q = kq.Quantizer(n, device=dev)
    pk = torch.zeros(n, dtype=torch.int32, device=dev)
    pw = torch.zeros(n, dtype=torch.int32, device=dev)
    pn = torch.zeros(1, dtype=torch.int32, device=dev)
    ws2 = torch.zeros(kq.kq_workspace_size(n, 256), dtype=torch.uint8, device=dev)
    lab2 = torch.zeros(n, dtype=torch.uint8, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    idx = q.idx[:n]

    def timed(fn, reps=5):
        ts = []
        for r in range(reps + 2):
            flush.fill_(r & 255)
            a, b = torch.cuda.Event(True), torch.cuda.Event(True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            if r >= 2:
                ts.append(a.elapsed_time(b))
        return float(np.median(ts))

    rows = []
    sweep = {}
    for K in (2, 4, 8, 16, 32, 64, 128, 256):
        kq.kq_histogram(rgb, q.keys, q.weights, q.n_unique, q.ws)
        c0 = torch.zeros(3 * K, dtype=torch.float64, device=dev)
        kq.kq_seed(q.keys, q.weights, q.n_unique, K, "FGY", SEED, c0, q.ws)
        c_w, c_k = c0.clone(), c0.clone()
        pal_w = torch.zeros(3 * K, dtype=torch.uint8, device=dev)
        pal_k = torch.zeros(3 * K, dtype=torch.uint8, device=dev)

        def wsm():
            kq.kq_histogram(rgb, q.keys, q.weights, q.n_unique, q.ws)
            c_w.copy_(c0)
            kq.kq_lloyd(q.keys, q.weights, q.n_unique, K, c_w, -1.0, 20, q.labels, pal_w, q.ws, stats=q.stats)
            kq.kq_map(rgb, pal_w, K, idx, q.ws, sse_num=q.sse_num)

        def km():
            kq.kq_pixel_keys(rgb, pk, pw, pn)
            c_k.copy_(c0)
            kq.kq_lloyd(pk, pw, pn, K, c_k, -1.0, 20, lab2, pal_k, ws2, stats=q.stats, flags=kq.LLOYD_DENSE)
            kq.kq_map(rgb, pal_k, K, idx, q.ws, sse_num=q.sse_num)

        t_w = timed(wsm)
        st_w = kq.parse_stats(q.stats)
        nu = int(q.n_unique.item())
        sweep[str(K)] = t_w
        if K >= 32:
            t_k = timed(km, reps=3)
            st_k = kq.parse_stats(q.stats)
            same = bool(torch.equal(c_w, c_k) and torch.equal(pal_w, pal_k))
            rows.append({"K": K, "ndc_wsm_per_pixel_per_pass": st_w["ndc"] / (n * 20.0),
                         "ndc_wsm_per_colour_per_pass": st_w["ndc"] / (nu * 20.0), "ndc_km": st_k["ndc"] / (n * 20.0),
                         "ms_wsm": t_w, "ms_km": t_k, "speedup": t_k / t_w, "same_centres": same})
    # 2:1 subsampling before the unique-colour sampling (Section 2.2): palette from
    # the pixels with even x and y, every pixel mapped; time and MSE beside the full run
    sub = []
    h, w = wl.height, wl.width
    for K in (64, 256):
        c = torch.zeros(3 * K, dtype=torch.float64, device=dev)
        pal = torch.zeros(3 * K, dtype=torch.uint8, device=dev)
        out = {}
        for stride in (1, 2):
            def run():
                kq.kq_histogram_strided(rgb, h, w, stride, q.keys, q.weights, q.n_unique, q.ws)
                kq.kq_seed(q.keys, q.weights, q.n_unique, K, SCHEME, SEED, c, q.ws)
                kq.kq_lloyd(q.keys, q.weights, q.n_unique, K, c, wl.eps, wl.max_iter, q.labels, pal, q.ws,
                            stats=q.stats)
                if stride != 1:
                    kq.kq_histogram(rgb, q.keys, q.weights, q.n_unique, q.ws)
                kq.kq_map(rgb, pal, K, idx, q.ws, sse_num=q.sse_num)

            t = timed(run)
            out[stride] = {"ms": t, "mse": int(q.sse_num.item()) / n, "iters": kq.parse_stats(q.stats)["iters"]}
        sub.append({"K": K, "full": out[1], "sub2": out[2], "mse_ratio": out[2]["mse"] / out[1]["mse"],
                    "speedup": out[1]["ms"] / out[2]["ms"]})
    sp = [r["speedup"] for r in rows]
    line = {"metric": "Table 1 analogue: k-means / WSM time, 20 passes from the same Forgy centres",
            "value": float(np.mean(sp)), "unit": "x", "n_gpus": world, "steps": 5, "warmup": 2,
            "ms_per_step": rows[-1]["ms_wsm"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "paper_512 image 0 (%dx%d, N'=%d), Forgy seeds, 20 fixed passes, times include "
                                   "the histogram (WSM) and the mapping (both)" % (wl.height, wl.width, nu),
                       "l2": "flushed between runs"},
            "rows": rows, "wsm_ms_by_K": sweep, "subsampling_2to1": sub, "gpu_launches": None}
    if rank == 0:
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- extra measurements of the default run
# The headline is the 512 x 512 image; the same JSON line also carries the kernels on
# the 4096 x 4096 image (where the histogram and mapping bandwidth targets apply), a
# size-stratified subset of the batched workload against the plain per-image path at
# the same MSE, and a short serving trace against the plain server.
EXTRA_BATCH = 64            # every 8th image, by size, of the 512-image batch spec
EXTRA_SERVE_POOL = 12       # serving: images the requests pick from
EXTRA_SERVE_RATE = 200.0    # req/s
EXTRA_SERVE_SECONDS = 3.0
EXTRA_OVERLOAD_RATE = 2000.0  # req/s: a short overload, where throughput counts
EXTRA_OVERLOAD_SECONDS = 1.0


def _gen_workload_image(args):
    from paper_1101_0395_gb300 import synth

    name, index = args
    return synth.WORKLOADS[name].make(index)


def extra_inputs():
    """The extras' synthetic inputs, generated on all host cores (spawned workers, so
    that no CUDA state is forked); called after the timed region."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor

    from paper_1101_0395_gb300 import synth

    spec = synth.batch_spec(512)
    order = sorted(range(len(spec.sizes)), key=lambda i: spec.sizes[i][0] * spec.sizes[i][1])
    pick = order[::len(order) // EXTRA_BATCH][:EXTRA_BATCH]
    sub = synth.BatchSpec([spec.sizes[i] for i in pick], [spec.ks[i] for i in pick], [spec.seeds[i] for i in pick])
    pool = synth.batch_spec(EXTRA_SERVE_POOL, side_lo=256, side_hi=4096, seed=4101, k_uniform_range=(8, 256))
    with ProcessPoolExecutor(max_workers=os.cpu_count(), mp_context=mp.get_context("spawn")) as ex:
        big = ex.submit(_gen_workload_image, ("large_4096", 0))
        bf = [ex.submit(_gen_batch_image, (h, w, sd)) for (h, w), sd in zip(sub.sizes, sub.seeds)]
        sf = [ex.submit(_gen_batch_image, (h, w, sd)) for (h, w), sd in zip(pool.sizes, pool.seeds)]
        return big.result(), (sub, [f.result() for f in bf]), (pool, [f.result() for f in sf])


def _median_ms(fn, flush, stream, reps=10, warm=3):
    import torch

    ts = []
    for r in range(reps + warm):
        flush.fill_(r & 255)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        if r >= warm:
            ts.append(a.elapsed_time(b))
    return float(statistics.median(ts))


def extra_large(img, K, dev, fp32_peak, hbm_peak, alu_peak) -> dict:
    """The 4096 x 4096 image: histogram and mapping against HBM, the full search
    against the FP32 peak, seeding and pruned Lloyd times, the whole pipeline."""
    import torch

    from paper_1101_0395_gb300 import kq, synth

    wl = synth.WORKLOADS["large_4096"]
    n = img.size // 3
    q = kq.Quantizer(n, device=dev)
    rgb = torch.from_numpy(img.reshape(-1)).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    c = q.centers[:3 * K]
    pal = q.palette[:3 * K]
    t_hist = _median_ms(lambda: kq.kq_histogram(rgb, q.keys, q.weights, q.n_unique, q.ws), flush, stream)
    nu = int(q.n_unique.item())
    t_seed = _median_ms(lambda: kq.kq_seed(q.keys, q.weights, q.n_unique, K, SCHEME, SEED, c, q.ws), flush, stream,
                        reps=5)
    c0 = c.clone()

    def lloyd(P, flags, eps):
        def f():
            c.copy_(c0)
            kq.kq_lloyd(q.keys, q.weights, q.n_unique, K, c, eps, P, q.labels, pal, q.ws, stats=q.stats, flags=flags)
        return f

    d1 = _median_ms(lloyd(1, kq.LLOYD_DENSE, -1.0), flush, stream, reps=5)
    d5 = _median_ms(lloyd(5, kq.LLOYD_DENSE, -1.0), flush, stream, reps=5)
    t_lloyd = _median_ms(lloyd(wl.max_iter, 0, wl.eps), flush, stream, reps=5)
    st = kq.parse_stats(q.stats)
    t_map = _median_ms(lambda: kq.kq_map(rgb, pal, K, q.idx[:n], q.ws,
                                         sse_num=q.sse_num), flush, stream)
    map_ndc = kq.kq_map_ndc_read(q.ws)
    t_all = _median_ms(lambda: q.quantize(rgb, K, SCHEME, SEED, wl.eps, wl.max_iter), flush, stream, reps=5)
    if kq.kq_status_read(q.ws) != kq.KQ_OK:
        raise RuntimeError("device status after the 4096x4096 runs: %s" % kq.strerror(kq.kq_status_read(q.ws)))
    hist_b, map_b = 3.0 * n + 8.0 * nu, 4.0 * n + 8.0 * nu
    pass_flop = float(FLOP_PER_DIST) * nu * K
    kpp_ops = 5.0 * nu * K
    return {
        "workload": "large_4096: one 4096x4096 synthetic RGB8 image (512 regions plus global ramps), K=%d, %s seeds, "
                    "eps=%g, <=%d passes; L2 flushed before every timed call" % (K, SCHEME, wl.eps, wl.max_iter),
        "n_pixels": n, "n_unique": nu,
        "pipeline": {"ms": t_all, "mpix_per_s": n / (t_all * 1e-3) / 1e6},
        "histogram": {"ms": t_hist, "achieved": hist_b / (t_hist * 1e-3) / 1e9, "unit": "GB/s", "peak": hbm_peak,
                      "frac": hist_b / (t_hist * 1e-3) / 1e9 / hbm_peak,
                      "algorithmic": "3 B per pixel + 8 B per unique colour"},
        "map": {"ms": t_map, "achieved": map_b / (t_map * 1e-3) / 1e9, "unit": "GB/s", "peak": hbm_peak,
                "frac": map_b / (t_map * 1e-3) / 1e9 / hbm_peak, "ndc": map_ndc,
                "ndc_per_colour": map_ndc / max(1, nu),
                "algorithmic": "3 B in + 1 B out per pixel + 8 B per unique colour"},
        "assignment_dense": {"one_pass_ms": d1, "five_pass_ms": d5,
                             "achieved_5_passes": 5 * pass_flop / (d5 * 1e-3) / 1e12, "unit": "TFLOP/s",
                             "peak": fp32_peak, "frac_5_passes": 5 * pass_flop / (d5 * 1e-3) / 1e12 / fp32_peak,
                             "frac_marginal_pass": pass_flop / ((d5 - d1) / 4 * 1e-3) / 1e12 / fp32_peak
                             if d5 > d1 else None,
                             "algorithmic": "%d FLOP per distance x N' x K per pass" % FLOP_PER_DIST},
        "seed_kpp": {"ms": t_seed, "us_per_round": 1e3 * t_seed / K,
                     "achieved": kpp_ops / (t_seed * 1e-3) / 1e12, "unit": "Tops/s", "peak": alu_peak,
                     "frac": kpp_ops / (t_seed * 1e-3) / 1e12 / alu_peak,
                     "algorithmic": "5 integer operations per unique colour per round (distance by dp4a, "
                                    "norm terms, minimum, weighted sum)"},
        "lloyd_pruned": {"ms": t_lloyd, "passes": st["iters"], "ndc_per_colour_per_pass": st["ndc"] / max(1, nu * st["iters"]),
                         "dense_equivalent_gdist_per_s": nu * K * st["iters"] / (t_lloyd * 1e-3) / 1e9},
    }


def extra_batched(sub, imgs, dev) -> dict:
    """The batched form (one persistent launch, autotuned, CUDA graph) against the
    plain per-image path on the same GPU and images, at the same MSE."""
    import numpy as np
    import torch

    from paper_1101_0395_gb300 import kq

    n_px = [im.size // 3 for im in imgs]
    bq = kq.BatchQuantizer(n_px, sub.ks, SCHEME, sub.seeds, 1e-4, 100, device=dev)
    for i, im in enumerate(imgs):
        bq.rgb(i).copy_(torch.from_numpy(im.reshape(-1)))
    torch.cuda.synchronize()
    bq.tune()
    bq.capture()
    stream = torch.cuda.current_stream()
    for _ in range(3):
        bq.replay()
    torch.cuda.synchronize()
    ts = []
    for _ in range(5):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        bq.replay()
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    ms = float(statistics.median(ts))
    res = bq.results()
    if np.any(res["status"] != kq.KQ_OK):
        raise RuntimeError("batch item errors: %s" % np.unique(res["status"]))
    q = kq.Quantizer(max(n_px), device=dev)
    sse_loop = []
    lt = []
    for rep in range(3):
        sse_loop.clear()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for i in range(len(imgs)):
            r = q.quantize(bq.rgb(i), sub.ks[i], SCHEME, sub.seeds[i], 1e-4, 100)
            sse_loop.append(r.sse_num.clone())
        b.record(stream)
        torch.cuda.synchronize()
        if rep:
            lt.append(a.elapsed_time(b))
    loop_ms = float(min(lt))
    sse_b = res["sse_num"].astype(np.int64)
    sse_l = np.array([int(x.item()) for x in sse_loop], dtype=np.int64)
    shape = {"cluster": bq.cfg.cluster, "split_pixels": bq.cfg.split_pixels, "images_on_clusters": bq.n_big}
    del bq
    torch.cuda.empty_cache()
    return {"workload": "%d of the 512 batch images (every 8th by size: %d..%d px), K from {16..256}, %s seeds, "
                        "eps=1e-4, <=100 passes" % (len(imgs), min(n_px), max(n_px), SCHEME),
            "images": len(imgs), "n_pixels": int(sum(n_px)), "launch_shape": shape,
            "batched": {"ms": ms, "img_per_s": len(imgs) / (ms * 1e-3), "mpix_per_s": sum(n_px) / (ms * 1e-3) / 1e6,
                        "mse": float(sse_b.sum() / sum(n_px))},
            "per_image_path": {"ms": loop_ms, "img_per_s": len(imgs) / (loop_ms * 1e-3),
                               "mpix_per_s": sum(n_px) / (loop_ms * 1e-3) / 1e6,
                               "mse": float(sse_l.sum() / sum(n_px))},
            "speedup": loop_ms / ms, "same_sse_images": int((sse_b == sse_l).sum())}


def extra_serving(pool, imgs, dev) -> dict:
    """A short Poisson trace through the server (continuous batching, memory
    admission) and through the plain per-image server, same requests."""
    import torch

    from paper_1101_0395_gb300 import kq, serve, synth

    arrivals = serve.poisson_arrivals(EXTRA_SERVE_RATE, EXTRA_SERVE_SECONDS, 4101)
    u = synth.uniform(4101, 40, 2 * max(1, arrivals.size))
    picks = (u[0::2] * len(imgs)).astype(int)
    ks = 8 + (u[1::2] * 249).astype(int).clip(0, 248)
    h_imgs = [torch.from_numpy(im.reshape(-1)).pin_memory() for im in imgs]
    max_px = max(im.size // 3 for im in imgs)

    def requests(count=None):
        out = []
        for i in range(arrivals.size if count is None else count):
            out.append(serve.Request(rid=i, rgb=h_imgs[int(picks[i])], K=int(ks[i]), scheme=SCHEME, seed=1000 + i,
                                     arrival=float(arrivals[i]) if count is None else 0.0))
        return out

    n_px = [im.size // 3 for im in imgs]
    bq = kq.BatchQuantizer(n_px, [int(k) for k in ks[:len(imgs)]], SCHEME, list(range(len(imgs))), device=dev)
    for i in range(len(imgs)):
        bq.rgb(i).copy_(h_imgs[i])
    bq.tune()
    cluster, split = bq.cfg.cluster, bq.cfg.split_pixels
    del bq
    torch.cuda.empty_cache()
    srv = serve.Server(serve.CudaBackend(cluster, split, device=dev, solo_max_pixels=max_px), 16 << 30, streams=2,
                       max_wave=64, solo_queue=SOLO_QUEUE)
    for r in requests(8):
        srv.submit(r)
    srv.drain()
    srv.finished.clear()
    reqs = requests()
    out = serve.run_trace(srv, reqs)
    waves, solo = srv.waves, srv.backend.solo_waves

    def live_server():
        be = serve.LiveBackend(cluster, split, device=dev, idle_us=20000, capacity=4096)
        return serve.LiveServer(be, 16 << 30, 2 << 30), be

    lsrv, lbe = live_server()
    for r in requests(8):
        lsrv.submit(r)
    lsrv.drain()
    lsrv.finished.clear()
    lreqs = requests()
    lout = serve.run_trace(lsrv, lreqs)
    lsame = sum(int(a.result["sse_num"]) == int(b.result["sse_num"]) for a, b in zip(reqs, lreqs))

    # overload: the same request mix arriving 10x faster, through the wave server,
    # the live server and one offline batch of the same images
    oarr = serve.poisson_arrivals(EXTRA_OVERLOAD_RATE, EXTRA_OVERLOAD_SECONDS, 4102)

    def oreqs():
        return [serve.Request(rid=i, rgb=h_imgs[int(picks[i % len(picks)])], K=int(ks[i % len(ks)]), scheme=SCHEME,
                              seed=1000 + i, arrival=float(oarr[i])) for i in range(oarr.size)]
    wo = serve.run_trace(srv, oreqs())
    lo_reqs = oreqs()
    lo = serve.run_trace(lsrv, lo_reqs)
    llaunches = lbe.launches
    lbe.close()
    del srv, lsrv, lbe
    torch.cuda.empty_cache()
    ob = oreqs()[:256]  # the first 256 requests of the same mix
    bq = kq.BatchQuantizer([r.rgb.numel() // 3 for r in ob], [r.K for r in ob], SCHEME, [r.seed for r in ob],
                           device=dev)
    for i, r in enumerate(ob):
        bq.rgb(i).copy_(r.rgb)
    bq.plan(kq.BatchConfig(cluster, 0, split))
    bq.run()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    bq.run()
    t1.record()
    torch.cuda.synchronize()
    ob_ms = t0.elapsed_time(t1)
    ob_px = sum(r.rgb.numel() // 3 for r in ob)
    del bq
    torch.cuda.empty_cache()
    plain = serve.Server(serve.PlainBackend(max_px, device=dev), 1 << 30, streams=1, max_wave=1)
    for r in requests(4):
        plain.submit(r)
    plain.drain()
    plain.finished.clear()
    preqs = requests()
    pout = serve.run_trace(plain, preqs)
    same = sum(int(a.result["sse_num"]) == int(b.result["sse_num"]) for a, b in zip(reqs, preqs))
    return {"workload": "Poisson arrivals at %g req/s for %g s; image side log-uniform 256-4096 (pool of %d), K uniform "
                        "8..256, %s seeds, eps=1e-4, <=100 passes" % (EXTRA_SERVE_RATE, EXTRA_SERVE_SECONDS, len(imgs),
                                                                     SCHEME),
            "requests": len(reqs),
            "server": {"p50_ms": out["p50_ms"], "p99_ms": out["p99_ms"], "img_per_s": out["img_per_s"],
                       "mpix_per_s": out["mpix_per_s"], "waves": waves, "solo_waves": solo},
            "live_server": {"p50_ms": lout["p50_ms"], "p99_ms": lout["p99_ms"], "img_per_s": lout["img_per_s"],
                            "mpix_per_s": lout["mpix_per_s"], "same_sse_requests": lsame},
            "overload": {"workload": "the same mix at %g req/s for %g s (%d requests)"
                                     % (EXTRA_OVERLOAD_RATE, EXTRA_OVERLOAD_SECONDS, oarr.size),
                         "server": {"p50_ms": wo["p50_ms"], "p99_ms": wo["p99_ms"], "img_per_s": wo["img_per_s"],
                                    "mpix_per_s": wo["mpix_per_s"]},
                         "live_server": {"p50_ms": lo["p50_ms"], "p99_ms": lo["p99_ms"], "img_per_s": lo["img_per_s"],
                                         "mpix_per_s": lo["mpix_per_s"], "launches": llaunches},
                         "offline_batch": {"images": len(ob), "ms": ob_ms, "mpix_per_s": ob_px / ob_ms / 1e3,
                                           "img_per_s": len(ob) / ob_ms * 1e3,
                                           "note": "the first 256 requests as one kq_batch_run, inputs resident"}},
            "plain_server": {"p50_ms": pout["p50_ms"], "p99_ms": pout["p99_ms"], "img_per_s": pout["img_per_s"],
                             "mpix_per_s": pout["mpix_per_s"]},
            "same_sse_requests": same}


def run_reference(args, rank, world) -> None:
    """The reference arm: the FP64 CPU oracle on the same workload."""
    if rank != 0:
        return
    import oracle  # noqa: F401
    from paper_1101_0395_gb300 import synth

    if args.workload == "serving":
        print(json.dumps({"impl": "reference", "unavailable": "the oracle is a batch program; it has no request "
                                                              "loop to time under arrivals"}), flush=True)
        return
    if args.workload == "batched":
        spec = synth.batch_spec(args.count)
        order = sorted(range(len(spec.sizes)), key=lambda i: spec.sizes[i][0] * spec.sizes[i][1])
        pick = order[::max(1, len(order) // 8)]
        sub = synth.BatchSpec([spec.sizes[i] for i in pick], [spec.ks[i] for i in pick],
                              [spec.seeds[i] for i in pick])
        imgs = batch_images(sub)
        mean_px = sum(h * w for h, w in spec.sizes) / len(spec.sizes)
        times = []
        for _ in range(max(1, args.steps)):
            cb = batched_cpu_baseline(imgs, sub, budget_s=1e9)
            times.append(cb)
        v = sum(c["value"] for c in times) / len(times)
        v = v * (sum(im.size // 3 for im in imgs) / len(imgs)) / mean_px
        line = {"metric": "batched img/s", "value": v, "unit": "img/s", "n_gpus": args.gpus, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 / v, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
                "config": batched_config(spec, [h * w for h, w in spec.sizes]),
                "cpu_baseline": {"value": v, "unit": "img/s", "kind": "oracle", "cores": 1,
                                 "sample": "%d size-stratified images of the batch per step, scaled to the batch's "
                                           "mean image size" % len(imgs)},
                "e2e": {"value": v, "unit": "img/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    wl = synth.WORKLOADS[args.workload]
    img = wl.make(0)
    K = args.K
    n = img.size // 3
    import oracle as orc

    for _ in range(max(0, args.warmup)):
        orc.quantize(img, K, SCHEME, SEED, wl.eps, wl.max_iter)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        out = orc.quantize(img, K, SCHEME, SEED, wl.eps, wl.max_iter)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = n / (ms * 1e-3) / 1e6
    line = {"metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": workload_config(wl, img, K, out["keys"].size, out["iters"]),
            "cpu_baseline": {"value": value, "unit": "Mpix/s", "kind": "oracle", "cores": 1,
                             "sample": "whole quantizations of the %dx%d image, one per step" % img.shape[:2]},
            "e2e": {"value": value, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gpu(args, rank, world, local) -> None:
    import numpy as np
    import torch

    from paper_1101_0395_gb300 import kq, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = synth.WORKLOADS[args.workload]
    K = args.K
    img = wl.make(rank)
    n = img.size // 3
    q = kq.Quantizer(n, device=dev)
    rgb = torch.from_numpy(img.reshape(-1)).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def stage_calls(src, quant):
        kq.kq_histogram(src, quant.keys, quant.weights, quant.n_unique, quant.ws)
        yield
        c = quant.centers[:3 * K]
        kq.kq_seed(quant.keys, quant.weights, quant.n_unique, K, SCHEME, SEED, c, quant.ws, conv_eps=wl.eps,
                   max_iter=wl.max_iter)
        yield
        pal = quant.palette[:3 * K]
        kq.kq_lloyd(quant.keys, quant.weights, quant.n_unique, K, c, wl.eps, wl.max_iter, quant.labels, pal,
                    quant.ws, stats=quant.stats)
        yield
        kq.kq_map(src, pal, K, quant.idx[:n], quant.ws,
                  sse_num=quant.sse_num)
        yield

    launches_per_step = (kq.launches("kq_histogram", n) + kq.launches("kq_seed", n, SCHEME, K)
                         + kq.launches("kq_lloyd") + kq.launches("kq_map", n))

    for _ in range(max(3, args.warmup)):
        for _ in stage_calls(rgb, q):
            pass
    torch.cuda.synchronize()
    st = kq.parse_stats(q.stats)
    n_unique = int(q.n_unique.item())
    status = kq.kq_status_read(q.ws)
    if status != kq.KQ_OK:
        raise RuntimeError("device status after warm-up: %s" % kq.strerror(status))

    steps = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(steps)]
    props = torch.cuda.get_device_properties(dev)
    gpu_id = "GPU-%s" % props.uuid if getattr(props, "uuid", None) else str(local)
    clocks = ClockSampler(gpu_id)
    clocks.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for s in range(steps):
        flush.fill_(s & 255)
        e = ev[s]
        e[0].record(stream)
        for j, _ in enumerate(stage_calls(rgb, q)):
            e[j + 1].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    step_ms = [e[0].elapsed_time(e[4]) for e in ev]
    stage_ms = [[e[j].elapsed_time(e[j + 1]) for e in ev] for j in range(4)]
    ms_local = sum(step_ms) / steps
    ms_max = reduce_max(ms_local, world)
    value = aggregate(n, world, ms_max)
    stage_mean = [sum(x) / steps for x in stage_ms]

    # ---- end to end through the public API with host buffers
    h_rgb = torch.from_numpy(img.reshape(-1).copy()).pin_memory()
    h_idx = torch.empty(n, dtype=torch.uint8).pin_memory()
    h_pal = torch.empty(3 * K, dtype=torch.uint8).pin_memory()
    h_stats = torch.empty(64, dtype=torch.uint8).pin_memory()
    d_rgb = torch.empty(3 * n, dtype=torch.uint8, device=dev)
    e2e_steps = max(10, min(steps, 100))
    e2e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(e2e_steps)]
    for s in range(e2e_steps + 3):
        if s >= 3:
            flush.fill_(s & 255)
            e2e_ev[s - 3][0].record(stream)
        d_rgb.copy_(h_rgb, non_blocking=True)
        res = q.quantize(d_rgb, K, SCHEME, SEED, wl.eps, wl.max_iter)
        h_idx.copy_(res.idx, non_blocking=True)
        h_pal.copy_(res.palette.view(-1), non_blocking=True)
        h_stats.copy_(res.stats, non_blocking=True)
        if s >= 3:
            e2e_ev[s - 3][1].record(stream)
    torch.cuda.synchronize()
    e2e_ms = reduce_max(sum(a.elapsed_time(b) for a, b in e2e_ev) / e2e_steps, world)
    if not np.array_equal(h_idx.numpy(), q.idx[:n].cpu().numpy()):
        raise RuntimeError("end-to-end result differs from the device-resident run")

    # ---- roofline of the dominant kernel
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz") or 2070.0)
    fp32_peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12  # TFLOP/s
    alu_peak = fp32_peak / 2.0  # one 32-bit integer operation per lane per clock
    hbm_peak = float(peaks.get("hbm_gbs") or 6800.0)
    hbm_source = "MEASURED_PEAKS hbm_gbs" if peaks.get("hbm_gbs") else "fallback 6800 GB/s (MEASURED_PEAKS.json absent)"
    names = ["kq_histogram", "kq_seed", "kq_lloyd", "kq_map"]
    dom = max(range(4), key=lambda j: stage_mean[j])
    lloyd_s = stage_mean[2] * 1e-3
    gdist_actual = st["ndc"] / lloyd_s / 1e9
    gdist_dense = n_unique * K * st["iters"] / lloyd_s / 1e9
    if dom == 2:
        achieved = st["ndc"] * FLOP_PER_DIST / lloyd_s / 1e12
        traffic, tsrc = profile_traffic("lloyd_kernel_%s_k%d.txt" % (wl.name.replace("_", ""), K))
        roof = {"kernel": "lloyd_kernel (kq_lloyd: one persistent launch, all passes)", "bound": "alu",
                "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                "traffic": traffic, "traffic_source": tsrc,
                "peak_source": "derived: %d SMs x 128 FP32 lanes x 2 FLOP x %.0f MHz (max SM clock, measured)"
                               % (props.multi_processor_count, sm_max),
                "algorithmic": "%d FLOP per distance x NDC %d" % (FLOP_PER_DIST, st["ndc"])}
    elif dom == 1:
        # k-means++ in one thread-block cluster of 16 CTAs: K dependent rounds, each
        # refreshing the exact integer D^2 of every unique colour (5 integer operations:
        # dp4a distance, two norm terms, minimum, weighted sum) and drawing the next
        # centre through two cross-CTA exchanges (every warp's total pushed to every CTA,
        # then the sampled key pushed back by the CTA holding it).  The colours live in
        # registers, so DRAM is idle; the exchanges' latency sets the round time.
        ops = 5.0 * n_unique * K
        achieved = ops / (stage_mean[1] * 1e-3) / 1e12
        cl = 16
        traffic, tsrc = profile_traffic("seed_far_cluster_%s_k%d.txt" % (wl.name.replace("_", ""), K))
        roof = {"kernel": "seed_far_cluster (kq_seed, k-means++: one 16-CTA cluster, st.async/mbarrier exchanges)",
                "bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "Tops/s",
                "frac": achieved / alu_peak, "traffic": traffic, "traffic_source": tsrc,
                "peak_source": "derived: %d SMs x 128 lanes x 1 op x %.0f MHz (max SM clock, measured)"
                               % (props.multi_processor_count, sm_max),
                "algorithmic": "5 integer ops per unique colour per round x %d rounds" % K,
                "frac_of_cluster_sms": achieved / (alu_peak * cl / props.multi_processor_count),
                "latency": {"us_per_round": 1e3 * stage_mean[1] / K, "rounds": K,
                            "exchanges_per_round": 2,
                            "note": "latency-bound: per round one push of every warp total to every CTA, one "
                                    "push of the sampled key; the cluster's 16 SMs idle between them"}}
    else:
        byts = (3.0 * n + 8.0 * n_unique) if dom == 0 else (4.0 * n + 8.0 * n_unique)
        achieved = byts / (stage_mean[dom] * 1e-3) / 1e9
        roof = {"kernel": names[dom], "bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": None, "peak_source": hbm_source,
                "algorithmic": "pixels 3 B in (+1 B out) + 8 B per unique colour"}

    # ---- the other kernels against their own rooflines (after the timed region)
    def ev_ms(fn, reps=10):
        ts = []
        for r in range(reps + 3):
            flush.fill_(r & 255)
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            fn()
            t1.record(stream)
            torch.cuda.synchronize()
            if r >= 3:
                ts.append(t0.elapsed_time(t1))
        return float(np.median(ts))

    c_seed = q.centers[:3 * K]
    kq.kq_seed(q.keys, q.weights, q.n_unique, K, SCHEME, SEED, c_seed, q.ws, conv_eps=wl.eps, max_iter=wl.max_iter)
    c0 = c_seed.clone()

    def dense(P):
        def f():
            c_seed.copy_(c0)
            kq.kq_lloyd(q.keys, q.weights, q.n_unique, K, c_seed, -1.0, P, q.labels, q.palette[:3 * K], q.ws,
                        stats=q.stats, flags=kq.LLOYD_DENSE)
        return f

    d1, d5 = ev_ms(dense(1)), ev_ms(dense(5))
    pass_flop = float(FLOP_PER_DIST) * n_unique * K
    marg = (d5 - d1) / 4.0
    hist_b, map_b = 3.0 * n + 8.0 * n_unique, 4.0 * n + 8.0 * n_unique
    kernels = {
        "assignment_dense": {
            "kernel": "lloyd_kernel with pruning off (full search of all K centres), K=%d, N'=%d" % (K, n_unique),
            "bound": "fp32", "peak": fp32_peak, "unit": "TFLOP/s",
            "one_pass_ms": d1, "five_pass_ms": d5, "marginal_pass_ms": marg,
            "achieved_5_passes": 5 * pass_flop / (d5 * 1e-3) / 1e12,
            "frac_5_passes": 5 * pass_flop / (d5 * 1e-3) / 1e12 / fp32_peak,
            "achieved_marginal_pass": pass_flop / (marg * 1e-3) / 1e12 if marg > 0 else None,
            "frac_marginal_pass": pass_flop / (marg * 1e-3) / 1e12 / fp32_peak if marg > 0 else None,
            "algorithmic": "%d FLOP per distance x N' x K per pass; the marginal pass is (5 passes - 1 pass) / 4, "
                           "which leaves out the launch and the one-time set-up" % FLOP_PER_DIST},
        "histogram": {"bound": "hbm", "achieved": hist_b / (stage_mean[0] * 1e-3) / 1e9, "peak": hbm_peak,
                      "unit": "GB/s", "frac": hist_b / (stage_mean[0] * 1e-3) / 1e9 / hbm_peak,
                      "algorithmic": "3 B per pixel + 8 B per unique colour"},
        "map": {"bound": "hbm", "achieved": map_b / (stage_mean[3] * 1e-3) / 1e9, "peak": hbm_peak,
                "unit": "GB/s", "frac": map_b / (stage_mean[3] * 1e-3) / 1e9 / hbm_peak,
                "algorithmic": "3 B in + 1 B out per pixel + 8 B per unique colour (palette table included)"},
    }

    line = {"metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": world, "steps": steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(wl, img, K, n_unique, st["iters"]),
            "clocks": {k: clk[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
            "e2e": {"value": aggregate(n, world, e2e_ms), "unit": "Mpix/s", "h2d_bytes_per_step": 3 * n,
                    "d2h_bytes_per_step": n + 3 * K + 64},
            "gpu_launches": launches_per_step * steps,
            "roofline": roof,
            "gdist_evals_per_s": {"actual": gdist_actual, "dense_equivalent": gdist_dense, "unit": "G/s",
                                  "ndc_per_colour_per_pass": st["ndc"] / max(1, n_unique * st["iters"])},
            "stages_ms": dict(zip(names, stage_mean)),
            "kernels": kernels,
            "wall_s_timed_region": wall, "clock_samples": clk["samples"]}
    if rank == 0 and world == 1 and args.workload == WORKLOAD and not args.no_extras:
        big, (sub, bimgs), (pool, simgs) = extra_inputs()
        line["extras"] = {"large_4096": extra_large(big, K, dev, fp32_peak, hbm_peak, alu_peak),
                          "batched_subset": extra_batched(sub, bimgs, dev),
                          "serving_short": extra_serving(pool, simgs, dev),
                          "peaks": {"hbm_gbs": hbm_peak, "hbm_source": hbm_source, "fp32_tflops": fp32_peak,
                                    "alu_tops": alu_peak}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(img, K, wl.eps, wl.max_iter)
    if rank == 0:
        print(json.dumps(line), flush=True)


def main(argv=None) -> None:
    args = parse_args(argv)
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        backend = "nccl" if args.impl == "kq" else "gloo"
        if backend == "nccl":
            import torch

            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        elif args.workload == "batched":
            run_batched(args, rank, world, local)
        elif args.workload == "serving":
            run_serving(args, rank, world, local)
        elif args.workload == "table1":
            run_table1(args, rank, world, local)
        else:
            run_gpu(args, rank, world, local)
    finally:
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()


if __name__ == "__main__":
    main()
