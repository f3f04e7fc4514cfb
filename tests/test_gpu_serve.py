"""Serving on the GPU: requests admitted by device memory and batched
continuously give, request by request, exactly the result they give alone;
mapping and histogram are checked against the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1101_0395_gb300 import kq, serve, synth
from tests.gpu_helpers import require_cuda

pytestmark = pytest.mark.gpu

SIZES = [(64, 64, 16, "KPP"), (300, 200, 128, "KPP"), (90, 120, 32, "MMX"), (256, 256, 256, "KPP"),
         (40, 30, 8, "VAR"), (180, 240, 64, "DEN"), (128, 96, 200, "KPP"), (20, 20, 12, "FGY"),
         (220, 160, 48, "SFF"), (140, 150, 100, "MMX")]


def _requests():
    out = []
    for i, (h, w, K, s) in enumerate(SIZES):
        img = synth.batch_image(h, w, 9100 + i)
        out.append(serve.Request(rid=i, rgb=img.reshape(-1), K=K, scheme=s, seed=31 + i, arrival=0.0004 * i))
    return out


def _fields(r):
    return (r.idx.tobytes(), r.palette.tobytes(), r.centers.tobytes(),
            tuple(r.result[f].tobytes() for f in ("status", "n_unique", "lloyd", "sse_num")))


def test_same_result_alone_and_in_the_mix():
    require_cuda()
    C = kq.kq_batch_max_cluster()
    backend = serve.CudaBackend(cluster=min(C, 4), split_pixels=30000)
    one = max(serve.request_layout(h * w, K, kq.kq_batch_scratch_bytes)[1] for h, w, K, _ in SIZES)
    pool = 3 * one  # memory admits about three requests at a time
    srv = serve.Server(backend, pool, streams=2, max_wave=3)
    mix = _requests()
    stats = serve.run_trace(srv, mix)
    assert stats["requests"] == len(SIZES)
    assert srv.arena.peak <= pool and srv.waves >= 4 and srv.max_running == 2
    alone_srv = serve.Server(serve.CudaBackend(cluster=min(C, 4), split_pixels=30000), one, streams=1, max_wave=1)
    for r in mix:
        a = serve.Request(rid=r.rid, rgb=r.rgb, K=r.K, scheme=r.scheme, seed=r.seed)
        alone_srv.submit(a)
        alone_srv.drain()
        assert a.result["status"] == kq.KQ_OK and r.result["status"] == kq.KQ_OK
        assert _fields(a) == _fields(r), r.rid
    # the served results themselves, against the oracle
    for r in mix[:4]:
        img = r.rgb.reshape(-1, 3)
        keys, _ = oracle.histogram(img)
        assert r.result["n_unique"] == keys.size
        oidx, osse = oracle.map_pixels(img, r.palette)
        assert np.array_equal(r.idx, oidx) and r.result["sse_num"] == osse


def test_lone_requests_take_the_whole_gpu_and_agree_within_tolerance():
    """With solo mode a request that finds the device idle runs through the four
    single-image calls on the whole GPU; in a busy mix it runs in a batch wave.
    Both are the same method: the final MSE agrees within 1e-5 relative, and when
    the stop test fires at the same pass the palettes are equal and the centres
    agree within 1e-3."""
    require_cuda()
    C = kq.kq_batch_max_cluster()
    max_px = max(h * w for h, w, _, _ in SIZES)
    one = max(serve.request_layout(h * w, K, kq.kq_batch_scratch_bytes)[1] for h, w, K, _ in SIZES)
    srv = serve.Server(serve.CudaBackend(min(C, 4), 30000, solo_max_pixels=max_px), 4 * one, streams=2,
                       max_wave=4)
    mix = _requests()
    for r in mix:
        r.arrival = 0.0
    serve.run_trace(srv, mix)
    alone_be = serve.CudaBackend(min(C, 4), 30000, solo_max_pixels=max_px)
    alone_srv = serve.Server(alone_be, one, streams=1, max_wave=1)
    for r in mix:
        a = serve.Request(rid=r.rid, rgb=r.rgb, K=r.K, scheme=r.scheme, seed=r.seed)
        alone_srv.submit(a)
        alone_srv.drain()
        assert a.result["status"] == kq.KQ_OK and r.result["status"] == kq.KQ_OK
        assert a.result["n_unique"] == r.result["n_unique"]
        sa, sm = int(a.result["sse_num"]), int(r.result["sse_num"])
        assert abs(sa - sm) <= 1e-5 * max(sa, 1)
        if a.result["lloyd"]["iters"] == r.result["lloyd"]["iters"]:
            assert np.array_equal(a.palette, r.palette)
            assert np.max(np.abs(a.centers - r.centers)) <= 1e-3
    assert alone_be.solo_waves == len(mix)


def test_live_server_same_result_as_alone():
    """Requests admitted into a running launch (LiveServer) give exactly the
    results they give alone, with memory admitting a few at a time and a
    four-slot queue ring."""
    require_cuda()
    C = kq.kq_batch_max_cluster()
    be = serve.LiveBackend(cluster=min(C, 4), split_pixels=30000, idle_us=5000, capacity=4)
    lay = [serve.live_layout(h * w, K, kq.kq_batch_scratch_bytes, False) for h, w, K, _ in SIZES]
    srv = serve.LiveServer(be, pool_bytes=3 * max(x[3] for x in lay), host_bytes=3 * max(x[1] for x in lay))
    mix = _requests()
    stats = serve.run_trace(srv, mix)
    be.close()
    # memory bounds what is in flight (small requests pack more densely than the largest)
    assert stats["requests"] == len(SIZES) and srv.max_inflight >= 2
    assert srv.host_arena.peak <= srv.host_arena.size and srv.dev_arena.peak <= srv.dev_arena.size
    assert srv.host_arena.in_use == 0 and srv.dev_arena.in_use == 0
    one = max(serve.request_layout(h * w, K, kq.kq_batch_scratch_bytes)[1] for h, w, K, _ in SIZES)
    alone_srv = serve.Server(serve.CudaBackend(cluster=min(C, 4), split_pixels=30000), one, streams=1, max_wave=1)
    for r in mix:
        a = serve.Request(rid=r.rid, rgb=r.rgb, K=r.K, scheme=r.scheme, seed=r.seed)
        alone_srv.submit(a)
        alone_srv.drain()
        assert r.result["status"] == kq.KQ_OK
        assert _fields(a) == _fields(r), r.rid
