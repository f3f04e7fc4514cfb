"""Host-side logic of bench.py on CPU: the max-over-ranks timing reduction and
the whole-job aggregate, exercised with two gloo ranks (no GPU)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, loc = bench.dist_env()
    assert (r, w, loc) == (rank, world, rank)
    bench.barrier(world)
    slowest = bench.reduce_max(10.0 + rank, world)   # rank 1 is the slower one
    out[rank] = bench.aggregate(1000, world, slowest)
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    # 2 ranks x 1000 px per step / 11 ms = 0.1818 Mpix/s on both ranks
    assert out[0] == out[1] == pytest.approx(2000 / 11e-3 / 1e6)


def test_single_rank_defaults():
    args = bench.parse_args([])
    assert args.gpus == 1 and args.warmup >= 3 and args.impl == "kq" and args.K == 256
    assert bench.reduce_max(3.5, 1) == 3.5
    assert bench.aggregate(262144, 1, 2.0) == pytest.approx(131.072)
