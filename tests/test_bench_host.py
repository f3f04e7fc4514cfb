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


def test_profile_traffic_follows_the_source_hash(tmp_path, monkeypatch):
    """roofline.traffic comes from a committed ncu summary only while the kernel's
    source still has the hash recorded there."""
    import hashlib

    src = tmp_path / "k.cu"
    src.write_text("__global__ void k() {}\n")
    (tmp_path / "profiles").mkdir()
    digest = hashlib.sha256(src.read_bytes()).hexdigest()
    (tmp_path / "profiles" / "k.txt").write_text(
        "# summary\nsource_sha256: %s  (k.cu)\ntraffic_bytes_per_launch: 123456\n" % digest)
    (tmp_path / "profiles" / "nolines.txt").write_text("# nothing recorded\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    traffic, why = bench.profile_traffic("k.txt")
    assert traffic == 123456 and "unchanged" in why
    src.write_text("__global__ void k() { }\n")  # the kernel changed
    traffic, why = bench.profile_traffic("k.txt")
    assert traffic is None and "changed" in why
    assert bench.profile_traffic("absent.txt")[0] is None
    assert bench.profile_traffic("nolines.txt")[0] is None


def test_committed_profiles_name_existing_sources():
    """Every committed summary that records a traffic figure names a source file
    of the repository and gives an integer byte count."""
    import glob

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    seen = 0
    for path in glob.glob(os.path.join(root, "profiles", "*.txt")):
        lines = open(path).read().splitlines()
        sha = [ln for ln in lines if ln.startswith("source_sha256:")]
        tr = [ln for ln in lines if ln.startswith("traffic_bytes_per_launch:")]
        assert len(sha) == len(tr) <= 1, path
        if sha:
            seen += 1
            assert os.path.exists(os.path.join(root, sha[0].split()[2].strip("()"))), path
            assert int(tr[0].split()[1]) > 0
    assert seen >= 4
