"""The multi-rank logic of bench.py on CPU (gloo, world size 2).

The path does not shard: under torchrun every rank solves its own instance
(replicas), the job's time is the slowest rank's (a MAX all-reduce) and its
throughput counts the units of all ranks; the reference arm runs on rank 0
only.  These tests run that logic with the gloo backend on 127.0.0.1."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method="env://")
    try:
        assert bench.rank_env() == (world, rank, rank)
        dist.barrier()
        local_ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
        ms = bench.job_ms(local_ms, world, "cpu")
        out.put((rank, ms, bench.job_throughput(3, world, ms)))
    finally:
        dist.destroy_process_group()


def test_job_time_is_the_slowest_rank_and_throughput_counts_all_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(out.get(timeout=10) for _ in range(2))
    for rank, ms, thr in got:
        assert ms == 150.0
        assert thr == pytest.approx(2 * 3 / 0.150)


def test_single_rank_needs_no_process_group(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.rank_env() == (1, 0, 0)
    assert bench.job_ms(42.0, 1, "cpu") == 42.0
    assert bench.job_throughput(5, 1, 1000.0) == pytest.approx(5.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    class Args:
        workload = "n65536_d64"
        steps = 1
        warmup = 0

    assert bench.run_reference(Args()) is None
    assert capsys.readouterr().out == ""
