"""The benchmark's multi-rank logic on CPU with gloo, world size 2: per-rank problems
differ (weak scaling over gate blocks), the job time is the slowest rank's, the job
throughput counts every rank's transforms, and the reference arm runs on rank 0 only."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = bench._workload("small", rank)
        ms = [100.0 + 50.0 * rank, 7.0 - rank]
        got = bench.max_over_ranks(ms, "cpu", world)
        q.put((rank, w.seed, got, bench.job_throughput(world, w.n_ranges, w.n_ipp, got[0]), bench._dist()))
    finally:
        dist.destroy_process_group()


def test_two_ranks_weak_scaling_and_max_timing():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, g0, v0, d0), (r1, s1, g1, v1, d1) = res
    assert s0 != s1                                   # independent gate blocks per rank
    assert g0 == g1 == [150.0, 7.0]                   # slowest rank's time, element-wise
    assert v0 == v1 == pytest.approx(2 * 64 * 100 / 0.150)
    assert d0 == (2, 0, 0) and d1 == (2, 1, 1)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    class A:
        workload, n_ranges, n_ipp = "small", None, None

    assert bench.run_reference(A()) == 0              # returns at once, prints nothing
