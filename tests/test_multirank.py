"""The multi-rank logic on CPU with gloo, world size 2 (not run on several GPUs here: every
GPU call of this project has one GPU).

* weak scaling: per-rank problems differ, the job time is the slowest rank's, the job
  throughput counts every rank's transforms, the reference arm runs on rank 0 only;
* strong scaling (one workload split by gates): contiguous gate blocks, each rank's echo
  sub-span covers exactly the samples its gates read, and the gathered blocks equal the
  single-rank [n_ranges][nfft] layout;
* ``--gpus N`` against the launcher's world size.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_2311_18737_gb300 import shard


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


def test_gate_blocks_are_contiguous_and_balanced():
    for n, world in [(1000, 1), (1000, 2), (1000, 3), (1000, 8), (7, 8), (152, 4)]:
        b = shard.gate_blocks(n, world)
        assert len(b) == world
        assert b[0][0] == 0 and sum(c for _, c in b) == n
        for (f0, c0), (f1, _) in zip(b, b[1:]):
            assert f1 == f0 + c0
        cs = [c for _, c in b]
        assert max(cs) - min(cs) <= 1 and cs == sorted(cs, reverse=True)


@pytest.mark.parametrize("start,step,code_len", [(0, 25, 16384), (3, 25, 1024), (5, 7, 700), (0, 1, 8)])
def test_echo_span_covers_exactly_the_block_windows(start, step, code_len):
    n_ranges = 37
    full_stride = (start + (n_ranges - 1) * step + code_len + 127) // 128 * 128
    for first, count in shard.gate_blocks(n_ranges, 3):
        sp = shard.echo_span(first, count, start, step, code_len)
        assert sp["s0"] % 4 == 0 and sp["echo_stride"] % 4 == 0 and 0 <= sp["range_start"] < 4
        assert sp["s0"] + sp["echo_stride"] <= full_stride          # inside the original row
        s_first = start + first * step
        assert sp["s0"] + sp["range_start"] == s_first
        # the block's windows inside the sub-row, relative start + (count-1) step + L <= stride
        assert sp["range_start"] + (count - 1) * step + code_len <= sp["echo_stride"]
        assert sp["s1"] == s_first + (count - 1) * step + code_len
        assert sp["echo_stride"] - (sp["s1"] - sp["s0"]) < 4         # no more than the rounding


def _gather_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n_ranges, nfft = 37, 16
        blocks = shard.gate_blocks(n_ranges, world)
        first, count = blocks[rank]
        # fake per-gate payload: value = 1000 * global gate + bin
        local = (1000.0 * torch.arange(first, first + count, dtype=torch.float64)[:, None]
                 + torch.arange(nfft, dtype=torch.float64)[None, :])
        got = shard.gather_gate_blocks(local, blocks, rank, world)
        q.put((rank, None if got is None else got.numpy()))
    finally:
        dist.destroy_process_group()


def test_two_ranks_strong_scaling_gather_equals_single_rank_layout():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gather_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[1] is None
    want = 1000.0 * np.arange(37)[:, None] + np.arange(16)[None, :]
    np.testing.assert_array_equal(res[0], want)


def test_strong_scaling_throughput_counts_the_one_workload():
    assert bench.job_throughput(4, 1000, 100, 1000.0, strong=True) == pytest.approx(1000 * 100)
    assert bench.job_throughput(4, 1000, 100, 1000.0) == pytest.approx(4 * 1000 * 100)


@pytest.mark.parametrize("gpus,world,launched,action", [
    (1, 1, False, "run"), (8, 8, True, "run"), (2, 1, False, "relaunch"), (8, 1, False, "relaunch"),
    (2, 1, True, "error"), (4, 2, True, "error"), (1, 2, True, "error"), (0, 1, False, "error")])
def test_gpus_flag_against_world_size(gpus, world, launched, action):
    assert bench.world_check(gpus, world, launched) == action
