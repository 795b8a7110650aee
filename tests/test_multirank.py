"""The N > 1 benchmark path on CPU: two gloo ranks (no GPU).

The IG path shards into independent perspectives, so ranks run replicas
with no data-path collective; the only exchange is the max of the per-rank
times.  These tests run that exchange, the whole-job throughput and the
rank-0-only reference arm as two real processes.
"""

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        mine = [12.5, 40.0][rank]                         # per-rank timed region, ms
        slowest = bench.max_over_ranks(mine, dist)
        value = bench.job_throughput(1024 * 10, world, slowest)
        w = bench.build_workload("exact64", rank)         # replicas draw their own batch
        out.put((rank, slowest, value, int(w.grid.astype("int64").sum())))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time_and_sum_the_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [40.0, 40.0]                 # both ranks see the slowest rank's time
    assert got[0][2] == got[1][2] == pytest.approx(2 * 10240 / 0.040)
    assert got[0][3] != got[1][3]                              # different scenes per rank


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(7.0, None) == 7.0
    assert bench.job_throughput(100, 1, 50.0) == pytest.approx(2000.0)


def test_reference_arm_runs_on_rank_zero_only(capsys, monkeypatch):
    class Args:
        workload, steps, warmup, gpus = "exact64", 1, 0, 2
    monkeypatch.setenv("RANK", "1")
    bench.run_reference(Args())                                # rank 1: returns without work or output
    assert capsys.readouterr().out == ""
