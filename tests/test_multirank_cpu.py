"""The N > 1 path of bench.py on CPU: replicas on world_size 2 gloo ranks.

A single grid does not shard without an exchange (every z line spans the
grid), so N GPUs run N independent replicas: the only cross-rank steps are
the barrier and the maximum of the ranks' times, and the job's rate counts
every rank's units.  These tests run that host logic on two gloo processes,
and check that the reference arm leaves ranks other than 0 without work.
"""
import os
import socket

import pytest

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seconds = 1.0 + 0.5 * rank            # rank 1 is the slow one
        job = bench.max_over_ranks(seconds, world)
        rate = bench.job_rate(300.0, world, job)
        dist.barrier()
        out.put((rank, job, rate))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_on_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks see the slower rank's time, and the rate counts both ranks' units
    assert [r[1] for r in res] == [1.5, 1.5]
    assert [r[2] for r in res] == [400.0, 400.0]


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(2.5, 1) == 2.5
    assert bench.job_rate(10.0, 1, 2.0) == 5.0


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    args = bench.parse()
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
