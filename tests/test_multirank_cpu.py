"""The N > 1 path of bench.py on CPU: replicas on world_size 2 gloo ranks.

A single grid does not shard without an exchange (every z line spans the
grid), so N GPUs run N independent replicas: the only cross-rank steps are
the barrier and the maximum of the ranks' times, and the job's rate counts
every rank's units.  These tests run that host logic on two gloo processes,
and check that the reference arm leaves ranks other than 0 without work.
The batched form shards by member instead (paper_2110_13368_gb300.shard):
every rank computes the same placement from the members' sizes, with no
exchange.
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


class _Member:
    def __init__(self, nx, ny, nz, n_sub, precision=64):
        self.nx, self.ny, self.nz, self.n_sub, self.precision = nx, ny, nz, n_sub, precision


def _members(seed=0, n=256):
    # sizes as the batched workload draws them: edges 32..96, 1..4 substrates
    import numpy as np
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        nx, ny, nz = (int(v) for v in rng.integers(32, 97, size=3))
        out.append(_Member(nx, ny, nz, int(rng.integers(1, 5))))
    return out


def test_lpt_partition_is_complete_disjoint_and_within_graham_bound():
    from paper_2110_13368_gb300 import shard
    ms = _members()
    costs = [shard.member_cost(m.nx, m.ny, m.nz, m.n_sub) for m in ms]
    for n_ranks in (1, 2, 3, 8):
        parts = shard.lpt_partition(costs, n_ranks)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(ms)))
        loads = [sum(costs[i] for i in p) for p in parts]
        lower = max(sum(costs) / n_ranks, max(costs))   # no placement beats this
        assert max(loads) <= 4.0 / 3.0 * lower
    # one rank takes everything; more ranks than members leave some empty
    assert shard.lpt_partition([5.0, 1.0], 1) == [[0, 1]]
    assert shard.lpt_partition([5.0, 1.0], 3) == [[0], [1], []]
    with pytest.raises(ValueError):
        shard.lpt_partition([1.0], 0)


def _shard_rank_main(rank, world, port, out):
    import torch.distributed as dist
    from paper_2110_13368_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = _members()
        mine = shard.problems_for_rank(ms, rank, world)
        ids = [ms.index(m) for m in mine]
        gathered = [None] * world
        dist.all_gather_object(gathered, ids)     # test only: the placement needs no exchange
        out.put((rank, gathered))
    finally:
        dist.destroy_process_group()


def test_ranks_place_the_batch_alike_without_exchange():
    """Each of two gloo ranks computes its own share of the 256 members from
    their sizes alone; gathered afterwards, the shares are disjoint, cover
    every member, and every rank saw the same placement."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    g0, g1 = res[0][1], res[1][1]
    assert g0 == g1
    assert not set(g0[0]) & set(g0[1])
    assert sorted(g0[0] + g0[1]) == list(range(256))
