"""Host side of the z-slab decomposition (paper_2110_13368_gb300.slabs and
bfvm_create_slab's argument checks), without a GPU: the layer partition,
the cell-to-slab assignment, and the exchange between the three calls of a
slab step on two gloo ranks."""
import os
import socket

import numpy as np
import pytest

from paper_2110_13368_gb300 import slabs


def test_partition_covers_the_layers_in_nearly_equal_slabs():
    for nz in (1, 2, 7, 17, 200):
        for n in range(1, min(nz, 9) + 1):
            z = slabs.partition(nz, n)
            assert z[0] == 0 and z[-1] == nz and len(z) == n + 1
            depth = np.diff(z)
            assert depth.min() >= 1 and depth.max() - depth.min() <= 1
    with pytest.raises(ValueError):
        slabs.partition(3, 4)
    with pytest.raises(ValueError):
        slabs.partition(3, 0)


def test_cells_go_to_the_slab_of_their_voxel_layer():
    """Brute force: the slab whose layer range holds min(floor(z / dx), nz - 1),
    including cells on slab boundaries and on the grid's top face."""
    dx, nz = 20.0, 17
    z = [0, 1, 9, 17]
    rng = np.random.default_rng(2)
    pz = np.concatenate([rng.uniform(0, nz * dx, 500), np.array(z) * dx,
                         np.array(z[1:-1]) * dx - 1e-9])
    got = slabs.cell_slabs(pz, dx, z)
    for p, g in zip(pz, got):
        layer = min(int(np.floor(p / dx)), nz - 1)
        want = [j for j in range(len(z) - 1) if z[j] <= layer < z[j + 1]]
        assert [g] == want, (p, g, want)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class _FakeSlab:
    """Stands in for a slab context: forward writes the rank's own values,
    backward and finish record what they were given, so the test sees the
    order of calls and gathers of step_distributed."""

    def __init__(self, rank, world):
        import torch
        self.slab, self.n_slabs = rank, world
        self.send = torch.zeros((2, 3, 4), dtype=torch.float64)
        self.log = []

    def forward(self):
        self.send.fill_(10.0 * (self.slab + 1))
        self.log.append(("forward",))

    def backward(self, gathered):
        self.log.append(("backward", gathered.clone()))
        self.send.fill_(-(self.slab + 1.0))

    def finish(self, gathered):
        self.log.append(("finish", gathered.clone()))


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s = _FakeSlab(rank, world)
        slabs.step_distributed(s, 2)
        summary = [(e[0], None if len(e) == 1 else e[1][:, 0, 0, 0].tolist()) for e in s.log]
        bad = None
        try:
            slabs.step_distributed(_FakeSlab((rank + 1) % world, world), 1)
        except ValueError as ex:
            bad = str(ex)
        out.put((rank, summary, bad))
    finally:
        dist.destroy_process_group()


def test_step_distributed_gathers_in_rank_order_on_two_gloo_ranks():
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
    one_step = [("forward", None), ("backward", [10.0, 20.0]), ("finish", [-1.0, -2.0])]
    for rank, summary, bad in res:
        assert summary == one_step * 2, (rank, summary)
        assert bad is not None and "slab" in bad


@pytest.mark.parametrize("z_starts,slab,msg", [
    ([1, 5, 9], 0, "z_starts[0]"),
    ([0, 5, 5, 9], 1, "at least one z layer"),
    ([0, 5, 9], 2, "slab must be"),
    ([0, 5, 9], -1, "slab must be"),
])
def test_create_slab_rejects_bad_partitions_on_host(z_starts, slab, msg):
    from paper_2110_13368_gb300 import build, bfvm
    build.build()
    with pytest.raises(bfvm.BfvmError) as ei:
        bfvm.bfvm_create_slab(4, 4, z_starts, slab, 20.0, 0.01, [1e5], [0.1], [0], [0.0])
    assert ei.value.status == 1
    assert msg in str(ei.value)
