"""A grid decomposed along z into slabs (bfvm_create_slab and the three
calls of a slab step) computes the whole grid's step: the slabs' fields,
put back together, match the oracle's run of the whole grid at 1e-12.

Slabs are stepped in one process on one device (the gathers are stacks of
the slabs' send buffers), and as two processes sharing the device with a
gloo all-gather between the calls (each process owns one slab; nothing on
the GPU waits for the other process: the exchange is between the calls)."""
import os
import socket
import tempfile

import numpy as np
import pytest

import oracle
from paper_2110_13368_gb300 import inputs
from tests.helpers import need_gpu, rel_inf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bf():
    need_gpu()
    from paper_2110_13368_gb300 import build, bfvm
    build.build()
    return bfvm


def _problem(nx=13, ny=11, nz=17, steps=5, seed=6, n_cells=260):
    p = inputs.make_problem(nx, ny, nz, n_sub=2, D=[6e4, 2e3], lam=[0.1, 0.02],
                            bc_kind=[1, 0], bc_value=[38.0, 0.0], n_cells=n_cells,
                            U=[10.0, 1.0], S=[0.5, 6.0], rho_star=[38.0, 2.0], steps=steps,
                            seed=seed)
    if n_cells >= 20:
        # cells on the grid's z faces and on slab boundaries (layers 1, 8, 9)
        p.pos[:4, 2] = [0.0, nz * p.dx, 1 * p.dx, 9 * p.dx]
        p.pos[4:8, 2] = 8 * p.dx + np.array([0.0, 1e-9, 0.5, 0.999999]) * p.dx
    return p


def _run_slabs(p, z_starts, steps):
    import torch
    from paper_2110_13368_gb300 import slabs
    parts = [slabs.Slab.from_problem(p, z_starts, j) for j in range(len(z_starts) - 1)]
    slabs.step_together(parts, steps)
    out = torch.cat([s.get_density() for s in parts], dim=1).cpu().numpy()
    for s in parts:
        s.close()
    return out


@pytest.mark.parametrize("z_starts", [[0, 17], [0, 9, 17], [0, 1, 9, 17], [0, 6, 12, 16, 17],
                                      [0, 3, 5, 7, 9, 11, 13, 15, 17]])
def test_slabs_match_the_whole_grid_oracle(bf, z_starts):
    p = _problem()
    got = _run_slabs(p, z_starts, p.steps)
    err = rel_inf(got, oracle.run(p))
    assert np.all(err <= 1e-12), (z_starts, err)


@pytest.mark.parametrize("grid,z_starts", [((1, 1, 7), [0, 3, 7]), ((2, 2, 2), [0, 1, 2]),
                                           ((40, 3, 33), [0, 11, 22, 33]),
                                           ((5, 37, 64), [0, 32, 64])])
def test_slabs_on_thin_and_long_grids(bf, grid, z_starts):
    nx, ny, nz = grid
    p = _problem(nx, ny, nz, steps=3, n_cells=0)
    got = _run_slabs(p, z_starts, p.steps)
    err = rel_inf(got, oracle.run(p))
    assert np.all(err <= 1e-12), (grid, z_starts, err)


def test_slab_contexts_reject_whole_grid_calls(bf):
    import torch
    p = _problem(steps=1)
    from paper_2110_13368_gb300 import slabs
    s = slabs.Slab.from_problem(p, [0, 9, 17], 1)
    for call in (lambda: bf.bfvm_step(s.handle, 1), lambda: bf.bfvm_record(s.handle, 2),
                 lambda: bf.bfvm_set_option(s.handle, bf.OPT_VARIANT, 1),
                 lambda: bf.bfvm_set_option(s.handle, bf.OPT_DIMS, 2)):
        with pytest.raises(bf.BfvmError) as ei:
            call()
        assert ei.value.status == 4
    # a cell whose voxel layer lies in the other slab
    bad = [torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
           for a in (np.array([[30.0, 30.0, 5.0]]), p.vol[:1], p.S[:1], p.U[:1], p.rho_star[:1])]
    with pytest.raises(bf.BfvmError) as ei:
        s.set_cells(*bad)
    assert ei.value.status == 1 and "slab" in str(ei.value)
    s.close()
    ordinary = bf.Sim.from_problem(p)
    with pytest.raises(bf.BfvmError) as ei:
        bf.bfvm_slab_forward(ordinary.handle, torch.zeros((2, 11, 13), dtype=torch.float64,
                                                          device="cuda"))
    assert ei.value.status == 4
    ordinary.close()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _slab_rank(rank, world, port, z_starts, out_dir):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        from paper_2110_13368_gb300 import bfvm, slabs
        bfvm.load_library()
        p = _problem()
        s = slabs.Slab.from_problem(p, z_starts, rank)
        slabs.step_distributed(s, p.steps)
        np.save(os.path.join(out_dir, f"slab{rank}.npy"), s.get_density().cpu().numpy())
        s.close()
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_processes_one_slab_each_with_gloo_exchange(bf):
    import torch.multiprocessing as mp
    z_starts = [0, 7, 17]
    ctx = mp.get_context("spawn")
    with tempfile.TemporaryDirectory() as d:
        port = _free_port()
        procs = [ctx.Process(target=_slab_rank, args=(r, 2, port, z_starts, d)) for r in range(2)]
        for pr in procs:
            pr.start()
        for pr in procs:
            pr.join(timeout=300)
            assert pr.exitcode == 0
        got = np.concatenate([np.load(os.path.join(d, f"slab{r}.npy")) for r in range(2)], axis=1)
    p = _problem()
    err = rel_inf(got, oracle.run(p))
    assert np.all(err <= 1e-12), err
