"""Moving cells: bfvm_update_cells re-bins the cells on the device between
diffusion steps (a mechanics cadence), with no host round trip.  Each
segment of steps must equal the oracle run from the previous field with
that segment's cells."""
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


def _moved(p, rng, step_um):
    """The cells after a mechanics step: a random displacement (kept inside
    the domain), a volume change, and new rates."""
    ext = np.array([p.nx, p.ny, p.nz]) * p.dx
    pos = np.clip(p.pos + rng.normal(0.0, step_um, p.pos.shape), 0.0, ext)
    vol = p.vol * rng.uniform(0.9, 1.1, p.vol.shape)
    U = p.U * rng.uniform(0.5, 1.5, p.U.shape)
    S = p.S * rng.uniform(0.5, 1.5, p.S.shape)
    return p.with_(pos=pos, vol=vol, U=U, S=S)


@pytest.mark.parametrize("precision,variant,tol", [(64, 1, 1e-12), (64, 0, 1e-12), (32, None, 1e-5)])
@pytest.mark.parametrize("fused", [2, 0])
def test_cells_move_every_few_steps(bf, precision, variant, tol, fused):
    import torch
    rng = np.random.default_rng(8)
    p = inputs.make_problem(30, 26, 22, n_sub=2, D=[1e5, 2e3], lam=[0.1, 0.01],
                            bc_kind=[1, 0], bc_value=[38.0, 0.0], n_cells=800,
                            cell_mode="sphere", sphere_radius=150.0, U=[10.0, 0.5],
                            S=[0.0, 10.0], rho_star=[1.0, 3.0], steps=4, seed=3)
    sim = bf.Sim.from_problem(p, precision=precision)
    if variant is not None:
        sim.set_option(bf.OPT_VARIANT, variant)
    sim.set_option(bf.OPT_FUSED_STEP, fused)
    ref = p.rho0
    cur = p
    dev = sim.device
    for seg in range(5):
        if seg:
            cur = _moved(cur, rng, 15.0 if seg != 3 else 400.0)   # segment 3: big jumps
            t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
            sim.update_cells(t(cur.pos), t(cur.vol), t(cur.S), t(cur.U), t(cur.rho_star))
        sim.step(cur.steps)
        ref = oracle.run(cur, rho0=ref)
    got = sim.get_density().double().cpu().numpy()
    info = sim.info()
    sim.close()
    assert info["n_source_voxels"] > 0
    err = rel_inf(got, ref)
    assert np.all(err <= tol), (precision, variant, fused, err)


def test_cell_update_rules_and_device_check(bf):
    import torch
    p = inputs.make_problem(12, 10, 9, n_sub=1, D=[1e4], lam=[0.1], n_cells=50, U=[1.0],
                            S=[0.5], rho_star=[2.0], steps=2, seed=4)
    dev = torch.device("cuda")
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    sim = bf.Sim.from_problem(p)
    with pytest.raises(bf.BfvmError) as ei:                      # a different count
        sim.update_cells(t(p.pos[:10]), t(p.vol[:10]), t(p.S[:10]), t(p.U[:10]),
                         t(p.rho_star[:10]))
    assert ei.value.status == 1
    bad = p.pos.copy()
    bad[7, 1] = -5.0                                             # outside the domain
    sim.update_cells(t(bad), t(p.vol), t(p.S), t(p.U), t(p.rho_star))
    sim.step(1)
    with pytest.raises(bf.BfvmError) as ei:
        sim.sync()
    assert ei.value.status == 1
    sim.sync()                                                   # reported once
    sim.record(2)
    with pytest.raises(bf.BfvmError) as ei:                      # not while recording
        sim.update_cells(t(p.pos), t(p.vol), t(p.S), t(p.U), t(p.rho_star))
    assert ei.value.status == 4
    sim.close()
    empty = bf.Sim.from_problem(p.with_(pos=None, vol=None, S=None, U=None, rho_star=None))
    with pytest.raises(bf.BfvmError) as ei:
        empty.update_cells(t(p.pos), t(p.vol), t(p.S), t(p.U), t(p.rho_star))
    assert ei.value.status == 4
    empty.close()
