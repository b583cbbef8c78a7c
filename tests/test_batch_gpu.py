"""GPU parity of the batched form: many uneven members advanced by one
launch per phase must each match the oracle run of that member alone."""
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


def small_batch(n_inst=7, steps=6, seed=3):
    probs = inputs.batch_256(seed=seed, n_inst=n_inst, steps=steps, edge_lo=5, edge_hi=23,
                             cells_lo=20, cells_hi=300)
    # one Dirichlet member and one with a long line to exercise both paths
    probs[1] = inputs.make_problem(17, 9, 12, n_sub=2, D=[1e5, 4e3], lam=[0.1, 0.02],
                                   bc_kind=[1, 0], bc_value=[38.0, 0.0], n_cells=80,
                                   U=[10.0, 1.0], S=[0.0, 5.0], rho_star=[1.0, 2.0],
                                   steps=steps, seed=9)
    return probs


@pytest.mark.parametrize("precision,tol", [(64, 1e-12), (32, 1e-5)])
def test_batch_members_match_oracle(bf, precision, tol):
    probs = small_batch()
    sims = [bf.Sim.from_problem(p, precision=precision) for p in probs]
    batch = bf.Batch(sims)
    info = batch.info()
    assert info["members"] == len(probs)
    batch.step(probs[0].steps)
    batch.sync()
    for p, s in zip(probs, sims):
        got = s.get_density().double().cpu().numpy()
        ref = oracle.run(p)
        err = rel_inf(got, ref)
        assert np.all(err <= tol), (p.name, err)
    batch.close()
    for s in sims:
        s.close()


def test_batch_across_periods_and_graphs(bf):
    """Steps that cross the common rescale period, in odd chunks."""
    probs = small_batch(n_inst=4, steps=13, seed=5)
    sims = [bf.Sim.from_problem(p) for p in probs]
    for s in sims:
        s.set_option(bf.OPT_PERIOD, 4)
    batch = bf.Batch(sims)
    assert batch.info()["period"] == 4
    for n in (5, 3, 5):
        batch.step(n)
    batch.sync()
    for p, s in zip(probs, sims):
        got = s.get_density().cpu().numpy()
        assert np.all(rel_inf(got, oracle.run(p, n_steps=13)) <= 1e-12), p.name
    batch.close()


@pytest.mark.slow
@pytest.mark.parametrize("precision,tol", [(64, 1e-12), (32, 1e-5)])
def test_batch_256_full_size_sampled_members(bf, precision, tol):
    """The 256-member workload in the launch configuration the benchmark
    times, 200 steps, in FP64 and in FP32; eight members (and the smallest)
    are checked against the FP64 oracle, at 1e-12 and 1e-5."""
    probs = inputs.batch_256(seed=0, precision=precision)
    sims = [bf.Sim.from_problem(p) for p in probs]
    batch = bf.Batch(sims)
    batch.step(probs[0].steps)
    batch.sync()
    rng = np.random.default_rng(0)
    pick = sorted(rng.choice(len(probs), size=8, replace=False))
    sizes = np.array([p.updates_per_step for p in probs])
    pick = sorted(set(pick) | {int(np.argmin(sizes))})
    for i in pick:
        got = sims[i].get_density().double().cpu().numpy()
        ref = oracle.run(probs[i])
        assert np.all(rel_inf(got, ref) <= tol), (i, rel_inf(got, ref))
    batch.close()
    for s in sims:
        s.close()


def test_batch_rejects_mixed_precision(bf):
    p = inputs.make_problem(8, 8, 8, steps=1)
    a = bf.Sim.from_problem(p, precision=64)
    b = bf.Sim.from_problem(p, precision=32)
    with pytest.raises(bf.BfvmError):
        bf.Batch([a, b])
    a.close()
    b.close()


def pcr_batch(steps=5):
    """Members whose x lines span every PCR register layout (1 to 4 elements
    per lane, lines of 1 and 2 voxels, 128 voxels), Dirichlet and zero-flux
    substrates side by side."""
    edges = [(1, 3, 4), (2, 5, 3), (7, 6, 5), (33, 4, 3), (64, 3, 5), (100, 4, 4), (128, 3, 3)]
    probs = []
    for i, (nx, ny, nz) in enumerate(edges):
        probs.append(inputs.make_problem(nx, ny, nz, n_sub=2, D=[2e4 * (i + 1), 3e2],
                                         lam=[0.1, 0.01 * (i + 1)], bc_kind=[i % 2, 0],
                                         bc_value=[38.0, 0.0], n_cells=10 + 5 * i,
                                         U=[10.0, 1.0], S=[0.5, 5.0], rho_star=[1.0, 2.0],
                                         steps=steps, seed=20 + i))
    return probs


@pytest.mark.parametrize("precision,variant,tol", [(64, 1, 1e-12), (64, 0, 1e-12), (32, None, 1e-5)])
@pytest.mark.parametrize("x_algo,x_warps,yz_warps", [(1, 4, 2), (1, 8, 4), (0, 2, 4)])
def test_batch_line_block_shapes_match_oracle(bf, precision, variant, tol, x_algo, x_warps,
                                              yz_warps):
    """Every line-block shape the autotuner may pick (PCR or Thomas for the
    x lines, CTA sizes) gives each member's oracle result, in the rescaled
    and plain FP64 forms and in FP32."""
    probs = pcr_batch()
    sims = [bf.Sim.from_problem(p, precision=precision) for p in probs]
    if variant is not None:
        for s in sims:
            s.set_option(bf.OPT_VARIANT, variant)
    batch = bf.Batch(sims)
    batch.set_option(bf.BATCH_OPT_ONE_LAUNCH, 0)   # the tuned per-phase launches
    batch.set_shape(0, x_algo, x_warps)
    batch.set_shape(1, 0, yz_warps)
    batch.set_shape(2, 0, yz_warps)
    assert batch.shape(0)[:2] == (x_algo, x_warps)
    batch.step(probs[0].steps)
    batch.sync()
    for p, s in zip(probs, sims):
        got = s.get_density().double().cpu().numpy()
        err = rel_inf(got, oracle.run(p))
        assert np.all(err <= tol), (p.name, x_algo, err)
    batch.close()
    for s in sims:
        s.close()


def test_batch_autotuner_measures_and_leaves_fields(bf):
    """The tuner times Thomas on every axis and PCR on the x lines, keeps a
    valid shape, and runs its trials on copies: the members' fields are
    unchanged by bfvm_batch_create.  Unsupported shapes are rejected."""
    import torch
    probs = pcr_batch()
    sims = [bf.Sim.from_problem(p) for p in probs]
    before = [s.get_density().clone() for s in sims]
    batch = bf.Batch(sims)
    for s, b0 in zip(sims, before):
        assert torch.equal(s.get_density(), b0)
    algo, warps, ms = batch.shape(0)
    assert algo in (0, 1) and warps in (2, 4, 8)
    assert ms[0] > 0 and ms[1] > 0
    for axis in (1, 2):
        algo, warps, ms = batch.shape(axis)
        assert algo == 0 and ms[0] > 0 and ms[1] == -1
    with pytest.raises(bf.BfvmError):
        batch.set_shape(1, 1, 4)            # PCR only for x lines
    with pytest.raises(bf.BfvmError):
        batch.set_shape(0, 0, 9)
    batch.close()
    big = [bf.Sim.from_problem(inputs.make_problem(130, 3, 3, n_sub=1, D=[1e4], lam=[0.1],
                                                   bc_kind=[0], bc_value=[0.0], steps=1))]
    b2 = bf.Batch(big)
    assert b2.shape(0)[2][1] == -1          # x lines over 128 voxels: no PCR candidate
    with pytest.raises(bf.BfvmError):
        b2.set_shape(0, 1, 4)
    b2.close()
    for s in sims + big:
        s.close()


@pytest.mark.parametrize("precision,variant,tol", [(64, 1, 1e-12), (64, 0, 1e-12), (32, None, 1e-5)])
def test_one_launch_batch_matches_oracle_and_per_phase_launches(bf, precision, variant, tol):
    """The one-launch batched step (every member's x, y, z tasks, shells and
    sources in one persistent launch) against each member's oracle run and
    against the per-phase launches of the same batch, in the rescaled and
    plain FP64 forms and in FP32; members of uneven shapes, a Dirichlet
    member, lines of 1 to 128 voxels; steps crossing the rescale period."""
    probs = small_batch(n_inst=6, steps=13, seed=11) + pcr_batch(steps=13)
    results = []
    for one in (1, 0):
        sims = [bf.Sim.from_problem(p, precision=precision) for p in probs]
        if variant is not None:
            for s in sims:
                s.set_option(bf.OPT_VARIANT, variant)
        if precision == 64 and variant == 1:
            for s in sims:
                s.set_option(bf.OPT_PERIOD, 4)
        batch = bf.Batch(sims)
        batch.set_option(bf.BATCH_OPT_ONE_LAUNCH, one)
        launches0 = batch.info()["launches"]
        for n in (5, 3, 5):
            batch.step(n)
        batch.sync()
        per_step = (batch.info()["launches"] - launches0) / 13
        if one:
            assert per_step == 1.0, per_step
        results.append([s.get_density().double().cpu().numpy() for s in sims])
        batch.close()
        for s in sims:
            s.close()
    for p, a, b in zip(probs, *results):
        ref = oracle.run(p)
        assert np.all(rel_inf(a, ref) <= tol), (p.name, rel_inf(a, ref))
        assert np.all(rel_inf(a, b) <= tol), (p.name, rel_inf(a, b))


def test_one_launch_batch_wait_gives_up_with_status(bf):
    """Batch option 2 makes every dependency wait of the one-launch step
    unreachable: the waits give up after the given polls, bfvm_batch_sync
    reports BFVM_ETIMEOUT, and after the option is cleared steps from a fresh
    field are correct again."""
    import torch
    probs = small_batch(n_inst=4, steps=2, seed=13)
    sims = [bf.Sim.from_problem(p) for p in probs]
    batch = bf.Batch(sims)
    batch.set_option(bf.BATCH_OPT_WAIT_TEST, 200)
    batch.step(1)
    with pytest.raises(bf.BfvmError) as ei:
        batch.sync()
    assert ei.value.status == 5
    batch.set_option(bf.BATCH_OPT_WAIT_TEST, 0)
    batch.close()
    for p, s in zip(probs, sims):
        s.set_density(torch.as_tensor(p.rho0, dtype=s.dtype, device="cuda"))
    batch = bf.Batch(sims)
    batch.step(2)
    batch.sync()
    for p, s in zip(probs, sims):
        got = s.get_density().cpu().numpy()
        assert np.all(rel_inf(got, oracle.run(p)) <= 1e-12), p.name
    batch.close()
    for s in sims:
        s.close()



def mixed_2d_batch(steps=7):
    """2-D members (x lines of 1 to 128 voxels, Dirichlet and zero-flux
    substrates) next to 3-D members; with any 2-D member the batch runs the
    plain form."""
    probs = []
    for i, (nx, ny) in enumerate([(1, 9), (5, 7), (33, 20), (64, 3), (128, 17), (47, 61)]):
        probs.append(inputs.make_problem(nx, ny, 1, n_sub=2, D=[2e4 * (i + 1), 3e2],
                                         lam=[0.1, 0.01 * (i + 1)], bc_kind=[(i + 1) % 2, 0],
                                         bc_value=[38.0, 0.0], n_cells=10 + 5 * i,
                                         U=[10.0, 1.0], S=[0.5, 5.0], rho_star=[1.0, 2.0],
                                         steps=steps, seed=40 + i, dims=2))
    probs.append(inputs.make_problem(17, 9, 12, n_sub=2, D=[1e5, 4e3], lam=[0.1, 0.02],
                                     bc_kind=[1, 0], bc_value=[38.0, 0.0], n_cells=80,
                                     U=[10.0, 1.0], S=[0.0, 5.0], rho_star=[1.0, 2.0],
                                     steps=steps, seed=9))
    probs.append(inputs.make_problem(30, 4, 5, n_sub=2, D=[3e4, 1e3], lam=[0.2, 0.05],
                                     bc_kind=[0, 1], bc_value=[0.0, 20.0], n_cells=40,
                                     U=[5.0, 1.0], S=[1.0, 2.0], rho_star=[3.0, 9.0],
                                     steps=steps, seed=11))
    return probs


@pytest.mark.parametrize("precision,tol", [(64, 1e-12), (32, 1e-5)])
@pytest.mark.parametrize("mode", ["one_launch", "pcr_x", "thomas"])
def test_batch_with_2d_members_matches_oracle(bf, precision, tol, mode):
    """2-D members in a batch (no z sweep, the four-edge shell) beside 3-D
    members: the one-launch step and the per-phase launches with PCR or
    Thomas x lines, each member against its own oracle run."""
    probs = mixed_2d_batch()
    sims = [bf.Sim.from_problem(p, precision=precision) for p in probs]
    batch = bf.Batch(sims)
    if mode == "one_launch":
        batch.set_option(bf.BATCH_OPT_ONE_LAUNCH, 1)
    else:
        batch.set_option(bf.BATCH_OPT_ONE_LAUNCH, 0)
        batch.set_shape(0, 1 if mode == "pcr_x" else 0, 4)
        batch.set_shape(1, 0, 4)
        batch.set_shape(2, 0, 4)
    launches0 = batch.info()["launches"]
    for n in (3, 4):
        batch.step(n)
    batch.sync()
    if mode == "one_launch":
        assert (batch.info()["launches"] - launches0) / 7 == 1.0
    for p, s in zip(probs, sims):
        got = s.get_density().double().cpu().numpy()
        err = rel_inf(got, oracle.run(p))
        assert np.all(err <= tol), (p.name, p.nx, p.ny, p.nz, mode, err)
    batch.close()
    for s in sims:
        s.close()
