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
def test_batch_256_full_size_sampled_members(bf):
    """The 256-member workload in the launch configuration the benchmark
    times, 200 steps; eight members are checked against the oracle."""
    probs = inputs.batch_256(seed=0)
    sims = [bf.Sim.from_problem(p) for p in probs]
    batch = bf.Batch(sims)
    batch.step(probs[0].steps)
    batch.sync()
    rng = np.random.default_rng(0)
    pick = sorted(rng.choice(len(probs), size=8, replace=False))
    sizes = np.array([p.updates_per_step for p in probs])
    pick = sorted(set(pick) | {int(np.argmin(sizes))})
    for i in pick:
        got = sims[i].get_density().cpu().numpy()
        ref = oracle.run(probs[i])
        assert np.all(rel_inf(got, ref) <= 1e-12), (i, rel_inf(got, ref))
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
