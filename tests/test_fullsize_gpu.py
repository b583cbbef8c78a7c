"""Parity at the full benchmark size, in the launch configuration bench.py
times: the 200^3 x 2 tumour workload (250 000 cells), FP64 and FP32, and
the 1000^2 x 2 form of the 2-D variant, against the oracle on the whole
field."""
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


@pytest.fixture(scope="module")
def tumour10():
    p = inputs.tumour_200(steps=10)
    return p, oracle.run(p)


@pytest.mark.parametrize("precision,tol", [(64, 1e-12), (32, 1e-5)])
def test_tumour_200_ten_steps(bf, tumour10, precision, tol):
    p, ref = tumour10
    sim = bf.Sim.from_problem(p, precision=precision)
    sim.step(p.steps)
    got = sim.get_density().double().cpu().numpy()
    sim.close()
    err = rel_inf(got, ref)
    assert np.all(err <= tol), err


@pytest.mark.slow
def test_tumour_200_full_run_fp64(bf):
    """All 1000 steps of the benchmark workload, FP64, whole field."""
    p = inputs.tumour_200()
    ref = oracle.run(p)
    sim = bf.Sim.from_problem(p)
    sim.step(p.steps)
    got = sim.get_density().cpu().numpy()
    sim.close()
    err = rel_inf(got, ref)
    assert np.all(err <= 1e-12), err


@pytest.fixture(scope="module")
def two_d10():
    # the 2-D form bench.py times: 1000 x 1000 x 2, 20k cells
    p = inputs.make_problem(1000, 1000, 1, n_sub=2, D=[1e5, 1e3], lam=[0.1, 0.01],
                            bc_kind=[1, 0], bc_value=[38.0, 0.0], field_mode="zero",
                            n_cells=20_000, U=[10.0, 0.0], S=[0.0, 10.0],
                            rho_star=[1.0, 1.0], steps=10, seed=0, dims=2)
    return p, oracle.run(p)


@pytest.mark.parametrize("precision,tol", [(64, 1e-12), (32, 1e-5)])
def test_two_d_1000_ten_steps(bf, two_d10, precision, tol):
    """The 2-D variant at the size bench.py times (lines of 1000 voxels in
    16-voxel segments of the split line solve), whole field."""
    p, ref = two_d10
    sim = bf.Sim.from_problem(p, precision=precision)
    sim.step(p.steps)
    got = sim.get_density().double().cpu().numpy()
    sim.close()
    err = rel_inf(got, ref)
    assert np.all(err <= tol), err
