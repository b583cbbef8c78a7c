"""Parity at the full benchmark size, in the launch configuration bench.py
times: the 200^3 x 2 tumour workload (250 000 cells), FP64 and FP32,
against the oracle on the whole field."""
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
