"""bfvm_apply_sources_noalloc: the cell source update for callers that must
not allocate device memory (host loops that cannot take the stalls of
cudaMalloc / cudaFree, programs whose memory manager owns all device
memory).  Its result must equal the library's own step: with D = lambda = 0
every sweep of bfvm_step is exactly the identity, so one step is exactly one
source update.  Collected last on purpose; builds everything it needs, so it
also passes alone in a fresh process."""
import numpy as np
import pytest

from tests.helpers import need_gpu, rel_inf

pytestmark = pytest.mark.gpu


def _problem():
    from paper_2110_13368_gb300 import inputs
    p = inputs.make_problem(17, 13, 11, n_sub=2, D=0.0, lam=0.0, n_cells=600,
                            U=[10.0, 1.0], S=[2.0, 6.0], rho_star=[38.0, 3.0], seed=4, steps=2)
    # a few voxels with many cells, to exercise the in-order composition
    p.pos[:40] = (np.array([3, 4, 5]) + 0.5) * p.dx
    p.pos[40:60] = (np.array([16, 12, 10]) + 0.5) * p.dx
    rng = np.random.default_rng(1)
    p.S = rng.uniform(0, 8, p.S.shape)
    p.U = rng.uniform(0, 8, p.U.shape)
    return p


def test_noalloc_sources_match_step_on_two_calls_in_a_row():
    torch = need_gpu()
    from paper_2110_13368_gb300 import build, bfvm
    build.build()
    p = _problem()
    sim = bfvm.Sim.from_problem(p)
    sim.step(1)
    ref1 = sim.get_density().cpu().numpy()
    sim.step(1)
    ref2 = sim.get_density().cpu().numpy()
    sim.close()
    rho = torch.as_tensor(p.rho0, dtype=torch.float64, device="cuda").contiguous()
    cells = [torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
             for a in (p.pos, p.vol, p.S, p.U, p.rho_star)]
    bfvm.bfvm_apply_sources_noalloc(rho, p.nx, p.ny, p.nz, p.dx, p.dt, *cells)
    got1 = rho.cpu().numpy()
    assert np.all(rel_inf(got1, ref1) <= 1e-12), rel_inf(got1, ref1)
    bfvm.bfvm_apply_sources_noalloc(rho, p.nx, p.ny, p.nz, p.dx, p.dt, *cells)
    got2 = rho.cpu().numpy()
    assert np.all(rel_inf(got2, ref2) <= 1e-12), rel_inf(got2, ref2)
    assert np.abs(got2 - got1).max() > 0.0


def test_noalloc_rejects_more_cells_than_its_scratch():
    torch = need_gpu()
    from paper_2110_13368_gb300 import build, bfvm
    build.build()
    n = (1 << 18) + 1
    rho = torch.zeros((1, 4, 4, 4), dtype=torch.float64, device="cuda")
    pos = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    one = torch.ones(n, dtype=torch.float64, device="cuda")
    rates = torch.zeros((n, 1), dtype=torch.float64, device="cuda")
    with pytest.raises(bfvm.BfvmError) as ei:
        bfvm.bfvm_apply_sources_noalloc(rho, 4, 4, 4, 20.0, 0.01, pos, one, rates, rates, rates)
    assert ei.value.status == 1
    assert "262144" in bfvm.bfvm_last_error(None)
