"""bfvm_apply_sources_noalloc: the cell source update for callers that must
not allocate device memory (host loops that cannot take the stalls of
cudaMalloc / cudaFree, programs whose memory manager owns all device
memory).

Its result is checked two ways on two calls in a row:
  * against the oracle's source update (cells in ascending index order per
    voxel, FP64, on the same inputs);
  * against the library's own step: with D = lambda = 0 every sweep of
    bfvm_step is exactly the identity, so one step is exactly one source
    update.
Cell counts cover the single shared-memory sort block (600 cells), the
multi-block merge of the sort (about 5 000 cells) and the scratch's maximum
(262 144 cells), each with many cells piled into a few voxels.

Collected last on purpose; builds everything it needs, so it also passes
alone in a fresh process."""
import numpy as np
import pytest

import oracle
from tests.helpers import need_gpu, rel_inf

pytestmark = pytest.mark.gpu

MAX_CELLS = 1 << 18


def _problem(n_cells, grid=(17, 13, 11), seed=4):
    from paper_2110_13368_gb300 import inputs
    nx, ny, nz = grid
    p = inputs.make_problem(nx, ny, nz, n_sub=2, D=0.0, lam=0.0, n_cells=n_cells,
                            U=[10.0, 1.0], S=[2.0, 6.0], rho_star=[38.0, 3.0], seed=seed, steps=2)
    # a few voxels with many cells, to exercise the in-order composition
    k = max(40, n_cells // 50)
    p.pos[:k] = (np.array([min(3, nx - 1), min(4, ny - 1), min(5, nz - 1)]) + 0.5) * p.dx
    p.pos[k:k + k // 2] = (np.array([nx - 1, ny - 1, nz - 1]) + 0.5) * p.dx
    p.pos[k + k // 2:k + k // 2 + 7] = 0.0                       # on the domain's corner
    rng = np.random.default_rng(seed + 1)
    p.S = rng.uniform(0, 8, p.S.shape)
    p.U = rng.uniform(0, 8, p.U.shape)
    return p


def _cells(torch, p):
    return [torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
            for a in (p.pos, p.vol, p.S, p.U, p.rho_star)]


@pytest.mark.parametrize("n_cells,grid", [(600, (17, 13, 11)), (5003, (23, 19, 29)),
                                          (MAX_CELLS, (64, 48, 40))])
def test_noalloc_sources_match_oracle_and_step_on_two_calls_in_a_row(n_cells, grid):
    torch = need_gpu()
    from paper_2110_13368_gb300 import build, bfvm
    build.build()
    oracle.build()
    p = _problem(n_cells, grid)
    ora1 = oracle.apply_sources(p, p.rho0)
    ora2 = oracle.apply_sources(p, ora1)
    sim = bfvm.Sim.from_problem(p)
    sim.step(1)
    ref1 = sim.get_density().cpu().numpy()
    sim.step(1)
    ref2 = sim.get_density().cpu().numpy()
    sim.close()
    rho = torch.as_tensor(p.rho0, dtype=torch.float64, device="cuda").contiguous()
    cells = _cells(torch, p)
    bfvm.bfvm_apply_sources_noalloc(rho, p.nx, p.ny, p.nz, p.dx, p.dt, *cells)
    got1 = rho.cpu().numpy()
    assert np.all(rel_inf(got1, ora1) <= 1e-12), rel_inf(got1, ora1)
    assert np.all(rel_inf(got1, ref1) <= 1e-12), rel_inf(got1, ref1)
    bfvm.bfvm_apply_sources_noalloc(rho, p.nx, p.ny, p.nz, p.dx, p.dt, *cells)
    got2 = rho.cpu().numpy()
    assert np.all(rel_inf(got2, ora2) <= 1e-12), rel_inf(got2, ora2)
    assert np.all(rel_inf(got2, ref2) <= 1e-12), rel_inf(got2, ref2)
    assert np.abs(got2 - got1).max() > 0.0


def test_noalloc_rejects_more_cells_than_its_scratch():
    torch = need_gpu()
    from paper_2110_13368_gb300 import build, bfvm
    build.build()
    n = MAX_CELLS + 1
    rho = torch.zeros((1, 4, 4, 4), dtype=torch.float64, device="cuda")
    pos = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    one = torch.ones(n, dtype=torch.float64, device="cuda")
    rates = torch.zeros((n, 1), dtype=torch.float64, device="cuda")
    with pytest.raises(bfvm.BfvmError) as ei:
        bfvm.bfvm_apply_sources_noalloc(rho, 4, 4, 4, 20.0, 0.01, pos, one, rates, rates, rates)
    assert ei.value.status == 1
    assert "262144" in bfvm.bfvm_last_error(None)


def test_noalloc_binding_checks_shapes_dtypes_and_devices():
    """The C entry point takes the array sizes on trust; the binding refuses
    arrays of the wrong type, shape or place before calling it, and the field
    is left as it was."""
    torch = need_gpu()
    from paper_2110_13368_gb300 import build, bfvm
    build.build()
    p = _problem(50, (6, 5, 4))
    rho = torch.as_tensor(p.rho0, dtype=torch.float64, device="cuda").contiguous()
    before = rho.clone()
    pos, vol, S, U, rs = _cells(torch, p)
    bad_calls = [
        (rho.float(), pos, vol, S, U, rs),                 # FP32 field
        (rho[:1].contiguous(), pos, vol, S, U, rs),        # fewer substrates than S has
        (rho, pos[:, :2].contiguous(), vol, S, U, rs),     # positions not (n, 3)
        (rho, pos, vol[:-1], S, U, rs),                    # volumes too short
        (rho, pos, vol, S[:, :1].contiguous(), U, rs),     # rates not (n, n_sub)
        (rho, pos, vol, S, U.cpu(), rs),                   # host tensor
        (rho, pos, vol, S, U, rs.float()),                 # FP32 rho*
    ]
    for args in bad_calls:
        with pytest.raises(ValueError):
            bfvm.bfvm_apply_sources_noalloc(args[0], p.nx, p.ny, p.nz, p.dx, p.dt, *args[1:])
    with pytest.raises(ValueError):   # grid that does not match the field
        bfvm.bfvm_apply_sources_noalloc(rho, p.nx + 1, p.ny, p.nz, p.dx, p.dt, pos, vol, S, U, rs)
    assert torch.equal(rho, before)
