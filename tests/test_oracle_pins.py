"""Pins of the CPU oracle against facts that do not come from the oracle.

Each test fixes the oracle to mathematics the paper's Eq. 1 and the LOD
scheme determine: closed forms, invariants, library routines, brute force on
tiny grids, and convergence to the exact solution of the source ODE.  Each is
chosen so that a plausible slip (a dropped term, a wrong sign, a transposed
axis, a wrong Dirichlet layer, a wrong cell order) fails at least one.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from paper_2110_13368_gb300 import inputs


def _laplacian_from_fluxes(n):
    """Zero-flux 1-D finite-volume Laplacian built from face fluxes: one
    difference operator row per interior face, L = B^T B."""
    if n == 1:
        return np.zeros((1, 1))
    B = np.zeros((n - 1, n))
    for f in range(n - 1):
        B[f, f] = -1.0
        B[f, f + 1] = 1.0
    return B.T @ B


# ----------------------------------------------------------------- line matrix
@pytest.mark.parametrize("n", [1, 2, 3, 7, 50])
def test_line_matrix_is_flux_form(n):
    c, ell = 2.5, 0.1 * 0.01 / 3
    lo, di, up = oracle.line_matrix(n, c, ell)
    A = np.diag(di) + np.diag(lo[1:], -1) + np.diag(up[:-1], 1)
    ref = (1 + ell) * np.eye(n) + c * _laplacian_from_fluxes(n)
    np.testing.assert_array_equal(A, ref)
    # symmetric, column sums 1 + ell (mass balance of zero-flux faces)
    np.testing.assert_array_equal(A, A.T)
    np.testing.assert_allclose(A.sum(axis=0), 1 + ell, rtol=0, atol=1e-15)


@pytest.mark.parametrize("n", [2, 5, 16, 33])
def test_line_matrix_cosine_spectrum(n):
    c, ell = 0.7, 0.013
    lo, di, up = oracle.line_matrix(n, c, ell)
    A = np.diag(di) + np.diag(lo[1:], -1) + np.diag(up[:-1], 1)
    ev = np.sort(np.linalg.eigvalsh(A))
    k = np.arange(n)
    ref = np.sort(1 + ell + 2 * c * (1 - np.cos(np.pi * k / n)))
    np.testing.assert_allclose(ev, ref, rtol=1e-13, atol=1e-13)


# ------------------------------------------------------------------- Thomas
@pytest.mark.parametrize("n", [1, 2, 3, 10, 200])
def test_thomas_matches_banded_lapack(n):
    rng = np.random.default_rng(n)
    lo = -rng.uniform(0.1, 1.0, n)
    up = -rng.uniform(0.1, 1.0, n)
    lo[0] = 0.0
    up[-1] = 0.0
    di = 1.0 + np.abs(lo) + np.abs(up) + rng.uniform(0.0, 1.0, n)
    rhs = rng.standard_normal(n)
    x = oracle.tridiag_solve(lo, di, up, rhs)
    ab = np.zeros((3, n))
    ab[0, 1:] = up[:-1]
    ab[1] = di
    ab[2, :-1] = lo[1:]
    ref = sla.solve_banded((1, 1), ab, rhs)
    np.testing.assert_allclose(x, ref, rtol=1e-13, atol=1e-13)


# ---------------------------------------------------------- P1 uniform field
def test_uniform_field_decays_by_closed_form():
    p = inputs.make_problem(9, 6, 11, D=1e5, lam=0.1, field_mode="zero")
    p.rho0[:] = 38.0
    r = oracle.run(p, n_steps=1)
    ell = p.lam[0] * p.dt / 3
    np.testing.assert_allclose(r, 38.0 * (1 + ell) ** -3, rtol=1e-14, atol=0)
    r5 = oracle.run(p, n_steps=5)
    np.testing.assert_allclose(r5, 38.0 * (1 + ell) ** -15, rtol=1e-13, atol=0)


# ---------------------------------------------------------- P2 Fourier modes
@pytest.mark.parametrize("dims,ks", [((12, 7, 9), (3, 1, 2)), ((5, 16, 3), (0, 5, 2)),
                                     ((1, 6, 10), (0, 2, 7))])
def test_cosine_modes_are_eigenfunctions(dims, ks):
    nx, ny, nz = dims
    p = inputs.make_problem(nx, ny, nz, D=3e4, lam=0.05, field_mode="zero")
    cx = np.cos(np.pi * ks[0] * (np.arange(nx) + 0.5) / nx)
    cy = np.cos(np.pi * ks[1] * (np.arange(ny) + 0.5) / ny)
    cz = np.cos(np.pi * ks[2] * (np.arange(nz) + 0.5) / nz)
    mode = cz[:, None, None] * cy[None, :, None] * cx[None, None, :]
    p.rho0[0] = mode
    c = p.D[0] * p.dt / p.dx ** 2
    ell = p.lam[0] * p.dt / 3
    fac = 1.0
    for n, k in zip(dims, ks):
        fac /= 1 + ell + 2 * c * (1 - np.cos(np.pi * k / n))
    r = oracle.run(p, n_steps=1)[0]
    np.testing.assert_allclose(r, fac * mode, rtol=0, atol=1e-14 * np.abs(mode).max())
    # three steps: factor cubed
    r3 = oracle.run(p, n_steps=3)[0]
    np.testing.assert_allclose(r3, fac ** 3 * mode, rtol=0, atol=1e-14 * np.abs(mode).max())


# ---------------------------------------------------- P3 mass conservation
def test_mass_conserved_without_decay():
    p = inputs.make_problem(13, 8, 10, n_sub=2, D=[1e5, 3e2], lam=0.0, seed=3)
    m0 = p.rho0.sum(axis=(1, 2, 3))
    r = oracle.run(p, n_steps=7)
    np.testing.assert_allclose(r.sum(axis=(1, 2, 3)), m0, rtol=1e-13)
    # and the field really moved
    assert np.abs(r - p.rho0).max() > 0.1


# ------------------------------------------------------ P4 dense LU, tiny grids
def _dense_step_operators(p):
    nx, ny, nz = p.nx, p.ny, p.nz
    mats = []
    for s in range(p.n_sub):
        c = p.D[s] * p.dt / p.dx ** 2
        ell = p.lam[s] * p.dt / 3
        Ix, Iy, Iz = np.eye(nx), np.eye(ny), np.eye(nz)
        Ax = (1 + ell) * Ix + c * _laplacian_from_fluxes(nx)
        Ay = (1 + ell) * Iy + c * _laplacian_from_fluxes(ny)
        Az = (1 + ell) * Iz + c * _laplacian_from_fluxes(nz)
        # flattened index (z, y, x), x fastest
        mats.append([np.kron(Iz, np.kron(Iy, Ax)), np.kron(Iz, np.kron(Ay, Ix)),
                     np.kron(Az, np.kron(Iy, Ix))])
    return mats


def _dense_shell_mask(nx, ny, nz):
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return ((x == 0) | (x == nx - 1) | (y == 0) | (y == ny - 1) | (z == 0)
            | (z == nz - 1)).ravel()


def _dense_run(p, n_steps):
    mats = _dense_step_operators(p)
    lus = [[sla.lu_factor(M) for M in ms] for ms in mats]
    shell = _dense_shell_mask(p.nx, p.ny, p.nz)
    rho = p.rho0.reshape(p.n_sub, -1).copy()
    vvox = p.dx ** 3
    for _ in range(n_steps):
        for s in range(p.n_sub):
            u = rho[s]
            dir_ = p.bc_kind[s] == 1
            if dir_:
                u[shell] = p.bc_value[s]
            for a in range(3):
                u = sla.lu_solve(lus[s][a], u)
                if dir_:
                    u[shell] = p.bc_value[s]
            rho[s] = u
        # sources, one cell at a time in index order (Eq. 1, implicit)
        for i in range(p.n_cells):
            v = [min(int(np.floor(p.pos[i, a] / p.dx)), n - 1)
                 for a, n in enumerate((p.nx, p.ny, p.nz))]
            lin = (v[2] * p.ny + v[1]) * p.nx + v[0]
            w = p.dt * p.vol[i] / vvox
            for s in range(p.n_sub):
                rho[s, lin] = ((rho[s, lin] + w * p.S[i, s] * p.rho_star[i, s])
                               / (1 + w * (p.S[i, s] + p.U[i, s])))
    return rho.reshape(p.rho0.shape)


@pytest.mark.parametrize("dims", [(3, 4, 5), (1, 1, 7), (2, 2, 2), (5, 1, 3), (4, 6, 1)])
def test_dense_lu_tiny_grids(dims):
    nx, ny, nz = dims
    p = inputs.make_problem(nx, ny, nz, n_sub=3, D=[1e5, 2e3, 4e4],
                            lam=[0.1, 0.0, 0.9], bc_kind=[1, 0, 1],
                            bc_value=[38.0, 0.0, 5.0], n_cells=6, U=[10.0, 1.0, 0.0],
                            S=[0.0, 3.0, 7.0], rho_star=[1.0, 38.0, 2.0], seed=11)
    ref = _dense_run(p, 3)
    got = oracle.run(p, n_steps=3)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * np.abs(ref).max())


# --------------------------------------------------------------- P5 sources
def _single_voxel_problem(dt, S, U, rho_star, vol, n_cells):
    p = inputs.make_problem(1, 1, 1, n_sub=1, D=0.0, lam=0.0, dt=dt,
                            field_mode="zero")
    p.rho0[:] = 5.0
    p.pos = np.full((n_cells, 3), 10.0)
    p.vol = np.asarray(vol, dtype=np.float64).reshape(n_cells)
    p.S = np.asarray(S, dtype=np.float64).reshape(n_cells, 1)
    p.U = np.asarray(U, dtype=np.float64).reshape(n_cells, 1)
    p.rho_star = np.asarray(rho_star, dtype=np.float64).reshape(n_cells, 1)
    return p


def test_single_cell_geometric_closed_form():
    p = _single_voxel_problem(0.01, [3.0], [2.0], [7.0], [2494.0], 1)
    w = 0.01 * 2494.0 / 20.0 ** 3
    fp = 3.0 * 7.0 / (3.0 + 2.0)
    for n in (1, 4, 50):
        got = oracle.run(p, n_steps=n)[0, 0, 0, 0]
        ref = fp + (5.0 - fp) * (1 + w * 5.0) ** (-n)
        assert got == pytest.approx(ref, rel=1e-13)
    # long run reaches the fixed point S rho* / (S + U)
    got = oracle.run(p, n_steps=200000)[0, 0, 0, 0]
    assert got == pytest.approx(fp, rel=1e-12)


def test_sources_converge_to_exact_ode_solution():
    """With D = lambda = 0, Eq. 1 in one voxel is the linear ODE
    d rho/dt = sum_i (V_i/V_vox) (S_i (rho*_i - rho) - U_i rho);
    the implicit steps converge to its exponential solution at first order."""
    T = 0.2
    S, U, rs, V = [4.0, 0.5], [1.0, 6.0], [9.0, 2.0], [30000.0, 20000.0]
    k = sum(v / 8000.0 * (s + u) for v, s, u in zip(V, S, U))
    src = sum(v / 8000.0 * s * r for v, s, r in zip(V, S, rs))
    exact = src / k + (5.0 - src / k) * np.exp(-k * T)
    errs = []
    for dt in (0.002, 0.001, 0.0005):
        p = _single_voxel_problem(dt, S, U, rs, V, 2)
        got = oracle.run(p, n_steps=int(round(T / dt)))[0, 0, 0, 0]
        errs.append(abs(got - exact))
    assert errs[0] / errs[1] == pytest.approx(2.0, rel=0.05)
    assert errs[1] / errs[2] == pytest.approx(2.0, rel=0.05)


def test_co_located_cells_apply_in_index_order():
    cells = dict(S=[4.0, 0.0], U=[0.0, 9.0], rho_star=[10.0, 0.0], vol=[6000.0, 6000.0])
    p = _single_voxel_problem(0.05, cells["S"], cells["U"], cells["rho_star"], cells["vol"], 2)
    both = oracle.run(p, n_steps=1)[0, 0, 0, 0]
    pa = _single_voxel_problem(0.05, [4.0], [0.0], [10.0], [6000.0], 1)
    after_a = oracle.run(pa, n_steps=1)[0, 0, 0, 0]
    pb = _single_voxel_problem(0.05, [0.0], [9.0], [0.0], [6000.0], 1)
    a_then_b = oracle.run(pb, rho0=np.full((1, 1, 1, 1), after_a), n_steps=1)[0, 0, 0, 0]
    assert both == a_then_b
    swapped = _single_voxel_problem(0.05, [0.0, 4.0], [9.0, 0.0], [0.0, 10.0], [6000.0, 6000.0], 2)
    assert oracle.run(swapped, n_steps=1)[0, 0, 0, 0] != pytest.approx(both, rel=1e-6)


def test_cell_voxel_mapping_faces_and_clamp():
    p = inputs.make_problem(4, 5, 6, dx=20.0, field_mode="zero")
    assert oracle.cell_voxel(p, [0.0, 0.0, 0.0]) == 0
    assert oracle.cell_voxel(p, [20.0, 0.0, 0.0]) == 1          # face -> higher voxel
    assert oracle.cell_voxel(p, [19.999999, 0.0, 0.0]) == 0
    assert oracle.cell_voxel(p, [80.0, 100.0, 120.0]) == (5 * 5 + 4) * 4 + 3  # clamp
    assert oracle.cell_voxel(p, [30.0, 45.0, 61.0]) == (3 * 5 + 2) * 4 + 1


# ---------------------------------------------------------- P6 Dirichlet
def test_dirichlet_shell_and_monotone_steady_state():
    p = inputs.make_problem(10, 9, 8, D=1e5, lam=0.0, bc_kind=1, bc_value=38.0,
                            field_mode="zero")
    shell = _dense_shell_mask(10, 9, 8).reshape(8, 9, 10)
    r1 = oracle.run(p, n_steps=1)[0]
    assert np.all(r1[shell] == 38.0)
    # only the outermost layer is held: the next layer is strictly between 0 and 38
    assert 0.0 < r1[1:-1, 1:-1, 1:-1].max() < 38.0
    prev = r1
    for _ in range(6):
        nxt = oracle.run(p, rho0=prev[None], n_steps=20)[0]
        assert np.all(nxt >= prev - 1e-12)
        prev = nxt
    assert np.abs(prev - 38.0).max() < 1e-6


# ---------------------------------------------------------- P7 adjoint
def _small_adjoint_problem():
    p = inputs.make_problem(6, 5, 4, n_sub=2, D=[2e4, 8e2], lam=[0.2, 0.05],
                            bc_kind=[1, 0], bc_value=[38.0, 0.0], n_cells=9,
                            U=[10.0, 2.0], S=[1.0, 6.0], rho_star=[38.0, 3.0],
                            seed=5, steps=5, dt=0.02)
    return p


def test_adjoint_field_gradient_dot_product():
    """The step is affine in rho, so <dL/drho0, v> = <w, run(rho0+v) - run(rho0)>
    exactly for L = <w, rho_final>."""
    p = _small_adjoint_problem()
    rng = np.random.default_rng(2)
    w = rng.standard_normal(p.rho0.shape)
    v = rng.standard_normal(p.rho0.shape)
    out = oracle.adjoint(p, w, checkpoint_every=2)
    lhs = np.vdot(out["g0"], v)
    rhs = np.vdot(w, oracle.run(p, rho0=p.rho0 + v) - oracle.run(p))
    assert lhs == pytest.approx(rhs, rel=1e-10)
    np.testing.assert_array_equal(out["rho_final"], oracle.run(p))


def test_adjoint_parameter_gradients_match_central_differences():
    p = _small_adjoint_problem()
    rng = np.random.default_rng(4)
    target = p.rho0 * 0.5 + rng.uniform(0, 1, p.rho0.shape)

    def loss(q):
        return float(((oracle.run(q) - target) ** 2).sum())

    g = 2.0 * (oracle.run(p) - target)
    out = oracle.adjoint(p, g, checkpoint_every=3)

    def fd(make):
        h_rel = 1e-5
        lp = loss(make(1 + h_rel))
        lm = loss(make(1 - h_rel))
        return lp, lm, h_rel

    for s in range(p.n_sub):
        for key, attr in (("dD", "D"), ("dlambda", "lam")):
            base = getattr(p, attr)

            def make(f, s=s, attr=attr, base=base):
                v = base.copy()
                v[s] *= f
                return p.with_(**{attr: v})
            lp, lm, h = fd(make)
            est = (lp - lm) / (2 * h * base[s])
            assert out[key][s] == pytest.approx(est, rel=2e-6), (key, s)
    for i in (0, 4, 8):
        for s in range(p.n_sub):
            for key, attr in (("dS", "S"), ("dU", "U")):
                base = getattr(p, attr)
                h = 1e-4 * max(abs(base[i, s]), 1e-2)

                def mk(delta, i=i, s=s, attr=attr, base=base):
                    v = base.copy()
                    v[i, s] += delta
                    return p.with_(**{attr: v})
                est = (loss(mk(h)) - loss(mk(-h))) / (2 * h)
                assert out[key][i, s] == pytest.approx(est, rel=1e-6, abs=1e-9), (key, i, s)


def test_oracle_threads_do_not_change_bits():
    p = inputs.make_problem(17, 9, 12, n_sub=2, n_cells=40, seed=8)
    a = oracle.run(p, n_steps=3, n_threads=1)
    b = oracle.run(p, n_steps=3, n_threads=4)
    np.testing.assert_array_equal(a, b)


# ------------------------------------------------------------ 2-D variant
def test_2d_uniform_field_decays_by_closed_form():
    """2-D variant: two sweeps, each with half of the decay: (1 + lambda dt/2)^-2."""
    p = inputs.make_problem(9, 6, 1, D=1e5, lam=0.1, field_mode="zero", dims=2)
    p.rho0[:] = 38.0
    ell = p.lam[0] * p.dt / 2
    np.testing.assert_allclose(oracle.run(p, n_steps=1), 38.0 * (1 + ell) ** -2, rtol=1e-14)
    np.testing.assert_allclose(oracle.run(p, n_steps=4), 38.0 * (1 + ell) ** -8, rtol=1e-13)


@pytest.mark.parametrize("dims,ks", [((12, 7), (3, 1)), ((5, 16), (0, 5)), ((1, 9), (0, 4))])
def test_2d_cosine_modes_are_eigenfunctions(dims, ks):
    nx, ny = dims
    p = inputs.make_problem(nx, ny, 1, D=3e4, lam=0.05, field_mode="zero", dims=2)
    cx = np.cos(np.pi * ks[0] * (np.arange(nx) + 0.5) / nx)
    cy = np.cos(np.pi * ks[1] * (np.arange(ny) + 0.5) / ny)
    mode = (cy[:, None] * cx[None, :])[None]
    p.rho0[0] = mode
    c = p.D[0] * p.dt / p.dx ** 2
    ell = p.lam[0] * p.dt / 2
    fac = 1.0
    for n, k in zip(dims, ks):
        fac /= 1 + ell + 2 * c * (1 - np.cos(np.pi * k / n))
    r = oracle.run(p, n_steps=2)[0]
    np.testing.assert_allclose(r, fac ** 2 * mode, rtol=0, atol=1e-14 * np.abs(mode).max())


def _dense_run_2d(p, n_steps):
    nx, ny = p.nx, p.ny
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    shell = ((x == 0) | (x == nx - 1) | (y == 0) | (y == ny - 1)).ravel()
    rho = p.rho0.reshape(p.n_sub, -1).copy()
    vvox = p.dx ** 3
    for _ in range(n_steps):
        for s in range(p.n_sub):
            c = p.D[s] * p.dt / p.dx ** 2
            ell = p.lam[s] * p.dt / 2
            Ax = (1 + ell) * np.eye(nx) + c * _laplacian_from_fluxes(nx)
            Ay = (1 + ell) * np.eye(ny) + c * _laplacian_from_fluxes(ny)
            ops = [np.kron(np.eye(ny), Ax), np.kron(Ay, np.eye(nx))]
            u = rho[s]
            dir_ = p.bc_kind[s] == 1
            if dir_:
                u[shell] = p.bc_value[s]
            for M in ops:
                u = sla.lu_solve(sla.lu_factor(M), u)
                if dir_:
                    u[shell] = p.bc_value[s]
            rho[s] = u
        for i in range(p.n_cells):
            v = [min(int(np.floor(p.pos[i, a] / p.dx)), n - 1) for a, n in enumerate((nx, ny, 1))]
            lin = v[1] * nx + v[0]
            w = p.dt * p.vol[i] / vvox
            for s in range(p.n_sub):
                rho[s, lin] = ((rho[s, lin] + w * p.S[i, s] * p.rho_star[i, s])
                               / (1 + w * (p.S[i, s] + p.U[i, s])))
    return rho.reshape(p.rho0.shape)


@pytest.mark.parametrize("dims", [(3, 4), (1, 7), (2, 2), (6, 5)])
def test_2d_dense_lu_tiny_grids(dims):
    """2-D step against Kronecker-assembled dense solves with the 2-D shell
    (four edges, not the z layer) and the same cell sources."""
    nx, ny = dims
    p = inputs.make_problem(nx, ny, 1, n_sub=3, D=[1e5, 2e3, 4e4], lam=[0.1, 0.0, 0.9],
                            bc_kind=[1, 0, 1], bc_value=[38.0, 0.0, 5.0], n_cells=5,
                            U=[10.0, 1.0, 0.0], S=[0.0, 3.0, 7.0], rho_star=[1.0, 38.0, 2.0],
                            seed=13, dims=2)
    ref = _dense_run_2d(p, 3)
    got = oracle.run(p, n_steps=3)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * np.abs(ref).max())


def test_2d_equals_3d_step_without_decay():
    """With lambda = 0 and zero-flux faces the 3-D step on an nx x ny x 1
    grid is the 2-D step (the z line matrix is [1]); mass is conserved."""
    p3 = inputs.make_problem(11, 8, 1, n_sub=2, D=[1e5, 3e2], lam=0.0, n_cells=7,
                             U=[2.0, 0.0], S=[0.0, 4.0], rho_star=[1.0, 2.0], seed=4)
    p2 = p3.with_(dims=2)
    np.testing.assert_array_equal(oracle.run(p2, n_steps=5), oracle.run(p3, n_steps=5))
    q = p3.with_(pos=None, vol=None, S=None, U=None, rho_star=None, dims=2)
    m0 = q.rho0.sum(axis=(1, 2, 3))
    np.testing.assert_allclose(oracle.run(q, n_steps=6).sum(axis=(1, 2, 3)), m0, rtol=1e-13)


# ------------------------------------------------------- Dirichlet nodes
def _dense_run_nodes(p, n_steps):
    """_dense_run with the node projection after every shell projection."""
    mats = _dense_step_operators(p)
    lus = [[sla.lu_factor(M) for M in ms] for ms in mats]
    shell = _dense_shell_mask(p.nx, p.ny, p.nz)
    vox, sub, val = p.nodes
    rho = p.rho0.reshape(p.n_sub, -1).copy()
    vvox = p.dx ** 3

    def project(s, u):
        if p.bc_kind[s] == 1:
            u[shell] = p.bc_value[s]
        for i in range(len(vox)):          # index order: the later node holds
            if sub[i] == s:
                u[vox[i]] = val[i]
        return u

    for _ in range(n_steps):
        for s in range(p.n_sub):
            u = project(s, rho[s])
            for a in range(3):
                u = project(s, sla.lu_solve(lus[s][a], u))
            rho[s] = u
        for i in range(p.n_cells):
            v = [min(int(np.floor(p.pos[i, a] / p.dx)), n - 1)
                 for a, n in enumerate((p.nx, p.ny, p.nz))]
            lin = (v[2] * p.ny + v[1]) * p.nx + v[0]
            w = p.dt * p.vol[i] / vvox
            for s in range(p.n_sub):
                rho[s, lin] = ((rho[s, lin] + w * p.S[i, s] * p.rho_star[i, s])
                               / (1 + w * (p.S[i, s] + p.U[i, s])))
    return rho.reshape(p.rho0.shape)


@pytest.mark.parametrize("dims", [(4, 5, 3), (1, 1, 6), (3, 3, 3)])
def test_nodes_dense_lu_tiny_grids(dims):
    """Dirichlet nodes (one on the shell, two on one voxel with different
    values) against Kronecker-assembled dense solves with the projections."""
    nx, ny, nz = dims
    p = inputs.make_problem(nx, ny, nz, n_sub=2, D=[1e5, 2e3], lam=[0.1, 0.02],
                            bc_kind=[1, 0], bc_value=[38.0, 0.0], n_cells=4, U=[10.0, 1.0],
                            S=[0.0, 3.0], rho_star=[1.0, 2.0], seed=17)
    n_vox = nx * ny * nz
    vox = np.array([n_vox // 2, 0, n_vox - 1, n_vox - 1], dtype=np.int64)
    sub = np.array([0, 1, 1, 1], dtype=np.int32)
    val = np.array([50.0, 7.0, 3.0, 9.0])
    p = p.with_(nodes=(vox, sub, val))
    ref = _dense_run_nodes(p, 3)
    got = oracle.run(p, n_steps=3)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    assert got[1].ravel()[n_vox - 1] == 9.0 or p.n_cells  # the later node holds


def test_node_fills_a_closed_box_monotonically():
    """Zero flux, no decay, no cells, one vessel column at V: by the maximum
    principle of the implicit steps every voxel rises monotonically, stays
    in [0, V], and the box fills towards V."""
    p = inputs.make_problem(7, 6, 5, D=1e5, lam=0.0, field_mode="zero")
    p = p.with_(nodes=inputs.vessel_nodes(7, 6, 5, value=38.0))
    prev = p.rho0.copy()
    for _ in range(10):
        cur = oracle.run(p, rho0=prev, n_steps=1)
        assert np.all(cur >= prev - 1e-12) and np.all(cur <= 38.0 + 1e-12)
        prev = cur
    # the deficit decays geometrically (the nodes act between sweeps only)
    d100 = 38.0 - oracle.run(p, n_steps=100).min()
    d400 = 38.0 - oracle.run(p, n_steps=400).min()
    assert 0 < d400 < 1e-3 and d400 < d100 * 1e-2


def test_node_on_shell_at_the_shell_value_changes_nothing():
    p = inputs.make_problem(6, 5, 4, n_sub=1, D=3e4, lam=0.1, bc_kind=[1], bc_value=[38.0],
                            n_cells=5, U=[1.0], S=[0.0], rho_star=[1.0], seed=2)
    q = p.with_(nodes=(np.array([0, 5], dtype=np.int64), np.array([0, 0], dtype=np.int32),
                       np.array([38.0, 38.0])))
    np.testing.assert_array_equal(oracle.run(q, n_steps=4), oracle.run(p, n_steps=4))


def test_nodes_on_dirichlet_faces_dense_lu():
    """Nodes on every face, an edge and a corner of a Dirichlet substrate at
    values other than the boundary's: the node projection follows the shell
    projection, so the solve of the line a face node ends sees the node's
    value there.  Against the dense solves, and the interior next to a face
    node does depend on its value."""
    nx, ny, nz = 5, 6, 4
    p = inputs.make_problem(nx, ny, nz, n_sub=2, D=[1e5, 2e3], lam=[0.1, 0.02],
                            bc_kind=[1, 0], bc_value=[38.0, 0.0], n_cells=4, U=[10.0, 1.0],
                            S=[0.0, 3.0], rho_star=[1.0, 2.0], seed=23)

    def v(x, y, z):
        return x + nx * (y + ny * z)

    faces = [v(0, 2, 1), v(nx - 1, 3, 2), v(2, 0, 2), v(1, ny - 1, 1), v(3, 2, 0),
             v(2, 4, nz - 1), v(0, 0, 2), v(nx - 1, ny - 1, nz - 1)]
    vox = np.array(faces + [v(2, 2, 2)], dtype=np.int64)
    sub = np.zeros(len(vox), dtype=np.int32)
    val = np.array([50.0, 20.0, 60.0, 10.0, 45.0, 30.0, 99.0, 5.0, 40.0])
    q = p.with_(nodes=(vox, sub, val))
    ref = _dense_run_nodes(q, 3)
    got = oracle.run(q, n_steps=3)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    val2 = val.copy()
    val2[0] = 38.0                        # the x = 0 face node at the boundary value
    other = oracle.run(p.with_(nodes=(vox, sub, val2)), n_steps=1)
    first = oracle.run(q, n_steps=1)
    assert abs(first[0, 1, 2, 1] - other[0, 1, 2, 1]) > 1e-3   # its x line's neighbour


# ------------------------------- adjoint of the 2-D variant and of Dirichlet nodes
def _adjoint_ext_problems():
    """A 2-D problem and a 3-D problem with Dirichlet nodes (interior, on a
    Dirichlet face, on a cell's voxel, on the zero-flux substrate)."""
    p2 = inputs.make_problem(7, 6, 1, n_sub=2, D=[2e4, 8e2], lam=[0.2, 0.05],
                             bc_kind=[1, 0], bc_value=[38.0, 0.0], n_cells=7,
                             U=[10.0, 2.0], S=[1.0, 6.0], rho_star=[38.0, 3.0],
                             seed=6, steps=5, dt=0.02, dims=2)
    p3 = _small_adjoint_problem()
    nx, ny = p3.nx, p3.ny

    def v(x, y, z):
        return x + nx * (y + ny * z)

    vox = [v(2, 2, 1), v(0, 2, 2), v(3, 0, 1), oracle.cell_voxel(p3, p3.pos[0]), v(1, 1, 1)]
    sub = [0, 0, 0, 1, 1]
    val = [45.0, 50.0, 20.0, 4.0, 2.5]
    p3 = p3.with_(nodes=(np.array(vox, dtype=np.int64), np.array(sub, dtype=np.int32),
                         np.array(val)))
    return {"2d": p2, "nodes": p3}


@pytest.mark.parametrize("kind", ["2d", "nodes"])
def test_adjoint_ext_field_gradient_dot_product(kind):
    """The 2-D step and the step with nodes are affine in rho as well:
    <dL/drho0, v> = <w, run(rho0 + v) - run(rho0)> for L = <w, rho_final>."""
    p = _adjoint_ext_problems()[kind]
    rng = np.random.default_rng(12)
    w = rng.standard_normal(p.rho0.shape)
    v = rng.standard_normal(p.rho0.shape)
    out = oracle.adjoint(p, w, checkpoint_every=2)
    lhs = np.vdot(out["g0"], v)
    rhs = np.vdot(w, oracle.run(p, rho0=p.rho0 + v) - oracle.run(p))
    assert lhs == pytest.approx(rhs, rel=1e-10)
    np.testing.assert_array_equal(out["rho_final"], oracle.run(p))
    if kind == "nodes":   # a node's value does not depend on the initial field
        n_vox = p.nx * p.ny * p.nz
        vox, sub, _ = p.nodes
        g0 = out["g0"].reshape(p.n_sub, n_vox)
        assert np.all(g0[sub, vox] == 0.0)


@pytest.mark.parametrize("kind", ["2d", "nodes"])
def test_adjoint_ext_parameter_gradients_match_central_differences(kind):
    p = _adjoint_ext_problems()[kind]
    rng = np.random.default_rng(14)
    target = p.rho0 * 0.5 + rng.uniform(0, 1, p.rho0.shape)

    def loss(q):
        return float(((oracle.run(q) - target) ** 2).sum())

    g = 2.0 * (oracle.run(p) - target)
    out = oracle.adjoint(p, g, checkpoint_every=3)
    h_rel = 1e-5
    for s in range(p.n_sub):
        for key, attr in (("dD", "D"), ("dlambda", "lam")):
            base = getattr(p, attr)

            def make(f, s=s, attr=attr, base=base):
                val = base.copy()
                val[s] *= f
                return p.with_(**{attr: val})
            est = (loss(make(1 + h_rel)) - loss(make(1 - h_rel))) / (2 * h_rel * base[s])
            assert out[key][s] == pytest.approx(est, rel=2e-6), (kind, key, s)
    for i in (0, 3, 6):
        for s in range(p.n_sub):
            for key, attr in (("dS", "S"), ("dU", "U")):
                base = getattr(p, attr)
                h = 1e-4 * max(abs(base[i, s]), 1e-2)

                def mk(delta, i=i, s=s, attr=attr, base=base):
                    val = base.copy()
                    val[i, s] += delta
                    return p.with_(**{attr: val})
                est = (loss(mk(h)) - loss(mk(-h))) / (2 * h)
                assert out[key][i, s] == pytest.approx(est, rel=1e-6, abs=1e-9), (kind, key, i, s)


def test_adjoint_ext_without_nodes_is_the_3d_adjoint():
    """oracle_adjoint_ext with dims 3 and no nodes gives oracle_adjoint's bits."""
    p = _small_adjoint_problem()
    rng = np.random.default_rng(3)
    w = rng.standard_normal(p.rho0.shape)
    a = oracle.adjoint(p, w, checkpoint_every=2)
    q = p.with_(nodes=(np.array([0], dtype=np.int64), np.array([0], dtype=np.int32),
                       np.array([38.0])))    # a node on the shell at the shell value
    b = oracle.adjoint(q, w, checkpoint_every=2)
    for k in ("dD", "dlambda", "dS", "dU", "g0", "rho_final"):
        np.testing.assert_array_equal(a[k], b[k])
