"""The seeded synthetic workloads match the configurations they stand in for
(grid, substrates, coefficients, boundaries, cells, steps), and a seed fixes
every array.  These are the inputs of the parity tests, the smoke check and
the benchmark, so a drift here would change what every measurement means."""
import numpy as np

from paper_2110_13368_gb300 import inputs


def test_plain_50_config():
    p = inputs.plain_50()
    assert (p.nx, p.ny, p.nz) == (50, 50, 50) and p.rho0.shape == (1, 50, 50, 50)
    assert p.dx == 20.0 and p.dt == 0.01 and p.steps == 100 and p.precision == 64
    assert np.allclose(p.D, [1e5]) and np.allclose(p.lam, [0.1])
    assert list(p.bc_kind) == [0]                                  # zero-flux
    assert p.rho0.min() >= 37.0 and p.rho0.max() <= 39.0          # 38 + U(-1, 1)
    assert abs(p.rho0.mean() - 38.0) < 0.01
    assert p.n_cells == 1000
    assert np.allclose(p.vol, 2494.0)
    assert np.allclose(p.U, 10.0) and np.allclose(p.S, 0.0)
    ext = 50 * 20.0
    assert p.pos.min() >= 0.0 and p.pos.max() <= ext               # uniform in the domain


def test_tumour_200_config():
    p = inputs.tumour_200(steps=1000)
    assert (p.nx, p.ny, p.nz) == (200, 200, 200) and p.rho0.shape == (2, 200, 200, 200)
    assert p.dx == 20.0 and p.dt == 0.01 and p.steps == 1000
    assert np.allclose(p.D, [1e5, 1e3]) and np.allclose(p.lam, [0.1, 0.01])
    assert list(p.bc_kind) == [1, 0] and np.allclose(p.bc_value[0], 38.0)   # oxygen Dirichlet 38
    assert not p.rho0.any()                                        # both start at 0
    assert p.n_cells == 250_000
    centre = np.array([100 * 20.0] * 3)
    r = np.linalg.norm(p.pos - centre, axis=1)
    assert r.max() <= 1500.0                                       # central sphere, radius 1500
    assert r.max() > 1400.0                                        # and it fills the sphere
    assert abs(p.vol.mean() - 2494.0) < 5.0 and abs(p.vol.std() - 250.0) < 5.0   # N(2494, 250)
    assert np.allclose(p.U[:, 0], 10.0) and np.allclose(p.U[:, 1], 0.0)          # oxygen uptake
    assert np.allclose(p.S[:, 0], 0.0) and np.allclose(p.S[:, 1], 10.0)          # factor secretion
    assert np.allclose(p.rho_star, 1.0)


def test_fp32_form_uses_the_same_arrays():
    a, b = inputs.plain_50(), inputs.plain_50()
    assert np.array_equal(a.rho0, b.rho0) and np.array_equal(a.pos, b.pos)
    t64 = inputs.tumour(40, 2000, 300.0, steps=2)
    t32 = inputs.tumour(40, 2000, 300.0, steps=2, precision=32)
    assert t32.precision == 32
    for f in ("rho0", "pos", "vol", "U", "S", "rho_star"):
        assert np.array_equal(getattr(t64, f), getattr(t32, f))


def test_batch_members_draw_from_the_stated_ranges():
    ms = inputs.batch_256(n_inst=12, steps=200)      # the first 12 members of the 256
    assert len(ms) == 12
    for m in ms:
        assert 32 <= min(m.nx, m.ny, m.nz) and max(m.nx, m.ny, m.nz) <= 96
        assert 1 <= m.n_sub <= 4 and m.rho0.shape == (m.n_sub, m.nz, m.ny, m.nx)
        assert np.all((m.D >= 1e2) & (m.D <= 1e5))
        assert np.all((m.lam >= 1e-3) & (m.lam <= 1.0))
        assert 1000 <= m.n_cells <= 20000
        assert np.all((m.U >= 0.1) & (m.U <= 10.0)) and np.all((m.S >= 0.1) & (m.S <= 10.0))
        assert m.dt == 0.01 and m.steps == 200 and not np.any(m.bc_kind)
    assert len({(m.nx, m.ny, m.nz, m.n_sub) for m in ms}) > 6      # uneven sizes
    again = inputs.batch_256(n_inst=12, steps=200)
    assert all(np.array_equal(a.rho0, b.rho0) for a, b in zip(ms, again))


def test_adjoint_problem_and_its_perturbed_target():
    p, q = inputs.adjoint_problem(n=20, n_cells=500, steps=4)
    assert (p.nx, p.ny, p.nz) == (20, 20, 20) and p.n_sub == 1 and p.n_cells == 500
    assert (q.nx, q.ny, q.nz, q.n_cells) == (p.nx, p.ny, p.nz, p.n_cells)
    assert np.array_equal(p.pos, q.pos)                             # same cells
    changed = [f for f in ("D", "lam", "U", "S") if not np.array_equal(getattr(p, f), getattr(q, f))]
    assert changed                                                 # perturbed parameters


def test_seed_fixes_every_array():
    a = inputs.make_problem(9, 8, 7, n_sub=2, D=[1e5, 1e3], lam=[0.1, 0.01], n_cells=40,
                            U=[10.0, 0.5], S=[0.0, 10.0], rho_star=[1.0, 3.0], seed=11)
    b = inputs.make_problem(9, 8, 7, n_sub=2, D=[1e5, 1e3], lam=[0.1, 0.01], n_cells=40,
                            U=[10.0, 0.5], S=[0.0, 10.0], rho_star=[1.0, 3.0], seed=11)
    c = inputs.make_problem(9, 8, 7, n_sub=2, D=[1e5, 1e3], lam=[0.1, 0.01], n_cells=40,
                            U=[10.0, 0.5], S=[0.0, 10.0], rho_star=[1.0, 3.0], seed=12)
    assert np.array_equal(a.rho0, b.rho0) and np.array_equal(a.pos, b.pos)
    assert not np.array_equal(a.pos, c.pos)
