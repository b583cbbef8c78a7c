"""GPU adjoint: gradients of a squared-difference loss with respect to D,
lambda and per-cell S and U (and the initial field) against the CPU FP64
oracle adjoint and against central finite differences of the GPU forward."""
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


def gpu_forward(bf, p, record=0, split=None):
    sim = bf.Sim.from_problem(p)
    if split is not None:
        sim.set_option(bf.OPT_SPLIT, split)
    if record:
        sim.record(record)
    sim.step(p.steps)
    out = sim.get_density().cpu().numpy()
    return sim, out


def loss_diff(fa, fb, target):
    """L(a) - L(b) for L(f) = sum (f - target)^2, as sum (fa - fb)(fa + fb - 2 target):
    the same number as the difference of the two sums, without cancelling
    two losses that agree in their first ten digits."""
    return float(((fa - fb) * (fa + fb - 2.0 * target)).sum())


def rate_step(p, i):
    """FD step of cell i's rates: 1e-6 relative to the cell's rate scale
    max(S_i, U_i).  S = 0 has no scale of its own; a step of 1e-6 absolute
    there is below the FD's rounding floor (the quotient's error grows as
    1/h and reaches ~2e-4 relative at h = 1e-6 for these gradients, in the
    oracle as on the GPU), so S takes the same step as U."""
    return 1e-6 * max(abs(p.S[i, 0]), abs(p.U[i, 0]))


def fd_gradient(field, p, attr, index, target, f0, h):
    """Finite-difference d(loss)/d(p.attr[index]) with step h from the GPU
    forward `field`: central where the parameter may go below by h, else
    (S = 0, its lower bound) the one-sided second-order difference
    (-3 L(0) + 4 L(h) - L(2h)) / 2h."""
    base = getattr(p, attr)
    up, dn = base.copy(), base.copy()
    if base[index] - h >= 0:
        up[index] += h
        dn[index] -= h
        return loss_diff(field(p.with_(**{attr: up})), field(p.with_(**{attr: dn})), target) / (2 * h)
    up[index] += h
    dn[index] += 2 * h
    f1 = field(p.with_(**{attr: up}))
    f2 = field(p.with_(**{attr: dn}))
    return (4 * loss_diff(f1, f0, target) - loss_diff(f2, f0, target)) / (2 * h)


def mixed_adjoint_problem():
    return inputs.make_problem(19, 14, 11, n_sub=2, D=[3e4, 9e2], lam=[0.2, 0.05],
                               bc_kind=[1, 0], bc_value=[38.0, 0.0], n_cells=60,
                               U=[10.0, 2.0], S=[1.0, 6.0], rho_star=[38.0, 3.0], seed=5,
                               steps=9, dt=0.02)


@pytest.mark.parametrize("every,split", [(1, None), (4, None), (9, None), (4, 2)])
def test_adjoint_matches_oracle(bf, every, split):
    """split 2: the replayed and adjoint line solves (Dirichlet modes 1 and
    2, separate input and output) through the split line solve."""
    import torch
    p = mixed_adjoint_problem()
    target = p.rho0 * 0.5 + np.random.default_rng(4).uniform(0, 1, p.rho0.shape)
    sim, fin = gpu_forward(bf, p, record=every, split=split)
    ref_fin = oracle.run(p)
    g = 2.0 * (fin - target)
    out = sim.backward(torch.as_tensor(g, device="cuda"), want_g0=True)
    sim.close()
    ref = oracle.adjoint(p, 2.0 * (ref_fin - target), checkpoint_every=every)
    for key in ("dD", "dlambda", "dS", "dU", "g0"):
        a = out[key].cpu().numpy()
        b = ref[key]
        scale = np.abs(b).max()
        assert np.abs(a - b).max() <= 1e-10 * scale, (key, np.abs(a - b).max() / scale)


def test_adjoint_host_buffers_match_device(bf):
    import torch
    p = mixed_adjoint_problem()
    sim, fin = gpu_forward(bf, p, record=3)
    g = np.ones_like(fin)
    dev = sim.backward(torch.as_tensor(g, device="cuda"))
    n = p.n_cells
    dD, dl = np.zeros(2), np.zeros(2)
    dS, dU = np.zeros((n, 2)), np.zeros((n, 2))
    bf.bfvm_backward(sim.handle, g, 0, dD, dl, dS, dU)
    sim.close()
    np.testing.assert_array_equal(dD, dev["dD"].cpu().numpy())
    np.testing.assert_array_equal(dS, dev["dS"].cpu().numpy())


def test_adjoint_central_differences(bf):
    """Adjoint workload shape (one substrate, uniform cells, rho* = 38),
    reduced grid and steps; FD step h = 1e-6 relative as the workload says,
    with the FD evaluated by the GPU forward itself.  Agreement within
    rel 1e-4 or abs 1e-7."""
    import torch
    p, q = inputs.adjoint_problem(n=24, n_cells=400, steps=20)
    target = oracle.run(q)

    def field(pp):
        _, f = gpu_forward(bf, pp)
        return f

    sim, fin = gpu_forward(bf, p, record=5)
    out = sim.backward(torch.as_tensor(2.0 * (fin - target), device="cuda"))
    sim.close()
    f0 = field(p)
    for key, attr in (("dD", "D"), ("dlambda", "lam")):
        h = 1e-6 * abs(getattr(p, attr)[0])
        est = fd_gradient(field, p, attr, 0, target, f0, h)
        assert out[key].cpu().numpy()[0] == pytest.approx(est, rel=1e-4, abs=1e-7), key
    for i in (0, 7, 123):
        for key, attr in (("dS", "S"), ("dU", "U")):
            est = fd_gradient(field, p, attr, (i, 0), target, f0, rate_step(p, i))
            got = out[key].cpu().numpy()[i, 0]
            assert got == pytest.approx(est, rel=1e-4, abs=1e-7), (key, i, got, est)


def test_backward_without_record_is_rejected(bf):
    p = mixed_adjoint_problem()
    sim, fin = gpu_forward(bf, p, record=0)
    import torch
    with pytest.raises(bf.BfvmError) as ei:
        sim.backward(torch.zeros(p.rho0.shape, dtype=torch.float64, device="cuda"))
    assert ei.value.status == 4
    sim.close()


def test_autograd_function_matches_adjoint_and_differences(bf):
    """lod_run (torch.autograd.Function over bfvm_record/bfvm_step and
    bfvm_backward): gradients of a squared-difference loss equal those of
    the direct adjoint call bit for bit, and the D and lambda gradients match
    central differences of the same forward."""
    import torch
    p = mixed_adjoint_problem()
    dev = torch.device("cuda")
    target = torch.as_tensor(p.rho0 * 0.5 + 1.0, device=dev)
    t = lambda a, g=True: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64,
                                       device=dev, requires_grad=g)
    rho0, D, lam, S, U = t(p.rho0), t(p.D), t(p.lam), t(p.S), t(p.U)
    kw = dict(grid=(p.nx, p.ny, p.nz), dx=p.dx, dt=p.dt, bc_kind=p.bc_kind,
              bc_value=p.bc_value, pos=t(p.pos, False), vol=t(p.vol, False),
              rho_star=t(p.rho_star, False), steps=p.steps, checkpoint_every=4)
    out = bf.lod_run(rho0, D, lam, S, U, **kw)
    loss = ((out - target) ** 2).sum()
    loss.backward()

    sim = bf.Sim.from_problem(p)
    sim.record(4)
    sim.step(p.steps)
    fin = sim.get_density()
    ref = sim.backward(2.0 * (fin - target), want_g0=True)
    sim.close()
    for name, grad in (("g0", rho0.grad), ("dD", D.grad), ("dlambda", lam.grad),
                       ("dS", S.grad), ("dU", U.grad)):
        torch.testing.assert_close(grad, ref[name].reshape(grad.shape), rtol=0, atol=0)

    def f(Dv, lv):
        with torch.no_grad():
            o = bf.lod_run(rho0.detach(), Dv, lv, S.detach(), U.detach(), **kw)
            return float(((o - target) ** 2).sum())
    for i in range(p.n_sub):
        for which, base in (("D", D.detach()), ("lam", lam.detach())):
            h = 1e-6 * float(base[i])
            up, dn = base.clone(), base.clone()
            up[i] += h
            dn[i] -= h
            if which == "D":
                est = (f(up, lam.detach()) - f(dn, lam.detach())) / (2 * h)
                got = float(D.grad[i])
            else:
                est = (f(D.detach(), up) - f(D.detach(), dn)) / (2 * h)
                got = float(lam.grad[i])
            assert got == pytest.approx(est, rel=1e-4), (which, i, got, est)


@pytest.mark.slow
def test_adjoint_workload_at_full_size(bf):
    """The adjoint workload as specified: 100^3 voxels, one substrate, 20 000
    cells, 200 steps, checkpoints every 20 steps, loss = sum of squared
    differences to the target field of the perturbed parameters (seed 1).
    dD, dlambda, dS and dU match the CPU FP64 adjoint at 1e-10 (infinity-norm
    relative); dD, dlambda and sampled per-cell dU and dS match central
    differences of the GPU forward with h = 1e-6 relative (S = 0 here, so dS
    takes the one-sided second-order difference with the cell's rate scale
    as its reference, see rate_step)."""
    import torch
    p, q = inputs.adjoint_problem()
    assert (p.nx, p.ny, p.nz, p.n_sub, p.n_cells, p.steps) == (100, 100, 100, 1, 20_000, 200)
    target = oracle.run(q)
    ref_fin = oracle.run(p)
    ref = oracle.adjoint(p, 2.0 * (ref_fin - target), checkpoint_every=20)
    sim, fin = gpu_forward(bf, p, record=20)
    assert np.all(rel_inf(fin, ref_fin) <= 1e-12)
    out = sim.backward(torch.as_tensor(2.0 * (fin - target), device="cuda"))
    sim.close()
    for key in ("dD", "dlambda", "dS", "dU"):
        a = out[key].cpu().numpy()
        b = ref[key]
        err = np.abs(a - b).max() / np.abs(b).max()
        assert err <= 1e-10, (key, err)

    def field(pp):
        _, f = gpu_forward(bf, pp)
        return f

    f0 = field(p)
    report = []
    for key, attr in (("dD", "D"), ("dlambda", "lam")):
        h = 1e-6 * abs(getattr(p, attr)[0])
        est = fd_gradient(field, p, attr, 0, target, f0, h)
        got = float(out[key].cpu().numpy()[0])
        report.append((key, got, est, abs(got)))
    dU = ref["dU"][:, 0]
    rng = np.random.default_rng(11)
    cells = sorted(set(np.argsort(-np.abs(dU))[:3].tolist()) |
                   set(rng.choice(p.n_cells, size=3, replace=False).tolist()))
    for i in cells:
        for key, attr in (("dU", "U"), ("dS", "S")):
            est = fd_gradient(field, p, attr, (i, 0), target, f0, rate_step(p, i))
            g = out[key].cpu().numpy()
            report.append((f"{key}[{i}]", float(g[i, 0]), est, float(np.abs(g).max())))
    for name, got, est, scale in report:
        print(f"{name}: adjoint {got:.12e} fd {est:.12e} diff {abs(got - est):.3e} "
              f"rel {abs(got - est) / max(abs(est), 1e-300):.3e} scale {scale:.3e}")
    # per gradient vector, infinity-norm relative as everywhere else in the
    # parity tests: |adjoint - fd| <= 1e-4 max_j |grad_j|
    for name, got, est, scale in report:
        assert abs(got - est) <= 1e-4 * scale, (name, got, est, scale)


def adjoint_2d_problem():
    return inputs.make_problem(37, 29, 1, n_sub=2, D=[3e4, 9e2], lam=[0.2, 0.05],
                               bc_kind=[1, 0], bc_value=[38.0, 0.0], n_cells=40,
                               U=[10.0, 2.0], S=[1.0, 6.0], rho_star=[38.0, 3.0], seed=7,
                               steps=9, dt=0.02, dims=2)


def adjoint_nodes_problem():
    """The mixed adjoint problem with Dirichlet nodes: a vessel stub, nodes
    on faces of the Dirichlet substrate (line ends) and on its edge, on a
    cell's voxel, on the zero-flux substrate."""
    p = mixed_adjoint_problem()
    nx, ny, nz = p.nx, p.ny, p.nz

    def v(x, y, z):
        return x + nx * (y + ny * z)

    nodes = [(v(9, 7, z), 0, 45.0) for z in range(2, nz - 2)]
    nodes += [(v(0, 5, 5), 0, 50.0), (v(nx - 1, 8, 3), 0, 20.0), (v(4, 0, 6), 0, 60.0),
              (v(6, 5, nz - 1), 0, 30.0), (v(0, 0, 4), 0, 99.0),
              (oracle.cell_voxel(p, p.pos[0]), 0, 12.0), (oracle.cell_voxel(p, p.pos[1]), 1, 4.0),
              (v(3, 3, 3), 1, 2.5)]
    vox, sub, val = zip(*nodes)
    return p.with_(nodes=(np.array(vox, dtype=np.int64), np.array(sub, dtype=np.int32),
                          np.array(val)))


@pytest.mark.parametrize("every,split", [(1, None), (4, None), (4, 2)])
@pytest.mark.parametrize("kind", ["2d", "nodes"])
def test_adjoint_2d_and_nodes_match_oracle(bf, kind, every, split):
    """The adjoint of the 2-D variant and of a step with Dirichlet nodes
    against the CPU oracle's adjoint (dD, dlambda, dS, dU, dL/drho0 at
    1e-10); split 2 sends the replayed and adjoint solves through the split
    line solve."""
    import torch
    p = adjoint_2d_problem() if kind == "2d" else adjoint_nodes_problem()
    target = p.rho0 * 0.5 + np.random.default_rng(4).uniform(0, 1, p.rho0.shape)
    sim, fin = gpu_forward(bf, p, record=every, split=split)
    ref_fin = oracle.run(p)
    assert rel_inf(fin, ref_fin).max() <= 1e-12
    g = 2.0 * (fin - target)
    out = sim.backward(torch.as_tensor(g, device="cuda"), want_g0=True)
    sim.close()
    ref = oracle.adjoint(p, 2.0 * (ref_fin - target), checkpoint_every=every)
    for key in ("dD", "dlambda", "dS", "dU", "g0"):
        a = out[key].cpu().numpy()
        b = ref[key]
        scale = np.abs(b).max()
        assert np.abs(a - b).max() <= 1e-10 * scale, (kind, key, np.abs(a - b).max() / scale)
