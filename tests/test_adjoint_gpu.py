"""GPU adjoint: gradients of a squared-difference loss with respect to D,
lambda and per-cell S and U (and the initial field) against the CPU FP64
oracle adjoint and against central finite differences of the GPU forward."""
import numpy as np
import pytest

import oracle
from paper_2110_13368_gb300 import inputs
from tests.helpers import need_gpu

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
    with the FD evaluated by the GPU forward itself."""
    import torch
    p, q = inputs.adjoint_problem(n=24, n_cells=400, steps=20)
    target = oracle.run(q)

    def loss(pp):
        _, f = gpu_forward(bf, pp)
        return float(((f - target) ** 2).sum())

    sim, fin = gpu_forward(bf, p, record=5)
    out = sim.backward(torch.as_tensor(2.0 * (fin - target), device="cuda"))
    sim.close()
    for key, attr in (("dD", "D"), ("dlambda", "lam")):
        base = getattr(p, attr)
        h = 1e-6 * abs(base[0])
        lp = loss(p.with_(**{attr: base + h}))
        lm = loss(p.with_(**{attr: base - h}))
        est = (lp - lm) / (2 * h)
        assert out[key].cpu().numpy()[0] == pytest.approx(est, rel=1e-4), key
    l0 = loss(p)
    for i in (0, 7, 123):
        for key, attr in (("dS", "S"), ("dU", "U")):
            base = getattr(p, attr)
            h = 1e-6 * max(abs(base[i, 0]), 1.0)
            v1, v2 = base.copy(), base.copy()
            if base[i, 0] - h >= 0:
                v1[i, 0] += h
                v2[i, 0] -= h
                est = (loss(p.with_(**{attr: v1})) - loss(p.with_(**{attr: v2}))) / (2 * h)
            else:
                # S = 0 in this workload: one-sided, second order
                v1[i, 0] += h
                v2[i, 0] += 2 * h
                est = (-3 * l0 + 4 * loss(p.with_(**{attr: v1})) - loss(p.with_(**{attr: v2}))) / (2 * h)
            got = out[key].cpu().numpy()[i, 0]
            assert got == pytest.approx(est, rel=2e-4, abs=1e-6), (key, i, got, est)


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
