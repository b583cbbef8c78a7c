"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Tolerance: per-substrate infinity-norm relative error <= 1e-12 for FP64 and
<= 1e-5 for the FP32 field.  Sizes span several 32-line warp blocks with
ragged tails, lines of length 1 and 2, lines longer than the shared-memory
staging, both sweep forms (plain and rescaled), mid-period reads of the
rescaled field, and Dirichlet and zero-flux substrates side by side.
"""
import numpy as np
import pytest

import oracle
from paper_2110_13368_gb300 import inputs
from tests.helpers import need_gpu, rel_inf, rel_l2

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5


@pytest.fixture(scope="module")
def bf():
    need_gpu()
    from paper_2110_13368_gb300 import build, bfvm
    build.build()
    return bfvm


def run_gpu(bf, p, steps=None, precision=None, variant=None, period=None, graphs=None,
            cells_on_device=True, grid_limit=None, sweep_kernel=None):
    sim = bf.Sim.from_problem(p, precision=precision, cells_on_device=cells_on_device)
    if grid_limit is not None:
        sim.set_option(bf.OPT_GRID_LIMIT, grid_limit)
    if sweep_kernel is not None:
        sim.set_option(bf.OPT_SWEEP_KERNEL, sweep_kernel)
    if variant is not None:
        sim.set_option(bf.OPT_VARIANT, variant)
    if period is not None:
        sim.set_option(bf.OPT_PERIOD, period)
    if graphs is not None:
        sim.set_option(bf.OPT_GRAPHS, graphs)
    sim.step(p.steps if steps is None else steps)
    out = sim.get_density().double().cpu().numpy()
    info = sim.info()
    sim.close()
    return out, info


def mixed(nx, ny, nz, n_cells=200, steps=6, seed=1, **kw):
    args = dict(n_sub=2, D=[1e5, 2e3], lam=[0.1, 0.01], bc_kind=[1, 0],
                bc_value=[38.0, 0.0], n_cells=n_cells, U=[10.0, 0.5], S=[0.0, 10.0],
                rho_star=[1.0, 3.0], steps=steps, seed=seed)
    args.update(kw)
    return inputs.make_problem(nx, ny, nz, **args)


CASES = {
    "ragged_37x45x50": lambda: mixed(37, 45, 50),
    "cube_33": lambda: mixed(33, 33, 33, n_cells=500, steps=9),
    "thin_1x1x7": lambda: mixed(1, 1, 7, n_cells=3),
    "thin_2x3x1": lambda: mixed(2, 3, 1, n_cells=4),
    "thin_5x1x3": lambda: mixed(5, 1, 3, n_cells=4),
    "flat_64x2x40": lambda: mixed(64, 2, 40),
    "long_x_300": lambda: mixed(300, 6, 5, n_cells=50, steps=3),
    "long_z_260": lambda: mixed(9, 7, 260, n_cells=50, steps=3),
    "no_cells_3sub": lambda: inputs.make_problem(23, 17, 29, n_sub=3, D=[1e5, 3e2, 4e4],
                                                 lam=[0.1, 0.0, 0.9], bc_kind=[1, 0, 1],
                                                 bc_value=[38.0, 0.0, 5.0], steps=5, seed=2),
    "plain_50_fullsteps": lambda: inputs.plain_50(),
}


@pytest.mark.parametrize("sweep_kernel", [0, 1])
@pytest.mark.parametrize("grid_limit", [0, 1, 3])
@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("case", sorted(CASES))
def test_fp64_matches_oracle(bf, case, variant, grid_limit, sweep_kernel):
    """grid_limit 1 or 3 caps the persistent sweeps at that many CTAs, so
    every warp (pair) walks many 32-line blocks; sweep_kernel selects the
    warp-pair (0) or one-warp (1) FP64 sweep."""
    p = CASES[case]()
    ref = oracle.run(p)
    got, info = run_gpu(bf, p, variant=variant, grid_limit=grid_limit, sweep_kernel=sweep_kernel)
    assert info["variant"] == variant
    err = rel_inf(got, ref)
    assert np.all(err <= TOL64), (case, variant, err)


FUSED_CASES = ["ragged_37x45x50", "cube_33", "thin_1x1x7", "thin_2x3x1", "flat_64x2x40",
               "long_z_260", "no_cells_3sub", "plain_50_fullsteps"]


# (precision, variant): the rescaled and the plain FP64 form, the FP32 form
FORMS = {"fp64_rescaled": (64, 1), "fp64_plain": (64, 0), "fp32": (32, 0)}


@pytest.mark.parametrize("form", sorted(FORMS))
@pytest.mark.parametrize("grid_limit", [0, 1, 2])
@pytest.mark.parametrize("case", FUSED_CASES)
def test_one_launch_step_matches_per_axis_launches(bf, case, grid_limit, form):
    """The step's three sweeps as one persistent launch (option 8) compute
    each line exactly as the per-axis launches do, so the fields agree bit
    for bit, and both agree with the oracle.  One or two CTAs make every
    pair take many tasks of all three axes, with dependency waits at the
    axis boundaries (single-substrate cases) and pairs of tasks of different
    line lengths (non-cubic grids)."""
    p = CASES[case]()
    ref = oracle.run(p)
    precision, variant = FORMS[form]
    outs, counts = [], []
    for fused in (2, 0):
        sim = bf.Sim.from_problem(p, precision=precision)
        if precision == 64:
            sim.set_option(bf.OPT_VARIANT, variant)
        sim.set_option(bf.OPT_SWEEP_KERNEL, 0)
        sim.set_option(bf.OPT_FUSED_STEP, fused)
        if grid_limit:
            sim.set_option(bf.OPT_GRID_LIMIT, grid_limit)
        n0 = sim.info()["launches"]
        sim.step(p.steps)
        sim.sync()
        launches = sim.info()["launches"] - n0
        outs.append(sim.get_density().cpu().numpy())
        counts.append(launches)
        sim.close()
        assert launches > 0
    assert counts[0] < counts[1]                 # the one launch ran
    np.testing.assert_array_equal(outs[0], outs[1])
    tol = TOL64 if precision == 64 else TOL32
    assert np.all(rel_inf(outs[0].astype(np.float64), ref) <= tol), rel_inf(outs[0], ref)


@pytest.mark.parametrize("precision", [64, 32])
def test_one_launch_step_wait_gives_up_with_status(bf, precision):
    """The dependency waits of the one-launch step are bounded: with option 9
    no wait can be satisfied, each gives up after a few polls, the kernel
    still finishes, and the next synchronising call reports BFVM_ETIMEOUT.
    Normal operation afterwards is unaffected."""
    p = inputs.make_problem(12, 10, 8, n_sub=1, D=[2e4], lam=[0.1], bc_kind=[0],
                            bc_value=[0.0], n_cells=20, U=[1.0], S=[0.5], rho_star=[2.0],
                            steps=2, seed=5)
    sim = bf.Sim.from_problem(p, precision=precision)
    with pytest.raises(bf.BfvmError):
        sim.set_option(bf.OPT_FUSED_STEP, 3)
    sim.set_option(bf.OPT_FUSED_STEP, 2)
    sim.set_option(bf.OPT_WAIT_TEST, 200)
    sim.step(1)
    with pytest.raises(bf.BfvmError) as ei:
        sim.sync()
    assert ei.value.status == 5
    sim.sync()                                   # the flag was cleared
    sim.set_option(bf.OPT_WAIT_TEST, 0)
    torch = __import__("torch")
    sim.set_density(torch.as_tensor(p.rho0, device=sim.device).to(sim.dtype))
    sim.step(p.steps)
    got = sim.get_density().double().cpu().numpy()
    sim.close()
    assert np.all(rel_inf(got, oracle.run(p)) <= (TOL64 if precision == 64 else TOL32))


def test_rescaled_across_periods_and_mid_period_reads(bf):
    """Short rescale period: the renormalising z sweep runs several times and
    the field is read while it still carries a scale."""
    p = mixed(30, 26, 22, n_cells=300, steps=11)
    for steps in (1, 2, 3, 7, 11):
        ref = oracle.run(p, n_steps=steps)
        got, info = run_gpu(bf, p, steps=steps, variant=1, period=3)
        assert info["period"] == 3
        assert np.all(rel_inf(got, ref) <= TOL64), (steps, rel_inf(got, ref))


def test_step_calls_compose(bf):
    """bfvm_step(a); bfvm_step(b) equals bfvm_step(a + b) of the oracle."""
    p = mixed(20, 19, 18, n_cells=100, steps=10)
    ref = oracle.run(p, n_steps=10)
    sim = bf.Sim.from_problem(p)
    sim.set_option(bf.OPT_PERIOD, 4)
    for n in (3, 1, 4, 2):
        sim.step(n)
    got = sim.get_density().cpu().numpy()
    sim.close()
    assert np.all(rel_inf(got, ref) <= TOL64)


def test_graphs_off_matches_graphs_on(bf):
    p = mixed(25, 24, 23, n_cells=150, steps=40)
    a, _ = run_gpu(bf, p, graphs=1)
    b, _ = run_gpu(bf, p, graphs=0)
    np.testing.assert_array_equal(a, b)


def test_deterministic_repeat(bf):
    p = mixed(31, 30, 29, n_cells=400, steps=8)
    a, _ = run_gpu(bf, p)
    b, _ = run_gpu(bf, p)
    np.testing.assert_array_equal(a, b)


def test_host_cells_equal_device_cells(bf):
    p = mixed(19, 21, 17, n_cells=250, steps=4)
    a, _ = run_gpu(bf, p, cells_on_device=True)
    b, _ = run_gpu(bf, p, cells_on_device=False)
    np.testing.assert_array_equal(a, b)


def test_checkpoint_resume_is_bitwise(bf):
    """get_density / set_density round trip is an exact resume (plain form)."""
    p = mixed(24, 22, 20, n_cells=120, steps=6)
    whole, _ = run_gpu(bf, p, variant=0)
    s1 = bf.Sim.from_problem(p)
    s1.set_option(bf.OPT_VARIANT, 0)
    s1.step(2)
    mid = s1.get_density().cpu().numpy()
    s1.close()
    s2 = bf.Sim.from_problem(p.with_(rho0=mid))
    s2.set_option(bf.OPT_VARIANT, 0)
    s2.step(4)
    resumed = s2.get_density().cpu().numpy()
    s2.close()
    np.testing.assert_array_equal(whole, resumed)


def test_co_located_cells_keep_index_order(bf):
    """Many cells in few voxels: the composed maps must follow cell index."""
    p = mixed(6, 5, 4, n_cells=0, steps=3)
    rng = np.random.default_rng(9)
    n = 400
    vox = rng.integers(0, 3, size=(n, 3))
    p.pos = (vox + 0.5) * p.dx
    p.vol = np.full(n, 2494.0)
    p.U = rng.uniform(0, 10, size=(n, 2))
    p.S = rng.uniform(0, 10, size=(n, 2))
    p.rho_star = rng.uniform(0, 40, size=(n, 2))
    ref = oracle.run(p)
    got, _ = run_gpu(bf, p)
    assert np.all(rel_inf(got, ref) <= TOL64)


def test_cells_on_faces_and_domain_max(bf):
    p = mixed(10, 9, 8, n_cells=0, steps=2)
    pos = np.array([[0.0, 0.0, 0.0], [20.0, 40.0, 60.0], [200.0, 180.0, 160.0],
                    [199.999, 0.0, 159.9999], [100.0, 100.0, 100.0]])
    n = len(pos)
    p.pos = pos
    p.vol = np.full(n, 3000.0)
    p.U = np.full((n, 2), 4.0)
    p.S = np.full((n, 2), 2.0)
    p.rho_star = np.full((n, 2), 7.0)
    ref = oracle.run(p)
    got, _ = run_gpu(bf, p)
    assert np.all(rel_inf(got, ref) <= TOL64)


@pytest.mark.parametrize("grid_limit", [0, 1])
@pytest.mark.parametrize("case", ["ragged_37x45x50", "cube_33", "thin_1x1x7", "long_x_300",
                                  "long_z_260", "plain_50_fullsteps"])
def test_fp32_matches_fp64_oracle(bf, case, grid_limit):
    p = CASES[case]()
    ref = oracle.run(p)
    got, info = run_gpu(bf, p, precision=32, grid_limit=grid_limit)
    assert info["precision"] == 32
    err = rel_inf(got, ref)
    assert np.all(err <= TOL32), (case, err, rel_l2(got, ref))


def test_zero_steps_and_empty_cells(bf):
    p = mixed(12, 11, 10, n_cells=0, steps=0)
    got, _ = run_gpu(bf, p, steps=0)
    np.testing.assert_array_equal(got, p.rho0)
    got1, _ = run_gpu(bf, p, steps=2)
    assert np.all(rel_inf(got1, oracle.run(p, n_steps=2)) <= TOL64)


def test_invalid_cells_rejected(bf):
    p = mixed(8, 8, 8, n_cells=5, steps=1)
    sim = bf.Sim.from_problem(p.with_(pos=None))
    bad = p.pos.copy()
    bad[2, 1] = 8 * 20.0 + 1.0
    with pytest.raises(bf.BfvmError) as ei:
        sim.set_cells(bad, p.vol, p.S, p.U, p.rho_star)
    assert ei.value.status == 1
    vol = p.vol.copy()
    vol[0] = 0.0
    with pytest.raises(bf.BfvmError):
        sim.set_cells(p.pos, vol, p.S, p.U, p.rho_star)
    S = p.S.copy()
    S[1, 0] = np.nan
    with pytest.raises(bf.BfvmError):
        sim.set_cells(p.pos, p.vol, S, p.U, p.rho_star)
    rho = p.rho0.copy()
    rho[0, 1, 2, 3] = np.inf
    with pytest.raises(bf.BfvmError) as ei:
        sim.set_density(rho)
    assert ei.value.status == 6
    with pytest.raises(bf.BfvmError) as ei:
        bf.bfvm_backward(sim.handle, np.zeros(p.rho0.shape), 0, np.zeros(2), np.zeros(2),
                         None, None)
    assert ei.value.status == 4
    # the context still works after the rejected calls
    sim.set_cells(p.pos, p.vol, p.S, p.U, p.rho_star)
    sim.step(1)
    got = sim.get_density().cpu().numpy()
    sim.close()
    assert np.all(rel_inf(got, oracle.run(p)) <= TOL64)


# ------------------------------------------------------------ 2-D variant
CASES_2D = {
    "ragged_37x45": lambda: mixed(37, 45, 1, dims=2),
    "thin_1x9": lambda: mixed(1, 9, 1, n_cells=3, dims=2),
    "thin_2x3": lambda: mixed(2, 3, 1, n_cells=4, dims=2),
    "flat_64x2": lambda: mixed(64, 2, 1, dims=2),
    "long_x_300": lambda: mixed(300, 6, 1, n_cells=50, steps=3, dims=2),
    "long_y_1000": lambda: mixed(3, 1000, 1, n_cells=50, steps=3, dims=2),
    "no_cells_3sub": lambda: inputs.make_problem(23, 17, 1, n_sub=3, D=[1e5, 3e2, 4e4],
                                                 lam=[0.1, 0.0, 0.9], bc_kind=[1, 0, 1],
                                                 bc_value=[38.0, 0.0, 5.0], steps=5, seed=2,
                                                 dims=2),
}


@pytest.mark.parametrize("split,grid_limit", [(1, 0), (0, 0), (0, 2)])
@pytest.mark.parametrize("precision,tol", [(64, TOL64), (32, TOL32)])
@pytest.mark.parametrize("case", sorted(CASES_2D))
def test_2d_variant_matches_oracle(bf, case, precision, tol, split, grid_limit):
    """The 2-D variant (option 10): x and y sweeps with half the decay each
    and the four-edge Dirichlet shell, against the 2-D oracle; lines from 1
    voxel to longer than shared memory.  split 1 (the default) runs the
    split line solve, split 0 the warp-pair and one-thread-per-line sweeps
    (grid_limit 2 makes their pairs walk many blocks)."""
    p = CASES_2D[case]()
    ref = oracle.run(p)
    sim = bf.Sim.from_problem(p, precision=precision)
    sim.set_option(bf.OPT_SPLIT, split)
    if grid_limit:
        sim.set_option(bf.OPT_GRID_LIMIT, grid_limit)
    info = sim.info()
    assert info["dims"] == 2 and info["variant"] == 0
    sim.step(p.steps)
    got = sim.get_density().double().cpu().numpy()
    sim.close()
    err = rel_inf(got, ref)
    assert np.all(err <= tol), (case, precision, err)


@pytest.mark.parametrize("precision,tol", [(64, TOL64), (32, TOL32)])
@pytest.mark.parametrize("case", sorted(CASES))
def test_split_line_solve_matches_oracle(bf, case, precision, tol):
    """The split line solve (option 11 = 2) on every 3-D case of the plain
    forms: segments of 8 elements or more (ragged last segments, single
    segments for short lines, up to 38 segments for 300-voxel lines), whole
    shell lines, Dirichlet ends; each axis is joined through the segments'
    end values, so any slip in the scans or the tabulated products shows
    against the oracle."""
    p = CASES[case]()
    ref = oracle.run(p)
    sim = bf.Sim.from_problem(p, precision=precision)
    if precision == 64:
        sim.set_option(bf.OPT_VARIANT, 0)
        sim.set_option(bf.OPT_FUSED_STEP, 0)
    sim.set_option(bf.OPT_SPLIT, 2)
    n0 = sim.info()["launches"]
    sim.step(p.steps)
    sim.sync()
    launches = sim.info()["launches"] - n0
    got = sim.get_density().double().cpu().numpy()
    sim.close()
    assert launches >= 9 * p.steps                # three per axis
    err = rel_inf(got, ref)
    assert np.all(err <= tol), (case, precision, err)


def test_split_option_rules(bf):
    sim = bf.Sim.from_problem(mixed(6, 5, 4))
    for bad in (-1, 3):
        with pytest.raises(bf.BfvmError) as ei:
            sim.set_option(bf.OPT_SPLIT, bad)
        assert ei.value.status == 1
    sim.close()


def test_2d_variant_option_rules(bf):
    p3 = mixed(10, 9, 4)
    sim = bf.Sim.from_problem(p3)
    with pytest.raises(bf.BfvmError) as ei:
        sim.set_option(bf.OPT_DIMS, 2)                  # nz != 1
    assert ei.value.status == 1
    sim.close()
    p = mixed(10, 9, 1, dims=2)
    sim = bf.Sim.from_problem(p)
    with pytest.raises(bf.BfvmError):
        sim.set_option(bf.OPT_VARIANT, 1)               # rescaled form needs the z sweep
    sim.record(2)                                       # the 2-D adjoint records
    with pytest.raises(bf.BfvmError) as ei:
        sim.set_option(bf.OPT_DIMS, 3)                  # not while recording
    assert ei.value.status == 4
    sim.record(0)
    bf.Batch([sim]).close()                             # 2-D members batch
    # back to 3-D on the same single-layer grid: the 3-D step again
    sim.set_option(bf.OPT_DIMS, 3)
    import torch
    sim.set_density(torch.as_tensor(p.rho0, device=sim.device))
    sim.step(p.steps)
    got = sim.get_density().cpu().numpy()
    sim.close()
    ref = oracle.run(p.with_(dims=3))
    assert np.all(rel_inf(got, ref) <= TOL64)


# ---------------------------------------------------- Dirichlet nodes
def _with_nodes(p, extra_dup=True):
    n_vox = p.nx * p.ny * p.nz
    vox, sub, val = inputs.vessel_nodes(p.nx, p.ny, p.nz, substrate=0, value=45.0)
    vox = list(vox) + [0, n_vox // 3]
    sub = list(sub) + [1, 1]
    val = list(val) + [2.0, 7.0]
    if extra_dup:                       # a repeat on one voxel: the later value holds
        vox.append(n_vox // 3)
        sub.append(1)
        val.append(11.0)
    return p.with_(nodes=(np.array(vox, dtype=np.int64), np.array(sub, dtype=np.int32),
                          np.array(val)))


NODE_CASES = {
    "ragged_37x45x50": lambda: _with_nodes(mixed(37, 45, 50)),
    "cube_33": lambda: _with_nodes(mixed(33, 33, 33, n_cells=300, steps=9)),
    "thin_1x1x7": lambda: _with_nodes(mixed(1, 1, 7, n_cells=3)),
    "long_z_260": lambda: _with_nodes(mixed(9, 7, 260, n_cells=50, steps=3)),
}


@pytest.mark.parametrize("precision,variant,period,tol",
                         [(64, 1, 0, TOL64), (64, 1, 3, TOL64), (64, 0, 0, TOL64),
                          (32, None, 0, TOL32)])
@pytest.mark.parametrize("case", sorted(NODE_CASES))
def test_dirichlet_nodes_match_oracle(bf, case, precision, variant, period, tol):
    """Dirichlet nodes (a vessel column, a node on the shell, a repeated
    node) in the rescaled form across rescale periods, the plain form and
    FP32, against the oracle."""
    p = NODE_CASES[case]()
    ref = oracle.run(p)
    sim = bf.Sim.from_problem(p, precision=precision)
    if variant is not None:
        sim.set_option(bf.OPT_VARIANT, variant)
    if period:
        sim.set_option(bf.OPT_PERIOD, period)
    sim.step(p.steps)
    got = sim.get_density().double().cpu().numpy()
    sim.close()
    err = rel_inf(got, ref)
    assert np.all(err <= tol), (case, precision, variant, err)


def test_dirichlet_node_rules(bf):
    p = mixed(10, 9, 8)
    sim = bf.Sim.from_problem(p)
    with pytest.raises(bf.BfvmError) as ei:
        bf.bfvm_set_dirichlet_nodes(sim.handle, [10 * 9 * 8], [0], [1.0])    # voxel out of range
    assert ei.value.status == 1
    with pytest.raises(bf.BfvmError):
        bf.bfvm_set_dirichlet_nodes(sim.handle, [3], [2], [1.0])             # substrate out of range
    with pytest.raises(bf.BfvmError):
        bf.bfvm_set_dirichlet_nodes(sim.handle, [3], [0], [float("nan")])
    bf.bfvm_set_dirichlet_nodes(sim.handle, [3], [0], [1.0])
    sim.record(2)                                                            # nodes record
    bf.bfvm_set_dirichlet_nodes(sim.handle, [4], [1], [2.0])                 # also while recording
    sim.record(0)
    with pytest.raises(bf.BfvmError):
        bf.Batch([sim])
    bf.bfvm_set_dirichlet_nodes(sim.handle, [], [], [])                      # removed again
    sim.record(2)
    sim.close()


# -------------------------------- Dirichlet nodes on shell faces, in one launch
def _with_face_nodes(p):
    """Nodes where the shell and the sweeps meet them: on each face of the
    Dirichlet substrate 0 (a line end of a solved line, at a value other
    than the boundary's), on an edge and a corner, a short interior vessel,
    on cells' voxels, on the zero-flux substrate 1's boundary and inside it,
    and a repeat."""
    nx, ny, nz = p.nx, p.ny, p.nz

    def v(x, y, z):
        return x + nx * (y + ny * z)

    nodes = [
        (v(0, ny // 3, nz // 2), 0, 50.0), (v(nx - 1, ny // 2, nz // 3), 0, 20.0),
        (v(nx // 3, 0, nz // 2), 0, 60.0), (v(nx // 2, ny - 1, 1), 0, 10.0),
        (v(nx // 4, ny // 4, 0), 0, 45.0), (v(nx // 2, ny // 3, nz - 1), 0, 30.0),
        (v(0, 0, nz // 2), 0, 99.0), (v(nx - 1, ny - 1, nz - 1), 0, 5.0),
        (v(0, ny // 2, nz // 4), 1, 7.0), (v(nx // 2, ny // 2, nz // 2), 1, 3.0),
    ]
    nodes += [(v(nx // 2, ny // 2, z), 0, 45.0) for z in range(2, nz - 2)]
    for i in range(min(3, len(p.pos))):      # on cells' voxels, both substrates
        nodes.append((oracle.cell_voxel(p, p.pos[i]), i % 2, 12.0 + i))
    nodes.append((v(nx // 2, ny // 2, nz // 2), 1, 4.0))   # the later one holds
    vox, sub, val = zip(*nodes)
    return p.with_(nodes=(np.array(vox, dtype=np.int64), np.array(sub, dtype=np.int32),
                          np.array(val, dtype=np.float64)))


FACE_NODE_CASES = {
    "ragged_37x45x50": lambda: _with_face_nodes(mixed(37, 45, 50)),
    "cube_33": lambda: _with_face_nodes(mixed(33, 33, 33, n_cells=300, steps=9)),
    "long_z_260": lambda: _with_face_nodes(mixed(9, 7, 260, n_cells=50, steps=3)),
}


@pytest.mark.parametrize("precision,variant,period,tol",
                         [(64, 1, 0, TOL64), (64, 1, 3, TOL64), (64, 0, 0, TOL64),
                          (32, None, 0, TOL32)])
@pytest.mark.parametrize("fused", [1, 0])
@pytest.mark.parametrize("case", sorted(FACE_NODE_CASES))
def test_face_nodes_match_oracle(bf, case, fused, precision, variant, period, tol):
    """Nodes on the Dirichlet shell's faces enter the solve of the line they
    end with their own value; with option 8 at its default the FP64 forms
    run the step as one launch plus the node fill ahead of it."""
    p = FACE_NODE_CASES[case]()
    ref = oracle.run(p)
    sim = bf.Sim.from_problem(p, precision=precision)
    if variant is not None:
        sim.set_option(bf.OPT_VARIANT, variant)
    if period:
        sim.set_option(bf.OPT_PERIOD, period)
    sim.set_option(bf.OPT_FUSED_STEP, fused)
    sim.step(p.steps)
    got = sim.get_density().double().cpu().numpy()
    sim.close()
    err = rel_inf(got, ref)
    assert np.all(err <= tol), (case, fused, precision, variant, err)


@pytest.mark.parametrize("opt,value", [("OPT_SWEEP_KERNEL", 1), ("OPT_SPLIT", 2)])
def test_face_nodes_other_sweep_kernels(bf, opt, value):
    """The one-warp-per-line sweeps and the split line solve take the node
    values at line ends too (plain FP64 form, where the split solve runs)."""
    p = FACE_NODE_CASES["ragged_37x45x50"]()
    ref = oracle.run(p)
    sim = bf.Sim.from_problem(p)
    sim.set_option(bf.OPT_VARIANT, 0)
    sim.set_option(getattr(bf, opt), value)
    sim.step(p.steps)
    got = sim.get_density().cpu().numpy()
    sim.close()
    assert np.all(rel_inf(got, ref) <= TOL64)


@pytest.mark.parametrize("variant,period", [(1, 0), (1, 3), (0, 0)])
@pytest.mark.parametrize("grid_limit", [0, 3])
def test_nodes_one_launch_matches_per_axis_bitwise(bf, variant, period, grid_limit):
    """With nodes the one-launch step (node fill, then one launch) gives the
    per-axis launches' field bit for bit, in fewer launches; CTA caps make
    the warp pairs walk many tasks, so node patches and the epilogue's node
    chunks meet many interleavings."""
    p = _with_face_nodes(mixed(37, 45, 50, steps=7))
    outs, counts = [], []
    for fused in (2, 0):
        sim = bf.Sim.from_problem(p)
        sim.set_option(bf.OPT_VARIANT, variant)
        if period:
            sim.set_option(bf.OPT_PERIOD, period)
        sim.set_option(bf.OPT_FUSED_STEP, fused)
        if grid_limit:
            sim.set_option(bf.OPT_GRID_LIMIT, grid_limit)
        n0 = sim.info()["launches"]
        sim.step(p.steps)
        sim.sync()
        counts.append(sim.info()["launches"] - n0)
        outs.append(sim.get_density().cpu().numpy())
        sim.close()
    assert counts[0] < counts[1]
    np.testing.assert_array_equal(outs[0], outs[1])
    assert np.all(rel_inf(outs[0], oracle.run(p)) <= TOL64)
