"""Plain FP64 CPU oracle of the LOD diffusion-decay-source step (Eq. 1).

TEST INFRASTRUCTURE ONLY.  Only the tests, the package's ``smoke()`` check and
the CPU-baseline leg of ``bench.py`` import this module.  The library path
never does, and this module imports nothing from the library.

The arithmetic lives in ``oracle.c`` (plain C, FP64, every operation rounded
on its own: the build disables floating-point contraction so that x86 and Arm
hosts give the same bits).  This file builds it with gcc and wraps it with
ctypes.

Functions and the passages they follow:

* ``line_matrix``     -- the per-axis implicit diffusion-decay matrix of Eq. 1
                         (zero-flux cell-centred finite volumes, LOD decay
                         share lambda*dt/3).
* ``tridiag_solve``   -- textbook Thomas algorithm (the x/y/z diffusion
                         sweeps of "Using OpenACC programming model").
* ``apply_dirichlet`` -- the Dirichlet condition of "Elements of Parallelism".
* ``axis_solve``      -- one LOD sweep along one axis.
* ``cell_voxel``      -- voxel of a cell (cell-centred grid, origin 0).
* ``apply_sources``   -- the delta source term of Eq. 1, implicit, cells in
                         ascending index order.
* ``run``             -- n full steps.
* ``adjoint``         -- literal reverse of ``run`` (gradients of a loss with
                         respect to D, lambda, per-cell S and U).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (gcc, OpenMP if present).
    BFVM_ORACLE_LIB names a prebuilt library to load instead (the mutation
    test loads copies of the oracle with planted mistakes that way)."""
    override = os.environ.get("BFVM_ORACLE_LIB")
    if override:
        return override
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
            "-shared", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_line_matrix.argtypes = [ctypes.c_int, ctypes.c_double,
                                               ctypes.c_double, _dp, _dp, _dp]
            lib.oracle_line_matrix.restype = None
            lib.oracle_tridiag_solve.argtypes = [ctypes.c_int, _dp, _dp, _dp,
                                                 _dp, _dp, _dp]
            lib.oracle_tridiag_solve.restype = None
            lib.oracle_apply_dirichlet.argtypes = [ctypes.c_int] * 4 + [_ip, _dp, _dp]
            lib.oracle_apply_dirichlet.restype = None
            lib.oracle_axis_solve.argtypes = ([ctypes.c_int] * 5 + [ctypes.c_double] * 2
                                              + [_dp, _dp, _dp, ctypes.c_int])
            lib.oracle_axis_solve.restype = None
            lib.oracle_cell_voxel.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double, _dp]
            lib.oracle_cell_voxel.restype = ctypes.c_int64
            lib.oracle_apply_sources.argtypes = ([ctypes.c_int] * 4 + [ctypes.c_double] * 2
                                                 + [ctypes.c_int64] + [_dp] * 6)
            lib.oracle_apply_sources.restype = None
            common = ([ctypes.c_int] * 3 + [ctypes.c_double] * 2 + [ctypes.c_int]
                      + [_dp, _dp, _ip, _dp, ctypes.c_int64, _dp, _dp, _dp, _dp, _dp])
            lib.oracle_run.argtypes = common + [ctypes.c_int, ctypes.c_int, _dp]
            lib.oracle_run.restype = ctypes.c_int
            lib.oracle_run_2d.argtypes = common + [ctypes.c_int, ctypes.c_int, _dp]
            lib.oracle_run_2d.restype = ctypes.c_int
            _lp = ctypes.POINTER(ctypes.c_int64)
            lib.oracle_run_nodes.argtypes = (common + [ctypes.c_int64, _lp, _ip, _dp]
                                             + [ctypes.c_int, ctypes.c_int, _dp])
            lib.oracle_run_nodes.restype = ctypes.c_int
            lib.oracle_apply_dirichlet_2d.argtypes = [ctypes.c_int] * 3 + [_ip, _dp, _dp]
            lib.oracle_apply_dirichlet_2d.restype = None
            lib.oracle_axis_solve_2d.argtypes = ([ctypes.c_int] * 4 + [ctypes.c_double] * 2
                                                 + [_dp, _dp, _dp])
            lib.oracle_axis_solve_2d.restype = None
            lib.oracle_adjoint.argtypes = common + [ctypes.c_int] * 3 + [_dp] * 8
            lib.oracle_adjoint.restype = ctypes.c_int
            lib.oracle_adjoint_ext.argtypes = ([ctypes.c_int] + common
                                               + [ctypes.c_int64, _lp, _ip, _dp]
                                               + [ctypes.c_int] * 3 + [_dp] * 8)
            lib.oracle_adjoint_ext.restype = ctypes.c_int
            lib.oracle_max_threads.argtypes = []
            lib.oracle_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def line_matrix(n: int, c: float, ell: float):
    """(lower, diag, upper) of the line matrix along one axis."""
    lib = _load()
    lo, di, up = (np.zeros(n) for _ in range(3))
    lib.oracle_line_matrix(n, c, ell, _d(lo), _d(di), _d(up))
    return lo, di, up


def tridiag_solve(lower, diag, upper, rhs):
    lib = _load()
    lower, diag, upper, rhs = (_f64(v) for v in (lower, diag, upper, rhs))
    n = rhs.shape[0]
    x = np.zeros(n)
    work = np.zeros(n)
    lib.oracle_tridiag_solve(n, _d(lower), _d(diag), _d(upper), _d(rhs), _d(x), _d(work))
    return x


class _Cells:
    def __init__(self, p, n_sub):
        n = 0 if p.pos is None else int(p.pos.shape[0])
        self.n = n
        if n == 0:
            z = np.zeros(1)
            self.pos = np.zeros(3)
            self.vol = z
            self.S = z.copy()
            self.U = z.copy()
            self.rho_star = z.copy()
        else:
            self.pos = _f64(p.pos, (n, 3))
            self.vol = _f64(p.vol, (n,))
            self.S = _f64(p.S, (n, n_sub))
            self.U = _f64(p.U, (n, n_sub))
            self.rho_star = _f64(p.rho_star, (n, n_sub))


def _common(p):
    n_sub = int(len(p.D))
    D = _f64(p.D)
    lam = _f64(p.lam)
    kind = np.ascontiguousarray(p.bc_kind, dtype=np.int32)
    val = _f64(p.bc_value)
    cells = _Cells(p, n_sub)
    keep = (D, lam, kind, val, cells)
    args = [int(p.nx), int(p.ny), int(p.nz), float(p.dx), float(p.dt), n_sub,
            _d(D), _d(lam), kind.ctypes.data_as(_ip), _d(val), ctypes.c_int64(cells.n),
            _d(cells.pos), _d(cells.vol), _d(cells.S), _d(cells.U), _d(cells.rho_star)]
    return args, keep


def run(p, rho0=None, n_steps=None, n_threads: int = 0):
    """Field after n_steps (default p.steps) full steps from rho0 (default p.rho0);
    the 2-D variant (oracle_run_2d) when the problem's `dims` is 2."""
    lib = _load()
    rho = _f64(p.rho0 if rho0 is None else rho0).copy()
    steps = int(p.steps if n_steps is None else n_steps)
    args, keep = _common(p)
    nodes = getattr(p, "nodes", None)
    if nodes is not None and len(nodes[0]) > 0:
        if getattr(p, "dims", 3) == 2:
            raise ValueError("Dirichlet nodes are defined for the 3-D step")
        vox = np.ascontiguousarray(nodes[0], dtype=np.int64)
        sub = np.ascontiguousarray(nodes[1], dtype=np.int32)
        val = _f64(nodes[2])
        rc = lib.oracle_run_nodes(*args, ctypes.c_int64(len(vox)),
                                  vox.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                  sub.ctypes.data_as(_ip), _d(val), steps,
                                  int(n_threads or max_threads()), _d(rho))
        if rc != 0:
            raise ValueError(f"oracle_run_nodes failed ({rc})")
        del keep
        return rho
    fn = lib.oracle_run_2d if getattr(p, "dims", 3) == 2 else lib.oracle_run
    rc = fn(*args, steps, int(n_threads or max_threads()), _d(rho))
    if rc != 0:
        raise ValueError(f"oracle_run failed ({rc})")
    del keep
    return rho


def adjoint(p, g_final, rho0=None, n_steps=None, checkpoint_every: int = 20,
            n_threads: int = 0):
    """Gradients of L given dL/drho_final; returns dict with dD, dlambda, dS, dU, g0, rho_final."""
    lib = _load()
    rho0 = _f64(p.rho0 if rho0 is None else rho0)
    steps = int(p.steps if n_steps is None else n_steps)
    n_sub = len(p.D)
    n = 0 if p.pos is None else int(p.pos.shape[0])
    g_final = _f64(g_final)
    dD = np.zeros(n_sub)
    dl = np.zeros(n_sub)
    dS = np.zeros(max(n, 1) * n_sub)
    dU = np.zeros(max(n, 1) * n_sub)
    g0 = np.zeros_like(rho0)
    fin = np.zeros_like(rho0)
    args, keep = _common(p)
    tail = [steps, int(checkpoint_every), int(n_threads or max_threads()), _d(rho0),
            _d(g_final), _d(dD), _d(dl), _d(dS), _d(dU), _d(g0), _d(fin)]
    nodes = getattr(p, "nodes", None)
    dims = int(getattr(p, "dims", 3))
    if dims == 2 or (nodes is not None and len(nodes[0]) > 0):
        # the 2-D variant, or Dirichlet nodes (oracle_adjoint_ext)
        if nodes is None or len(nodes[0]) == 0:
            vox = np.zeros(1, dtype=np.int64)
            sub = np.zeros(1, dtype=np.int32)
            val = np.zeros(1)
            n_nodes = 0
        else:
            vox = np.ascontiguousarray(nodes[0], dtype=np.int64)
            sub = np.ascontiguousarray(nodes[1], dtype=np.int32)
            val = _f64(nodes[2])
            n_nodes = len(vox)
        rc = lib.oracle_adjoint_ext(dims, *args, ctypes.c_int64(n_nodes),
                                    vox.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                    sub.ctypes.data_as(_ip), _d(val), *tail)
    else:
        rc = lib.oracle_adjoint(*args, *tail)
    if rc != 0:
        raise ValueError(f"oracle_adjoint failed ({rc})")
    del keep
    return {"dD": dD, "dlambda": dl, "dS": dS[: n * n_sub].reshape(n, n_sub),
            "dU": dU[: n * n_sub].reshape(n, n_sub), "g0": g0, "rho_final": fin}


def apply_dirichlet(p, rho):
    lib = _load()
    rho = _f64(rho).copy()
    kind = np.ascontiguousarray(p.bc_kind, dtype=np.int32)
    val = _f64(p.bc_value)
    lib.oracle_apply_dirichlet(int(p.nx), int(p.ny), int(p.nz), len(p.D),
                               kind.ctypes.data_as(_ip), _d(val), _d(rho))
    return rho


def axis_solve(p, rho, axis: int, n_threads: int = 1):
    lib = _load()
    rho = _f64(rho).copy()
    D = _f64(p.D)
    lam = _f64(p.lam)
    lib.oracle_axis_solve(int(axis), int(p.nx), int(p.ny), int(p.nz), len(p.D),
                          float(p.dx), float(p.dt), _d(D), _d(lam), _d(rho), int(n_threads))
    return rho


def cell_voxel(p, pos) -> int:
    lib = _load()
    pos = _f64(pos, (3,))
    return int(lib.oracle_cell_voxel(int(p.nx), int(p.ny), int(p.nz), float(p.dx), _d(pos)))


def apply_sources(p, rho):
    lib = _load()
    rho = _f64(rho).copy()
    n_sub = len(p.D)
    cells = _Cells(p, n_sub)
    lib.oracle_apply_sources(int(p.nx), int(p.ny), int(p.nz), n_sub, float(p.dx),
                             float(p.dt), ctypes.c_int64(cells.n), _d(cells.pos),
                             _d(cells.vol), _d(cells.S), _d(cells.U),
                             _d(cells.rho_star), _d(rho))
    return rho


def apply_dirichlet_2d(p, rho):
    """The 2-D Dirichlet shell (the four edges of an nx x ny x 1 grid)."""
    lib = _load()
    rho = _f64(rho).copy()
    kind = np.ascontiguousarray(p.bc_kind, dtype=np.int32)
    val = _f64(p.bc_value)
    lib.oracle_apply_dirichlet_2d(int(p.nx), int(p.ny), len(p.D), kind.ctypes.data_as(_ip),
                                  _d(val), _d(rho))
    return rho


def axis_solve_2d(p, rho, axis: int):
    """One 2-D line solve (decay share lambda dt / 2) along x (0) or y (1)."""
    lib = _load()
    rho = _f64(rho).copy()
    D = _f64(p.D)
    lam = _f64(p.lam)
    lib.oracle_axis_solve_2d(int(axis), int(p.nx), int(p.ny), len(p.D), float(p.dx),
                             float(p.dt), _d(D), _d(lam), _d(rho))
    return rho
