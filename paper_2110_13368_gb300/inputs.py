"""Seeded synthetic inputs for the transport step (no step arithmetic here).

Both the library's tests and benchmarks and the CPU oracle's tests draw their
inputs from this module, so that the two sides always see identical arrays.
It holds only random draws and problem descriptions: no line matrix, no
solve, no source formula.

Every generator uses ``numpy.random.default_rng(seed)`` and draws in a fixed
order: initial field, then cell positions, then volumes, then rates.

The five named workloads:

* ``plain_50``     -- 50^3 voxels (dx = 20 um), one substrate
                      (D = 1e5 um^2/min, lambda = 0.1/min), zero-flux,
                      initial field 38 + U(-1, 1), 1000 uniformly placed
                      cells, V = 2494 um^3, U = 10/min, S = 0, dt = 0.01 min,
                      100 steps.
* ``tumour_200``   -- 200^3 voxels, oxygen (D = 1e5, lambda = 0.1, Dirichlet
                      38 on all faces) and a secreted factor (D = 1e3,
                      lambda = 0.01, zero-flux), field starts at 0; 250 000
                      cells uniform in a central sphere of radius 1500 um,
                      V ~ N(2494, 250) (clipped > 0), oxygen U = 10, factor
                      S = 10, rho* = 1; 1000 steps.  This mirrors the
                      paper's cancer-immune sample ("Profiling", "Input
                      Datasets"): oxygen diffusing in from the boundary and
                      consumed by a tumour, plus a tumour-secreted factor.
* ``tumour_200`` in FP32 -- same arrays, precision 32.
* ``batch_256``    -- 256 independent problems, grid edges U{32..96} per axis,
                      1..4 substrates, D log-uniform [1e2, 1e5], lambda
                      log-uniform [1e-3, 1], 1k..20k uniform cells with
                      uptake/secretion log-uniform [0.1, 10]; dx = 20,
                      zero-flux, field 38 + U(-1, 1), V = 2494, rho* = 1,
                      200 steps.
* ``adjoint_100``  -- 100^3, one substrate as ``plain_50`` otherwise, 20 000
                      cells, rho* = 38, 200 steps; the target field comes from
                      the same problem with D, lambda and every U_i multiplied
                      by exp(0.1 z), z ~ N(0, 1) drawn with seed 1.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import List, Optional

import numpy as np

V_CELL = 2494.0


@dataclass
class Problem:
    nx: int
    ny: int
    nz: int
    dx: float
    dt: float
    D: np.ndarray
    lam: np.ndarray
    bc_kind: np.ndarray
    bc_value: np.ndarray
    rho0: np.ndarray                  # [n_sub][nz][ny][nx] float64
    pos: Optional[np.ndarray] = None  # [n][3]
    vol: Optional[np.ndarray] = None  # [n]
    S: Optional[np.ndarray] = None    # [n][n_sub]
    U: Optional[np.ndarray] = None
    rho_star: Optional[np.ndarray] = None
    steps: int = 1
    precision: int = 64
    name: str = ""
    meta: dict = field(default_factory=dict)
    dims: int = 3                     # 2: the 2-D variant (nz == 1, x and y sweeps only)
    nodes: Optional[tuple] = None     # Dirichlet nodes: (voxel x+nx(y+ny z), substrate, value)

    @property
    def n_sub(self) -> int:
        return int(len(self.D))

    @property
    def n_cells(self) -> int:
        return 0 if self.pos is None else int(self.pos.shape[0])

    @property
    def n_vox(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def updates_per_step(self) -> int:
        return self.n_vox * self.n_sub

    def with_(self, **kw) -> "Problem":
        return replace(self, **kw)


def _arr(v, dtype=np.float64):
    return np.ascontiguousarray(np.asarray(v, dtype=dtype))


def uniform_cells(rng, n, extent):
    """n positions uniform in [0, extent) per axis (extent = (Lx, Ly, Lz))."""
    return rng.uniform(0.0, 1.0, size=(n, 3)) * np.asarray(extent, dtype=np.float64)


def sphere_cells(rng, n, centre, radius):
    """n positions uniform in a ball: direction from a normalised N(0,1)^3,
    radius R u^(1/3)."""
    d = rng.standard_normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = radius * rng.uniform(0.0, 1.0, size=n) ** (1.0 / 3.0)
    return np.asarray(centre, dtype=np.float64)[None, :] + d * r[:, None]


def make_problem(nx, ny, nz, *, n_sub=1, D=1e5, lam=0.1, dx=20.0, dt=0.01,
                 bc_kind=0, bc_value=38.0, field_mode="noise", n_cells=0,
                 cell_mode="uniform", sphere_radius=None, vol_mode="fixed",
                 U=10.0, S=0.0, rho_star=38.0, steps=1, seed=0, precision=64,
                 name="custom", dims=3):
    """A generic problem; scalars broadcast over substrates, per-cell rates
    are the given constants broadcast to [n_cells][n_sub]."""
    rng = np.random.default_rng(seed)
    D = _arr(np.broadcast_to(D, (n_sub,)))
    lam = _arr(np.broadcast_to(lam, (n_sub,)))
    kind = _arr(np.broadcast_to(bc_kind, (n_sub,)), np.int32)
    val = _arr(np.broadcast_to(bc_value, (n_sub,)))
    shape = (n_sub, nz, ny, nx)
    if field_mode == "noise":
        rho0 = 38.0 + rng.uniform(-1.0, 1.0, size=shape)
    elif field_mode == "zero":
        rho0 = np.zeros(shape)
    else:
        raise ValueError(field_mode)
    if dims == 2 and nz != 1:
        raise ValueError("the 2-D variant needs nz == 1")
    p = Problem(nx, ny, nz, float(dx), float(dt), D, lam, kind, val, _arr(rho0),
                steps=int(steps), precision=int(precision), name=name, dims=int(dims))
    if n_cells > 0:
        extent = (nx * dx, ny * dx, nz * dx)
        if cell_mode == "uniform":
            pos = uniform_cells(rng, n_cells, extent)
        elif cell_mode == "sphere":
            pos = sphere_cells(rng, n_cells, np.asarray(extent) / 2.0, sphere_radius)
        else:
            raise ValueError(cell_mode)
        if vol_mode == "fixed":
            vol = np.full(n_cells, V_CELL)
        else:
            vol = np.clip(rng.normal(V_CELL, 250.0, size=n_cells), 1e-6, None)
        p.pos = _arr(pos)
        p.vol = _arr(vol)
        p.U = _arr(np.broadcast_to(U, (n_cells, n_sub)))
        p.S = _arr(np.broadcast_to(S, (n_cells, n_sub)))
        p.rho_star = _arr(np.broadcast_to(rho_star, (n_cells, n_sub)))
    return p


def plain_50(seed: int = 0, steps: int = 100) -> Problem:
    return make_problem(50, 50, 50, n_sub=1, D=1e5, lam=0.1, bc_kind=0,
                        field_mode="noise", n_cells=1000, cell_mode="uniform",
                        U=10.0, S=0.0, rho_star=38.0, steps=steps, seed=seed,
                        name="plain_50^3x1_fp64")


def tumour(n: int = 200, n_cells: int = 250_000, radius: float = 1500.0,
           seed: int = 0, steps: int = 1000, precision: int = 64) -> Problem:
    """Oxygen (Dirichlet 38) + secreted factor (zero-flux) on n^3 voxels with a
    central spherical tumour of n_cells cells."""
    p = make_problem(n, n, n, n_sub=2, D=[1e5, 1e3], lam=[0.1, 0.01],
                     bc_kind=[1, 0], bc_value=[38.0, 0.0], field_mode="zero",
                     n_cells=n_cells, cell_mode="sphere", sphere_radius=radius,
                     vol_mode="normal", U=[10.0, 0.0], S=[0.0, 10.0],
                     rho_star=[1.0, 1.0], steps=steps, seed=seed,
                     precision=precision, name=f"tumour_{n}^3x2_fp{precision}")
    return p


def tumour_200(seed: int = 0, steps: int = 1000, precision: int = 64) -> Problem:
    return tumour(200, 250_000, 1500.0, seed=seed, steps=steps, precision=precision)


def batch_256(seed: int = 0, n_inst: int = 256, steps: int = 200,
              precision: int = 64, edge_lo: int = 32, edge_hi: int = 96,
              cells_lo: int = 1000, cells_hi: int = 20000) -> List[Problem]:
    """Independent problems of uneven sizes.  Per instance, draws in order:
    grid edges, substrate count, D, lambda, cell count, then the instance's
    field, positions and rates."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_inst):
        nx, ny, nz = (int(v) for v in rng.integers(edge_lo, edge_hi + 1, size=3))
        n_sub = int(rng.integers(1, 5))
        D = 10.0 ** rng.uniform(2.0, 5.0, size=n_sub)
        lam = 10.0 ** rng.uniform(-3.0, 0.0, size=n_sub)
        n_cells = int(rng.integers(cells_lo, cells_hi + 1))
        rho0 = 38.0 + rng.uniform(-1.0, 1.0, size=(n_sub, nz, ny, nx))
        pos = uniform_cells(rng, n_cells, (nx * 20.0, ny * 20.0, nz * 20.0))
        vol = np.full(n_cells, V_CELL)
        U = 10.0 ** rng.uniform(-1.0, 1.0, size=(n_cells, n_sub))
        S = 10.0 ** rng.uniform(-1.0, 1.0, size=(n_cells, n_sub))
        p = Problem(nx, ny, nz, 20.0, 0.01, _arr(D), _arr(lam),
                    np.zeros(n_sub, np.int32), np.zeros(n_sub), _arr(rho0),
                    pos=_arr(pos), vol=_arr(vol), S=_arr(S), U=_arr(U),
                    rho_star=_arr(np.ones((n_cells, n_sub))), steps=steps,
                    precision=precision, name=f"batch[{k}]")
        out.append(p)
    return out


def adjoint_problem(n: int = 100, n_cells: int = 20_000, steps: int = 200,
                    seed: int = 0, perturb_seed: int = 1):
    """(problem, perturbed problem) for the adjoint workload.  The perturbed
    problem differs only in D, lambda and U (each times exp(0.1 z))."""
    p = make_problem(n, n, n, n_sub=1, D=1e5, lam=0.1, bc_kind=0,
                     field_mode="noise", n_cells=n_cells, cell_mode="uniform",
                     U=10.0, S=0.0, rho_star=38.0, steps=steps, seed=seed,
                     name=f"adjoint_{n}^3x1_fp64")
    rng = np.random.default_rng(perturb_seed)
    zD = rng.standard_normal(p.n_sub)
    zl = rng.standard_normal(p.n_sub)
    zU = rng.standard_normal(p.U.shape)
    q = p.with_(D=_arr(p.D * np.exp(0.1 * zD)), lam=_arr(p.lam * np.exp(0.1 * zl)),
                U=_arr(p.U * np.exp(0.1 * zU)), name=p.name + "_target")
    return p, q


def vessel_nodes(nx, ny, nz, substrate=0, value=38.0, x=None, y=None):
    """A straight vessel along z at (x, y) (default the grid centre): one
    Dirichlet node per voxel of that column holding `substrate` at `value`."""
    x = nx // 2 if x is None else x
    y = ny // 2 if y is None else y
    vox = np.array([x + nx * (y + ny * z) for z in range(nz)], dtype=np.int64)
    return (vox, np.full(nz, substrate, dtype=np.int32), np.full(nz, float(value)))
