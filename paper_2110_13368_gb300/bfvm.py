"""Thin ctypes binding of libbfvm (include/bfvm.h), same names as the C ABI.

Argument marshalling only: every step of the transport path runs in the
library's CUDA kernels.  PyTorch supplies device memory and streams.  If the
compiled library is missing the import of a binding function raises; there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libbfvm.so")

BFVM_OK = 0
STATUS_NAMES = {0: "BFVM_OK", 1: "BFVM_EINVAL", 2: "BFVM_ENOMEM", 3: "BFVM_ECUDA",
                4: "BFVM_ESTATE", 5: "BFVM_ETIMEOUT", 6: "BFVM_ENONFINITE"}
BC_ZERO_FLUX = 0
BC_DIRICHLET = 1

OPT_VARIANT = 1
OPT_PERIOD = 2
OPT_FUSE_SOURCES = 3
OPT_GRAPHS = 4
OPT_TIME_KERNELS = 5
OPT_GRID_LIMIT = 6
OPT_SWEEP_KERNEL = 7
OPT_FUSED_STEP = 8
OPT_WAIT_TEST = 9
OPT_DIMS = 10
OPT_SPLIT = 11

EXPORTED = ["bfvm_create", "bfvm_destroy", "bfvm_set_density", "bfvm_get_density",
            "bfvm_set_cells", "bfvm_step", "bfvm_sync", "bfvm_record", "bfvm_backward",
            "bfvm_last_error", "bfvm_status_string", "bfvm_get_info", "bfvm_set_option",
            "bfvm_kernel_times",
            "bfvm_batch_create", "bfvm_batch_step", "bfvm_batch_sync", "bfvm_batch_destroy",
            "bfvm_batch_last_error", "bfvm_batch_info", "bfvm_batch_shape",
            "bfvm_batch_set_shape", "bfvm_apply_sources_noalloc", "bfvm_set_dirichlet_nodes",
            "bfvm_update_cells", "bfvm_fp64_fma_rate", "bfvm_create_slab", "bfvm_batch_set_option",
            "bfvm_slab_forward", "bfvm_slab_backward", "bfvm_slab_finish"]


class BfvmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None

_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64


def load_library(path: Optional[str] = None):
    """Load libbfvm.so (built by paper_2110_13368_gb300.build)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libbfvm is not built ({p} missing); run "
                               "paper_2110_13368_gb300.build.build() first")
        lib = ctypes.CDLL(p)
        lib.bfvm_create.argtypes = [ctypes.POINTER(_vp), _i32, _i32, _i32, ctypes.c_double,
                                    ctypes.c_double, _i32, _dp, _dp,
                                    ctypes.POINTER(_i32), _dp, _i32, _vp]
        lib.bfvm_destroy.argtypes = [_vp]
        lib.bfvm_destroy.restype = None
        lib.bfvm_set_density.argtypes = [_vp, _vp, _i32]
        lib.bfvm_get_density.argtypes = [_vp, _vp, _i32]
        lib.bfvm_set_cells.argtypes = [_vp, _i64, _vp, _vp, _vp, _vp, _vp, _i32]
        lib.bfvm_update_cells.argtypes = [_vp, _i64, _vp, _vp, _vp, _vp, _vp]
        lib.bfvm_update_cells.restype = ctypes.c_int
        lib.bfvm_set_dirichlet_nodes.argtypes = [_vp, _i64, _vp, _vp, _vp, _i32]
        lib.bfvm_set_dirichlet_nodes.restype = ctypes.c_int
        lib.bfvm_step.argtypes = [_vp, _i32]
        lib.bfvm_sync.argtypes = [_vp]
        lib.bfvm_record.argtypes = [_vp, _i32]
        lib.bfvm_backward.argtypes = [_vp, _vp, _i32, _vp, _vp, _vp, _vp, _vp, _i32]
        lib.bfvm_last_error.argtypes = [_vp]
        lib.bfvm_last_error.restype = ctypes.c_char_p
        lib.bfvm_status_string.argtypes = [_i32]
        lib.bfvm_status_string.restype = ctypes.c_char_p
        lib.bfvm_get_info.argtypes = [_vp, ctypes.POINTER(_i64)]
        lib.bfvm_set_option.argtypes = [_vp, _i32, _i64]
        lib.bfvm_kernel_times.argtypes = [_vp, _vp, _vp, _i32]
        lib.bfvm_batch_create.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i32, _vp]
        lib.bfvm_batch_step.argtypes = [_vp, _i32]
        lib.bfvm_batch_sync.argtypes = [_vp]
        lib.bfvm_batch_destroy.argtypes = [_vp]
        lib.bfvm_batch_destroy.restype = None
        lib.bfvm_batch_last_error.argtypes = [_vp]
        lib.bfvm_batch_last_error.restype = ctypes.c_char_p
        lib.bfvm_batch_info.argtypes = [_vp, ctypes.POINTER(_i64)]
        lib.bfvm_batch_info.restype = ctypes.c_int
        lib.bfvm_batch_shape.argtypes = [_vp, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32), _dp]
        lib.bfvm_batch_shape.restype = ctypes.c_int
        lib.bfvm_batch_set_shape.argtypes = [_vp, _i32, _i32, _i32]
        lib.bfvm_batch_set_shape.restype = ctypes.c_int
        lib.bfvm_batch_set_option.argtypes = [_vp, _i32, _i64]
        lib.bfvm_batch_set_option.restype = ctypes.c_int
        lib.bfvm_apply_sources_noalloc.argtypes = ([_vp] + [_i32] * 4 + [ctypes.c_double] * 2
                                                   + [_i64] + [_vp] * 5 + [_vp])
        lib.bfvm_apply_sources_noalloc.restype = ctypes.c_int
        lib.bfvm_fp64_fma_rate.argtypes = [_i32, _i32, _i64, _vp, _dp, _dp]
        lib.bfvm_fp64_fma_rate.restype = ctypes.c_int
        lib.bfvm_create_slab.argtypes = [ctypes.POINTER(_vp), _i32, _i32, _i32,
                                         ctypes.POINTER(_i32), _i32, ctypes.c_double,
                                         ctypes.c_double, _i32, _dp, _dp, ctypes.POINTER(_i32),
                                         _dp, _vp]
        lib.bfvm_slab_forward.argtypes = [_vp, _vp]
        lib.bfvm_slab_backward.argtypes = [_vp, _vp, _vp]
        lib.bfvm_slab_finish.argtypes = [_vp, _vp]
        for name in ("bfvm_create_slab", "bfvm_slab_forward", "bfvm_slab_backward",
                     "bfvm_slab_finish"):
            getattr(lib, name).restype = ctypes.c_int
        for name in ("bfvm_create", "bfvm_set_density", "bfvm_get_density", "bfvm_set_cells",
                     "bfvm_step", "bfvm_sync", "bfvm_record", "bfvm_backward", "bfvm_get_info",
                     "bfvm_set_option", "bfvm_kernel_times", "bfvm_batch_create", "bfvm_batch_step",
                     "bfvm_batch_sync"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def _check(status: int, handle=None, batch=False):
    if status != BFVM_OK:
        lib = load_library()
        if batch:
            msg = lib.bfvm_batch_last_error(handle)
        else:
            msg = lib.bfvm_last_error(handle)
        raise BfvmError(status, (msg or b"").decode())


def _f64(a, n=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def _ptr(buf):
    """(pointer, on_device, keepalive) for a torch tensor or numpy array."""
    try:
        import torch
        if isinstance(buf, torch.Tensor):
            if not buf.is_contiguous():
                raise ValueError("tensor must be contiguous")
            return ctypes.c_void_p(buf.data_ptr()), int(buf.is_cuda), buf
    except ImportError:  # pragma: no cover
        pass
    arr = np.ascontiguousarray(buf)
    return ctypes.c_void_p(arr.ctypes.data), 0, arr


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


# ------------------------------------------------------------------ C names
def bfvm_create(nx, ny, nz, dx_um, dt_min, D, lam, bc_kind, bc_value, precision=64,
                stream=None):
    lib = load_library()
    n_sub = len(D)
    D = _f64(D, n_sub)
    lam = _f64(lam, n_sub)
    kind = np.ascontiguousarray(np.asarray(bc_kind, dtype=np.int32))
    val = _f64(bc_value, n_sub)
    if kind.size != n_sub:
        raise ValueError("bc_kind length")
    h = _vp()
    st = lib.bfvm_create(ctypes.byref(h), int(nx), int(ny), int(nz), float(dx_um),
                         float(dt_min), n_sub, D.ctypes.data_as(_dp), lam.ctypes.data_as(_dp),
                         kind.ctypes.data_as(ctypes.POINTER(_i32)), val.ctypes.data_as(_dp),
                         int(precision), _stream_handle(stream))
    _check(st, None)
    return h


def bfvm_destroy(h):
    load_library().bfvm_destroy(h)


def bfvm_set_density(h, rho):
    p, dev, keep = _ptr(rho)
    _check(load_library().bfvm_set_density(h, p, dev), h)
    del keep


def bfvm_get_density(h, out):
    p, dev, keep = _ptr(out)
    _check(load_library().bfvm_get_density(h, p, dev), h)
    return out


def bfvm_set_cells(h, pos, vol, S, U, rho_star):
    n = 0 if pos is None else int(np.shape(pos)[0])
    if n == 0:
        _check(load_library().bfvm_set_cells(h, 0, None, None, None, None, None, 0), h)
        return
    ps = [_ptr(a) for a in (pos, vol, S, U, rho_star)]
    devs = {d for _, d, _ in ps}
    if len(devs) != 1:
        raise ValueError("cell arrays must all be on the host or all on the device")
    _check(load_library().bfvm_set_cells(h, n, *[p for p, _, _ in ps], devs.pop()), h)
    del ps


def bfvm_update_cells(h, pos, vol, S, U, rho_star):
    """Re-bin the cells of the last bfvm_set_cells from new device arrays
    (same count), on the stream, without allocating or synchronising."""
    ps = [_ptr(a) for a in (pos, vol, S, U, rho_star)]
    if any(d != 1 for _, d, _ in ps):
        raise ValueError("bfvm_update_cells takes device tensors only")
    n = int(pos.shape[0])
    _check(load_library().bfvm_update_cells(h, n, *[p for p, _, _ in ps]), h)
    del ps


def bfvm_set_dirichlet_nodes(h, voxel, substrate, value):
    """Dirichlet nodes (int64 voxel x + nx (y + ny z), int32 substrate, FP64
    value), all on the host or all on the device; empty arrays remove them."""
    n = 0 if voxel is None else int(np.shape(voxel)[0])
    if n == 0:
        _check(load_library().bfvm_set_dirichlet_nodes(h, 0, None, None, None, 0), h)
        return
    try:
        import torch
        if isinstance(voxel, torch.Tensor):
            ps = [_ptr(voxel.to(torch.int64).contiguous()), _ptr(substrate.to(torch.int32).contiguous()),
                  _ptr(value.to(torch.float64).contiguous())]
        else:
            raise TypeError
    except (ImportError, TypeError):
        ps = [_ptr(np.ascontiguousarray(voxel, dtype=np.int64)),
              _ptr(np.ascontiguousarray(substrate, dtype=np.int32)),
              _ptr(np.ascontiguousarray(value, dtype=np.float64))]
    devs = {d for _, d, _ in ps}
    if len(devs) != 1:
        raise ValueError("node arrays must all be on the host or all on the device")
    _check(load_library().bfvm_set_dirichlet_nodes(h, n, ps[0][0], ps[1][0], ps[2][0],
                                                   devs.pop()), h)
    del ps


def bfvm_step(h, n_steps):
    _check(load_library().bfvm_step(h, int(n_steps)), h)


def bfvm_sync(h):
    _check(load_library().bfvm_sync(h), h)


def bfvm_record(h, checkpoint_every):
    _check(load_library().bfvm_record(h, int(checkpoint_every)), h)


def bfvm_backward(h, g_final, checkpoint_every, dD, dlambda, dS, dU, g0=None):
    ptrs = [_ptr(a) for a in (g_final, dD, dlambda)]
    dev = ptrs[0][1]
    extra = [_ptr(a) if a is not None else (None, dev, None) for a in (dS, dU, g0)]
    for _, d, _ in ptrs + extra:
        if d != dev:
            raise ValueError("all gradient buffers must be on the same side (host or device)")
    _check(load_library().bfvm_backward(h, ptrs[0][0], int(checkpoint_every), ptrs[1][0],
                                        ptrs[2][0], extra[0][0], extra[1][0], extra[2][0], dev), h)
    del ptrs, extra


def bfvm_get_info(h):
    info = (_i64 * 16)()
    _check(load_library().bfvm_get_info(h, info), h)
    keys = ["precision", "nx", "ny", "nz", "n_sub", "pitch", "n_source_voxels",
            "steps_taken", "variant", "period", "launches", "recorded_steps", "dims"]
    return {k: int(info[i]) for i, k in enumerate(keys)}


def bfvm_set_option(h, key, value):
    _check(load_library().bfvm_set_option(h, int(key), int(value)), h)


def bfvm_kernel_times(h, reset=True):
    """(ms[5], launches[5]) per kernel kind: x, y, z sweep, sources and
    shell, and the three sweeps as one launch."""
    ms = (ctypes.c_double * 5)()
    n = (_i64 * 5)()
    _check(load_library().bfvm_kernel_times(h, ms, n, int(bool(reset))), h)
    return list(ms), list(n)


def bfvm_status_string(status):
    return load_library().bfvm_status_string(int(status)).decode()


def bfvm_last_error(h=None):
    return (load_library().bfvm_last_error(h) or b"").decode()


def bfvm_batch_create(handles, stream=None):
    lib = load_library()
    arr = (_vp * len(handles))(*[h.value if isinstance(h, _vp) else h for h in handles])
    b = _vp()
    st = lib.bfvm_batch_create(ctypes.byref(b), arr, len(handles), _stream_handle(stream))
    if st != BFVM_OK:
        raise BfvmError(st, "bfvm_batch_create failed (mixed precision, a member mid-period "
                            "or recording, or out of memory)")
    return b


def bfvm_batch_step(b, n_steps):
    _check(load_library().bfvm_batch_step(b, int(n_steps)), b, batch=True)


def bfvm_batch_sync(b):
    _check(load_library().bfvm_batch_sync(b), b, batch=True)


def bfvm_batch_destroy(b):
    load_library().bfvm_batch_destroy(b)


def bfvm_batch_info(b):
    info = (_i64 * 8)()
    _check(load_library().bfvm_batch_info(b, info), b, batch=True)
    keys = ["members", "precision", "rescaled", "period", "tasks_per_step", "source_entries",
            "launches", "state"]
    return {k: int(info[i]) for i, k in enumerate(keys)}


def bfvm_batch_shape(b, axis):
    """(algo, warps per CTA, [best Thomas ms, best PCR ms]) of an axis; algo
    0 Thomas, 1 PCR; times -1 where not measured."""
    algo, warps = _i32(), _i32()
    ms = (ctypes.c_double * 2)()
    _check(load_library().bfvm_batch_shape(b, int(axis), ctypes.byref(algo), ctypes.byref(warps),
                                           ms), b, batch=True)
    return int(algo.value), int(warps.value), [ms[0], ms[1]]


def bfvm_batch_set_shape(b, axis, algo, warps):
    _check(load_library().bfvm_batch_set_shape(b, int(axis), int(algo), int(warps)), b, batch=True)


BATCH_OPT_ONE_LAUNCH = 1
BATCH_OPT_WAIT_TEST = 2


def bfvm_batch_set_option(b, key, value):
    _check(load_library().bfvm_batch_set_option(b, int(key), int(value)), b, batch=True)


def bfvm_create_slab(nx, ny, z_starts, slab, dx_um, dt_min, D, lam, bc_kind, bc_value,
                     stream=None):
    """Context of z-slab `slab` of a grid decomposed along z (slab j holds
    the global layers [z_starts[j], z_starts[j+1]))."""
    lib = load_library()
    n_sub = len(D)
    zs = np.ascontiguousarray(np.asarray(z_starts, dtype=np.int32))
    D = _f64(D, n_sub)
    lam = _f64(lam, n_sub)
    kind = np.ascontiguousarray(np.asarray(bc_kind, dtype=np.int32))
    val = _f64(bc_value, n_sub)
    h = _vp()
    st = lib.bfvm_create_slab(ctypes.byref(h), int(nx), int(ny), int(zs.size - 1),
                              zs.ctypes.data_as(ctypes.POINTER(_i32)), int(slab), float(dx_um),
                              float(dt_min), n_sub, D.ctypes.data_as(_dp), lam.ctypes.data_as(_dp),
                              kind.ctypes.data_as(ctypes.POINTER(_i32)), val.ctypes.data_as(_dp),
                              _stream_handle(stream))
    _check(st, None)
    return h


def _dev_f64(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 \
            or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def bfvm_slab_forward(h, send):
    """x, y sweeps and the z forward of the slab; send: (n_sub, ny, nx)."""
    _check(load_library().bfvm_slab_forward(h, _dev_f64(send, "send")), h)


def bfvm_slab_backward(h, gathered, send):
    """gathered: (n_slabs, n_sub, ny, nx) of every slab's forward values."""
    _check(load_library().bfvm_slab_backward(h, _dev_f64(gathered, "gathered"),
                                             _dev_f64(send, "send")), h)


def bfvm_slab_finish(h, gathered):
    """gathered: (n_slabs, n_sub, ny, nx) of every slab's backward values."""
    _check(load_library().bfvm_slab_finish(h, _dev_f64(gathered, "gathered")), h)


def bfvm_fp64_fma_rate(warps_per_sm, chains, iters, stream=None):
    """(FP64 FMAs per second, timed ms) of independent FMA chains on every
    SM of the current device (the FP64-pipe roofline's denominator)."""
    rate = ctypes.c_double()
    ms = ctypes.c_double()
    st = load_library().bfvm_fp64_fma_rate(int(warps_per_sm), int(chains), int(iters),
                                           _stream_handle(stream), ctypes.byref(rate),
                                           ctypes.byref(ms))
    _check(st, None)
    return float(rate.value), float(ms.value)


def bfvm_apply_sources_noalloc(rho, nx, ny, nz, dx_um, dt_min, pos, vol, S, U, rho_star,
                               stream=None):
    """Cell source/uptake update on a dense FP64 device field, in place,
    without any device allocation (for callers that must not allocate; see
    include/bfvm.h).  All arrays are contiguous float64 CUDA tensors on one
    device: rho (n_sub, nz, ny, nx), pos (n, 3), vol (n,), S, U and rho_star
    (n, n_sub).  The C entry point takes the sizes on trust, so they are
    checked here, before the call."""
    import torch
    arrs = {"rho": rho, "pos": pos, "vol": vol, "S": S, "U": U, "rho_star": rho_star}
    for name, a in arrs.items():
        if not isinstance(a, torch.Tensor) or not a.is_cuda:
            raise ValueError(f"bfvm_apply_sources_noalloc: {name} must be a CUDA tensor")
        if a.dtype != torch.float64:
            raise ValueError(f"bfvm_apply_sources_noalloc: {name} must be float64, got {a.dtype}")
        if not a.is_contiguous():
            raise ValueError(f"bfvm_apply_sources_noalloc: {name} must be contiguous")
        if a.device != rho.device:
            raise ValueError(f"bfvm_apply_sources_noalloc: {name} is on {a.device}, "
                             f"rho on {rho.device}")
    nx, ny, nz = int(nx), int(ny), int(nz)
    if rho.dim() != 4 or tuple(rho.shape[1:]) != (nz, ny, nx):
        raise ValueError(f"bfvm_apply_sources_noalloc: rho must be (n_sub, {nz}, {ny}, {nx}), "
                         f"got {tuple(rho.shape)}")
    n_sub = int(rho.shape[0])
    if pos.dim() != 2 or pos.shape[1] != 3:
        raise ValueError(f"bfvm_apply_sources_noalloc: pos must be (n, 3), got {tuple(pos.shape)}")
    n_cells = int(pos.shape[0])
    if tuple(vol.shape) != (n_cells,):
        raise ValueError(f"bfvm_apply_sources_noalloc: vol must be ({n_cells},), "
                         f"got {tuple(vol.shape)}")
    for name, a in (("S", S), ("U", U), ("rho_star", rho_star)):
        if tuple(a.shape) != (n_cells, n_sub):
            raise ValueError(f"bfvm_apply_sources_noalloc: {name} must be ({n_cells}, {n_sub}), "
                             f"got {tuple(a.shape)}")
    if torch.cuda.current_device() != rho.device.index:
        raise ValueError("bfvm_apply_sources_noalloc: the tensors' device must be the current "
                         "CUDA device")
    ptrs = [_ptr(a) for a in (rho, pos, vol, S, U, rho_star)]
    st = load_library().bfvm_apply_sources_noalloc(
        ptrs[0][0], nx, ny, nz, n_sub, float(dx_um), float(dt_min), n_cells,
        ptrs[1][0], ptrs[2][0], ptrs[3][0], ptrs[4][0], ptrs[5][0], _stream_handle(stream))
    _check(st, None)
    del ptrs


class Batch:
    """Many Sim members advanced together by the batched launches."""

    def __init__(self, sims, stream=None):
        import torch
        self.sims = list(sims)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.handle = bfvm_batch_create([s.handle for s in self.sims], self.stream)

    def step(self, n=1):
        bfvm_batch_step(self.handle, n)

    def sync(self):
        bfvm_batch_sync(self.handle)

    def info(self):
        return bfvm_batch_info(self.handle)

    def shape(self, axis):
        return bfvm_batch_shape(self.handle, axis)

    def set_option(self, key, value):
        bfvm_batch_set_option(self.handle, key, value)

    def set_shape(self, axis, algo, warps):
        bfvm_batch_set_shape(self.handle, axis, algo, warps)

    def close(self):
        if getattr(self, "handle", None) is not None:
            bfvm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------- convenience
class Sim:
    """One simulation context with torch-owned buffers.

    ``Sim.from_problem(p)`` creates the context for a Problem of
    ``paper_2110_13368_gb300.inputs`` and uploads its field and cells.
    """

    def __init__(self, nx, ny, nz, dx, dt, D, lam, bc_kind, bc_value, precision=64,
                 stream=None, device=None):
        import torch
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else device
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.shape = (len(D), nz, ny, nx)
        self.precision = int(precision)
        self.dtype = torch.float64 if precision == 64 else torch.float32
        self.n_cells = 0
        self.handle = bfvm_create(nx, ny, nz, dx, dt, D, lam, bc_kind, bc_value, precision,
                                  self.stream)

    @classmethod
    def from_problem(cls, p, precision=None, stream=None, cells_on_device=True):
        import torch
        prec = p.precision if precision is None else precision
        s = cls(p.nx, p.ny, p.nz, p.dx, p.dt, p.D, p.lam, p.bc_kind, p.bc_value, prec, stream)
        if getattr(p, "dims", 3) == 2:
            s.set_option(OPT_DIMS, 2)
        if getattr(p, "nodes", None) is not None and len(p.nodes[0]) > 0:
            bfvm_set_dirichlet_nodes(s.handle, *p.nodes)
        s.set_density(torch.as_tensor(p.rho0, dtype=s.dtype, device=s.device))
        if p.n_cells:
            arrs = [p.pos, p.vol, p.S, p.U, p.rho_star]
            if cells_on_device:
                arrs = [torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64,
                                        device=s.device) for a in arrs]
            s.set_cells(*arrs)
        return s

    def set_density(self, rho):
        bfvm_set_density(self.handle, rho)

    def get_density(self, out=None):
        import torch
        if out is None:
            out = torch.empty(self.shape, dtype=self.dtype, device=self.device)
        bfvm_get_density(self.handle, out)
        return out

    def set_cells(self, pos, vol, S, U, rho_star):
        bfvm_set_cells(self.handle, pos, vol, S, U, rho_star)
        self.n_cells = 0 if pos is None else int(pos.shape[0])

    def update_cells(self, pos, vol, S, U, rho_star):
        bfvm_update_cells(self.handle, pos, vol, S, U, rho_star)

    def step(self, n=1):
        bfvm_step(self.handle, n)

    def sync(self):
        bfvm_sync(self.handle)

    def record(self, every):
        bfvm_record(self.handle, every)

    def backward(self, g_final, checkpoint_every=0, want_g0=False):
        import torch
        n_sub = self.shape[0]
        dev = g_final.device
        dD = torch.zeros(n_sub, dtype=torch.float64, device=dev)
        dl = torch.zeros(n_sub, dtype=torch.float64, device=dev)
        dS = torch.zeros((max(self.n_cells, 1), n_sub), dtype=torch.float64, device=dev)
        dU = torch.zeros_like(dS)
        g0 = torch.zeros(self.shape, dtype=torch.float64, device=dev) if want_g0 else None
        bfvm_backward(self.handle, g_final.contiguous(), checkpoint_every, dD, dl, dS, dU, g0)
        out = {"dD": dD, "dlambda": dl, "dS": dS[: self.n_cells], "dU": dU[: self.n_cells]}
        if want_g0:
            out["g0"] = g0
        return out

    def info(self):
        return bfvm_get_info(self.handle)

    def set_option(self, key, value):
        bfvm_set_option(self.handle, key, value)

    def close(self):
        if getattr(self, "handle", None) is not None:
            bfvm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------- autograd
_LOD_FN = None


def _lod_function():
    """torch.autograd.Function around a recorded forward run (bfvm_record +
    bfvm_step) and its hand-written adjoint (bfvm_backward)."""
    global _LOD_FN
    if _LOD_FN is not None:
        return _LOD_FN
    import torch

    class LODRun(torch.autograd.Function):
        @staticmethod
        def forward(ctx, rho0, D, lam, S, U, spec):
            nx, ny, nz = spec["grid"]
            sim = Sim(nx, ny, nz, spec["dx"], spec["dt"], D.detach().cpu().tolist(),
                      lam.detach().cpu().tolist(), spec["bc_kind"], spec["bc_value"], 64,
                      stream=spec.get("stream"), device=rho0.device)
            try:
                sim.set_density(rho0.detach().contiguous())
                if spec["pos"] is not None and spec["pos"].shape[0] > 0:
                    sim.set_cells(spec["pos"], spec["vol"], S.detach().contiguous(),
                                  U.detach().contiguous(), spec["rho_star"])
                sim.record(spec["checkpoint_every"])
                sim.step(spec["steps"])
                out = sim.get_density()
            except Exception:
                sim.close()
                raise
            ctx.sim = sim
            ctx.shapes = (D.shape, lam.shape, S.shape, U.shape)
            return out

        @staticmethod
        def backward(ctx, g):
            sim = ctx.sim
            try:
                grads = sim.backward(g.contiguous().to(torch.float64), want_g0=True)
            finally:
                sim.close()
                ctx.sim = None
            sD, sl, sS, sU = ctx.shapes
            dS = grads["dS"] if sim.n_cells else torch.zeros(sS, dtype=torch.float64, device=g.device)
            dU = grads["dU"] if sim.n_cells else torch.zeros(sU, dtype=torch.float64, device=g.device)
            return (grads["g0"], grads["dD"].reshape(sD), grads["dlambda"].reshape(sl),
                    dS.reshape(sS), dU.reshape(sU), None)

    _LOD_FN = LODRun
    return LODRun


def lod_run(rho0, D, lam, S, U, *, grid, dx, dt, bc_kind, bc_value, pos=None, vol=None,
            rho_star=None, steps=1, checkpoint_every=20, stream=None):
    """Differentiable FP64 run of `steps` LOD steps (Eq. 1) on the GPU.

    rho0 [n_sub, nz, ny, nx], D and lam [n_sub], S and U [n_cells, n_sub]:
    FP64 tensors (rho0, S, U on the GPU) that may require gradients; pos
    [n_cells, 3], vol [n_cells] and rho_star [n_cells, n_sub] are constants.
    Returns the field after the run.  The forward records a checkpoint every
    `checkpoint_every` steps; the backward replays each segment from its
    checkpoint and runs the library's adjoint kernels (bfvm_backward), giving
    d(loss)/d(rho0, D, lambda, S, U).  A context is created per call and
    released by the backward.
    """
    spec = {"grid": tuple(int(v) for v in grid), "dx": float(dx), "dt": float(dt),
            "bc_kind": list(bc_kind), "bc_value": list(bc_value), "pos": pos, "vol": vol,
            "rho_star": rho_star, "steps": int(steps), "checkpoint_every": int(checkpoint_every),
            "stream": stream}
    return _lod_function().apply(rho0, D, lam, S, U, spec)
