"""ctypes binding of libdg.so: same names as include/dg.h, marshalling only.

Host arrays are numpy float64/int32 arrays; device arrays are torch CUDA
tensors (their data pointer is passed with on_device = 1).  Streams are
passed as the integer handle of a torch.cuda.Stream (``stream.cuda_stream``).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

__all__ = ["DG_OK", "DG_PRECISION_FP64", "DG_PRECISION_MIXED", "DG_SOURCE_NONE",
           "DG_SOURCE_MANUFACTURED", "DG_SOURCE_VORTEX", "DgParams", "DGError", "lib", "library_path",
           "dg_create", "dg_destroy", "dg_set_mesh", "dg_set_state", "dg_get_state", "dg_rhs",
           "dg_lsrk_step", "dg_lsrk_steps", "dg_compute_dt", "dg_wall_forces",
           "dg_wall_forces_noalloc", "DG_NOALLOC_MAX_WALL_FACES", "dg_rigid_step",
           "dg_check_finite", "dg_set_source", "dg_node_coords", "dg_reference_operators",
           "dg_kernel_launches", "dg_last_error", "Solver", "EXPORTED", "dg_broken_gradient",
           "dg_set_stage_variant", "dg_stage_variant", "dg_set_fused_steps", "dg_set_barrier_limit",
           "dg_barrier_status", "dg_set_overintegration", "dg_overint_degree",
           "DgCase", "dg_batch_create", "dg_batch_destroy", "dg_batch_last_error",
           "dg_batch_kernel_launches", "dg_batch_stream", "dg_batch_case_size",
           "dg_batch_set_stage_variant", "dg_batch_stage_variant", "dg_batch_set_fused_steps", "dg_batch_node_coords",
           "dg_batch_set_state", "dg_batch_get_state", "dg_batch_run", "dg_batch_reset_history",
           "dg_batch_rigid", "BatchSolver",
           "dg_mlp_create", "dg_mlp_destroy", "dg_mlp_last_error", "dg_mlp_param_count",
           "dg_mlp_kernel_launches", "dg_mlp_set_params", "dg_mlp_get_params", "dg_mlp_forward",
           "dg_mlp_loss_grad", "dg_mlp_train", "dg_mlp_set_fused", "dg_mlp_is_fused", "Mlp"]

DG_OK = 0
DG_PRECISION_FP64, DG_PRECISION_MIXED = 0, 1
DG_SOURCE_NONE, DG_SOURCE_MANUFACTURED, DG_SOURCE_VORTEX = 0, 1, 2
DG_NOALLOC_MAX_WALL_FACES = 16384
STATUS = {0: "DG_OK", -1: "DG_EINVAL", -2: "DG_EMESH", -3: "DG_ECUDA", -4: "DG_ENONFINITE",
          -5: "DG_ETIMEOUT", -6: "DG_EUNSUPPORTED"}

_HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(_HERE, "libdg.so")

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)


class DgParams(C.Structure):
    _fields_ = [("p", C.c_int), ("precision", C.c_int), ("gamma", C.c_double), ("Pr", C.c_double),
                ("mu", C.c_double), ("theta", C.c_double), ("C1", C.c_double),
                ("rho_inf", C.c_double), ("u_inf", C.c_double), ("v_inf", C.c_double),
                ("p_inf", C.c_double), ("adiabatic_zero_heatflux", C.c_int)]


class DgCase(C.Structure):
    """dg_case of include/dg_batch.h."""
    _fields_ = [("p", C.c_int), ("Nv", C.c_int64), ("vx", _dp), ("vy", _dp), ("K", C.c_int64),
                ("EToV", _ip), ("EToE", _ip), ("EToF", _ip), ("bc", _ip), ("mu", C.c_double),
                ("M_r", C.c_double), ("C_r", C.c_double), ("K_r", C.c_double), ("mass", C.c_double),
                ("y0", C.c_double), ("ydot0", C.c_double)]


class DGError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__(f"{STATUS.get(status, status)}: {msg}")


# name -> (restype, argtypes)
EXPORTED = {
    "dg_create": (C.c_int, [C.POINTER(DgParams), C.c_void_p, C.POINTER(C.c_void_p)]),
    "dg_destroy": (C.c_int, [C.c_void_p]),
    "dg_set_mesh": (C.c_int, [C.c_void_p, C.c_int64, _dp, _dp, C.c_int64, _ip, _ip, _ip, _ip]),
    "dg_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "dg_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "dg_rhs": (C.c_int, [C.c_void_p, C.c_double, _dp, C.c_void_p, C.c_int]),
    "dg_lsrk_step": (C.c_int, [C.c_void_p, C.c_double, C.c_double, _dp]),
    "dg_lsrk_steps": (C.c_int, [C.c_void_p, C.c_double, C.c_double, _dp, C.c_int]),
    "dg_compute_dt": (C.c_int, [C.c_void_p, C.c_double, _dp, _dp]),
    "dg_wall_forces": (C.c_int, [C.c_void_p, _dp, _dp]),
    "dg_wall_forces_noalloc": (C.c_int, [C.c_void_p, _dp, _dp]),
    "dg_rigid_step": (C.c_int, [_dp, C.c_double, C.c_double, _dp, _dp]),
    "dg_check_finite": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "dg_set_source": (C.c_int, [C.c_void_p, C.c_int, _dp]),
    "dg_node_coords": (C.c_int, [C.c_void_p, _dp, _dp]),
    "dg_reference_operators": (C.c_int, [C.c_int, _dp, _dp, _dp, _dp, _dp, _ip]),
    "dg_kernel_launches": (C.c_int64, [C.c_void_p]),
    "dg_set_stage_variant": (C.c_int, [C.c_void_p, C.c_int]),
    "dg_stage_variant": (C.c_int, [C.c_void_p]),
    "dg_set_fused_steps": (C.c_int, [C.c_void_p, C.c_int]),
    "dg_set_overintegration": (C.c_int, [C.c_void_p, C.c_int]),
    "dg_overint_degree": (C.c_int, [C.c_int]),
    "dg_set_barrier_limit": (C.c_int, [C.c_void_p, C.c_uint32]),
    "dg_barrier_status": (C.c_int, [C.c_void_p]),
    "dg_last_error": (C.c_char_p, [C.c_void_p]),
    # include/dg_batch.h
    "dg_batch_create": (C.c_int, [C.POINTER(DgParams), C.c_int, C.POINTER(DgCase), C.POINTER(C.c_void_p)]),
    "dg_batch_destroy": (C.c_int, [C.c_void_p]),
    "dg_batch_last_error": (C.c_char_p, [C.c_void_p]),
    "dg_batch_kernel_launches": (C.c_int64, [C.c_void_p]),
    "dg_batch_stream": (C.c_void_p, [C.c_void_p]),
    "dg_batch_set_stage_variant": (C.c_int, [C.c_void_p, C.c_int]),
    "dg_batch_stage_variant": (C.c_int, [C.c_void_p, C.c_int]),
    "dg_batch_set_fused_steps": (C.c_int, [C.c_void_p, C.c_int]),
    "dg_batch_set_fixed_dt": (C.c_int, [C.c_void_p, _dp]),
    "dg_broken_gradient": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int]),
    "dg_batch_case_size": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int)]),
    "dg_batch_node_coords": (C.c_int, [C.c_void_p, C.c_int, _dp, _dp]),
    "dg_batch_set_state": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int]),
    "dg_batch_get_state": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int]),
    "dg_batch_run": (C.c_int, [C.c_void_p, C.c_double, C.c_int, C.c_int, C.c_void_p, C.c_int]),
    "dg_batch_reset_history": (C.c_int, [C.c_void_p]),
    "dg_batch_rigid": (C.c_int, [C.c_void_p, _dp]),
    # include/dg_mlp.h
    "dg_mlp_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_uint64, C.POINTER(C.c_void_p)]),
    "dg_mlp_destroy": (C.c_int, [C.c_void_p]),
    "dg_mlp_last_error": (C.c_char_p, [C.c_void_p]),
    "dg_mlp_param_count": (C.c_int64, [C.c_void_p]),
    "dg_mlp_kernel_launches": (C.c_int64, [C.c_void_p]),
    "dg_mlp_set_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "dg_mlp_get_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "dg_mlp_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "dg_mlp_loss_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "dg_mlp_train": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_float, C.c_void_p]),
    "dg_mlp_set_fused": (C.c_int, [C.c_void_p, C.c_int]),
    "dg_mlp_is_fused": (C.c_int, [C.c_void_p]),
}

_lib = None


def lib():
    """Load libdg.so; raises ImportError if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(library_path):
            raise ImportError(f"libdg.so not built ({library_path}); run "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(library_path)
        for name, (res, args) in EXPORTED.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _dptr(a):
    return a.ctypes.data_as(_dp)


def _arr_ptr(x):
    """(pointer, on_device) of a numpy array or torch tensor of float64."""
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be contiguous float64")
        return x.ctypes.data_as(C.c_void_p), 0
    if hasattr(x, "data_ptr"):
        import torch
        if x.dtype != torch.float64 or not x.is_contiguous():
            raise ValueError("device tensors must be contiguous float64")
        return C.c_void_p(x.data_ptr()), 1 if x.is_cuda else 0
    raise TypeError("expected a numpy array or a torch tensor")


def _check(st, ctx=None):
    if st != DG_OK:
        msg = lib().dg_last_error(ctx).decode() if ctx else ""
        raise DGError(st, msg)


def _vw(vw):
    return _f64(vw if vw is not None else (0.0, 0.0))


# ---- one Python function per C entry point --------------------------------

def dg_create(params: DgParams, stream=0):
    out = C.c_void_p()
    _check(lib().dg_create(C.byref(params), C.c_void_p(int(stream or 0)), C.byref(out)))
    return out


def dg_destroy(ctx):
    return lib().dg_destroy(ctx)


def dg_set_mesh(ctx, vx, vy, EToV, EToE, EToF, bc):
    vx, vy = _f64(vx), _f64(vy)
    EToV, EToE, EToF, bc = _i32(EToV), _i32(EToE), _i32(EToF), _i32(bc)
    _check(lib().dg_set_mesh(ctx, vx.size, _dptr(vx), _dptr(vy), EToV.shape[0],
                             EToV.ctypes.data_as(_ip), EToE.ctypes.data_as(_ip),
                             EToF.ctypes.data_as(_ip), bc.ctypes.data_as(_ip)), ctx)


def dg_set_state(ctx, U):
    ptr, dev = _arr_ptr(U)
    _check(lib().dg_set_state(ctx, ptr, dev), ctx)


def dg_get_state(ctx, U):
    ptr, dev = _arr_ptr(U)
    _check(lib().dg_get_state(ctx, ptr, dev), ctx)


def dg_rhs(ctx, t, vw, out):
    ptr, dev = _arr_ptr(out)
    _check(lib().dg_rhs(ctx, float(t), _dptr(_vw(vw)), ptr, dev), ctx)


def dg_lsrk_step(ctx, t, dt, vw=None):
    _check(lib().dg_lsrk_step(ctx, float(t), float(dt), _dptr(_vw(vw))), ctx)


def dg_lsrk_steps(ctx, t, dt, vw, nsteps):
    _check(lib().dg_lsrk_steps(ctx, float(t), float(dt), _dptr(_vw(vw)), int(nsteps)), ctx)


def dg_compute_dt(ctx, cfl, vw=None):
    out = np.zeros(1)
    _check(lib().dg_compute_dt(ctx, float(cfl), _dptr(_vw(vw)), _dptr(out)), ctx)
    return float(out[0])


def dg_wall_forces(ctx, xc=(0.0, 0.0)):
    out = np.zeros(3)
    _check(lib().dg_wall_forces(ctx, _dptr(_f64(xc)), _dptr(out)), ctx)
    return out


def dg_wall_forces_noalloc(ctx, xc=(0.0, 0.0)):
    """dg_wall_forces without device allocation: the partial sums live in a
    fixed array inside the library (at most DG_NOALLOC_MAX_WALL_FACES wall
    faces; concurrent calls on the GPU race on that array)."""
    out = np.zeros(3)
    _check(lib().dg_wall_forces_noalloc(ctx, _dptr(_f64(xc)), _dptr(out)), ctx)
    return out


def dg_broken_gradient(ctx, gx, gy, impl=0):
    """gx, gy: [K][4][Np] float64 arrays (host numpy or device torch tensors)."""
    px, dx = _arr_ptr(gx)
    py, dy = _arr_ptr(gy)
    if dx != dy:
        raise ValueError("gx and gy must both be on the host or both on the device")
    _check(lib().dg_broken_gradient(ctx, px, py, dx, int(impl)), ctx)


def dg_rigid_step(coeff, F, dt, state):
    """Returns (new_state, v_b); `state` is not modified."""
    st = _f64(state).copy()
    vb = np.zeros(1)
    _check(lib().dg_rigid_step(_dptr(_f64(coeff)), float(F), float(dt), _dptr(st), _dptr(vb)))
    return st, float(vb[0])


def dg_check_finite(ctx):
    ok = C.c_int(0)
    _check(lib().dg_check_finite(ctx, C.byref(ok)), ctx)
    return bool(ok.value)


def dg_set_source(ctx, kind, params=None):
    pa = _f64(params if params is not None else (0.0, 0.0))
    _check(lib().dg_set_source(ctx, int(kind), _dptr(pa)), ctx)


def dg_node_coords(ctx, K, Np):
    x = np.zeros((K, Np))
    y = np.zeros((K, Np))
    _check(lib().dg_node_coords(ctx, _dptr(x), _dptr(y)), ctx)
    return x, y


def dg_reference_operators(p):
    Np, Nfp = (p + 1) * (p + 2) // 2, p + 1
    r, s = np.zeros(Np), np.zeros(Np)
    Dr, Ds = np.zeros((Np, Np)), np.zeros((Np, Np))
    LIFT = np.zeros((Np, 3 * Nfp))
    Fmask = np.zeros((3, Nfp), dtype=np.int32)
    _check(lib().dg_reference_operators(int(p), _dptr(r), _dptr(s), _dptr(Dr), _dptr(Ds), _dptr(LIFT),
                                        Fmask.ctypes.data_as(_ip)))
    return dict(r=r, s=s, Dr=Dr, Ds=Ds, LIFT=LIFT, Fmask=Fmask)


def dg_kernel_launches(ctx):
    return int(lib().dg_kernel_launches(ctx))


def dg_set_stage_variant(ctx, variant):
    _check(lib().dg_set_stage_variant(ctx, int(variant)), ctx)


def dg_stage_variant(ctx):
    return int(lib().dg_stage_variant(ctx))


def dg_set_overintegration(ctx, on):
    _check(lib().dg_set_overintegration(ctx, int(bool(on))), ctx)


def dg_overint_degree(p):
    return int(lib().dg_overint_degree(int(p)))


def dg_set_fused_steps(ctx, on):
    _check(lib().dg_set_fused_steps(ctx, int(bool(on))), ctx)


def dg_set_barrier_limit(ctx, waits):
    _check(lib().dg_set_barrier_limit(ctx, int(waits)), ctx)


def dg_barrier_status(ctx):
    _check(lib().dg_barrier_status(ctx), ctx)


def dg_last_error(ctx):
    return lib().dg_last_error(ctx).decode()


class Solver:
    """A context with a mesh: the C calls as methods (no extra logic)."""

    def __init__(self, mesh, p, precision="fp64", stream=0, gamma=1.4, Pr=0.72, mu=1e-3,
                 C1=0.01, rho_inf=1.0, u_inf=1.0, v_inf=0.0, p_inf=1.0,
                 adiabatic_zero_heatflux=1, theta=0.0):
        prec = {"fp64": DG_PRECISION_FP64, "mixed": DG_PRECISION_MIXED}[precision]
        self.params = DgParams(p, prec, gamma, Pr, mu, theta, C1, rho_inf, u_inf, v_inf, p_inf,
                               int(adiabatic_zero_heatflux))
        self.p, self.K = p, mesh.K
        self.Np = (p + 1) * (p + 2) // 2
        self.ctx = dg_create(self.params, stream)
        dg_set_mesh(self.ctx, mesh.vx, mesh.vy, mesh.EToV, mesh.EToE, mesh.EToF, mesh.bc)

    def __del__(self):
        ctx = getattr(self, "ctx", None)
        if ctx is not None and _lib is not None:
            dg_destroy(ctx)
            self.ctx = None

    @property
    def shape(self):
        return (self.K, 4, self.Np)

    def node_coords(self):
        return dg_node_coords(self.ctx, self.K, self.Np)

    def set_state(self, U):
        dg_set_state(self.ctx, U if not isinstance(U, np.ndarray) else _f64(U))

    def get_state(self, out=None):
        out = np.zeros(self.shape) if out is None else out
        dg_get_state(self.ctx, out)
        return out

    def rhs(self, t=0.0, vw=None, out=None):
        out = np.zeros(self.shape) if out is None else out
        dg_rhs(self.ctx, t, vw, out)
        return out

    def step(self, t, dt, vw=None):
        dg_lsrk_step(self.ctx, t, dt, vw)

    def steps(self, t, dt, nsteps, vw=None):
        dg_lsrk_steps(self.ctx, t, dt, vw, nsteps)

    def dt(self, cfl, vw=None):
        return dg_compute_dt(self.ctx, cfl, vw)

    def wall_forces(self, xc=(0.0, 0.0)):
        return dg_wall_forces(self.ctx, xc)

    def broken_gradient(self, impl=0):
        """(d/dx, d/dy) of the current state, each [K][4][Np] (host arrays)."""
        gx, gy = np.zeros(self.shape), np.zeros(self.shape)
        dg_broken_gradient(self.ctx, gx, gy, impl)
        return gx, gy

    def check_finite(self):
        return dg_check_finite(self.ctx)

    def set_source(self, kind, params=None):
        dg_set_source(self.ctx, kind, params)

    @property
    def launches(self):
        return dg_kernel_launches(self.ctx)

    def set_variant(self, v):
        """Stage-kernel tile shape: 0 = tuned on first step, 1, 2 or 3 forced
        (3: tensor-core warp tiles)."""
        dg_set_stage_variant(self.ctx, v)

    @property
    def variant(self):
        return dg_stage_variant(self.ctx)

    def set_overint(self, on):
        """Cubature-integrated volume term (FP64 path)."""
        dg_set_overintegration(self.ctx, on)

    def set_fused(self, on):
        """One cooperative launch per step (five stages, grid barriers)."""
        dg_set_fused_steps(self.ctx, on)


# ---- include/dg_batch.h ---------------------------------------------------

def _bcheck(st, b=None):
    if st != DG_OK:
        raise DGError(st, lib().dg_batch_last_error(b).decode())


def dg_batch_create(params: DgParams, cases):
    """cases: a sequence of DgCase (their arrays must stay alive during the call)."""
    arr = (DgCase * len(cases))(*cases)
    out = C.c_void_p()
    _bcheck(lib().dg_batch_create(C.byref(params), len(cases), arr, C.byref(out)), None)
    return out


def dg_batch_destroy(b):
    return lib().dg_batch_destroy(b)


def dg_batch_last_error(b):
    return lib().dg_batch_last_error(b).decode()


def dg_batch_kernel_launches(b):
    return int(lib().dg_batch_kernel_launches(b))


def dg_batch_set_stage_variant(b, variant):
    _bcheck(lib().dg_batch_set_stage_variant(b, int(variant)), b)


def dg_batch_stage_variant(b, i):
    return int(lib().dg_batch_stage_variant(b, int(i)))


def dg_batch_set_fused_steps(b, on):
    """0 off, 1 (or True) one cooperative launch per degree group, 2 one for all groups."""
    _bcheck(lib().dg_batch_set_fused_steps(b, int(on)), b)


def dg_batch_set_fixed_dt(b, dt):
    """dt: per-case steps (sequence of ncases floats), or None for the CFL bound."""
    if dt is None:
        _bcheck(lib().dg_batch_set_fixed_dt(b, None), b)
        return
    arr = _f64(dt)
    _bcheck(lib().dg_batch_set_fixed_dt(b, _dptr(arr)), b)


def dg_batch_stream(b):
    """Integer handle of the batch's cudaStream_t."""
    return int(lib().dg_batch_stream(b) or 0)


def dg_batch_case_size(b, i):
    K, p = C.c_int64(0), C.c_int(0)
    _bcheck(lib().dg_batch_case_size(b, int(i), C.byref(K), C.byref(p)), b)
    return int(K.value), int(p.value)


def dg_batch_node_coords(b, i):
    K, p = dg_batch_case_size(b, i)
    Np = (p + 1) * (p + 2) // 2
    x, y = np.zeros((K, Np)), np.zeros((K, Np))
    _bcheck(lib().dg_batch_node_coords(b, int(i), _dptr(x), _dptr(y)), b)
    return x, y


def dg_batch_set_state(b, i, U):
    ptr, dev = _arr_ptr(U)
    _bcheck(lib().dg_batch_set_state(b, int(i), ptr, dev), b)


def dg_batch_get_state(b, i, U):
    ptr, dev = _arr_ptr(U)
    _bcheck(lib().dg_batch_get_state(b, int(i), ptr, dev), b)


def dg_batch_run(b, cfl, nsteps, use_graph=True, hist=None):
    """hist: optional torch CUDA float64 tensor [rows][ncases][8]."""
    hp, rows = None, 0
    if hist is not None:
        ptr, dev = _arr_ptr(hist)
        if not dev:
            raise ValueError("the history must be a device tensor")
        hp, rows = ptr, int(hist.shape[0])
    _bcheck(lib().dg_batch_run(b, float(cfl), int(nsteps), int(bool(use_graph)), hp, rows), b)


def dg_batch_reset_history(b):
    _bcheck(lib().dg_batch_reset_history(b), b)


def dg_batch_rigid(b, ncases):
    out = np.zeros((ncases, 10))
    _bcheck(lib().dg_batch_rigid(b, _dptr(out)), b)
    return out


class BatchSolver:
    """A batch of cases: the dg_batch_* calls as methods.

    Each case is a dict with keys mesh, p, mu, M_r, C_r, K_r, mass and
    optionally y0, ydot0; the other keyword arguments are the shared
    parameters (gamma, Pr, C1, far field, wall flag)."""

    def __init__(self, cases, gamma=1.4, Pr=0.72, C1=0.01, rho_inf=1.0, u_inf=1.0, v_inf=0.0,
                 p_inf=1.0, adiabatic_zero_heatflux=1):
        self.params = DgParams(0, DG_PRECISION_MIXED, gamma, Pr, 0.0, 0.0, C1, rho_inf, u_inf, v_inf,
                               p_inf, int(adiabatic_zero_heatflux))
        keep, descs = [], []
        for c in cases:
            m = c["mesh"]
            arrs = (_f64(m.vx), _f64(m.vy), _i32(m.EToV), _i32(m.EToE), _i32(m.EToF), _i32(m.bc))
            keep.append(arrs)
            vx, vy, EToV, EToE, EToF, bc = arrs
            descs.append(DgCase(int(c["p"]), vx.size, _dptr(vx), _dptr(vy), EToV.shape[0],
                                EToV.ctypes.data_as(_ip), EToE.ctypes.data_as(_ip),
                                EToF.ctypes.data_as(_ip), bc.ctypes.data_as(_ip), float(c["mu"]),
                                float(c["M_r"]), float(c["C_r"]), float(c["K_r"]), float(c["mass"]),
                                float(c.get("y0", 0.0)), float(c.get("ydot0", 0.0))))
        self.ncases = len(descs)
        self.b = dg_batch_create(self.params, descs)
        self.sizes = [dg_batch_case_size(self.b, i) for i in range(self.ncases)]

    def __del__(self):
        b = getattr(self, "b", None)
        if b is not None and _lib is not None:
            dg_batch_destroy(b)
            self.b = None

    def shape(self, i):
        K, p = self.sizes[i]
        return (K, 4, (p + 1) * (p + 2) // 2)

    def node_coords(self, i):
        return dg_batch_node_coords(self.b, i)

    def set_state(self, i, U):
        dg_batch_set_state(self.b, i, U if not isinstance(U, np.ndarray) else _f64(U))

    def get_state(self, i):
        out = np.zeros(self.shape(i))
        dg_batch_get_state(self.b, i, out)
        return out

    def run(self, cfl, nsteps, use_graph=True, hist=None):
        dg_batch_run(self.b, cfl, nsteps, use_graph, hist)

    def reset_history(self):
        dg_batch_reset_history(self.b)

    def rigid(self):
        """[ncases][10]: t, dt, y, y', y'', v_b, Fx, Fy, Mz, frozen."""
        return dg_batch_rigid(self.b, self.ncases)

    @property
    def launches(self):
        return dg_batch_kernel_launches(self.b)

    @property
    def stream(self):
        return dg_batch_stream(self.b)

    def set_variant(self, v):
        dg_batch_set_stage_variant(self.b, v)

    def variant(self, i):
        return dg_batch_stage_variant(self.b, i)

    def set_fused(self, on):
        """Fused steps: 1 = one cooperative launch per degree group and step,
        2 = one cooperative launch for all degree groups, 0 = off."""
        dg_batch_set_fused_steps(self.b, int(on))

    def set_fixed_dt(self, dt):
        """Per-case fixed steps (None: back to the CFL bound)."""
        if dt is not None:
            dt = np.broadcast_to(np.asarray(dt, dtype=np.float64), (self.ncases,))
        dg_batch_set_fixed_dt(self.b, dt)


# ---- include/dg_mlp.h -----------------------------------------------------

def _mcheck(st, m):
    if st != DG_OK:
        raise DGError(st, lib().dg_mlp_last_error(m).decode() if m else "")


def _f32_dev(x):
    """Pointer of a contiguous float32 CUDA tensor; the network runs on its
    own stream, so the caller's stream is synchronised first."""
    import torch
    if not (hasattr(x, "data_ptr") and x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()):
        raise ValueError("expected a contiguous float32 CUDA tensor")
    torch.cuda.current_stream(x.device).synchronize()
    return C.c_void_p(x.data_ptr())


def dg_mlp_create(n_in, width, depth, n_out, max_batch, seed=0):
    out = C.c_void_p()
    _mcheck(lib().dg_mlp_create(int(n_in), int(width), int(depth), int(n_out), int(max_batch), int(seed),
                                C.byref(out)), None)
    return out


def dg_mlp_destroy(m):
    return lib().dg_mlp_destroy(m)


def dg_mlp_last_error(m):
    return lib().dg_mlp_last_error(m).decode()


def dg_mlp_param_count(m):
    return int(lib().dg_mlp_param_count(m))


def dg_mlp_kernel_launches(m):
    return int(lib().dg_mlp_kernel_launches(m))


def dg_mlp_set_params(m, params):
    if isinstance(params, np.ndarray):
        a = np.ascontiguousarray(params, dtype=np.float32)
        _mcheck(lib().dg_mlp_set_params(m, a.ctypes.data_as(C.c_void_p), 0), m)
    else:
        _mcheck(lib().dg_mlp_set_params(m, _f32_dev(params), 1), m)


def dg_mlp_get_params(m):
    out = np.zeros(dg_mlp_param_count(m), dtype=np.float32)
    _mcheck(lib().dg_mlp_get_params(m, out.ctypes.data_as(C.c_void_p), 0), m)
    return out


def dg_mlp_forward(m, X, Y):
    _mcheck(lib().dg_mlp_forward(m, _f32_dev(X), int(X.shape[0]), _f32_dev(Y)), m)


def dg_mlp_loss_grad(m, X, T, grad, loss):
    _mcheck(lib().dg_mlp_loss_grad(m, _f32_dev(X), _f32_dev(T), int(X.shape[0]), _f32_dev(grad), _f32_dev(loss)), m)


def dg_mlp_train(m, X, T, nsteps, lr, loss_hist=None):
    lh = _f32_dev(loss_hist) if loss_hist is not None else None
    _mcheck(lib().dg_mlp_train(m, _f32_dev(X), _f32_dev(T), int(X.shape[0]), int(nsteps), float(lr), lh), m)


def dg_mlp_set_fused(m, on):
    _mcheck(lib().dg_mlp_set_fused(m, 1 if on else 0), m)


def dg_mlp_is_fused(m):
    return bool(lib().dg_mlp_is_fused(m))


class Mlp:
    """The surrogate network: the dg_mlp_* calls as methods (torch CUDA
    float32 tensors in and out)."""

    def __init__(self, n_in, width=128, depth=3, n_out=2, max_batch=8192, seed=0):
        self.n_in, self.n_out = n_in, n_out
        self.m = dg_mlp_create(n_in, width, depth, n_out, max_batch, seed)

    def __del__(self):
        m = getattr(self, "m", None)
        if m is not None and _lib is not None:
            dg_mlp_destroy(m)
            self.m = None

    @property
    def nparams(self):
        return dg_mlp_param_count(self.m)

    def set_params(self, p):
        dg_mlp_set_params(self.m, p)

    def get_params(self):
        return dg_mlp_get_params(self.m)

    def forward(self, X):
        import torch
        Y = torch.empty((X.shape[0], self.n_out), dtype=torch.float32, device=X.device)
        dg_mlp_forward(self.m, X, Y)
        return Y

    def loss_grad(self, X, T):
        import torch
        g = torch.empty(self.nparams, dtype=torch.float32, device=X.device)
        loss = torch.empty(1, dtype=torch.float32, device=X.device)
        dg_mlp_loss_grad(self.m, X, T, g, loss)
        return float(loss.item()), g

    def train(self, X, T, nsteps, lr, out=None):
        """nsteps Adam steps; returns the loss before each step, in `out`
        (a float32 CUDA tensor of at least nsteps values) if given.  Calls
        with the same X, T, out and lr reuse the captured step graph."""
        import torch
        hist = out if out is not None else torch.empty(max(nsteps, 1), dtype=torch.float32, device=X.device)
        if hist.numel() < nsteps or hist.dtype != torch.float32 or not hist.is_contiguous():
            raise ValueError("out must be a contiguous float32 tensor of at least nsteps values")
        dg_mlp_train(self.m, X, T, nsteps, lr, hist)
        return hist[:nsteps]

    @property
    def launches(self):
        return dg_mlp_kernel_launches(self.m)

    @property
    def fused(self):
        """True while the chunked implementation is in use."""
        return dg_mlp_is_fused(self.m)

    @fused.setter
    def fused(self, on):
        dg_mlp_set_fused(self.m, on)
