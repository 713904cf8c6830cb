"""CPU oracle for the nodal IP-DG Navier-Stokes right-hand side and LSRK step.

Oracle header: this package is test infrastructure.  It is a plain, slow,
FP64 statement of the method (paper Sec. 2) used only by ``tests/``, the
smoke check and the CPU-baseline leg of ``bench.py``.  It shares no code with
the CUDA library: the reference operators come from ``refelem`` (numpy /
scipy), the geometry and face matching from ``geometry`` and the per-node
arithmetic from ``dg_oracle.c`` compiled by ``build_oracle()``.

Functions without an independent pin are marked "parity unpinned" in their
docstrings; every other function is pinned by the CPU tests.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

from . import refelem, geometry

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_dp = C.POINTER(C.c_double)
_lp = C.POINTER(C.c_longlong)


def build_oracle(force: bool = False) -> str:
    """Compile dg_oracle.c into oracle/liboracle.so (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
               "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build_oracle()
        L = C.CDLL(_LIB)
        L.oracle_rhs.argtypes = [C.c_void_p, _dp, C.c_double, _dp, _dp]
        L.oracle_lsrk_step.argtypes = [C.c_void_p, _dp, C.c_double, C.c_double, _dp]
        L.oracle_face_sigma.argtypes = [C.c_void_p, _dp, _dp, _dp]
        L.oracle_broken_gradient.argtypes = [C.c_void_p, _dp, _dp, _dp]
        L.oracle_dt.argtypes = [C.c_void_p, _dp, C.c_double, _dp, _dp, _dp]
        L.oracle_wall_forces.argtypes = [C.c_void_p, _dp, _dp, _dp]
        L.oracle_penalty_norm.argtypes = [_dp, _dp, C.c_double, C.c_double, C.c_double]
        L.oracle_penalty_norm.restype = C.c_double
        L.oracle_roe.argtypes = [_dp, _dp, _dp, _dp, C.c_double, _dp, _dp, _dp]
        L.oracle_flux_n.argtypes = [_dp, _dp, _dp, C.c_double, _dp]
        L.oracle_G_blocks.argtypes = [_dp, C.c_double, C.c_double, C.c_double, _dp]
        L.oracle_newmark_step.argtypes = [_dp, C.c_double, C.c_double, _dp, _dp]
        L.oracle_lsrk_coeffs.argtypes = [_dp, _dp, _dp]
        L.oracle_manufactured_source.argtypes = [C.c_double] * 7 + [_dp]
        L.oracle_set_threads.argtypes = [C.c_int]
        L.oracle_get_threads.restype = C.c_int
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


class _Problem(C.Structure):
    _fields_ = [("p", C.c_int), ("Np", C.c_int), ("Nfp", C.c_int), ("K", C.c_int),
                ("Dr", _dp), ("Ds", _dp), ("Mhat", _dp), ("Minv", _dp),
                ("Fmask", _lp), ("M1D", _dp),
                ("rx", _dp), ("ry", _dp), ("sx", _dp), ("sy", _dp), ("J", _dp),
                ("nx", _dp), ("ny", _dp), ("sJ", _dp),
                ("EToE", _lp), ("EToF", _lp), ("bc", _lp), ("mapP", _lp),
                ("x", _dp), ("y", _dp),
                ("gamma", C.c_double), ("Pr", C.c_double), ("mu", C.c_double),
                ("theta", C.c_double), ("C1", C.c_double),
                ("rho_inf", C.c_double), ("u_inf", C.c_double), ("v_inf", C.c_double),
                ("p_inf", C.c_double), ("adiabatic_zero_heatflux", C.c_longlong),
                ("source_kind", C.c_longlong), ("src_kappa", C.c_double), ("src_C2", C.c_double),
                ("Nq", C.c_longlong), ("Vq", _dp), ("Vqr", _dp), ("Vqs", _dp), ("wq", _dp)]


class Problem:
    """A mesh, a polynomial degree and the physical parameters, ready for the
    oracle's C routines.  State arrays are float64 [K][4][Np]."""

    def __init__(self, mesh, p, gamma=1.4, Pr=0.72, mu=1e-3, C1=0.01, theta=0.0,
                 rho_inf=1.0, u_inf=1.0, v_inf=0.0, p_inf=1.0, adiabatic_zero_heatflux=1,
                 source=None, overint=0):
        if not 1 <= p <= 6:
            raise ValueError("oracle supports 1 <= p <= 6")
        ops = refelem.operators(p)
        self.ops = ops
        self.p, self.Np, self.Nfp, self.K = p, ops["Np"], ops["Nfp"], mesh.K
        geo = geometry.element_geometry(mesh.vx, mesh.vy, mesh.EToV, ops["r"], ops["s"])
        self.geo = geo
        mapP, worst = geometry.match_face_nodes(geo["x"], geo["y"], ops["Fmask"],
                                                mesh.EToE, mesh.EToF, mesh.bc)
        self.match_error = worst
        self.mesh = mesh
        keep = dict(Dr=_f64(ops["Dr"]), Ds=_f64(ops["Ds"]), Mhat=_f64(ops["M"]),
                    Minv=_f64(ops["Minv"]), Fmask=_i64(ops["Fmask"]), M1D=_f64(ops["M1D"]),
                    rx=_f64(geo["rx"]), ry=_f64(geo["ry"]), sx=_f64(geo["sx"]),
                    sy=_f64(geo["sy"]), J=_f64(geo["J"]), nx=_f64(geo["nx"]),
                    ny=_f64(geo["ny"]), sJ=_f64(geo["sJ"]), EToE=_i64(mesh.EToE),
                    EToF=_i64(mesh.EToF), bc=_i64(mesh.bc), mapP=_i64(mapP),
                    x=_f64(geo["x"]), y=_f64(geo["y"]))
        self._keep = keep
        s = _Problem()
        s.p, s.Np, s.Nfp, s.K = p, self.Np, self.Nfp, self.K
        for name, arr in keep.items():
            ptr = arr.ctypes.data_as(_lp if arr.dtype == np.int64 else _dp)
            setattr(s, name, ptr)
        s.gamma, s.Pr, s.mu, s.theta, s.C1 = gamma, Pr, mu, theta, C1
        s.rho_inf, s.u_inf, s.v_inf, s.p_inf = rho_inf, u_inf, v_inf, p_inf
        s.adiabatic_zero_heatflux = int(adiabatic_zero_heatflux)
        self.vortex = None
        if source is not None and source[0] == "vortex":
            # ("vortex", beta, x0, y0, L, u0, v0): S = -div F_v of the advected
            # vortex, added on the Python side (vortex_source.py)
            b, x0, y0, L, u0, v0 = (float(q) for q in source[1:7])
            self.vortex = dict(beta=b, center=(x0, y0), L=L, u0=u0, v0=v0)
        elif source is not None:        # ("manufactured", kappa, C2) of Sec. 3.1
            s.source_kind, s.src_kappa, s.src_C2 = 1, float(source[1]), float(source[2])
        if overint:                     # volume flux integrated with cubature(overint)
            oi = refelem.overint_operators(p, int(overint))
            for name in ("Vq", "Vqr", "Vqs", "wq"):
                keep[name] = _f64(oi[name])
                setattr(s, name, keep[name].ctypes.data_as(_dp))
            s.Nq = int(oi["Nq"])
        self._s = s
        self.params = dict(gamma=gamma, Pr=Pr, mu=mu, C1=C1, theta=theta, rho_inf=rho_inf,
                           u_inf=u_inf, v_inf=v_inf, p_inf=p_inf,
                           adiabatic_zero_heatflux=adiabatic_zero_heatflux)

    @property
    def x(self):
        return self.geo["x"]

    @property
    def y(self):
        return self.geo["y"]

    def _ptr(self):
        return C.byref(self._s)

    def vortex_source(self, t):
        """Nodal S(x, t) of the vortex source, [K][4][Np]."""
        from .vortex_source import vortex_viscous_source
        v = self.vortex
        S = vortex_viscous_source(self.x, self.y, t, self.params["gamma"], self.params["Pr"],
                                  self.params["mu"], v["beta"], v["center"], v["L"], v["u0"], v["v0"])
        return np.ascontiguousarray(np.transpose(S, (0, 2, 1)))

    def rhs(self, U, t=0.0, vw=(0.0, 0.0)):
        """dU/dt = M^-1 R(t, U) (Eq. dg_on_K), [K][4][Np]."""
        U = _f64(U)
        R = np.empty_like(U)
        vwa = _f64(vw)
        st = lib().oracle_rhs(self._ptr(), _p(U), float(t), _p(vwa), _p(R))
        if st != 0:
            raise RuntimeError(f"oracle_rhs failed ({st})")
        if self.vortex is not None:
            R += self.vortex_source(t)
        return R

    def lsrk_step(self, U, t, dt, vw=(0.0, 0.0)):
        """One five-stage 2N-storage step (Algorithm 1); returns the new state."""
        U = _f64(U).copy()
        if self.vortex is not None:
            # Algorithm 1 around the Python-side residual (time-dependent source)
            A, B, c = lsrk_coeffs()
            K1 = np.zeros_like(U)
            for i in range(5):
                K1 = A[i] * K1 + dt * self.rhs(U, t + c[i] * dt, vw)
                U = U + B[i] * K1
            return U
        vwa = _f64(vw)
        st = lib().oracle_lsrk_step(self._ptr(), _p(U), float(t), float(dt), _p(vwa))
        if st != 0:
            raise RuntimeError(f"oracle_lsrk_step failed ({st})")
        return U

    def run(self, U, t0, dt, nsteps, vw=(0.0, 0.0)):
        U = _f64(U).copy()
        t = t0
        for _ in range(nsteps):
            U = self.lsrk_step(U, t, dt, vw)
            t += dt
        return U

    def broken_gradient(self, U):
        """(Ux, Uy) = ((rx Dr + sx Ds) U, (ry Dr + sy Ds) U) per element, [K][4][Np] each."""
        U = _f64(U)
        Ux, Uy = np.empty_like(U), np.empty_like(U)
        lib().oracle_broken_gradient(self._ptr(), _p(U), _p(Ux), _p(Uy))
        return Ux, Uy

    def face_sigma(self, U, vw=(0.0, 0.0)):
        """Penalty sigma_e per face, [K][3] (Eq. penalty_final)."""
        U = _f64(U)
        out = np.empty((self.K, 3))
        vwa = _f64(vw)
        lib().oracle_face_sigma(self._ptr(), _p(U), _p(vwa), _p(out))
        return out

    def dt(self, U, cfl, vw=(0.0, 0.0)):
        """CFL / max_K Lambda_K (Eq. rayleigh_bound, readings in dg_oracle.c).
        Pinned against the spectral radius of the linearised residual and the
        p-ratios of the paper's dt table (tests/test_oracle_dt.py)."""
        U = _f64(U)
        lam = np.empty(self.K)
        out = np.zeros(1)
        vwa = _f64(vw)
        lib().oracle_dt(self._ptr(), _p(U), float(cfl), _p(vwa), _p(out), _p(lam))
        return float(out[0]), lam

    def wall_forces(self, U, xc=(0.0, 0.0)):
        """(Fx, Fy, Mz) of the fluid on the wall boundary."""
        U = _f64(U)
        out = np.zeros(3)
        xca = _f64(xc)
        lib().oracle_wall_forces(self._ptr(), _p(U), _p(xca), _p(out))
        return out


# ---- pointwise routines (for pins) ----------------------------------------

def penalty_norm(U, n, gamma=1.4, Pr=0.72, mu=1e-3):
    U, n = _f64(U), _f64(n)
    return lib().oracle_penalty_norm(_p(U), _p(n), gamma, Pr, mu)


def G_blocks(U, gamma=1.4, Pr=0.72, mu=1e-3):
    """The four 4x4 blocks as an array G[a, b, 4, 4]."""
    U = _f64(U)
    out = np.zeros(64)
    lib().oracle_G_blocks(_p(U), gamma, Pr, mu, _p(out))
    return out.reshape(2, 2, 4, 4)


def roe(Up, Um, n, vw=(0.0, 0.0), gamma=1.4):
    """(H, A_signed, A_abs) of the Roe flux at one face node."""
    Up, Um, n, vwa = _f64(Up), _f64(Um), _f64(n), _f64(vw)
    H = np.zeros(4)
    As = np.zeros(16)
    Aa = np.zeros(16)
    st = lib().oracle_roe(_p(Up), _p(Um), _p(n), _p(vwa), gamma, _p(H), _p(As), _p(Aa))
    if st != 0:
        raise RuntimeError("oracle_roe failed")
    return H, As.reshape(4, 4), Aa.reshape(4, 4)


def flux_n(U, n, vw=(0.0, 0.0), gamma=1.4):
    U, n, vwa = _f64(U), _f64(n), _f64(vw)
    F = np.zeros(4)
    lib().oracle_flux_n(_p(U), _p(n), _p(vwa), gamma, _p(F))
    return F


def newmark_step(coeff, F, dt, state):
    """One Newmark (1/4, 1/2) step; returns (new_state, v_b)."""
    c = _f64(coeff)
    s = _f64(state).copy()
    vb = np.zeros(1)
    lib().oracle_newmark_step(_p(c), float(F), float(dt), _p(s), _p(vb))
    return s, float(vb[0])


def manufactured_source(x, y, kappa=25.0, C2=200.0, gamma=1.4, Pr=0.72, mu=0.01):
    S = np.zeros(4)
    lib().oracle_manufactured_source(float(x), float(y), kappa, C2, gamma, Pr, mu, _p(S))
    return S


def manufactured_state(x, y, kappa=25.0, C2=200.0):
    """U = (w, w, w, w^2), w = sin(kappa (x + y)) + C2 (Sec. 3.1), shape (..., 4)."""
    w = np.sin(kappa * (np.asarray(x) + np.asarray(y))) + C2
    return np.stack([w, w, w, w * w], axis=-1)


def lsrk_coeffs():
    A, B, c = np.zeros(5), np.zeros(5), np.zeros(5)
    lib().oracle_lsrk_coeffs(_p(A), _p(B), _p(c))
    return A, B, c


def set_threads(n: int):
    lib().oracle_set_threads(int(n))


def get_threads() -> int:
    return int(lib().oracle_get_threads())
