"""Error measures shared by the GPU parity tests (CPU arithmetic only).

* rel_l2: relative L2 error per conserved field in the DG mass norm
  sum_K J_K u^T M u (reading R15);
* field_err: max-norm error of a residual per field, relative to that
  field's own largest entry;
* fp32_sensitivity: how much the oracle's own residual moves, per field and
  in the same relative measure, when its input state is rounded to FP32.
  The mixed path computes every residual from an FP32 copy of the state, so
  this is the floor of its error; the parity tests allow MIXED_SENS times it
  (FP32 arithmetic of the fluxes, the FP32 pressure and the split-TF32
  contractions add errors of the same kind; the largest ratio measured over
  p = 1..6, periodic and O-grid states and the three tile shapes was 6.3);
* inc_err: relative L2 error per field of the increment U_n - U_0, which a
  run that skipped its updates fails with error 1.

Tolerances:
  FP64 path: residual 1e-12 relative to its largest entry and 1e-11 per field
  (a field whose residual is small next to its largest flux term, as rho v1
  next to the pressure p_inf = 17.9 on the O-grid, is about 300 times more
  sensitive to rounding than its size: 1.3e-12 was measured there); state
  1e-12; increment 1e-9 (FP64 rounding of the state, 1e-16 |U|, against
  increments of 1e-6 |U| and more);
  mixed path: residual per field MIXED_SENS x the FP32 sensitivity (a fixed
  max-norm bound does not fit: the sensitivity grows with the number of
  elements sampled and with p, from 5e-7 on 50 elements at p = 1 to 5.6e-5
  on 32,768 elements at p = 4); state 2e-5 relative L2 per field (the bound
  the method is held to after 100 steps); increment 5e-4 (the increment is a
  sum of dt R, so it carries the residual's relative error, at most about
  2e-4 per field on the O-grid states).
"""
import numpy as np

MIXED_SENS = 10.0
INC_TOL = {"fp64": 1e-9, "mixed": 5e-4}
STATE_TOL = {"fp64": 1e-12, "mixed": 2e-5}
RHS_TOL_ALL_FP64 = 1e-12
RHS_TOL_FIELD_FP64 = 1e-11


def rel_l2(P, d, ref):
    J, M = P.geo["J"], P.ops["M"]
    num = np.einsum("k,kcn,nm,kcm->c", J, d, M, d)
    den = np.einsum("k,kcn,nm,kcm->c", J, ref, M, ref)
    return np.sqrt(num / den)


def inc_err(P, got, ref, U0):
    return rel_l2(P, got - ref, ref - U0)


def field_err(got, ref, scale=None):
    s = np.abs(ref).max(axis=(0, 2)) if scale is None else scale
    return np.abs(got - ref).max(axis=(0, 2)) / s


def all_err(got, ref):
    return np.abs(got - ref).max() / np.abs(ref).max()


def fp32_sensitivity(P, U, t=0.0, vw=(0.0, 0.0), scale=None):
    R = P.rhs(U, t, vw)
    R32 = P.rhs(U.astype(np.float32).astype(np.float64), t, vw)
    return field_err(R32, R, scale)


def check_rhs(P, U, got, precision, t=0.0, vw=(0.0, 0.0), ref=None):
    """Residual parity with the bounds of the precision; returns (all-field
    error, per-field errors, per-field bounds)."""
    ref = P.rhs(U, t, vw) if ref is None else ref
    ea, ef = all_err(got, ref), field_err(got, ref)
    if precision == "fp64":
        bound = np.full(4, RHS_TOL_FIELD_FP64)
        assert ea <= RHS_TOL_ALL_FP64, (ea, ef)
    else:
        bound = MIXED_SENS * fp32_sensitivity(P, U, t, vw)
    assert np.all(ef <= bound), (ef, bound)
    return ea, ef, bound
