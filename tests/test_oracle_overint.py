"""Pins of the over-integrated volume term (the volume flux integral of
Eq. dg_on_K evaluated with a cubature rule instead of the nodal
interpolant of the flux; Sec. 2.2, weak matrices).

* The cubature rule integrates every monomial up to its degree exactly
  (closed form over the reference triangle) and its weights sum to the area.
* At rest with a pressure linear in x (the Euler flux is then linear, so its
  nodal interpolant is exact) over-integration reproduces the collocated
  residual.
* Free stream is preserved and every field is conserved on periodic meshes.
* The aliasing error shrinks: against a much finer rule, the rule of degree
  3p is closer than the nodal interpolant.
"""
from fractions import Fraction
from math import factorial

import numpy as np
import pytest

import dg_inputs
import oracle
from dg_inputs.states import to_kcn
from oracle import refelem


def exact_monomial(a, b):
    """int over the reference triangle of (1 + r)^a (1 + s)^b = 2^(a+b+2) a! b! / (a+b+2)!."""
    return float(Fraction(2 ** (a + b + 2) * factorial(a) * factorial(b), factorial(a + b + 2)))


@pytest.mark.parametrize("deg", [1, 3, 6, 9, 12, 15, 18])
def test_cubature_exact_to_its_degree(deg):
    r, s, w = refelem.cubature(deg)
    assert abs(w.sum() - 2.0) < 1e-14
    assert np.all(w > 0)
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            got = np.sum(w * (1 + r) ** a * (1 + s) ** b)
            ref = exact_monomial(a, b)
            assert abs(got - ref) <= 1e-13 * max(1.0, ref), (deg, a, b)


def test_overint_equals_collocation_for_linear_flux():
    m = dg_inputs.periodic_square(5)
    for p in (2, 4):
        P0 = oracle.Problem(m, p, mu=0.0)
        P1 = oracle.Problem(m, p, mu=0.0, overint=3 * p)
        U = to_kcn(dg_inputs.free_stream(P0.x.shape, rho=1.0, u=0.0, v=0.0, p=1.0))
        U[:, 3] += 0.003 * (P0.x - 5.0) / 0.4      # energy, hence pressure, linear in x
        # (the jump this leaves across the periodic boundary enters both
        # residuals through the same face terms; only the volume terms differ)
        R0, R1 = P0.rhs(U), P1.rhs(U)
        assert np.abs(R1 - R0).max() <= 1e-11 * max(1.0, np.abs(R0).max())


@pytest.mark.parametrize("p", [1, 3, 5])
def test_overint_free_stream_and_conservation(p):
    m = dg_inputs.periodic_square(4)
    P = oracle.Problem(m, p, mu=5e-3, overint=3 * p)
    U = to_kcn(dg_inputs.free_stream(P.x.shape, rho=1.2, u=0.4, v=-0.2, p=1.5))
    assert np.abs(P.rhs(U)).max() < 1e-12
    U = dg_inputs.perturb(to_kcn(dg_inputs.isentropic_vortex(P.x, P.y)), seed=4, amp=2e-2)
    R = P.rhs(U)
    tot = np.einsum("k,kcn,nm->c", P.geo["J"], R, P.ops["M"])
    scale = np.einsum("k,kcn,nm->c", P.geo["J"], np.abs(R), P.ops["M"])
    assert np.all(np.abs(tot) <= 1e-13 * scale)


@pytest.mark.parametrize("p", [2, 3, 4])
def test_overint_reduces_aliasing(p):
    m = dg_inputs.periodic_square(4)
    U = None
    res = {}
    for deg in (0, 3 * p, 3 * p + 8):
        P = oracle.Problem(m, p, mu=1e-2, overint=deg)
        if U is None:
            U = dg_inputs.perturb(to_kcn(dg_inputs.isentropic_vortex(P.x, P.y, mach=0.5)), seed=5, amp=5e-2)
        res[deg] = P.rhs(U)
    fine = res[3 * p + 8]
    e_col = np.abs(res[0] - fine).max()
    e_oi = np.abs(res[3 * p] - fine).max()
    assert e_oi < 0.5 * e_col, (e_oi, e_col)
