"""Pins for the oracle's reference-element operators (Sec. 2.2, weak matrices).

Each check compares against mathematics that does not pass through the
oracle's construction: exact derivatives and integrals of monomials on the
reference triangle, Legendre-Gauss-Lobatto nodes and weights from numpy's
Legendre module, and the integration-by-parts identity of the weak matrices.
"""
import math
from fractions import Fraction

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from oracle import refelem

PS = [1, 2, 3, 4, 5, 6]


def tri_monomial_integral(a, b):
    """int over K^ of r^a s^b (K^ = {(-1,-1),(1,-1),(-1,1)}), by the Dirichlet
    integral int_{u,v>=0,u+v<=1} u^i v^j = i! j! / (i+j+2)! after r = 2u-1, s = 2v-1."""
    tot = Fraction(0)
    for i in range(a + 1):
        for j in range(b + 1):
            coef = math.comb(a, i) * 2 ** i * (-1) ** (a - i) * math.comb(b, j) * 2 ** j * (-1) ** (b - j)
            tot += Fraction(coef * math.factorial(i) * math.factorial(j), math.factorial(i + j + 2))
    return float(4 * tot)


def monomials(p):
    return [(a, b) for a in range(p + 1) for b in range(p + 1 - a)]


@pytest.mark.parametrize("p", PS)
def test_node_count_and_inside(p):
    r, s = refelem.nodes(p)
    assert r.size == (p + 1) * (p + 2) // 2
    assert np.all(r >= -1 - 1e-14) and np.all(s >= -1 - 1e-14) and np.all(r + s <= 1e-14)
    # vertices are nodes
    pts = set(zip(np.round(r, 12), np.round(s, 12)))
    for v in [(-1.0, -1.0), (1.0, -1.0), (-1.0, 1.0)]:
        assert v in pts


@pytest.mark.parametrize("p", PS)
def test_edge_nodes_are_lgl(p):
    """Warp-and-blend places the nodes of every edge at the LGL points."""
    r, s = refelem.nodes(p)
    inner = np.sort(npleg.Legendre.basis(p).deriv().roots().real)
    lgl = np.concatenate([[-1.0], inner, [1.0]])
    bottom = np.sort(r[np.abs(s + 1) < 1e-10])
    left = np.sort(s[np.abs(r + 1) < 1e-10])
    hyp = np.sort(s[np.abs(r + s) < 1e-10])
    for edge in (bottom, left, hyp):
        assert np.allclose(edge, lgl, atol=1e-13)


@pytest.mark.parametrize("p", PS)
def test_node_set_symmetric(p):
    """The node set is invariant under the reflection r <-> s of K^."""
    r, s = refelem.nodes(p)
    a = np.array(sorted(zip(np.round(r, 11), np.round(s, 11))))
    b = np.array(sorted(zip(np.round(s, 11), np.round(r, 11))))
    assert np.allclose(a, b, atol=1e-11)


@pytest.mark.parametrize("p", PS)
def test_differentiation_exact(p):
    o = refelem.operators(p)
    r, s = o["r"], o["s"]
    for a, b in monomials(p):
        f = r ** a * s ** b
        fr = a * r ** (a - 1) * s ** b if a > 0 else np.zeros_like(r)
        fs = b * r ** a * s ** (b - 1) if b > 0 else np.zeros_like(r)
        assert np.abs(o["Dr"] @ f - fr).max() < 1e-12 * max(1.0, np.abs(fr).max())
        assert np.abs(o["Ds"] @ f - fs).max() < 1e-12 * max(1.0, np.abs(fs).max())
    one = np.ones_like(r)
    assert np.abs(o["Dr"] @ one).max() < 1e-13
    assert np.abs(o["Ds"] @ one).max() < 1e-13


@pytest.mark.parametrize("p", PS)
def test_mass_matrix_exact(p):
    o = refelem.operators(p)
    r, s = o["r"], o["s"]
    M = o["M"]
    assert np.allclose(M, M.T, atol=1e-15)
    assert np.linalg.eigvalsh(M).min() > 0
    assert abs(M.sum() - 2.0) < 1e-13
    mons = monomials(p)
    for (a, b) in mons:
        for (c, d) in mons:
            f = r ** a * s ** b
            g = r ** c * s ** d
            assert abs(f @ M @ g - tri_monomial_integral(a + c, b + d)) < 1e-13


@pytest.mark.parametrize("p", PS)
def test_face_mass_rows_are_lgl_weights(p):
    o = refelem.operators(p)
    x = np.concatenate([[-1.0], np.sort(npleg.Legendre.basis(p).deriv().roots().real), [1.0]])
    w = 2.0 / (p * (p + 1) * npleg.legval(x, [0] * p + [1]) ** 2)
    for f in range(3):
        M1 = o["M1D"][f]
        assert np.allclose(np.sort(M1.sum(axis=0)), np.sort(w), atol=1e-14)
        assert abs(M1.sum() - 2.0) < 1e-14


@pytest.mark.parametrize("p", PS)
def test_integration_by_parts_identity(p):
    """M Dr + (M Dr)^T = sum_f n_r,f sJ_f E_f M1D_f E_f^T on K^ (and the same
    for s): int d_r(l_i l_j) = boundary integral.  Pins Dr, Ds, M, Fmask and
    the face mass matrices together."""
    o = refelem.operators(p)
    M, Dr, Ds, Fm, M1 = o["M"], o["Dr"], o["Ds"], o["Fmask"], o["M1D"]
    Np = o["Np"]
    # reference faces: s=-1 (n=(0,-1), sJ=1), r+s=0 (n=(1,1)/sqrt2, sJ=sqrt2), r=-1 (n=(-1,0), sJ=1)
    nr_sJ = [0.0, 1.0, -1.0]
    ns_sJ = [-1.0, 1.0, 0.0]
    Br = np.zeros((Np, Np))
    Bs = np.zeros((Np, Np))
    for f in range(3):
        B = np.zeros((Np, Np))
        B[np.ix_(Fm[f], Fm[f])] = M1[f]
        Br += nr_sJ[f] * B
        Bs += ns_sJ[f] * B
    assert np.abs(M @ Dr + (M @ Dr).T - Br).max() < 1e-13
    assert np.abs(M @ Ds + (M @ Ds).T - Bs).max() < 1e-13


@pytest.mark.parametrize("p", PS)
def test_lift_identity(p):
    o = refelem.operators(p)
    assert np.abs(o["M"] @ o["LIFT"] - o["Emat"]).max() < 1e-13
