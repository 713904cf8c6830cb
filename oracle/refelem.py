"""Reference-triangle operators for the CPU oracle (test infrastructure only).

Oracle header: this package is the plain, slow FP64 statement of the method
that the CUDA path is checked against.  Only tests, the smoke check and the
CPU-baseline leg of the benchmark may import it; the product never does.

Reference element K^ = {(-1,-1), (1,-1), (-1,1)} (Sec. 2.2).  The nodal basis
sits on the optimised interpolation points of the warp-and-blend construction
(Sec. 1, Sec. 2.2 "Weak matrices and nodal formulation"); the modal basis is
the Dubiner-Proriol-Koornwinder (PKD) orthonormal basis (Sec. 1), from which
the Vandermonde matrix V, the mass matrix M = (V V^T)^-1 and the
differentiation matrices Dr, Ds follow (Sec. 2.2, weak matrices).

Every operator here is built from library primitives (scipy Jacobi
polynomials and Gauss-Jacobi roots, numpy inverse) so that this code shares
nothing with the C++ builder inside the CUDA library.

Node ordering: node (n, m) has barycentric weight n/p on the vertex (-1, 1)
and m/p on the vertex (1, -1) before warping; nodes are numbered with n
outer (bottom row s = -1 first) and m inner (increasing r).  Both sides of
every parity test use this numbering.
"""
from __future__ import annotations

import functools
import math

import numpy as np
from scipy.special import eval_jacobi, gammaln, roots_jacobi

# Optimised blend parameter alpha(p) for p = 1..15 of the warp-and-blend node
# family (Hesthaven and Warburton, Nodal DG Methods, 2008, Table 6.1).
ALPHA_OPT = (0.0, 0.0, 1.4152, 0.1001, 0.2751, 0.9800, 1.0999, 1.2832,
             1.3648, 1.4773, 1.4959, 1.5743, 1.5770, 1.6223, 1.6258)


def np_count(p: int) -> int:
    """N_p = (p+1)(p+2)/2 (Sec. 2.2)."""
    return (p + 1) * (p + 2) // 2


def _jacobi_norm2(n, a, b):
    """h_n = int_{-1}^{1} (1-x)^a (1+x)^b (P_n^{(a,b)})^2 dx."""
    lg = ((a + b + 1) * math.log(2.0) - math.log(2 * n + a + b + 1)
          + gammaln(n + a + 1) + gammaln(n + b + 1)
          - gammaln(n + a + b + 1) - gammaln(n + 1))
    return math.exp(lg)


def jacobi_hat(x, a, b, n):
    """Orthonormal Jacobi polynomial P_n^{(a,b)} / sqrt(h_n)."""
    return eval_jacobi(n, a, b, np.asarray(x, dtype=np.float64)) / math.sqrt(_jacobi_norm2(n, a, b))


def jacobi_hat_deriv(x, a, b, n):
    """Derivative of jacobi_hat; uses d/dx P_n^{(a,b)} = (n+a+b+1)/2 P_{n-1}^{(a+1,b+1)}."""
    x = np.asarray(x, dtype=np.float64)
    if n == 0:
        return np.zeros_like(x)
    return (0.5 * (n + a + b + 1) * eval_jacobi(n - 1, a + 1, b + 1, x)
            / math.sqrt(_jacobi_norm2(n, a, b)))


def lgl_nodes(p: int) -> np.ndarray:
    """Legendre-Gauss-Lobatto nodes: -1, 1 and the roots of P_p' = c P_{p-1}^{(1,1)}."""
    if p == 1:
        return np.array([-1.0, 1.0])
    inner, _ = roots_jacobi(p - 1, 1.0, 1.0)
    return np.concatenate([[-1.0], np.sort(inner), [1.0]])


def _warp(p: int, t: np.ndarray) -> np.ndarray:
    """Edge warp: Lagrange interpolant (equispaced nodes) of the LGL displacement,
    divided by (1 - t^2) inside the edge and zero at its end points."""
    req = np.linspace(-1.0, 1.0, p + 1)
    disp = lgl_nodes(p) - req
    t = np.asarray(t, dtype=np.float64)
    w = np.zeros_like(t)
    for i in range(p + 1):
        li = np.ones_like(t)
        for j in range(p + 1):
            if j != i:
                li = li * (t - req[j]) / (req[i] - req[j])
        w = w + disp[i] * li
    inside = np.abs(t) < 1.0 - 1e-10
    out = np.zeros_like(t)
    out[inside] = w[inside] / (1.0 - t[inside] ** 2)
    return out


@functools.lru_cache(maxsize=None)
def nodes(p: int):
    """Warp-and-blend nodes (r, s) on K^ in the documented order."""
    alpha = ALPHA_OPT[p - 1] if p <= 15 else 5.0 / 3.0
    L1, L3 = [], []
    for n in range(p + 1):
        for m in range(p + 1 - n):
            L1.append(n / p)
            L3.append(m / p)
    L1 = np.array(L1)
    L3 = np.array(L3)
    L2 = 1.0 - L1 - L3
    sq3 = math.sqrt(3.0)
    # equilateral triangle: L2 at (-1,-1/sqrt3), L3 at (1,-1/sqrt3), L1 at (0,2/sqrt3)
    x = -L2 + L3
    y = (-L2 - L3 + 2.0 * L1) / sq3
    edges = [  # (blend weight, edge parameter, direction angle, opposite weight)
        (4.0 * L2 * L3, L3 - L2, 0.0, L1),
        (4.0 * L1 * L3, L1 - L3, 2.0 * math.pi / 3.0, L2),
        (4.0 * L1 * L2, L2 - L1, 4.0 * math.pi / 3.0, L3),
    ]
    for blend, t, ang, opp in edges:
        shift = blend * _warp(p, t) * (1.0 + (alpha * opp) ** 2)
        x = x + math.cos(ang) * shift
        y = y + math.sin(ang) * shift
    # back to barycentrics, then to (r, s) with L2 -> (-1,-1), L3 -> (1,-1), L1 -> (-1,1)
    B1 = (sq3 * y + 1.0) / 3.0
    B2 = (-3.0 * x - sq3 * y + 2.0) / 6.0
    B3 = (3.0 * x - sq3 * y + 2.0) / 6.0
    r = -B2 + B3 - B1
    s = -B2 - B3 + B1
    return r, s


def _collapsed(r, s):
    a = np.where(np.abs(1.0 - s) > 1e-14, 2.0 * (1.0 + r) / np.where(np.abs(1.0 - s) > 1e-14, 1.0 - s, 1.0) - 1.0, -1.0)
    return a, s


def _modes(p):
    return [(i, j) for i in range(p + 1) for j in range(p + 1 - i)]


def pkd(r, s, i, j):
    """Orthonormal PKD mode psi_ij = sqrt2 P^_i(a) P^_j^{(2i+1,0)}(b) (1-b)^i."""
    a, b = _collapsed(np.asarray(r, float), np.asarray(s, float))
    return math.sqrt(2.0) * jacobi_hat(a, 0, 0, i) * jacobi_hat(b, 2 * i + 1, 0, j) * (1.0 - b) ** i


def pkd_grad(r, s, i, j):
    """(d/dr, d/ds) psi_ij by the chain rule through a = 2(1+r)/(1-s) - 1, b = s."""
    a, b = _collapsed(np.asarray(r, float), np.asarray(s, float))
    fa, dfa = jacobi_hat(a, 0, 0, i), jacobi_hat_deriv(a, 0, 0, i)
    gb, dgb = jacobi_hat(b, 2 * i + 1, 0, j), jacobi_hat_deriv(b, 2 * i + 1, 0, j)
    om = 1.0 - b
    if i == 0:
        dr = np.zeros_like(a)
        ds = math.sqrt(2.0) * fa * dgb
    else:
        dr = 2.0 * math.sqrt(2.0) * dfa * gb * om ** (i - 1)
        ds = math.sqrt(2.0) * (dfa * (1.0 + a) * gb * om ** (i - 1)
                               + fa * (dgb * om ** i - i * gb * om ** (i - 1)))
    return dr, ds


@functools.lru_cache(maxsize=None)
def operators(p: int):
    """All reference operators for degree p as a dict of float64 arrays."""
    r, s = nodes(p)
    Np = np_count(p)
    modes = _modes(p)
    V = np.column_stack([pkd(r, s, i, j) for (i, j) in modes])
    Vr = np.column_stack([pkd_grad(r, s, i, j)[0] for (i, j) in modes])
    Vs = np.column_stack([pkd_grad(r, s, i, j)[1] for (i, j) in modes])
    Vinv = np.linalg.inv(V)
    Dr = Vr @ Vinv
    Ds = Vs @ Vinv
    Minv = V @ V.T
    M = np.linalg.inv(Minv)
    tol = 1e-10
    faces = [np.where(np.abs(s + 1.0) < tol)[0],
             np.where(np.abs(r + s) < tol)[0],
             np.where(np.abs(r + 1.0) < tol)[0]]
    Nfp = p + 1
    Fmask = np.array(faces, dtype=np.int64)
    assert Fmask.shape == (3, Nfp)
    tcoord = [r[faces[0]], s[faces[1]], s[faces[2]]]
    M1D = np.zeros((3, Nfp, Nfp))
    Emat = np.zeros((Np, 3 * Nfp))
    for f in range(3):
        V1 = np.column_stack([jacobi_hat(tcoord[f], 0, 0, n) for n in range(Nfp)])
        M1D[f] = np.linalg.inv(V1 @ V1.T)
        for k in range(Nfp):
            Emat[Fmask[f, k], f * Nfp:(f + 1) * Nfp] += M1D[f][k]
    LIFT = Minv @ Emat
    return dict(p=p, Np=Np, Nfp=Nfp, r=r, s=s, V=V, Dr=Dr, Ds=Ds, M=M,
                Minv=Minv, Fmask=Fmask, M1D=M1D, Emat=Emat, LIFT=LIFT)


@functools.lru_cache(maxsize=None)
def cubature(deg: int):
    """Collapsed-coordinate Gauss rule on the reference triangle, exact for
    polynomials of total degree <= deg: N = ceil((deg + 1) / 2) Gauss-Legendre
    points in a and N Gauss-Jacobi (1, 0) points in b, r = (1 + a)(1 - b)/2 - 1,
    s = b, weight w_a w_b / 2 (dr ds = (1 - b)/2 da db)."""
    n = (deg + 2) // 2
    a, wa = roots_jacobi(n, 0.0, 0.0)
    b, wb = roots_jacobi(n, 1.0, 0.0)
    A, B = np.meshgrid(a, b, indexing="ij")
    W = np.outer(wa, wb) / 2.0
    r = (1.0 + A) * (1.0 - B) / 2.0 - 1.0
    return r.ravel(), B.ravel(), W.ravel()


@functools.lru_cache(maxsize=None)
def overint_operators(p: int, deg: int):
    """Nodal basis values and (r, s) derivatives at the cubature points of
    `cubature(deg)`: Vq, Vqr, Vqs [Nq][Np] (ell_j and its derivatives at x_q)
    and the weights wq [Nq]."""
    ops = operators(p)
    rq, sq, wq = cubature(deg)
    modes = _modes(p)
    Vinv = np.linalg.inv(ops["V"])
    Vq = np.column_stack([pkd(rq, sq, i, j) for (i, j) in modes]) @ Vinv
    Vqr = np.column_stack([pkd_grad(rq, sq, i, j)[0] for (i, j) in modes]) @ Vinv
    Vqs = np.column_stack([pkd_grad(rq, sq, i, j)[1] for (i, j) in modes]) @ Vinv
    return dict(rq=rq, sq=sq, wq=wq, Vq=Vq, Vqr=Vqr, Vqs=Vqs, Nq=rq.size)
