"""Viscous source that makes the advected isentropic vortex an exact
Navier-Stokes solution (test infrastructure, part of the oracle).

The vortex U_v(x, t) (Shu's isentropic vortex carried by the free stream)
solves the Euler equations exactly, U_t + div F_c = 0.  With the viscous
flux of Sec. 2.1, F_v = G(U) grad U, the Navier-Stokes form
U_t + div (F_c - F_v) = S holds exactly for

    S(x, t) = - div F_v(U_v(x, t)).

This module evaluates S the plain way: U_v is written once in hyper-dual
arithmetic (a + b e1 + c e2 + d e1 e2 with e1^2 = e2^2 = 0), which returns
U, its derivatives along two directions and their mixed second derivative
exactly; the four G blocks are transcribed entry by entry from Sec. 2.1 in
first-order dual arithmetic, so that

    d/dx_i [ G_ij(U) d_j U ] = (dual part of) G_ij(U + e1 d_i U) (d_j U + e1 d_i d_j U)

and S = - sum_ij of those.  Nothing here is shared with the CUDA library,
which evaluates the same S from a closed form.
"""
from __future__ import annotations

import numpy as np


class HD:
    """Hyper-dual number with numpy components (a, b, c, d): a + b e1 + c e2 + d e1 e2."""

    def __init__(self, a, b=0.0, c=0.0, d=0.0):
        self.a, self.b, self.c, self.d = a, b, c, d

    @staticmethod
    def _w(o):
        return o if isinstance(o, HD) else HD(o)

    def __add__(self, o):
        o = HD._w(o)
        return HD(self.a + o.a, self.b + o.b, self.c + o.c, self.d + o.d)

    __radd__ = __add__

    def __neg__(self):
        return HD(-self.a, -self.b, -self.c, -self.d)

    def __sub__(self, o):
        return self + (-HD._w(o))

    def __rsub__(self, o):
        return HD._w(o) - self

    def __mul__(self, o):
        o = HD._w(o)
        return HD(self.a * o.a, self.a * o.b + self.b * o.a, self.a * o.c + self.c * o.a,
                  self.a * o.d + self.b * o.c + self.c * o.b + self.d * o.a)

    __rmul__ = __mul__

    def _fn(self, f0, f1, f2):
        """g(x) with g = f0, g' = f1, g'' = f2 evaluated at the real part."""
        return HD(f0, f1 * self.b, f1 * self.c, f1 * self.d + f2 * self.b * self.c)

    def recip(self):
        a = self.a
        return self._fn(1.0 / a, -1.0 / a ** 2, 2.0 / a ** 3)

    def __truediv__(self, o):
        return self * HD._w(o).recip()

    def __rtruediv__(self, o):
        return HD._w(o) * self.recip()

    def exp(self):
        e = np.exp(self.a)
        return self._fn(e, e, e)

    def pow(self, q):
        a = self.a
        return self._fn(a ** q, q * a ** (q - 1), q * (q - 1) * a ** (q - 2))


class D:
    """First-order dual number (value, derivative) with numpy components."""

    def __init__(self, v, e=0.0):
        self.v, self.e = v, e

    @staticmethod
    def _w(o):
        return o if isinstance(o, D) else D(o)

    def __add__(self, o):
        o = D._w(o)
        return D(self.v + o.v, self.e + o.e)

    __radd__ = __add__

    def __neg__(self):
        return D(-self.v, -self.e)

    def __sub__(self, o):
        return self + (-D._w(o))

    def __rsub__(self, o):
        return D._w(o) - self

    def __mul__(self, o):
        o = D._w(o)
        return D(self.v * o.v, self.v * o.e + self.e * o.v)

    __rmul__ = __mul__

    def __truediv__(self, o):
        o = D._w(o)
        return D(self.v / o.v, (self.e * o.v - self.v * o.e) / (o.v * o.v))

    def __rtruediv__(self, o):
        return D._w(o) / self


def vortex_hd(X, Y, t, gamma, beta, center, L, u0, v0):
    """Conserved state of the advected vortex at hyper-dual coordinates."""
    xc = center[0] + u0 * t
    yc = center[1] + v0 * t
    dx = X - xc
    dy = Y - yc
    # nearest periodic image: a constant shift taken from the real part
    dx = dx - L * np.round(dx.a / L)
    dy = dy - L * np.round(dy.a / L)
    r2 = dx * dx + dy * dy
    e = (1.0 - r2).exp()
    T = 1.0 - (gamma - 1.0) * beta ** 2 / (8.0 * gamma * np.pi ** 2) * e
    f = beta / (2.0 * np.pi) * (0.5 * (1.0 - r2)).exp()
    u = u0 - f * dy
    v = v0 + f * dx
    rho = T.pow(1.0 / (gamma - 1.0))
    p = rho * T
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    return [rho, rho * u, rho * v, E]


def G_apply(U, dU, j, i, gamma, Pr, mu):
    """(G_ij(U) dU)_row for the four rows, dual arithmetic (Sec. 2.1 blocks;
    i is the flux direction, j the derivative direction)."""
    rho, m1, m2, eps = U
    v1, v2 = m1 / rho, m2 / rho
    vv = v1 * v1 + v2 * v2
    c = mu / rho
    gp = gamma / Pr
    e_over = eps / rho
    d0, d1, d2, d3 = dU
    if (i, j) == (0, 0):                       # G11
        g41 = -1.0 / 3.0 * v1 * v1 - vv - gp * (e_over - vv)
        rows = [0.0 * d0,
                -4.0 / 3.0 * v1 * d0 + 4.0 / 3.0 * d1,
                -v2 * d0 + d2,
                g41 * d0 + (4.0 / 3.0 - gp) * v1 * d1 + (1.0 - gp) * v2 * d2 + gp * d3]
    elif (i, j) == (0, 1):                     # G12
        rows = [0.0 * d0,
                2.0 / 3.0 * v2 * d0 - 2.0 / 3.0 * d2,
                -v1 * d0 + d1,
                -1.0 / 3.0 * v1 * v2 * d0 + v2 * d1 - 2.0 / 3.0 * v1 * d2]
    elif (i, j) == (1, 0):                     # G21
        rows = [0.0 * d0,
                -v2 * d0 + d2,
                2.0 / 3.0 * v1 * d0 - 2.0 / 3.0 * d1,
                -1.0 / 3.0 * v1 * v2 * d0 - 2.0 / 3.0 * v2 * d1 + v1 * d2]
    else:                                      # G22
        g41 = -1.0 / 3.0 * v2 * v2 - vv - gp * (e_over - vv)
        rows = [0.0 * d0,
                -v1 * d0 + d1,
                -4.0 / 3.0 * v2 * d0 + 4.0 / 3.0 * d2,
                g41 * d0 + (1.0 - gp) * v1 * d1 + (4.0 / 3.0 - gp) * v2 * d2 + gp * d3]
    return [c * r for r in rows]


def vortex_viscous_source(x, y, t, gamma=1.4, Pr=0.72, mu=1e-3, beta=5.0, center=(5.0, 5.0),
                          L=10.0, u0=None, v0=0.0, mach=0.3):
    """S = -div F_v(U_v) at points (x, y), time t; returns shape (..., 4).
    u0 defaults to the free-stream speed M sqrt(gamma) of the vortex input."""
    if u0 is None:
        u0 = mach * np.sqrt(gamma)
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    one, zero = np.ones_like(x), np.zeros_like(x)
    S = [np.zeros_like(x) for _ in range(4)]
    for i in range(2):                         # flux direction, differentiated along e_i
        for j in range(2):                     # gradient direction
            ei = (one, zero) if i == 0 else (zero, one)
            ej = (one, zero) if j == 0 else (zero, one)
            X = HD(x, ei[0], ej[0], zero)
            Y = HD(y, ei[1], ej[1], zero)
            Uh = vortex_hd(X, Y, t, gamma, beta, center, L, u0, v0)
            U = [D(q.a, q.b) for q in Uh]                  # U and d_i U
            dU = [D(q.c, q.d) for q in Uh]                 # d_j U and d_i d_j U
            F = G_apply(U, dU, j, i, gamma, Pr, mu)
            for r in range(4):
                S[r] = S[r] - F[r].e
    return np.stack(S, axis=-1)
