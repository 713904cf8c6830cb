"""Pins for the oracle's viscous vortex source (config 2's source term):
S = -div F_v(U_v) of the advected isentropic vortex U_v, which makes U_v an
exact solution of the Navier-Stokes form of Sec. 2.1 with a source.

* S_rho = 0 (the continuity equation has no viscous part) and S vanishes far
  from the vortex core;
* S against central differences of F_v = G(U) grad U, with G from the C
  oracle's blocks (pinned against the textbook stress and heat flux) and
  U_v, grad U_v from the independent input generator;
* the DG residual of the exact vortex with the source approaches dU_v/dt =
  -(u0 d/dx + v0 d/dy) U_v under mesh refinement (like h^(p-1), the order of
  the residual's consistency for a second-order term), while without the
  source the mismatch stays at the size of S (large viscosity).
"""
import numpy as np

import dg_inputs
import oracle
from dg_inputs.states import to_kcn
from oracle.vortex_source import vortex_viscous_source

GAMMA, PR, MACH = 1.4, 0.72, 0.3
U0 = MACH * np.sqrt(GAMMA)


def vortex(x, y, t):
    return dg_inputs.isentropic_vortex(x, y, t, gamma=GAMMA, mach=MACH)


def test_continuity_row_zero_and_far_field():
    rng = np.random.default_rng(0)
    x, y = rng.uniform(0, 10, 200), rng.uniform(0, 10, 200)
    S = vortex_viscous_source(x, y, 0.3, GAMMA, PR, 1e-2)
    assert np.all(S[:, 0] == 0.0)
    far = vortex_viscous_source(np.array([0.2, 9.8]), np.array([0.1, 0.3]), 0.0, GAMMA, PR, 1e-2)
    assert np.abs(far).max() < 1e-7 * np.abs(S).max()


def grad_fd(x, y, t, h=1e-4):
    ux = (vortex(x + h, y, t) - vortex(x - h, y, t)) / (2 * h)
    uy = (vortex(x, y + h, t) - vortex(x, y - h, t)) / (2 * h)
    return ux, uy


def viscous_flux(x, y, t, mu):
    U = vortex(x, y, t)
    ux, uy = grad_fd(x, y, t)
    F = np.zeros(U.shape[:-1] + (2, 4))
    for n in range(U.shape[0]):
        G = oracle.G_blocks(U[n], GAMMA, PR, mu)
        F[n, 0] = G[0, 0] @ ux[n] + G[0, 1] @ uy[n]
        F[n, 1] = G[1, 0] @ ux[n] + G[1, 1] @ uy[n]
    return F


def test_source_against_finite_differences():
    mu, t, h = 2e-2, 0.41, 2e-3
    rng = np.random.default_rng(1)
    x = 5.0 + U0 * t + rng.uniform(-2, 2, 40)
    y = 5.0 + rng.uniform(-2, 2, 40)
    S = vortex_viscous_source(x, y, t, GAMMA, PR, mu)
    div = ((viscous_flux(x + h, y, t, mu)[:, 0] - viscous_flux(x - h, y, t, mu)[:, 0])
           + (viscous_flux(x, y + h, t, mu)[:, 1] - viscous_flux(x, y - h, t, mu)[:, 1])) / (2 * h)
    assert np.abs(S + div).max() < 1e-5 * np.abs(S).max()


def residual_mismatch(n, p, mu, with_source):
    mesh = dg_inputs.periodic_square(n)
    src = ("vortex", 5.0, 5.0, 5.0, 10.0, U0, 0.0) if with_source else None
    P = oracle.Problem(mesh, p, mu=mu, source=src)
    t = 0.2
    U = to_kcn(vortex(P.x, P.y, t))
    h = 1e-5
    Ut = -U0 * (to_kcn(vortex(P.x + h, P.y, t)) - to_kcn(vortex(P.x - h, P.y, t))) / (2 * h)
    d = P.rhs(U, t) - Ut
    J, M = P.geo["J"], P.ops["M"]
    return np.sqrt(np.einsum("k,kcn,nm,kcm->", J, d, M, d))


def test_exact_vortex_is_a_solution_with_the_source():
    mu, p = 0.05, 3
    e16, e32 = residual_mismatch(16, p, mu, True), residual_mismatch(32, p, mu, True)
    n16, n32 = residual_mismatch(16, p, mu, False), residual_mismatch(32, p, mu, False)
    # with the source the mismatch is the residual's truncation error, which
    # for the second-order viscous term falls like h^(p-1)
    assert np.log2(e16 / e32) > p - 1.2, (e16, e32)
    # without it the viscous term of the exact vortex remains
    assert n32 > 5 * e32 and n32 > 0.8 * n16, (n16, n32, e32)
