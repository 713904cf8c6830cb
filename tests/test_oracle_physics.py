"""Pins for the oracle's pointwise physics (Sec. 2.1, Sec. 2.2 fluxes, Sec. 3.1).

* G(U) grad U against the textbook Navier-Stokes stress and heat flux written
  from primitive-variable gradients (a wrong entry of any G block fails);
* the penalty spectral norm against numpy's SVD-based 2-norm;
* the Roe flux: consistency, the Rankine-Hugoniot property
  A (U+ - U-) = F_n(U+) - F_n(U-), full upwinding when every wave speed has one
  sign, antisymmetry under exchanging sides and flipping the normal, and the
  moving-wall eigenvalue shift;
* the manufactured source of Sec. 3.1 against central differences of the
  oracle's own fluxes evaluated on the exact solution.
"""
import numpy as np
import pytest

import oracle

GAMMA, PR, MU = 1.4, 0.72, 1e-3


def random_state(rng, mach=0.5):
    rho = rng.uniform(0.5, 2.0)
    v = rng.uniform(-1, 1, 2)
    p = rng.uniform(0.5, 2.0)
    c = np.sqrt(GAMMA * p / rho)
    v = v / np.linalg.norm(v) * mach * c * rng.uniform(0.1, 1.0)
    E = p / (GAMMA - 1) + 0.5 * rho * v @ v
    return np.array([rho, rho * v[0], rho * v[1], E])


def textbook_viscous_flux(U, Ux, Uy, gamma=GAMMA, Pr=PR, mu=MU):
    """Stress tau = mu (grad v + grad v^T - 2/3 div v I); energy flux
    v . tau + mu gamma/Pr grad(e_int), e_int = eps/rho - |v|^2/2 (unit c_v)."""
    rho, m1, m2, E = U
    v = np.array([m1, m2]) / rho
    G = np.array([Ux, Uy])               # G[d, c] = d_d U_c
    dv = np.zeros((2, 2))                 # dv[d, i] = d_d v_i
    for d in range(2):
        for i in range(2):
            dv[d, i] = (G[d, 1 + i] - v[i] * G[d, 0]) / rho
    div = dv[0, 0] + dv[1, 1]
    tau = mu * (dv.T + dv - 2.0 / 3.0 * div * np.eye(2))   # tau[i, j] = mu(d_j v_i + d_i v_j) - ...
    e = E / rho
    de = np.array([(G[d, 3] - e * G[d, 0]) / rho for d in range(2)])
    deint = de - np.array([v @ dv[d] for d in range(2)])
    F = np.zeros((2, 4))
    for d in range(2):
        F[d, 1] = tau[0, d]
        F[d, 2] = tau[1, d]
        F[d, 3] = v @ tau[:, d] + mu * gamma / Pr * deint[d]
    return F


def test_G_blocks_match_textbook_flux():
    rng = np.random.default_rng(1)
    for _ in range(200):
        U = random_state(rng)
        Ux, Uy = rng.normal(size=4), rng.normal(size=4)
        G = oracle.G_blocks(U, GAMMA, PR, MU)
        Fx = G[0, 0] @ Ux + G[0, 1] @ Uy
        Fy = G[1, 0] @ Ux + G[1, 1] @ Uy
        ref = textbook_viscous_flux(U, Ux, Uy)
        assert np.allclose(Fx, ref[0], rtol=1e-12, atol=1e-14)
        assert np.allclose(Fy, ref[1], rtol=1e-12, atol=1e-14)


def test_penalty_norm_is_spectral_norm():
    rng = np.random.default_rng(2)
    for _ in range(300):
        U = random_state(rng)
        th = rng.uniform(0, 2 * np.pi)
        n = np.array([np.cos(th), np.sin(th)])
        G = oracle.G_blocks(U, GAMMA, PR, MU)
        A = n[0] ** 2 * G[0, 0] + n[0] * n[1] * (G[0, 1] + G[1, 0]) + n[1] ** 2 * G[1, 1]
        ref = np.linalg.norm(A, 2)
        got = oracle.penalty_norm(U, n, GAMMA, PR, MU)
        assert abs(got - ref) <= 1e-13 * ref


def test_penalty_norm_velocity_block():
    """N G N^T restricted to the momentum rows/columns is (mu/rho)(I + n n^T/3):
    for a fluid at rest with zero energy-row coupling its norm bounds 4/3 mu/rho."""
    U = np.array([2.0, 0.0, 0.0, 0.0])       # e = 0, v = 0: only the momentum block survives
    for th in np.linspace(0, np.pi, 7):
        n = np.array([np.cos(th), np.sin(th)])
        got = oracle.penalty_norm(U, n, GAMMA, PR, MU)
        assert abs(got - max(4.0 / 3.0, GAMMA / PR) * MU / 2.0) < 1e-15


@pytest.mark.parametrize("vw", [(0.0, 0.0), (0.13, -0.21)])
def test_roe_consistency(vw):
    rng = np.random.default_rng(3)
    for _ in range(100):
        U = random_state(rng)
        n = rng.normal(size=2)
        n /= np.linalg.norm(n)
        H, _, _ = oracle.roe(U, U, n, vw)
        assert np.allclose(H, oracle.flux_n(U, n, vw), rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("vw", [(0.0, 0.0), (0.2, 0.05)])
def test_roe_rankine_hugoniot(vw):
    rng = np.random.default_rng(4)
    for _ in range(200):
        Up, Um = random_state(rng, 0.9), random_state(rng, 0.9)
        n = rng.normal(size=2)
        n /= np.linalg.norm(n)
        _, As, _ = oracle.roe(Up, Um, n, vw)
        dF = oracle.flux_n(Up, n, vw) - oracle.flux_n(Um, n, vw)
        assert np.allclose(As @ (Up - Um), dF, rtol=1e-11, atol=1e-12 * np.abs(dF).max())


def test_roe_supersonic_is_upwind():
    rng = np.random.default_rng(5)
    n = np.array([1.0, 0.0])
    for _ in range(50):
        # both states moving right at Mach ~2-3: every wave speed positive
        rho, p = rng.uniform(0.5, 2, 2)
        c = np.sqrt(GAMMA * p / rho)
        u = rng.uniform(2.0, 3.0) * c
        Up = np.array([rho, rho * u, 0.1 * rho, p / 0.4 + 0.5 * rho * (u * u + 0.01)])
        rho2, p2 = rho * 1.05, p * 0.97
        u2 = u * 1.02
        Um = np.array([rho2, rho2 * u2, 0.0, p2 / 0.4 + 0.5 * rho2 * u2 * u2])
        H, _, _ = oracle.roe(Up, Um, n)
        assert np.allclose(H, oracle.flux_n(Up, n), rtol=1e-12)
        H2, _, _ = oracle.roe(Um, Up, -n)
        assert np.allclose(H2, oracle.flux_n(Up, -n), rtol=1e-12)


def test_roe_antisymmetry_and_moving_frame():
    rng = np.random.default_rng(6)
    for _ in range(100):
        Up, Um = random_state(rng), random_state(rng)
        n = rng.normal(size=2)
        n /= np.linalg.norm(n)
        vw = rng.uniform(-0.2, 0.2, 2)
        H1, _, A1 = oracle.roe(Up, Um, n, vw)
        H2, _, _ = oracle.roe(Um, Up, -n, vw)
        assert np.allclose(H1, -H2, rtol=1e-12, atol=1e-13)
        # moving frame shifts every eigenvalue by -vw.n: A(vw) = A(0) - (vw.n) I
        _, As0, _ = oracle.roe(Up, Um, n, (0.0, 0.0))
        _, As1, _ = oracle.roe(Up, Um, n, vw)
        assert np.allclose(As1, As0 - (vw @ n) * np.eye(4), atol=1e-12)


def exact_fluxes(x, y, kappa, C2, gamma, Pr, mu):
    U = oracle.manufactured_state(x, y, kappa, C2)
    w = U[0]
    dw = kappa * np.cos(kappa * (x + y))
    dU = dw * np.array([1.0, 1.0, 1.0, 2.0 * w])
    Fcx = oracle.flux_n(U, [1.0, 0.0], gamma=gamma)
    Fcy = oracle.flux_n(U, [0.0, 1.0], gamma=gamma)
    G = oracle.G_blocks(U, gamma, Pr, mu)
    Fvx = G[0, 0] @ dU + G[0, 1] @ dU
    Fvy = G[1, 0] @ dU + G[1, 1] @ dU
    return Fcx - Fvx, Fcy - Fvy


def test_manufactured_source_by_central_differences():
    """S = div(F_c - F_v) for the steady solution of Sec. 3.1, checked with
    fourth-order central differences of the oracle's flux functions."""
    kappa, C2, gamma, Pr, mu = 25.0, 200.0, 1.4, 0.72, 0.01
    h = 1e-4
    rng = np.random.default_rng(7)
    for _ in range(20):
        x, y = rng.uniform(0, 1, 2)
        div = np.zeros(4)
        for d, (ex, ey) in enumerate([(1, 0), (0, 1)]):
            f = [exact_fluxes(x + k * h * ex, y + k * h * ey, kappa, C2, gamma, Pr, mu)[d]
                 for k in (-2, -1, 1, 2)]
            div += (f[0] - 8 * f[1] + 8 * f[2] - f[3]) / (12 * h)
        S = oracle.manufactured_source(x, y, kappa, C2, gamma, Pr, mu)
        assert np.allclose(S, div, rtol=1e-7, atol=1e-7 * np.abs(div).max())


def test_printed_source_coefficients_do_not_balance():
    """The printed source (1/2 k g1 and k g1 in front of cos) leaves a residual,
    which is why the oracle uses the derived coefficients."""
    kappa, C2, gamma = 25.0, 200.0, 1.4
    g1 = gamma - 1
    x, y = 0.1, 0.2
    phi = kappa * (x + y)
    printed_mom = kappa * g1 * np.sin(2 * phi) + (2 * kappa - 0.5 * kappa * g1 + 2 * kappa * C2 * g1) * np.cos(phi)
    S = oracle.manufactured_source(x, y, kappa, C2, gamma, 0.72, 0.01)
    assert abs(printed_mom - S[1]) > 1.0


def test_manufactured_mach_reading_of_eos():
    """With p = (gamma-1)(eps - rho |v|^2/2) the Sec. 3.1 state has Mach ~0.13,
    matching the stated Ma ~ 0.15; the printed form (gamma-1) rho (eps - v^2/2)
    would give Mach ~ 0.01."""
    gamma, C2 = 1.4, 200.0
    w = C2
    p = (gamma - 1) * (w * w - 0.5 * w * 2.0)
    mach = np.sqrt(2.0) / np.sqrt(gamma * p / w)
    assert 0.1 < mach < 0.16
    p_printed = (gamma - 1) * w * (w * w - 0.5 * 2.0)
    assert np.sqrt(2.0) / np.sqrt(gamma * p_printed / w) < 0.02
