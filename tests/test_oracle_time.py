"""Pins for the oracle's time integration (Algorithm 1), rigid-body step
(Eq. 1dof_oscillator), wall forces (Eq. lift_drag) and time step (Eq.
rayleigh_bound).

* LSRK: the 2N-storage coefficients, unrolled into a Butcher tableau, satisfy
  all eight order conditions of order 4; the stability polynomial matches
  exp(z) to fourth order; the oracle's DG step equals the same recursion
  written out here around the oracle's residual.
* Newmark average acceleration: exact energy conservation without damping and
  load, the known period elongation 2 arctan(w dt / 2), static offset F/K.
* Forces: zero for uniform pressure; Archimedes' law -g*Area for a linear
  pressure; 2 mu a Area for the shear flow v = (a y^2, 0) on the polygon.
* dt: scales linearly with the CFL number (its p-scaling, its size against
  the operator's spectral radius and the paper's dt table are pinned in
  test_oracle_dt.py).
"""
import numpy as np
import pytest

import dg_inputs
import oracle
from dg_inputs.states import to_kcn


def butcher_from_2n(A, B):
    s = len(A)
    a = np.zeros((s + 1, s))
    for i in range(1, s + 1):          # stage i+1 uses U after i register updates
        for j in range(i):
            acc = 0.0
            for m in range(j, i):
                prod = 1.0
                for l in range(j + 1, m + 1):
                    prod *= A[l]
                acc += B[m] * prod
            a[i, j] = acc
    return a[:s], a[s]


def test_lsrk_order_conditions():
    A, B, c = oracle.lsrk_coeffs()
    a, b = butcher_from_2n(A, B)
    cc = a.sum(axis=1)
    assert np.allclose(cc, c, atol=1e-12)
    conds = [
        (b.sum(), 1.0), (b @ cc, 1 / 2), (b @ cc ** 2, 1 / 3), (b @ a @ cc, 1 / 6),
        (b @ cc ** 3, 1 / 4), (b @ (cc * (a @ cc)), 1 / 8), (b @ a @ cc ** 2, 1 / 12),
        (b @ a @ a @ cc, 1 / 24)]
    for got, want in conds:
        assert abs(got - want) < 1e-12


def test_lsrk_linear_order():
    A, B, c = oracle.lsrk_coeffs()
    lam = -1.3 + 0.7j

    def run(n):
        dt = 1.0 / n
        y, k1 = 1.0 + 0j, 0j
        for _ in range(n):
            for i in range(5):
                k1 = A[i] * k1 + dt * lam * y
                y = y + B[i] * k1
        return abs(y - np.exp(lam))

    e1, e2 = run(20), run(40)
    assert 3.8 < np.log2(e1 / e2) < 4.3


def test_oracle_step_is_algorithm_1():
    m = dg_inputs.periodic_square(4)
    P = oracle.Problem(m, 2, mu=1e-2)
    U = dg_inputs.perturb(to_kcn(dg_inputs.isentropic_vortex(P.x, P.y)), seed=9, amp=1e-2)
    A, B, c = oracle.lsrk_coeffs()
    dt, vw = 2e-3, (0.03, 0.01)
    K0, K1 = U.copy(), np.zeros_like(U)
    for i in range(5):
        K1 = A[i] * K1 + dt * P.rhs(K0, 0.1 + c[i] * dt, vw)
        K0 = K0 + B[i] * K1
    got = P.lsrk_step(U, 0.1, dt, vw)
    assert np.abs(got - K0).max() < 1e-15 * np.abs(K0).max() * 10


def test_newmark_energy_and_period():
    M, Kr = 1.0, (2 * np.pi) ** 2
    w = np.sqrt(Kr / M)
    dt = 0.05
    st = np.array([0.3, 0.0, -Kr * 0.3 / M])
    e0 = 0.5 * M * st[1] ** 2 + 0.5 * Kr * st[0] ** 2
    ys = [st[0]]
    for _ in range(4000):
        st, _ = oracle.newmark_step((M, 0.0, Kr), 0.0, dt, st)
        ys.append(st[0])
        e = 0.5 * M * st[1] ** 2 + 0.5 * Kr * st[0] ** 2
        assert abs(e - e0) < 1e-12 * e0
    # numerical frequency wbar with wbar dt = 2 arctan(w dt / 2)
    wbar = 2 * np.arctan(w * dt / 2) / dt
    t = dt * np.arange(len(ys))
    assert np.allclose(ys, 0.3 * np.cos(wbar * t), atol=1e-9)


def test_newmark_static_load_and_vb():
    coeff = (1.0, 2.0, 25.0)
    st = np.zeros(3)
    ys = []
    for _ in range(3000):
        y_old = st[0]
        st, vb = oracle.newmark_step(coeff, 5.0, 0.01, st)
        assert abs(vb - (st[0] - y_old) / 0.01) < 1e-14
        ys.append(st[0])
    assert abs(ys[-1] - 5.0 / 25.0) < 1e-8


def ogrid_problem(p=2, mu=0.01):
    m = dg_inputs.ogrid_cylinder(24, 4, 0.5, 2.0, seed=2)
    return oracle.Problem(m, p, mu=mu, rho_inf=1.0, u_inf=0.0, v_inf=0.0, p_inf=1.0)


def polygon_area(n, r):
    return 0.5 * n * r * r * np.sin(2 * np.pi / n)


def test_forces_uniform_pressure_zero():
    P = ogrid_problem()
    U = to_kcn(dg_inputs.free_stream(P.x.shape, rho=1.0, u=0.0, v=0.0, p=3.0))
    F = P.wall_forces(U)
    assert np.abs(F).max() < 1e-13


def test_forces_archimedes():
    P = ogrid_problem()
    g = 0.7
    p = 5.0 + g * P.y
    U = np.stack([np.ones_like(p), 0 * p, 0 * p, p / 0.4], axis=-1)
    F = P.wall_forces(to_kcn(U))
    area = polygon_area(24, 0.5)
    assert abs(F[1] + g * area) < 1e-12
    assert abs(F[0]) < 1e-12 and abs(F[2]) < 1e-12


def test_forces_viscous_shear():
    mu, a = 0.01, 0.3
    P = ogrid_problem(p=2, mu=mu)
    y = P.y
    rho = np.ones_like(y)
    v1 = a * y * y
    E = 1.0 / 0.4 + 0.5 * rho * v1 * v1
    U = np.stack([rho, rho * v1, 0 * y, E], axis=-1)
    F = P.wall_forces(to_kcn(U))
    area = polygon_area(24, 0.5)
    assert abs(F[0] - 2 * mu * a * area) < 1e-12
    assert abs(F[1]) < 1e-12


def test_dt_scales_with_cfl():
    m = dg_inputs.periodic_square(4)
    P = oracle.Problem(m, 2, mu=1e-3)
    U = to_kcn(dg_inputs.isentropic_vortex(P.x, P.y))
    d1, lam = P.dt(U, 0.3)
    d2, _ = P.dt(U, 0.6)
    assert abs(d2 - 2 * d1) < 1e-15 * d2
    assert abs(d1 - 0.3 / lam.max()) < 1e-18
