"""Pins for the symmetric / non-symmetric interior-penalty variants
(theta = 1 / -1 in Eq. ip_flux, the H_theta terms of Eq. dg_on_K).

* theta terms vanish where the state is continuous: a globally linear state
  gives the same residual for every theta;
* they conserve every field (sum_i d l_i/dx = 0 on each element);
* the penalty scales as (1 + theta)^2 (Eq. penalty_final): SIP is 4 x IIP
  (the paper's tables show ~5; the equation is followed);
* rotation invariance with theta = 1;
* at a fluid at rest the momentum block of G is block-symmetric
  (G_jl^T = G_lj), so the linearised viscous operator restricted to the
  momentum fields is self-adjoint in the DG mass inner product exactly when
  theta = 1; theta = 0 and theta = -1 are not;
* the residual is affine in theta when sigma = 0;
* linearised spectrum at rest: IIP with C1 = 0.01 and SIP with C1 = 0.02
  have no eigenvalue with positive real part, SIP without penalty has;
* SIP convergence on the Sec. 3.1 manufactured solution reaches the
  paper's printed SIP rates (mesh m1) minus 0.45, with C1 = 1: under
  Eq. penalty_final taken literally (factor (1+theta)^2 = 4) SIP with the
  paper's C1 = 0.01 is unstable on these meshes (an eigenvalue of the
  linearised operator with positive real part; it blows up at t ~ 0.01),
  and C1 = 0.1 still leaves the p = 2 error ten times IIP's.
"""
import json
import os

import numpy as np
import pytest

import dg_inputs
import oracle
from dg_inputs.states import to_kcn

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "sec31_convergence_tables.json")))


def linear_state(P):
    x, y = P.x, P.y
    rho = 1.0 + 0.05 * x - 0.03 * y
    m1 = 0.3 + 0.02 * y
    m2 = -0.1 + 0.01 * x
    E = 2.5 + 0.04 * x + 0.02 * y
    return to_kcn(np.stack([rho, m1, m2, E], axis=-1))


@pytest.mark.parametrize("theta", [1.0, -1.0])
def test_theta_terms_vanish_on_continuous_state(theta):
    m = dg_inputs.ogrid_cylinder(16, 4, 0.5, 2.0, seed=1)
    kw = dict(mu=0.02, rho_inf=1.0, u_inf=0.3, v_inf=0.0, p_inf=1.0)
    P0 = oracle.Problem(m, 3, theta=0.0, C1=0.0, **kw)
    P1 = oracle.Problem(m, 3, theta=theta, C1=0.0, **kw)
    U = linear_state(P0)
    # interior faces see no jump; boundary faces do (ghost states), so compare
    # only elements without boundary faces
    interior = np.all(m.bc == 0, axis=1)
    R0, R1 = P0.rhs(U), P1.rhs(U)
    assert np.abs(R1[interior] - R0[interior]).max() < 1e-12 * np.abs(R0).max()


@pytest.mark.parametrize("theta", [1.0, -1.0])
def test_theta_conservation(theta):
    m = dg_inputs.periodic_square(6)
    P = oracle.Problem(m, 3, mu=1e-2, theta=theta)
    U = dg_inputs.perturb(to_kcn(dg_inputs.isentropic_vortex(P.x, P.y)), seed=3, amp=2e-2)
    R = P.rhs(U)
    tot = np.einsum("k,kcn,nm->c", P.geo["J"], R, P.ops["M"])
    scale = np.einsum("k,kcn,nm->c", P.geo["J"], np.abs(R), P.ops["M"])
    assert np.all(np.abs(tot) <= 1e-13 * scale)


def test_sip_penalty_is_four_times_iip():
    m = dg_inputs.periodic_square(5)
    Pi = oracle.Problem(m, 2, mu=1e-2, theta=0.0)
    Ps = oracle.Problem(m, 2, mu=1e-2, theta=1.0)
    U = dg_inputs.perturb(to_kcn(dg_inputs.isentropic_vortex(Pi.x, Pi.y)), seed=1, amp=1e-2)
    assert np.allclose(Ps.face_sigma(U), 4.0 * Pi.face_sigma(U), rtol=1e-14)


def test_theta_rotation_invariance():
    p = 3
    m = dg_inputs.periodic_square(5)
    P = oracle.Problem(m, p, mu=5e-3, theta=1.0)
    U = dg_inputs.perturb(to_kcn(dg_inputs.isentropic_vortex(P.x, P.y)), seed=5, amp=1e-2)
    mr = dg_inputs.Mesh(-m.vy.copy(), m.vx.copy(), m.EToV, m.EToE, m.EToF, m.bc, m.period)
    Pr = oracle.Problem(mr, p, mu=5e-3, theta=1.0)
    Ur = U.copy()
    Ur[:, 1], Ur[:, 2] = -U[:, 2], U[:, 1]
    R, Rr = P.rhs(U), Pr.rhs(Ur)
    expect = R.copy()
    expect[:, 1], expect[:, 2] = -R[:, 2], R[:, 1]
    assert np.abs(Rr - expect).max() < 1e-12 * np.abs(R).max()


SLOW = pytest.mark.skipif(os.environ.get("DG_SLOW_TESTS") != "1",
                          reason="set DG_SLOW_TESTS=1 (about 8 minutes)")


@pytest.mark.parametrize("p,meshes", [
    (2, (4, 8)),
    pytest.param(2, (8, 16), marks=[pytest.mark.slow, SLOW]),
    pytest.param(3, (8, 16), marks=[pytest.mark.slow, SLOW]),
])
def test_convergence_manufactured_sip(p, meshes):
    """SIP (C1 = 1) on the steady manufactured solution of Sec. 3.1, over the
    same time window as the IIP convergence test (200 IIP steps on 4^2), on
    two split-quad meshes.  Rate at least the paper's printed SIP r2 for mesh
    m1 minus 0.45 (p = 2 gives 2.14 on 4^2 -> 8^2 and 2.0 on 8^2 -> 16^2 over
    this short window; p = 3 gives 4.3 on 8^2 -> 16^2)."""
    kappa, C2, mu = 25.0, 200.0, 0.01
    L = 4 * np.pi / kappa
    m = dg_inputs.periodic_square(4, L=L)
    P = oracle.Problem(m, p, mu=mu, source=("manufactured", kappa, C2))
    T = 200 * P.dt(to_kcn(oracle.manufactured_state(P.x, P.y, kappa, C2)), 0.3)[0]
    errs, hs = [], []
    for n in meshes:
        m = dg_inputs.periodic_square(n, L=L)
        P = oracle.Problem(m, p, mu=mu, theta=1.0, C1=1.0, source=("manufactured", kappa, C2))
        U0 = to_kcn(oracle.manufactured_state(P.x, P.y, kappa, C2))
        dt0, _ = P.dt(U0, 0.3)
        ns = int(np.ceil(T / dt0))
        d = P.run(U0, 0.0, T / ns, ns) - U0
        errs.append(np.sqrt(np.einsum("k,kcn,nm,kcm->", P.geo["J"], d, P.ops["M"], d)))
        hs.append(L / n)
    rate = np.log(errs[0] / errs[1]) / np.log(hs[0] / hs[1])
    paper = {int(k): v for k, v in GOLDEN["r2_sip_m1"].items()}[p]
    assert rate >= paper - 0.45, (errs, rate)

def rest_problem(theta, C1, mu, p=2):
    m = dg_inputs.periodic_square(3, L=1.0)
    P = oracle.Problem(m, p, mu=mu, theta=theta, C1=C1)
    U0 = to_kcn(dg_inputs.free_stream(P.x.shape, rho=1.0, u=0.0, v=0.0, p=1.0))
    return P, U0


def jacobian(P, U0, cols, eps=1e-6):
    """Central-difference Jacobian of the residual, columns `cols`, all rows."""
    J = np.empty((U0.size, len(cols)))
    for a, i in enumerate(cols):
        Up = U0.copy().reshape(-1)
        Um = Up.copy()
        Up[i] += eps
        Um[i] -= eps
        J[:, a] = (P.rhs(Up.reshape(U0.shape)) - P.rhs(Um.reshape(U0.shape))).reshape(-1) / (2 * eps)
    return J


def momentum_viscous_asymmetry(theta):
    Jm = []
    for mu in (0.05, 0.0):
        P, U0 = rest_problem(theta, 0.02, mu)
        mom = np.arange(U0.size).reshape(P.K, 4, P.Np)[:, 1:3].reshape(-1)
        Jm.append(jacobian(P, U0, mom)[mom])
    D = Jm[0] - Jm[1]                   # viscous + penalty part (advection cancels)
    W = np.kron(np.diag(np.repeat(P.geo["J"], 2)), P.ops["M"])
    B = W @ D
    return np.abs(B - B.T).max() / np.abs(B).max()


def test_sip_momentum_operator_self_adjoint_at_rest():
    assert momentum_viscous_asymmetry(1.0) < 1e-8
    assert momentum_viscous_asymmetry(0.0) > 1e-2
    assert momentum_viscous_asymmetry(-1.0) > 1e-2


def test_residual_affine_in_theta_without_penalty():
    m = dg_inputs.ogrid_cylinder(16, 4, 0.5, 2.0, seed=2)
    kw = dict(mu=0.02, C1=0.0, rho_inf=1.0, u_inf=0.3, v_inf=0.0, p_inf=1.0)
    R = {}
    for th in (-1.0, 0.0, 1.0, 0.5):
        P = oracle.Problem(m, 3, theta=th, **kw)
        if th == -1.0:
            r = np.hypot(P.x, P.y)
            U = to_kcn(dg_inputs.free_stream(P.x.shape, rho=1.0, u=0.3, v=0.0, p=1.0))
            U = dg_inputs.perturb(U * (1 + 0.1 * np.sin(3 * r))[:, None, :], seed=4, amp=1e-2)
        R[th] = P.rhs(U)
    scale = np.abs(R[0.0]).max()
    assert np.abs(R[1.0] + R[-1.0] - 2 * R[0.0]).max() < 1e-11 * scale
    assert np.abs(R[0.5] - 0.5 * (R[0.0] + R[1.0])).max() < 1e-11 * scale
    assert np.abs(R[1.0] - R[0.0]).max() > 1e-6 * scale


@pytest.mark.parametrize("theta,C1,stable", [(0.0, 0.01, True), (1.0, 0.02, True), (1.0, 0.0, False)])
def test_linearised_spectrum_at_rest(theta, C1, stable):
    P, U0 = rest_problem(theta, C1, 0.05)
    ev = np.linalg.eigvals(jacobian(P, U0, range(U0.size), eps=1e-7))
    ratio = ev.real.max() / np.abs(ev.real).max()
    assert (ratio < 1e-8) == stable, (theta, C1, ratio)
