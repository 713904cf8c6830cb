"""Pins for the oracle's time-step bound Lambda_K (Eq. rayleigh_bound,
Eq. cfl_general; Appendix on the CFL condition).

The bound has free constants (C_grad, C_CFL) and the paper's dt table needs
the paper's own mesh, so the pins check what the paper fixes without them:

* G_K, read as the largest diffusivity of the system, equals the largest
  eigenvalue of N G N^T built from the G blocks (pinned against the textbook
  stress and heat flux elsewhere) at random states and normals;
* the Appendix closes by stating that the bound and the true size of the
  spatial operator differ by constants independent of p and of the PDE
  coefficients: Lambda = max_K Lambda_K divided by the spectral radius of the
  oracle's linearised residual (power iteration on finite-difference
  Jacobian-vector products, which never calls the bound) stays in a narrow
  band for p = 1..5 and two flow regimes;
* on an O-grid shaped like the paper's cylinder case (Re = 200, Ma = 0.1,
  about 20,000 triangles) the ratios dt(p) / dt(p+1) follow the paper's
  table of maximum stable steps within a factor 2 (the table was found by
  trial on a mesh that is not available, and the ratios move with the mesh's
  balance of advective and penalty stiffness), and the table's steps times
  the spectral radius of the oracle's operator land in the stability range
  of the five-stage Runge-Kutta scheme to within an order of magnitude.
"""
import json
import os

import numpy as np
import pytest

import dg_inputs
import oracle
from dg_inputs.states import free_stream, perturb

GOLD = os.path.join(os.path.dirname(__file__), "golden", "dt_max_table.json")
GAMMA, PR = 1.4, 0.72


def flow_state(P, mach):
    p_inf = 1.0 / (GAMMA * mach * mach)
    U = np.ascontiguousarray(free_stream((P.K, P.Np), p=p_inf).transpose(0, 2, 1))
    return perturb(U, 0, 1e-4)


def ogrid_problem(mesh, p, mach, Re):
    return oracle.Problem(mesh, p, mu=1.0 / Re, rho_inf=1.0, u_inf=1.0, v_inf=0.0,
                          p_inf=1.0 / (GAMMA * mach * mach))


def spectral_radius(P, U, iters=70, tail=25):
    """|lambda|_max of dR/dU at U: power iteration, growth rate averaged over
    the last iterations (complex pairs make single ratios oscillate)."""
    R0 = P.rhs(U)
    scale = np.abs(U).max(axis=(0, 2), keepdims=True)
    scale = np.maximum(scale, scale[:, 1:2])          # rho v may vanish
    v = np.random.default_rng(0).standard_normal(U.shape) * scale
    v /= np.linalg.norm(v / scale)
    logs = []
    for _ in range(iters):
        Jv = (P.rhs(U + 1e-7 * v) - R0) / 1e-7
        nv = np.linalg.norm(Jv / scale)
        logs.append(np.log(nv))
        v = Jv / nv
    return float(np.exp(np.mean(logs[-tail:])))


def test_diffusivity_is_largest_eigenvalue_of_NGNt():
    rng = np.random.default_rng(3)
    mu = 0.013
    for _ in range(20):
        rho = rng.uniform(0.3, 3.0)
        v = rng.uniform(-2, 2, 2)
        eps = rng.uniform(2.0, 60.0) + 0.5 * rho * v @ v
        U = np.array([rho, rho * v[0], rho * v[1], eps])
        G = oracle.G_blocks(U, GAMMA, PR, mu)
        th = rng.uniform(0, 2 * np.pi)
        n = np.array([np.cos(th), np.sin(th)])
        A = sum(n[a] * n[b] * G[a, b] for a in range(2) for b in range(2))
        ev = np.sort(np.linalg.eigvals(A).real)
        want = np.sort(np.array([0.0, 4 / 3, 1.0, GAMMA / PR]) * mu / rho)
        assert np.allclose(ev, want, rtol=1e-10, atol=1e-14)
        # and the spectral norm the penalty uses is far larger at low Mach
        assert np.linalg.norm(A, 2) > ev.max()


def test_lambda_tracks_operator_spectral_radius():
    mesh = dg_inputs.ogrid_cylinder(24, 8, 0.5, 5.0, seed=0)
    ratios = []
    for mach, Re in ((0.1, 200.0), (0.3, 100.0)):
        for p in range(1, 6):
            P = ogrid_problem(mesh, p, mach, Re)
            U = flow_state(P, mach)
            _, lam = P.dt(U, 0.3)
            ratios.append(lam.max() / spectral_radius(P, U))
    ratios = np.array(ratios)
    # an upper bound of the operator's size ...
    assert ratios.min() > 2.0, ratios
    # ... by a constant that neither p nor the flow moves by much
    assert ratios.max() < 10.0, ratios
    assert ratios.max() / ratios.min() < 2.0, ratios


@pytest.fixture(scope="module")
def paper_shaped_mesh():
    # about 20,000 triangles, first cell the wall arc length, far field at 30 D
    return dg_inputs.ogrid_cylinder(120, 84, 0.5, 30.0, seed=0)


def test_dt_ratios_follow_table(paper_shaped_mesh):
    table = json.load(open(GOLD))["dt_1e4"]
    want = np.array([table[str(p)] for p in range(1, 6)]) * 1e-4
    got = []
    for p in range(1, 6):
        P = ogrid_problem(paper_shaped_mesh, p, 0.1, 200.0)
        got.append(P.dt(flow_state(P, 0.1), 0.3)[0])
    got = np.array(got)
    r_got = got[:-1] / got[1:]
    r_want = want[:-1] / want[1:]
    q = r_got / r_want
    assert np.all((q > 0.5) & (q < 2.0)), (r_got, r_want)
    # the step always shrinks with p
    assert np.all(r_got > 1.0)


@pytest.mark.parametrize("p", [1, 4])
def test_table_steps_in_rk_stability_range(paper_shaped_mesh, p):
    table = json.load(open(GOLD))["dt_1e4"]
    P = ogrid_problem(paper_shaped_mesh, p, 0.1, 200.0)
    rho = spectral_radius(P, flow_state(P, 0.1), iters=60, tail=20)
    # the five-stage scheme is stable up to |z| of about 3.2 (left half plane)
    # to 4.7 (negative real axis); the paper's step on its own mesh sits at
    # that edge, so on a comparable mesh dt_table * rho is of that order
    z = table[str(p)] * 1e-4 * rho
    assert 1.0 < z < 40.0, z
