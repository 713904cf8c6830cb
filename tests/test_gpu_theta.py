"""GPU parity of the SIP / NIPG variants (theta = 1 / -1 in Eq. ip_flux).

The kernel variant with the theta terms of Eq. dg_on_K against the oracle:
residuals on the periodic square (p = 1..6) and on the O-grid with wall and
far-field faces, and 50 LSRK steps of SIP.  Tolerances as for IIP
(tests/_parity.py): residuals 1e-12 relative to the largest entry and 1e-11
per field (FP64), and per field 10 x the oracle's FP32 input sensitivity
(mixed).
"""
import numpy as np
import pytest

import dg_inputs
import oracle
from dg_inputs.states import to_kcn
from _parity import check_rhs

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-12, "mixed": 2e-5}


@pytest.fixture(scope="module")
def dg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_17917_gb300 import build
    build.build()
    import paper_2508_17917_gb300 as dg
    return dg


def stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


@pytest.mark.parametrize("theta", [1.0, -1.0, 0.5])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_rhs_periodic_theta(dg, p, precision, theta):
    mesh = dg_inputs.periodic_square(5)
    P = oracle.Problem(mesh, p, mu=5e-3, theta=theta, C1=0.05)
    U = to_kcn(dg_inputs.isentropic_vortex(P.x, P.y))
    U = dg_inputs.perturb(U, seed=3, amp=1e-2)
    vw = (0.05, 0.02)
    ref = P.rhs(U, vw=vw)
    s = dg.Solver(mesh, p, precision, stream=stream(), mu=5e-3, theta=theta, C1=0.05)
    s.set_state(U)
    got = s.rhs(0.0, vw)
    check_rhs(P, U, got, precision, 0.0, vw, ref)
    # the theta terms themselves, against the oracle's difference
    d_ref = ref - oracle.Problem(mesh, p, mu=5e-3, theta=0.0, C1=0.05 * (1 + theta) ** 2).rhs(U, vw=vw)
    s0 = dg.Solver(mesh, p, precision, stream=stream(), mu=5e-3, theta=0.0, C1=0.05 * (1 + theta) ** 2)
    s0.set_state(U)
    d_got = got - s0.rhs(0.0, vw)
    assert np.abs(d_got - d_ref).max() <= 50 * TOL[precision] * np.abs(d_ref).max(), \
        np.abs(d_got - d_ref).max() / np.abs(d_ref).max()


@pytest.mark.parametrize("theta", [1.0, -1.0])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("p", [2, 4])
def test_rhs_ogrid_theta(dg, p, precision, theta):
    mesh = dg_inputs.ogrid_cylinder(24, 8, 0.5, 4.0, seed=3)
    kw = dict(mu=0.01, rho_inf=1.0, u_inf=1.0, v_inf=0.0, p_inf=17.857142857142858, theta=theta, C1=0.05)
    P = oracle.Problem(mesh, p, **kw)
    r = np.hypot(P.x, P.y)
    U = to_kcn(dg_inputs.free_stream(P.x.shape, rho=1.0, u=1.0, v=0.0, p=kw["p_inf"]))
    U[:, 1] *= np.tanh(3 * (r - 0.5))
    U = dg_inputs.perturb(U, seed=12, amp=1e-3)
    vw = (0.0, 0.05)
    ref = P.rhs(U, vw=vw)
    s = dg.Solver(mesh, p, precision, stream=stream(), **kw)
    s.set_state(U)
    got = s.rhs(0.0, vw)
    check_rhs(P, U, got, precision, 0.0, vw, ref)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_sip_50_steps_and_dt(dg, precision):
    mesh = dg_inputs.periodic_square(8)
    p = 3
    P = oracle.Problem(mesh, p, mu=2e-3, theta=1.0, C1=0.1)
    U0 = dg_inputs.perturb(to_kcn(dg_inputs.isentropic_vortex(P.x, P.y)), seed=5, amp=1e-3)
    dt, _ = P.dt(U0, 0.3)
    s = dg.Solver(mesh, p, precision, stream=stream(), mu=2e-3, theta=1.0, C1=0.1)
    s.set_state(U0)
    assert abs(s.dt(0.3) - dt) <= 1e-12 * dt
    ref = P.run(U0, 0.0, dt, 50)
    s.steps(0.0, dt, 50)
    got = s.get_state()
    d = got - ref
    J, M = P.geo["J"], P.ops["M"]
    err = np.sqrt(np.einsum("k,kcn,nm,kcm->c", J, d, M, d) / np.einsum("k,kcn,nm,kcm->c", J, ref, M, ref))
    assert np.all(err <= (1e-12 if precision == "fp64" else 2e-5)), err
