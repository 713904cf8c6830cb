"""GPU parity of the over-integrated volume term (dg_set_overintegration,
FP64 path) against the oracle with the same cubature degree.

The library builds its own collapsed Gauss rule (Newton iteration on the
Jacobi polynomials) and the oracle takes scipy's; both are exact to the same
degree, so the residuals agree to FP64 rounding: 1e-12 relative, as for the
collocated FP64 path.
"""
import numpy as np
import pytest

import dg_inputs
import oracle
from dg_inputs.states import to_kcn

pytestmark = pytest.mark.gpu


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


def test_rule_degree(dg):
    assert [dg.dg_overint_degree(p) for p in range(1, 7)] == [3, 6, 9, 12, 15, 15]


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_rhs_periodic_overint(dg, p):
    mesh = dg_inputs.periodic_square(5)
    deg = dg.dg_overint_degree(p)
    P = oracle.Problem(mesh, p, mu=5e-3, overint=deg)
    U = dg_inputs.perturb(to_kcn(dg_inputs.isentropic_vortex(P.x, P.y, mach=0.5)), seed=3, amp=2e-2)
    vw = (0.05, -0.02)
    ref = P.rhs(U, vw=vw)
    s = dg.Solver(mesh, p, "fp64", stream=stream(), mu=5e-3)
    s.set_overint(True)
    s.set_state(U)
    got = s.rhs(0.0, vw)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    # and it is not the collocated residual
    col = oracle.Problem(mesh, p, mu=5e-3).rhs(U, vw=vw)
    assert np.abs(col - ref).max() > 1e-9 * np.abs(ref).max()


@pytest.mark.parametrize("p", [2, 4])
def test_rhs_ogrid_overint(dg, p):
    mesh = dg_inputs.ogrid_cylinder(24, 8, 0.5, 4.0, seed=3)
    kw = dict(mu=0.01, rho_inf=1.0, u_inf=1.0, v_inf=0.0, p_inf=17.857142857142858)
    P = oracle.Problem(mesh, p, overint=dg.dg_overint_degree(p), **kw)
    r = np.hypot(P.x, P.y)
    U = to_kcn(dg_inputs.free_stream(P.x.shape, rho=1.0, u=1.0, v=0.0, p=kw["p_inf"]))
    U[:, 1] *= np.tanh(3 * (r - 0.5))
    U = dg_inputs.perturb(U, seed=11, amp=1e-3)
    vw = (0.0, 0.05)
    ref = P.rhs(U, vw=vw)
    s = dg.Solver(mesh, p, "fp64", stream=stream(), **kw)
    s.set_overint(True)
    s.set_state(U)
    got = s.rhs(0.0, vw)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_overint_steps(dg):
    mesh = dg_inputs.periodic_square(8)
    p = 3
    P = oracle.Problem(mesh, p, mu=1e-3, overint=dg.dg_overint_degree(p))
    U0 = dg_inputs.perturb(to_kcn(dg_inputs.isentropic_vortex(P.x, P.y)), seed=1)
    dt, _ = P.dt(U0, 0.3)
    ref = P.run(U0, 0.0, dt, 20)
    s = dg.Solver(mesh, p, "fp64", stream=stream(), mu=1e-3)
    s.set_overint(True)
    s.set_state(U0)
    s.steps(0.0, dt, 20)
    d = s.get_state() - ref
    J, M = P.geo["J"], P.ops["M"]
    err = np.sqrt(np.einsum("k,kcn,nm,kcm->c", J, d, M, d) / np.einsum("k,kcn,nm,kcm->c", J, ref, M, ref))
    assert np.all(err <= 1e-12), err


def test_overint_rejected_on_mixed(dg):
    s = dg.Solver(dg_inputs.periodic_square(4), 2, "mixed", stream=stream())
    with pytest.raises(dg.DGError) as e:
        s.set_overint(True)
    assert e.value.status == -6
