"""p = 6 (Np = 28) on an 80,000-triangle seeded O-grid (200 x 200 cells,
r in [0.5, 30], wall and far field), Re = 150, M = 0.2: the library against
the oracle, in both precisions: the residual per field, three LSRK steps
(state and increment per field, wall forces) and the time step."""
import numpy as np
import pytest

import dg_inputs
import oracle
from dg_inputs.states import to_kcn
from _parity import INC_TOL, check_rhs, inc_err, rel_l2

pytestmark = pytest.mark.gpu
GAMMA, MACH, RE = 1.4, 0.2, 150.0
P_INF = 1.0 / (GAMMA * MACH * MACH)
KW = dict(mu=1.0 / RE, rho_inf=1.0, u_inf=1.0, v_inf=0.0, p_inf=P_INF)
TOL = {"fp64": 1e-12, "mixed": 2e-5}
FORCE_TOL = {"fp64": 1e-10, "mixed": 1e-4}


@pytest.fixture(scope="module")
def case():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_17917_gb300 import build
    build.build()
    mesh = dg_inputs.ogrid_cylinder(200, 200, 0.5, 30.0, seed=6)
    assert mesh.K == 80000
    P = oracle.Problem(mesh, 6, **KW)
    r = np.hypot(P.x, P.y)
    U = to_kcn(dg_inputs.free_stream(P.x.shape, rho=1.0, u=1.0, v=0.0, p=P_INF))
    damp = np.tanh(4.0 * (r - 0.5))
    U[:, 1] *= damp
    U[:, 2] = 0.1 * damp * np.sin(np.arctan2(P.y, P.x))     # some cross-flow, so no field is zero
    U[:, 3] = P_INF / (GAMMA - 1) + 0.5 * (U[:, 1] ** 2 + U[:, 2] ** 2) / U[:, 0]
    U0 = dg_inputs.perturb(U, seed=3, amp=1e-3)
    dt, _ = P.dt(U0, 0.3)
    ref = P.run(U0, 0.0, dt, 3)
    return mesh, P, U0, dt, ref, P.wall_forces(ref)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_p6_80k_three_steps(case, precision):
    import torch
    import paper_2508_17917_gb300 as dg
    mesh, P, U0, dt, ref, F_ref = case
    s = dg.Solver(mesh, 6, precision, stream=torch.cuda.current_stream().cuda_stream, **KW)
    s.set_state(U0)
    check_rhs(P, U0, s.rhs(0.0), precision)
    assert abs(s.dt(0.3) - dt) <= 1e-12 * dt
    s.steps(0.0, dt, 3)
    got = s.get_state()
    err = rel_l2(P, got - ref, ref)
    assert np.all(err <= TOL[precision]), err
    # the state moves by ~1e-6 of itself in three steps: the increment is
    # what tells an updated state from a stale one
    inc = inc_err(P, got, ref, U0)
    assert np.all(inc <= INC_TOL[precision]), inc
    F = s.wall_forces()
    assert np.all(np.abs(F - F_ref) <= FORCE_TOL[precision] * np.abs(F_ref).max()), (F, F_ref)
