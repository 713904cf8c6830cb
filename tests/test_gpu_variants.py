"""Both tile shapes of the mixed-precision stage kernel against the oracle:
one node per thread (variant 1) and two volume nodes plus two face nodes of
one face per thread (variant 2), forced through dg_set_stage_variant; and the
first-step tuner's choice.  Tolerances as for the mixed path
(tests/_parity.py): residuals, per field, 10 x the change of the oracle's
residual under FP32 rounding of its input state, at every p."""
import numpy as np
import pytest

import dg_inputs
import oracle
from dg_inputs.states import to_kcn
from _parity import check_rhs

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


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_rhs_periodic_variant(dg, p, variant):
    mesh = dg_inputs.periodic_square(5)
    P = oracle.Problem(mesh, p, mu=5e-3)
    U = dg_inputs.perturb(to_kcn(dg_inputs.isentropic_vortex(P.x, P.y)), seed=7, amp=1e-2)
    vw = (0.07, -0.03)
    ref = P.rhs(U, vw=vw)
    s = dg.Solver(mesh, p, "mixed", stream=stream(), mu=5e-3)
    s.set_variant(variant)
    assert s.variant == variant
    s.set_state(U)
    got = s.rhs(0.0, vw)
    check_rhs(P, U, got, "mixed", 0.0, vw, ref)


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("p", [2, 4, 6])
def test_rhs_ogrid_variant(dg, p, variant):
    mesh = dg_inputs.ogrid_cylinder(24, 8, 0.5, 4.0, seed=3)
    kw = dict(mu=0.01, rho_inf=1.0, u_inf=1.0, v_inf=0.0, p_inf=17.857142857142858)
    P = oracle.Problem(mesh, p, **kw)
    r = np.hypot(P.x, P.y)
    U = to_kcn(dg_inputs.free_stream(P.x.shape, rho=1.0, u=1.0, v=0.0, p=kw["p_inf"]))
    U[:, 1] *= np.tanh(3 * (r - 0.5))
    U = dg_inputs.perturb(U, seed=11, amp=1e-3)
    vw = (0.0, 0.05)
    ref = P.rhs(U, vw=vw)
    s = dg.Solver(mesh, p, "mixed", stream=stream(), **kw)
    s.set_variant(variant)
    s.set_state(U)
    got = s.rhs(0.0, vw)
    check_rhs(P, U, got, "mixed", 0.0, vw, ref)


@pytest.mark.parametrize("variant", [2, 0])
def test_vortex_steps_variant(dg, variant):
    mesh = dg_inputs.periodic_square(16)
    P = oracle.Problem(mesh, 2, mu=1e-3)
    U0 = dg_inputs.perturb(to_kcn(dg_inputs.isentropic_vortex(P.x, P.y)), seed=1)
    dt, _ = P.dt(U0, 0.3)
    ref = P.run(U0, 0.0, dt, 100)
    s = dg.Solver(mesh, 2, "mixed", stream=stream(), mu=1e-3)
    s.set_variant(variant)
    s.set_state(U0)
    s.steps(0.0, dt, 100)
    got = s.get_state()
    d = got - ref
    J, M = P.geo["J"], P.ops["M"]
    err = np.sqrt(np.einsum("k,kcn,nm,kcm->c", J, d, M, d) / np.einsum("k,kcn,nm,kcm->c", J, ref, M, ref))
    assert np.all(err <= 2e-5), err
    assert s.variant in (1, 2, 3)


def test_variant_two_rejected_on_fp64(dg):
    mesh = dg_inputs.periodic_square(4)
    s = dg.Solver(mesh, 2, "fp64", stream=stream())
    with pytest.raises(dg.DGError) as e:
        s.set_variant(2)
    assert e.value.status == -6
