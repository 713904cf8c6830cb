"""Fused steps: the five stages of Algorithm 1 in one cooperative launch with
grid barriers between stages (dg_set_fused_steps).

* The same result as five stage launches, for every tile shape, on the
  periodic vortex and on the O-grid with wall and far-field faces: equal to
  within 1e-9 of the largest state value (the fused kernels are separate
  instantiations, so the compiler may contract a multiply-add differently;
  seen: a 3.6e-12 relative difference after 10 steps at wall elements with
  the two-node shape, none elsewhere), and bit-identical from run to run.
* One launch per step.
* The bounded barrier wait: with a limit of zero waits every barrier gives
  up at once; the launch ends early, dg_barrier_status reports DG_ETIMEOUT,
  and after the limit is restored and the state reset the fused steps match
  again.  (No wait can run longer than the limit: nothing hangs.)
"""
import numpy as np
import pytest

import dg_inputs
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


def vortex_case():
    mesh = dg_inputs.periodic_square(32)
    return mesh, 4, dict(mu=1e-3), None


def ogrid_case():
    mesh = dg_inputs.ogrid_cylinder(40, 12, 0.5, 6.0, seed=4)
    kw = dict(mu=0.01, rho_inf=1.0, u_inf=1.0, v_inf=0.0, p_inf=17.857142857142858)
    return mesh, 3, kw, (0.0, 0.02)


def start(s, kw):
    x, y = s.node_coords()
    if "p_inf" in kw:
        U = to_kcn(dg_inputs.free_stream(x.shape, rho=1.0, u=1.0, v=0.0, p=kw["p_inf"]))
        U[:, 1] *= np.tanh(3 * (np.hypot(x, y) - 0.5))
    else:
        U = to_kcn(dg_inputs.isentropic_vortex(x, y))
    return dg_inputs.perturb(U, seed=2, amp=1e-3)


@pytest.mark.parametrize("variant", [1, 2, 3])
@pytest.mark.parametrize("case", [vortex_case, ogrid_case])
def test_fused_steps_match_five_launches(dg, case, variant):
    mesh, p, kw, vw = case()
    out = []
    for fused in (False, True, True):
        s = dg.Solver(mesh, p, "mixed", stream=stream(), **kw)
        s.set_variant(variant)
        s.set_fused(fused)
        U0 = start(s, kw)
        s.set_state(U0)
        dt = s.dt(0.3, vw)
        n0 = s.launches
        s.steps(0.0, dt, 10, vw)
        launches = s.launches - n0
        out.append(s.get_state())
        assert launches == (10 if fused else 50)
        dg.dg_barrier_status(s.ctx)
    assert np.array_equal(out[1], out[2])                      # deterministic
    assert np.abs(out[1] - out[0]).max() <= 1e-9 * np.abs(out[0]).max()
    assert np.all(np.isfinite(out[1]))


def test_barrier_wait_limit_reports_timeout(dg):
    mesh, p, kw, vw = vortex_case()
    ref = dg.Solver(mesh, p, "mixed", stream=stream(), **kw)
    ref.set_variant(1)
    ref.set_fused(True)
    U0 = start(ref, kw)
    ref.set_state(U0)
    dt = ref.dt(0.3)
    ref.steps(0.0, dt, 2)
    want = ref.get_state()

    s = dg.Solver(mesh, p, "mixed", stream=stream(), **kw)
    s.set_variant(1)
    s.set_fused(True)
    s.set_state(U0)
    dg.dg_set_barrier_limit(s.ctx, 0)            # every barrier wait gives up at once
    s.steps(0.0, dt, 1)
    with pytest.raises(dg.DGError) as e:
        dg.dg_barrier_status(s.ctx)
    assert e.value.status == -5
    dg.dg_barrier_status(s.ctx)                  # the flag was cleared
    dg.dg_set_barrier_limit(s.ctx, 1 << 24)
    s.set_state(U0)
    s.steps(0.0, dt, 2)
    assert np.array_equal(s.get_state(), want)


def test_fused_rejected_on_fp64(dg):
    s = dg.Solver(dg_inputs.periodic_square(4), 2, "fp64", stream=stream())
    with pytest.raises(dg.DGError) as e:
        s.set_fused(True)
    assert e.value.status == -6


def test_tc_copy_wait_limit_reports_or_completes(dg):
    """The tensor-core stage kernel stages its operator table and each warp's
    own element records with bulk copies on mbarriers, and every wait on them
    is bounded by the same limit as the grid barriers.  With a zero limit a
    wait gives up unless its copy has already landed, so the run either
    completes with the reference state or reports DG_ETIMEOUT from the
    synchronising state read; either way nothing hangs, and with the limit
    restored the context reproduces the reference bit for bit."""
    mesh, p, kw, vw = vortex_case()
    ref = dg.Solver(mesh, p, "mixed", stream=stream(), **kw)
    ref.set_variant(3)
    U0 = start(ref, kw)
    ref.set_state(U0)
    dt = ref.dt(0.3)
    ref.steps(0.0, dt, 2)
    want = ref.get_state()

    s = dg.Solver(mesh, p, "mixed", stream=stream(), **kw)
    s.set_variant(3)
    s.set_state(U0)
    dg.dg_set_barrier_limit(s.ctx, 0)
    s.steps(0.0, dt, 2)
    try:
        got = s.get_state()
        assert np.array_equal(got, want)
    except dg.DGError as e:
        assert e.status == -5
    dg.dg_barrier_status(s.ctx)                  # nothing left to report
    dg.dg_set_barrier_limit(s.ctx, 1 << 24)
    s.set_state(U0)
    s.steps(0.0, dt, 2)
    assert np.array_equal(s.get_state(), want)
