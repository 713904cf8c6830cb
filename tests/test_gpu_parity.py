"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Same seeded inputs on both sides; tolerances (derived in tests/_parity.py):
* FP64 path: residuals <= 1e-12 relative to the largest entry and <= 1e-11
  per field; state <= 1e-12 relative L2 per conserved field after 100 LSRK
  steps; increments U_n - U_0 <= 1e-9 per field;
* mixed path (FP32 arithmetic, FP64 state / pressure / registers): residuals,
  per field, <= 10 x the change of the oracle's own residual under FP32
  rounding of its input; state <= 2e-5; increments <= 5e-4 per field;
* time step, wall forces (FP64 on both sides): <= 1e-12 relative.
The increment checks are what a run that skipped its stage updates fails:
over a few steps the state moves by far less than 2e-5 of itself.
"""
import numpy as np
import pytest

import dg_inputs
import oracle
from dg_inputs.states import to_kcn
from _parity import (INC_TOL, STATE_TOL, check_rhs, fp32_sensitivity, field_err, inc_err,
                     MIXED_SENS, rel_l2)

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


def vortex_state(P, seed):
    U = to_kcn(dg_inputs.isentropic_vortex(P.x, P.y))
    return dg_inputs.perturb(U, seed=seed, amp=1e-3)


PREC_TOL = STATE_TOL


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_rhs_periodic(dg, p, precision):
    mesh = dg_inputs.periodic_square(5)
    P = oracle.Problem(mesh, p, mu=5e-3)
    U = dg_inputs.perturb(vortex_state(P, 1), seed=7, amp=1e-2)
    vw = (0.07, -0.03)
    ref = P.rhs(U, vw=vw)
    s = dg.Solver(mesh, p, precision, stream=stream(), mu=5e-3)
    s.set_state(U)
    got = s.rhs(0.0, vw)
    check_rhs(P, U, got, precision, 0.0, vw, ref)


@pytest.mark.parametrize("adiabatic", [1, 0])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("p", [2, 4])
def test_rhs_ogrid_wall_farfield(dg, p, precision, adiabatic):
    mesh = dg_inputs.ogrid_cylinder(24, 8, 0.5, 4.0, seed=3)
    kw = dict(mu=0.01, rho_inf=1.0, u_inf=1.0, v_inf=0.0, p_inf=17.857142857142858,
              adiabatic_zero_heatflux=adiabatic)
    P = oracle.Problem(mesh, p, **kw)
    r = np.hypot(P.x, P.y)
    # free stream with a smooth no-slip-like deficit near the wall and a perturbation
    U = to_kcn(dg_inputs.free_stream(P.x.shape, rho=1.0, u=1.0, v=0.0, p=kw["p_inf"]))
    U[:, 1] *= np.tanh(3 * (r - 0.5))
    U = dg_inputs.perturb(U, seed=11, amp=1e-3)
    vw = (0.0, 0.05)
    ref = P.rhs(U, vw=vw)
    s = dg.Solver(mesh, p, precision, stream=stream(), **kw)
    s.set_state(U)
    got = s.rhs(0.0, vw)
    check_rhs(P, U, got, precision, 0.0, vw, ref)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_rhs_manufactured_source(dg, precision):
    kappa, C2 = 25.0, 200.0
    mesh = dg_inputs.periodic_square(4, L=4 * np.pi / kappa)
    P = oracle.Problem(mesh, 3, mu=0.01, source=("manufactured", kappa, C2))
    U = dg_inputs.perturb(to_kcn(oracle.manufactured_state(P.x, P.y, kappa, C2)), seed=2, amp=1e-4)
    ref = P.rhs(U)
    # near the steady solution the flux terms cancel the source: measure the
    # error against the size of the terms that cancel
    P0 = oracle.Problem(mesh, 3, mu=0.01)
    scale = max(np.abs(ref).max(), np.abs(P0.rhs(U)).max())
    s = dg.Solver(mesh, 3, precision, stream=stream(), mu=0.01)
    s.set_source(dg.DG_SOURCE_MANUFACTURED, (kappa, C2))
    s.set_state(U)
    got = s.rhs(0.0)
    err = np.abs(got - ref).max() / scale
    # Mixed path: the state enters FP32 with relative rounding 2^-24 = 6e-8 of
    # |U|; for this state |E| / |variation of E| = C2 / 2 = 100, and the
    # derivative operators amplify by max_i sum_j |Dr_ij| h / 2 ~ 10 at p = 3,
    # so the residual is good to about 6e-8 * 100 * 10 = 6e-5 of its terms.
    assert err <= (1e-12 if precision == "fp64" else 2e-4), err
    # per field, against the size of the terms that cancel in that field
    fscale = np.maximum(np.abs(ref).max(axis=(0, 2)), np.abs(P0.rhs(U)).max(axis=(0, 2)))
    ef = field_err(got, ref, fscale)
    if precision == "fp64":
        assert np.all(ef <= 1e-11), ef
    else:
        assert np.all(ef <= MIXED_SENS * fp32_sensitivity(P, U, scale=fscale)), ef


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_manufactured_100_steps(dg, precision):
    """The manufactured steady state of Sec. 3.1 advanced 100 steps: state
    error within the path's tolerance (the residual-level FP32 error above is
    multiplied by dt, so the state keeps its digits)."""
    kappa, C2 = 25.0, 200.0
    mesh = dg_inputs.periodic_square(4, L=4 * np.pi / kappa)
    P = oracle.Problem(mesh, 3, mu=0.01, source=("manufactured", kappa, C2))
    U0 = dg_inputs.perturb(to_kcn(oracle.manufactured_state(P.x, P.y, kappa, C2)), seed=3, amp=1e-4)
    dt, _ = P.dt(U0, 0.3)
    ref = P.run(U0, 0.0, dt, 100)
    s = dg.Solver(mesh, 3, precision, stream=stream(), mu=0.01)
    s.set_source(dg.DG_SOURCE_MANUFACTURED, (kappa, C2))
    s.set_state(U0)
    s.steps(0.0, dt, 100)
    got = s.get_state()
    err = rel_l2(P, got - ref, ref)
    assert np.all(err <= PREC_TOL[precision]), err
    # near the steady state the net residual is the small remainder of
    # cancelling terms, so only the FP64 path resolves the increment itself
    if precision == "fp64":
        assert np.all(inc_err(P, got, ref, U0) <= INC_TOL[precision])


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_vortex_p2_100_steps(dg, precision, seed):
    """Isentropic vortex, p = 2, 16 x 16 split quads (K = 512), mu = 1e-3,
    100 LSRK steps at CFL 0.3 fixed at t = 0, seeded perturbation."""
    mesh = dg_inputs.periodic_square(16)
    P = oracle.Problem(mesh, 2, mu=1e-3)
    U0 = vortex_state(P, seed)
    dt, _ = P.dt(U0, 0.3)
    ref = P.run(U0, 0.0, dt, 100)
    s = dg.Solver(mesh, 2, precision, stream=stream(), mu=1e-3)
    s.set_state(U0)
    s.steps(0.0, dt, 100)
    got = s.get_state()
    err = rel_l2(P, got - ref, ref)
    assert np.all(err <= PREC_TOL[precision]), err
    assert np.all(inc_err(P, got, ref, U0) <= INC_TOL[precision])
    assert s.check_finite()


_FULL = {}


def _full_size_reference():
    """Oracle run of the benchmark workload: 100 steps (shared by the cases
    below; about 35 s on 16 host cores)."""
    if not _FULL:
        mesh = dg_inputs.periodic_square(128)
        P = oracle.Problem(mesh, 4, mu=1e-3)
        U0 = vortex_state(P, 0)
        dt, _ = P.dt(U0, 0.3)
        _FULL.update(mesh=mesh, P=P, U0=U0, dt=dt, ref=P.run(U0, 0.0, dt, 100))
    return _FULL


@pytest.mark.parametrize("precision,variant", [("fp64", 0), ("mixed", 0), ("mixed", 3)])
def test_vortex_p4_full_size_100_steps(dg, precision, variant):
    """p = 4, 128 x 128 split quads (K = 32,768), the benchmark's launch
    configuration (tile shape from the tuner; also the tensor-core shape
    forced): residual per field, then 100 steps, state and increment per
    field."""
    f = _full_size_reference()
    P, U0, ref = f["P"], f["U0"], f["ref"]
    s = dg.Solver(f["mesh"], 4, precision, stream=stream(), mu=1e-3)
    if variant:
        s.set_variant(variant)
    s.set_state(U0)
    check_rhs(P, U0, s.rhs(0.0), precision)
    s.steps(0.0, f["dt"], 100)
    got = s.get_state()
    err = rel_l2(P, got - ref, ref)
    assert np.all(err <= PREC_TOL[precision]), err
    inc = inc_err(P, got, ref, U0)
    assert np.all(inc <= INC_TOL[precision]), inc


@pytest.mark.parametrize("p", [2, 4])
def test_dt_matches_oracle(dg, p):
    mesh = dg_inputs.ogrid_cylinder(24, 8, 0.5, 4.0, seed=3)
    kw = dict(mu=0.01, rho_inf=1.0, u_inf=1.0, v_inf=0.0, p_inf=17.857142857142858)
    P = oracle.Problem(mesh, p, **kw)
    U = dg_inputs.perturb(to_kcn(dg_inputs.free_stream(P.x.shape, u=1.0, p=kw["p_inf"])), seed=4, amp=1e-2)
    vw = (0.0, 0.02)
    ref, _ = P.dt(U, 0.3, vw)
    s = dg.Solver(mesh, p, "fp64", stream=stream(), **kw)
    s.set_state(U)
    got = s.dt(0.3, vw)
    assert abs(got - ref) <= 1e-12 * ref


@pytest.mark.parametrize("p", [2, 4])
def test_wall_forces_match_oracle(dg, p):
    mesh = dg_inputs.ogrid_cylinder(24, 8, 0.5, 4.0, seed=3)
    kw = dict(mu=0.01, rho_inf=1.0, u_inf=1.0, v_inf=0.0, p_inf=17.857142857142858)
    P = oracle.Problem(mesh, p, **kw)
    r = np.hypot(P.x, P.y)
    U = to_kcn(dg_inputs.free_stream(P.x.shape, u=1.0, p=kw["p_inf"]))
    U[:, 1] *= np.tanh(3 * (r - 0.5)) * (1 + 0.1 * P.y)
    U = dg_inputs.perturb(U, seed=5, amp=1e-3)
    ref = P.wall_forces(U, (0.0, 0.0))
    s = dg.Solver(mesh, p, "mixed", stream=stream(), **kw)
    s.set_state(U)
    got = s.wall_forces((0.0, 0.0))
    assert np.all(np.abs(got - ref) <= 1e-12 * np.abs(ref).max()), (got, ref)


def test_free_stream_preserved_mixed(dg):
    mesh = dg_inputs.periodic_square(8)
    s = dg.Solver(mesh, 4, "mixed", stream=stream(), mu=1e-3)
    x, y = s.node_coords()
    U = to_kcn(dg_inputs.free_stream(x.shape, rho=1.0, u=0.35, v=0.1, p=1.0))
    s.set_state(U)
    R = s.rhs(0.0, (0.02, 0.0))
    # FP32 arithmetic: the discrete divergence of a constant flux vanishes only
    # to rounding (sum_j Dr_ij = 0 up to 2^-24 |Dr|), so the residual is at
    # the 1e-6 level and 10 steps of dt = 1e-3 move the state by <= 1e-7
    assert np.abs(R).max() < 1e-5
    s.steps(0.0, 1e-3, 10)
    assert np.abs(s.get_state() - U).max() < 1e-7


def test_check_finite_and_bad_mesh(dg):
    mesh = dg_inputs.periodic_square(4)
    s = dg.Solver(mesh, 2, "fp64", stream=stream())
    x, y = s.node_coords()
    U = to_kcn(dg_inputs.free_stream(x.shape))
    U[3, 2, 1] = np.nan
    s.set_state(U)
    assert not s.check_finite()
    bad = dg_inputs.periodic_square(4)
    bad.EToV = bad.EToV[:, [0, 2, 1]].copy()          # clockwise elements
    with pytest.raises(dg.DGError) as e:
        dg.Solver(bad, 2, "fp64", stream=stream())
    assert e.value.status == -2


def test_device_state_roundtrip_and_launch_count(dg):
    import torch
    mesh = dg_inputs.periodic_square(6)
    s = dg.Solver(mesh, 3, "mixed", stream=stream())
    x, y = s.node_coords()
    U = to_kcn(dg_inputs.isentropic_vortex(x, y, L=10.0))
    Ud = torch.tensor(U, device="cuda")
    s.set_state(Ud)
    n0 = s.launches
    s.steps(0.0, 1e-4, 4)
    # 5 stage launches per step; the first step also times the three tile
    # shapes of the mixed kernel at p <= 4 (5 residual-only launches each)
    assert s.launches - n0 == 20 + 15
    assert s.variant in (1, 2, 3)
    n1 = s.launches
    s.steps(0.0, 1e-4, 3)
    assert s.launches - n1 == 15
    out = torch.empty_like(Ud)
    dg.dg_get_state(s.ctx, out)
    torch.cuda.synchronize()
    assert np.allclose(out.cpu().numpy(), s.get_state())
