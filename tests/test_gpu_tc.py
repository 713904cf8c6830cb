"""The tensor-core stage kernel (dg_set_stage_variant 3: one warp per tile of
two elements, Dr / Ds / LIFT products as mma.sync TF32 with three products
of split operands) against the oracle.

Tolerances are those of the mixed path (tests/_parity.py): residuals, per
field, 10 x the change of the oracle's residual under FP32 rounding of its
input state (the floor of any path that reads an FP32 copy of the state),
at every p; 2e-5 relative L2 per field after 100 steps.  The split products are good to about 2^-21 of
sum |A||B| and the operands are taken relative to the element's first node,
so the contraction error stays below the FP32 rounding of the state that
bounds the other mixed kernels."""
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


def rel_l2(P, d, ref):
    J, M = P.geo["J"], P.ops["M"]
    return np.sqrt(np.einsum("k,kcn,nm,kcm->c", J, d, M, d) / np.einsum("k,kcn,nm,kcm->c", J, ref, M, ref))


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("n", [5, 7])
def test_rhs_periodic_tc(dg, p, n):
    # K = 50 and 98 elements: several warp tiles and a ragged last tile
    mesh = dg_inputs.periodic_square(n)
    P = oracle.Problem(mesh, p, mu=5e-3)
    U = dg_inputs.perturb(to_kcn(dg_inputs.isentropic_vortex(P.x, P.y)), seed=7, amp=1e-2)
    vw = (0.07, -0.03)
    ref = P.rhs(U, vw=vw)
    s = dg.Solver(mesh, p, "mixed", stream=stream(), mu=5e-3)
    s.set_variant(3)
    assert s.variant == 3
    s.set_state(U)
    got = s.rhs(0.0, vw)
    check_rhs(P, U, got, "mixed", 0.0, vw, ref)


@pytest.mark.parametrize("adiabatic", [1, 0])
@pytest.mark.parametrize("p", [2, 3, 4, 5, 6])
def test_rhs_ogrid_wall_farfield_tc(dg, p, adiabatic):
    mesh = dg_inputs.ogrid_cylinder(24, 8, 0.5, 4.0, seed=3)
    kw = dict(mu=0.01, rho_inf=1.0, u_inf=1.0, v_inf=0.0, p_inf=17.857142857142858,
              adiabatic_zero_heatflux=adiabatic)
    P = oracle.Problem(mesh, p, **kw)
    r = np.hypot(P.x, P.y)
    U = to_kcn(dg_inputs.free_stream(P.x.shape, rho=1.0, u=1.0, v=0.0, p=kw["p_inf"]))
    U[:, 1] *= np.tanh(3 * (r - 0.5))
    U = dg_inputs.perturb(U, seed=11, amp=1e-3)
    vw = (0.0, 0.05)
    ref = P.rhs(U, vw=vw)
    s = dg.Solver(mesh, p, "mixed", stream=stream(), **kw)
    s.set_variant(3)
    s.set_state(U)
    got = s.rhs(0.0, vw)
    check_rhs(P, U, got, "mixed", 0.0, vw, ref)


def test_rhs_manufactured_source_tc(dg):
    kappa, C2 = 25.0, 200.0
    mesh = dg_inputs.periodic_square(4, L=4 * np.pi / kappa)
    P = oracle.Problem(mesh, 3, mu=0.01, source=("manufactured", kappa, C2))
    U = dg_inputs.perturb(to_kcn(oracle.manufactured_state(P.x, P.y, kappa, C2)), seed=2, amp=1e-4)
    ref = P.rhs(U)
    scale = max(np.abs(ref).max(), np.abs(oracle.Problem(mesh, 3, mu=0.01).rhs(U)).max())
    s = dg.Solver(mesh, 3, "mixed", stream=stream(), mu=0.01)
    s.set_variant(3)
    s.set_source(dg.DG_SOURCE_MANUFACTURED, (kappa, C2))
    s.set_state(U)
    got = s.rhs(0.0)
    # same bound as the other mixed kernels: FP32 state rounding amplified by
    # |E| / |variation of E| = 100 and the derivative row sums
    assert np.abs(got - ref).max() / scale <= 2e-4


@pytest.mark.parametrize("p", [2, 4, 6])
def test_vortex_100_steps_tc(dg, p):
    mesh = dg_inputs.periodic_square(10)
    P = oracle.Problem(mesh, p, mu=1e-3)
    U0 = dg_inputs.perturb(to_kcn(dg_inputs.isentropic_vortex(P.x, P.y)), seed=1)
    dt, _ = P.dt(U0, 0.3)
    ref = P.run(U0, 0.0, dt, 100)
    s = dg.Solver(mesh, p, "mixed", stream=stream(), mu=1e-3)
    s.set_variant(3)
    s.set_state(U0)
    s.steps(0.0, dt, 100)
    err = rel_l2(P, s.get_state() - ref, ref)
    assert np.all(err <= 2e-5), err


@pytest.mark.parametrize("variant", [2, 3])
def test_ogrid_steps_tc(dg, variant):
    """Wall and far-field faces with a moving mesh over 20 steps against the
    oracle (the two-node kernel alongside, on the same bound).  The free
    stream crosses at 0.4 so that no momentum field is near zero (the
    relative L2 error of a field whose values are round-off-sized says
    nothing)."""
    mesh = dg_inputs.ogrid_cylinder(32, 10, 0.5, 6.0, seed=5)
    kw = dict(mu=0.01, rho_inf=1.0, u_inf=1.0, v_inf=0.4, p_inf=17.857142857142858)
    P = oracle.Problem(mesh, 4, **kw)
    U0 = to_kcn(dg_inputs.free_stream(P.x.shape, rho=1.0, u=1.0, v=0.4, p=kw["p_inf"]))
    damp = np.tanh(3 * (np.hypot(P.x, P.y) - 0.5))
    U0[:, 1] *= damp
    U0[:, 2] *= damp
    U0 = dg_inputs.perturb(U0, seed=4, amp=1e-3)
    vw = (0.0, 0.02)
    dt, _ = P.dt(U0, 0.3, vw=vw)
    ref = P.run(U0, 0.0, dt, 20, vw=vw)
    s = dg.Solver(mesh, 4, "mixed", stream=stream(), **kw)
    s.set_variant(variant)
    s.set_state(U0)
    s.steps(0.0, dt, 20, vw)
    err = rel_l2(P, s.get_state() - ref, ref)
    assert np.all(err <= 2e-5), err


def test_tc_rejected_on_fp64_two_node_on_theta(dg):
    s = dg.Solver(dg_inputs.periodic_square(4), 3, "mixed", stream=stream(), theta=1.0, C1=0.05)
    with pytest.raises(dg.DGError) as e:
        s.set_variant(2)
    assert e.value.status == -6
    s = dg.Solver(dg_inputs.periodic_square(4), 3, "fp64", stream=stream())
    with pytest.raises(dg.DGError) as e:
        s.set_variant(3)
    assert e.value.status == -6


@pytest.mark.parametrize("theta", [1.0, -1.0, 0.5])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_rhs_periodic_tc_theta(dg, p, theta):
    """SIP / NIPG (theta terms of Eq. dg_on_K) in the tensor-core shape:
    theta vectors lifted by MMA, the weak-form derivatives Wr, Ws by MMA,
    FP64 jumps."""
    mesh = dg_inputs.periodic_square(5)
    P = oracle.Problem(mesh, p, mu=5e-3, theta=theta, C1=0.05)
    U = dg_inputs.perturb(to_kcn(dg_inputs.isentropic_vortex(P.x, P.y)), seed=3, amp=1e-2)
    vw = (0.05, 0.02)
    ref = P.rhs(U, vw=vw)
    s = dg.Solver(mesh, p, "mixed", stream=stream(), mu=5e-3, theta=theta, C1=0.05)
    s.set_variant(3)
    assert s.variant == 3
    s.set_state(U)
    got = s.rhs(0.0, vw)
    check_rhs(P, U, got, "mixed", 0.0, vw, ref)


@pytest.mark.parametrize("theta", [1.0, -1.0])
@pytest.mark.parametrize("p", [2, 4, 6])
def test_rhs_ogrid_tc_theta(dg, p, theta):
    mesh = dg_inputs.ogrid_cylinder(24, 8, 0.5, 4.0, seed=3)
    kw = dict(mu=0.01, rho_inf=1.0, u_inf=1.0, v_inf=0.0, p_inf=17.857142857142858, theta=theta, C1=0.05)
    P = oracle.Problem(mesh, p, **kw)
    r = np.hypot(P.x, P.y)
    U = to_kcn(dg_inputs.free_stream(P.x.shape, rho=1.0, u=1.0, v=0.0, p=kw["p_inf"]))
    U[:, 1] *= np.tanh(3 * (r - 0.5))
    U = dg_inputs.perturb(U, seed=12, amp=1e-3)
    vw = (0.0, 0.05)
    ref = P.rhs(U, vw=vw)
    s = dg.Solver(mesh, p, "mixed", stream=stream(), **kw)
    s.set_variant(3)
    s.set_state(U)
    got = s.rhs(0.0, vw)
    check_rhs(P, U, got, "mixed", 0.0, vw, ref)


def test_sip_50_steps_tc(dg):
    mesh = dg_inputs.periodic_square(8)
    p = 3
    P = oracle.Problem(mesh, p, mu=2e-3, theta=1.0, C1=0.1)
    U0 = dg_inputs.perturb(to_kcn(dg_inputs.isentropic_vortex(P.x, P.y)), seed=5, amp=1e-3)
    dt, _ = P.dt(U0, 0.3)
    ref = P.run(U0, 0.0, dt, 50)
    s = dg.Solver(mesh, p, "mixed", stream=stream(), mu=2e-3, theta=1.0, C1=0.1)
    s.set_variant(3)
    s.set_state(U0)
    s.steps(0.0, dt, 50)
    err = rel_l2(P, s.get_state() - ref, ref)
    assert np.all(err <= 2e-5), err


def _drop_element(mesh, k_drop):
    """The mesh without element k_drop: an odd element count, so the last
    two-element warp tile holds one element; the faces the removal exposes
    become far-field faces."""
    from dg_inputs.meshes import BC_FARFIELD, BC_INTERIOR, Mesh, _connect
    keep = np.array([k for k in range(mesh.K) if k != k_drop])
    EToV = mesh.EToV[keep].copy()
    EToE, EToF, owner = _connect(EToV, np.arange(mesh.Nv))
    bc = np.full(EToV.shape, BC_INTERIOR, dtype=np.int32)
    old_bc = mesh.bc[keep]
    for (k, f) in owner.values():
        bc[k, f] = old_bc[k, f] if old_bc[k, f] != BC_INTERIOR else BC_FARFIELD
    return Mesh(mesh.vx, mesh.vy, EToV, EToE.astype(np.int32), EToF.astype(np.int32), bc, None, "dropped")


@pytest.mark.parametrize("variant", [1, 2, 3])
@pytest.mark.parametrize("p", [2, 4, 6])
def test_rhs_odd_element_count(dg, p, variant):
    """A ragged last tile in every tile shape (383 elements: the last warp
    tile of the tensor-core shape holds one element), walls and far field."""
    if variant == 2 and p == 6:
        pytest.skip("covered at p = 2, 4")
    mesh = _drop_element(dg_inputs.ogrid_cylinder(24, 8, 0.5, 4.0, seed=3), 100)
    assert mesh.K % 2 == 1
    kw = dict(mu=0.01, rho_inf=1.0, u_inf=1.0, v_inf=0.2, p_inf=17.857142857142858)
    P = oracle.Problem(mesh, p, **kw)
    r = np.hypot(P.x, P.y)
    U = to_kcn(dg_inputs.free_stream(P.x.shape, rho=1.0, u=1.0, v=0.2, p=kw["p_inf"]))
    U[:, 1] *= np.tanh(3 * (r - 0.5))
    U = dg_inputs.perturb(U, seed=13, amp=1e-3)
    vw = (0.0, 0.03)
    ref = P.rhs(U, vw=vw)
    s = dg.Solver(mesh, p, "mixed", stream=stream(), **kw)
    s.set_variant(variant)
    s.set_state(U)
    got = s.rhs(0.0, vw)
    check_rhs(P, U, got, "mixed", 0.0, vw, ref)
