"""dg_broken_gradient against the oracle's broken gradient (Sec. 2.2).

impl 0 (FP64 on the CUDA cores) within 1e-12 of each field's largest
gradient entry; impl 1 (tcgen05 kind::tf32 with three split products and
TMA-staged tiles) within 2e-5, the mixed path's bound (the split products
are good to about 2^-21 of sum |D||U - U_first|, the FP32 rounding of U -
U_first to 2^-24 of it).  Degrees 1..6, element counts that are and are not
whole 32-element tiles (the last tile's rows past K are read as zeros), the
O-grid with its small wall cells, and the benchmark mesh at full size."""
import numpy as np
import pytest

import dg_inputs
import oracle
from dg_inputs.states import to_kcn

pytestmark = pytest.mark.gpu
TOL = {0: 1e-12, 1: 2e-5}


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


def field_err(got, ref):
    return np.abs(got - ref).max(axis=(0, 2)) / np.abs(ref).max(axis=(0, 2))


def vortex(P, seed):
    return dg_inputs.perturb(to_kcn(dg_inputs.isentropic_vortex(P.x, P.y)), seed=seed, amp=1e-2)


@pytest.mark.parametrize("impl", [0, 1])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("n", [4, 5])
def test_gradient_periodic(dg, p, n, impl):
    # K = 32 (one whole tile) and K = 50 (a ragged second tile)
    mesh = dg_inputs.periodic_square(n)
    P = oracle.Problem(mesh, p, mu=1e-3)
    U = vortex(P, p)
    rx, ry = P.broken_gradient(U)
    s = dg.Solver(mesh, p, "fp64", stream=stream(), mu=1e-3)
    s.set_state(U)
    gx, gy = s.broken_gradient(impl)
    assert np.all(field_err(gx, rx) <= TOL[impl]), field_err(gx, rx)
    assert np.all(field_err(gy, ry) <= TOL[impl]), field_err(gy, ry)


@pytest.mark.parametrize("impl", [0, 1])
@pytest.mark.parametrize("p", [2, 4, 6])
def test_gradient_ogrid(dg, p, impl):
    mesh = dg_inputs.ogrid_cylinder(24, 8, 0.5, 4.0, seed=3)
    kw = dict(mu=0.01, rho_inf=1.0, u_inf=1.0, v_inf=0.0, p_inf=17.857142857142858)
    P = oracle.Problem(mesh, p, **kw)
    r = np.hypot(P.x, P.y)
    U = to_kcn(dg_inputs.free_stream(P.x.shape, rho=1.0, u=1.0, v=0.0, p=kw["p_inf"]))
    U[:, 1] *= np.tanh(3 * (r - 0.5))
    U[:, 2] = 0.05 * np.sin(np.arctan2(P.y, P.x))
    U = dg_inputs.perturb(U, seed=11, amp=1e-3)
    rx, ry = P.broken_gradient(U)
    s = dg.Solver(mesh, p, "mixed", stream=stream(), **kw)
    s.set_state(U)
    gx, gy = s.broken_gradient(impl)
    assert np.all(field_err(gx, rx) <= TOL[impl]), field_err(gx, rx)
    assert np.all(field_err(gy, ry) <= TOL[impl]), field_err(gy, ry)


def test_gradient_full_size_device_outputs(dg):
    """The benchmark mesh (K = 32,768, p = 4), both implementations into
    device tensors, against the oracle."""
    import torch
    mesh = dg_inputs.periodic_square(128)
    P = oracle.Problem(mesh, 4, mu=1e-3)
    U = vortex(P, 0)
    rx, ry = P.broken_gradient(U)
    s = dg.Solver(mesh, 4, "mixed", stream=stream(), mu=1e-3)
    s.set_state(U)
    for impl in (0, 1):
        gx = torch.empty(U.shape, dtype=torch.float64, device="cuda")
        gy = torch.empty_like(gx)
        dg.dg_broken_gradient(s.ctx, gx, gy, impl)
        torch.cuda.synchronize()
        assert np.all(field_err(gx.cpu().numpy(), rx) <= TOL[impl])
        assert np.all(field_err(gy.cpu().numpy(), ry) <= TOL[impl])


@pytest.mark.parametrize("p,n", [(6, 75), (3, 131)])
def test_gradient_many_tiles_ragged(dg, p, n):
    """Hundreds of tiles with a ragged last one (K = 11,250 at p = 6, 34,322
    at p = 3) into device outputs that start as NaN, so a row that no tile
    writes fails; a second call reuses the operator image uploaded by the
    first."""
    import torch
    mesh = dg_inputs.periodic_square(n)
    P = oracle.Problem(mesh, p, mu=1e-3)
    U = vortex(P, 1)
    rx, ry = P.broken_gradient(U)
    s = dg.Solver(mesh, p, "mixed", stream=stream(), mu=1e-3)
    s.set_state(U)
    gx = torch.full(U.shape, float("nan"), dtype=torch.float64, device="cuda")
    gy = torch.full(U.shape, float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):
        dg.dg_broken_gradient(s.ctx, gx, gy, 1)
        dg.dg_barrier_status(s.ctx)
        assert np.all(field_err(gx.cpu().numpy(), rx) <= TOL[1])
        assert np.all(field_err(gy.cpu().numpy(), ry) <= TOL[1])
        gx.fill_(float("nan"))
        gy.fill_(float("nan"))



def test_gradient_unaligned_device_outputs(dg):
    """Device outputs that start 8 bytes past a 16-byte boundary cannot take
    the bulk tile stores; the kernel stores rows instead, with the same
    results."""
    import torch
    mesh = dg_inputs.periodic_square(5)
    P = oracle.Problem(mesh, 4, mu=1e-3)
    U = vortex(P, 3)
    rx, ry = P.broken_gradient(U)
    s = dg.Solver(mesh, 4, "mixed", stream=stream(), mu=1e-3)
    s.set_state(U)
    n = U.size
    buf = torch.full((2 * n + 2,), float("nan"), dtype=torch.float64, device="cuda")
    gx, gy = buf[1:n + 1], buf[n + 2:]               # 8-byte and 16-byte aligned
    assert gx.data_ptr() % 16 == 8
    dg.dg_broken_gradient(s.ctx, gx, gy, 1)
    dg.dg_barrier_status(s.ctx)
    assert np.all(field_err(gx.cpu().numpy().reshape(U.shape), rx) <= TOL[1])
    assert np.all(field_err(gy.cpu().numpy().reshape(U.shape), ry) <= TOL[1])
