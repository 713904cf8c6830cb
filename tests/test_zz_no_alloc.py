"""dg_wall_forces_noalloc: the wall force and moment for callers that may not
allocate device memory when they ask for them (for example code whose device
memory is owned by another allocator, or a loop that must not risk the
synchronisation of a cudaFree).

The call keeps its partial sums in a fixed array inside the library instead
of a mesh buffer.  These checks go through the C ABI: two calls in a row must
reproduce dg_wall_forces within the FP64 tolerance of the other tests, and a
mesh with more wall faces than the array holds must be refused with a clear
message.  The file is named to be collected last.
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


def wall_state(x, y, p_inf):
    r = np.hypot(x, y)
    U = to_kcn(dg_inputs.free_stream(x.shape, u=1.0, p=p_inf))
    U[:, 1] *= np.tanh(3 * (r - 0.5)) * (1 + 0.1 * y)
    U[:, 2] += 0.05 * np.sin(2.0 * x)
    return dg_inputs.perturb(U, seed=21, amp=1e-3)


@pytest.mark.parametrize("p", [2, 4])
def test_noalloc_matches_wall_forces_twice(dg, p):
    mesh = dg_inputs.ogrid_cylinder(48, 6, 0.5, 3.0, seed=4)
    kw = dict(mu=0.01, rho_inf=1.0, u_inf=1.0, v_inf=0.0, p_inf=17.857142857142858)
    s = dg.Solver(mesh, p, "mixed", stream=stream(), **kw)
    x, y = s.node_coords()
    s.set_state(wall_state(x, y, kw["p_inf"]))
    for xc in [(0.0, 0.0), (0.1, -0.2)]:
        ref = s.wall_forces(xc)
        first = dg.dg_wall_forces_noalloc(s.ctx, xc)
        second = dg.dg_wall_forces_noalloc(s.ctx, xc)
        scale = np.abs(ref).max()
        assert np.all(np.abs(first - ref) <= 1e-12 * scale), (first, ref)
        assert np.all(np.abs(second - ref) <= 1e-12 * scale), (second, ref)


def test_noalloc_rejects_too_many_wall_faces(dg):
    n = dg.DG_NOALLOC_MAX_WALL_FACES + 16
    mesh = dg_inputs.ogrid_cylinder(n, 1, 0.5, 0.6, seed=0)
    s = dg.Solver(mesh, 1, "fp64", stream=stream(), mu=0.01, u_inf=0.0, p_inf=1.0)
    with pytest.raises(dg.DGError) as e:
        dg.dg_wall_forces_noalloc(s.ctx, (0.0, 0.0))
    assert e.value.status == -1
    assert "wall faces" in str(e.value) and "dg_wall_forces" in str(e.value)


def test_noalloc_at_the_limit_allocates_nothing(dg):
    """Exactly DG_NOALLOC_MAX_WALL_FACES wall faces (the largest accepted
    size): the result matches dg_wall_forces, and after a first call (which
    looks up the array's address) further calls leave the device's free
    memory unchanged -- any cudaMalloc would take at least one 2 MB page."""
    import torch
    n = dg.DG_NOALLOC_MAX_WALL_FACES
    mesh = dg_inputs.ogrid_cylinder(n, 1, 0.5, 0.6, seed=0)
    kw = dict(mu=0.01, rho_inf=1.0, u_inf=1.0, v_inf=0.0, p_inf=17.857142857142858)
    s = dg.Solver(mesh, 1, "fp64", stream=stream(), **kw)
    x, y = s.node_coords()
    s.set_state(wall_state(x, y, kw["p_inf"]))
    ref = s.wall_forces((0.0, 0.0))
    first = dg.dg_wall_forces_noalloc(s.ctx, (0.0, 0.0))
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    again = [dg.dg_wall_forces_noalloc(s.ctx, (0.0, 0.0)) for _ in range(3)]
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    scale = np.abs(ref).max()
    for got in [first] + again:
        assert np.all(np.abs(got - ref) <= 1e-12 * scale), (got, ref)
