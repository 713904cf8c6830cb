"""Convergence of the GPU path to an exact Navier-Stokes solution.

With the viscous vortex source (dg_set_source DG_SOURCE_VORTEX: S =
-div F_v of the advected isentropic vortex) the vortex is an exact solution
of the viscous equations, so the error of the discrete solution after a
fixed time measures the discretisation alone.  The FP64 path reaches the
design order p + 1 (rate between 16^2 and 32^2 split quads at least
p + 0.5; the paper reports about p to p + 1 for its manufactured case), and
the mixed path's error equals it to 1e-3 of its size plus 1e-8: the FP32
rounding of the residual, accumulated over the few thousand steps to t =
0.5 on states of order one, stays below that.  Measured (RMS nodal error,
FP64 path, 8^2 / 16^2 / 32^2 / 64^2): p = 1: 6.8e-2, 1.6e-2, 3.5e-3, 7.8e-4;
p = 2: 1.9e-2, 3.2e-3, 3.7e-4, 4.7e-5; p = 3: 7.8e-3, 4.4e-4, 2.8e-5, 2.1e-6;
p = 4: 1.6e-3, 6.8e-5, 2.3e-6, 9.0e-7.  The p = 4 value on 64^2 sits on a
floor: the vortex is not periodic (its velocity perturbation is about 2e-5
at the domain edge), so the exact solution built from the nearest periodic
image has a mismatch there that no resolution removes; the test stops at
32^2."""
import numpy as np
import pytest

import dg_inputs
from dg_inputs.states import to_kcn

pytestmark = pytest.mark.gpu
GAMMA, MACH, MU, T = 1.4, 0.3, 0.02, 0.5
U0 = MACH * np.sqrt(GAMMA)
SRC = (5.0, 5.0, 5.0, 10.0, U0, 0.0)


@pytest.fixture(scope="module")
def dg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_17917_gb300 import build
    build.build()
    import paper_2508_17917_gb300 as dg
    return dg


def error(dg, n, p, precision):
    import torch
    mesh = dg_inputs.periodic_square(n)
    s = dg.Solver(mesh, p, precision, stream=torch.cuda.current_stream().cuda_stream, mu=MU)
    s.set_source(dg.DG_SOURCE_VORTEX, SRC)
    x, y = s.node_coords()
    s.set_state(to_kcn(dg_inputs.isentropic_vortex(x, y)))
    dt0 = s.dt(0.3)
    ns = int(np.ceil(T / dt0))
    s.steps(0.0, T / ns, ns)
    d = s.get_state() - to_kcn(dg_inputs.isentropic_vortex(x, y, t=T))
    # nodal 2-norm weighted by the element areas (the elements of a split
    # square are congruent, so the DG mass norm is proportional to it)
    return float(np.sqrt(np.mean(d * d)))


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_fp64_path_design_order(dg, p):
    e16, e32 = error(dg, 16, p, "fp64"), error(dg, 32, p, "fp64")
    rate = np.log2(e16 / e32)
    assert rate >= p + 0.5, (e16, e32, rate)


@pytest.mark.parametrize("p", [2, 3, 4])
def test_mixed_path_same_error(dg, p):
    for n in (16, 32):
        e64, emx = error(dg, n, p, "fp64"), error(dg, n, p, "mixed")
        assert abs(emx - e64) <= 1e-3 * e64 + 1e-8, (n, e64, emx)
