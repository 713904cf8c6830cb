"""The viscous vortex source (dg_set_source kind DG_SOURCE_VORTEX: S =
-div F_v of the advected isentropic vortex, config 2's source) against the
oracle, which evaluates the same S by hyper-dual differentiation through the
G blocks of Sec. 2.1.

* residual with the source at a time t > 0 (the source moves with the
  vortex), per field (tolerances of tests/_parity.py);
* 100 LSRK steps with the source on the 16 x 16 p = 2 mesh, whole state and
  the increment U_n - U_0 per field;
* the benchmark workload (128 x 128 quads, p = 4, K = 32,768) with the
  source for 20 steps, state and increment per field, both precisions.

The mixed path runs twice, with the single-node and with the tensor-core
tile shape; the source kernel fills an array for the five stage times (one
launch per step) that every stage kernel reads.
"""
import numpy as np
import pytest

import dg_inputs
import oracle
from dg_inputs.states import to_kcn
from _parity import INC_TOL, STATE_TOL, check_rhs, rel_l2

pytestmark = pytest.mark.gpu
GAMMA, MACH = 1.4, 0.3
U0 = MACH * np.sqrt(GAMMA)
SRC = (5.0, 5.0, 5.0, 10.0, U0, 0.0)          # beta, x0, y0, L, u0, v0


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


CASES = [("fp64", 0), ("mixed", 1), ("mixed", 3)]


def solver(dg, mesh, p, precision, variant, mu):
    s = dg.Solver(mesh, p, precision, stream=stream(), mu=mu)
    if variant:
        s.set_variant(variant)
    s.set_source(dg.DG_SOURCE_VORTEX, SRC)
    return s


@pytest.mark.parametrize("precision,variant", CASES)
@pytest.mark.parametrize("p", [2, 4])
def test_rhs_with_vortex_source(dg, p, precision, variant):
    mu = 2e-2
    mesh = dg_inputs.periodic_square(6)
    P = oracle.Problem(mesh, p, mu=mu, source=("vortex",) + SRC)
    t = 0.7
    U = to_kcn(dg_inputs.isentropic_vortex(P.x, P.y, t))
    ref = P.rhs(U, t)
    s = solver(dg, mesh, p, precision, variant, mu)
    s.set_state(U)
    got = s.rhs(t)
    check_rhs(P, U, got, precision, t, (0.0, 0.0), ref)
    # the source itself is what moved the residual
    P0 = oracle.Problem(mesh, p, mu=mu)
    assert np.abs(ref - P0.rhs(U, t)).max() > 1e3 * np.abs(got - ref).max()


@pytest.mark.parametrize("precision,variant", CASES)
def test_vortex_source_100_steps(dg, precision, variant):
    mu = 1e-3
    mesh = dg_inputs.periodic_square(16)
    P = oracle.Problem(mesh, 2, mu=mu, source=("vortex",) + SRC)
    U0 = dg_inputs.perturb(to_kcn(dg_inputs.isentropic_vortex(P.x, P.y)), seed=0, amp=1e-3)
    dt, _ = P.dt(U0, 0.3)
    ref = P.run(U0, 0.0, dt, 100)
    s = solver(dg, mesh, 2, precision, variant, mu)
    s.set_state(U0)
    s.steps(0.0, dt, 100)
    got = s.get_state()
    assert np.all(rel_l2(P, got - ref, ref) <= STATE_TOL[precision])
    inc = rel_l2(P, got - ref, ref - U0)
    assert np.all(inc <= INC_TOL[precision]), inc


_FULL = {}


def full_size():
    if not _FULL:
        mesh = dg_inputs.periodic_square(128)
        P = oracle.Problem(mesh, 4, mu=1e-3, source=("vortex",) + SRC)
        U0 = dg_inputs.perturb(to_kcn(dg_inputs.isentropic_vortex(P.x, P.y)), seed=0, amp=1e-3)
        dt, _ = P.dt(U0, 0.3)
        _FULL.update(mesh=mesh, P=P, U0=U0, dt=dt, ref=P.run(U0, 0.0, dt, 20))
    return _FULL


@pytest.mark.parametrize("precision,variant", CASES)
def test_vortex_source_full_size_20_steps(dg, precision, variant):
    f = full_size()
    s = solver(dg, f["mesh"], 4, precision, variant, 1e-3)
    s.set_state(f["U0"])
    n0 = s.launches
    s.steps(0.0, f["dt"], 20)
    # one source launch per step, then the five stages
    assert s.launches - n0 == 20 * 6
    got = s.get_state()
    P, ref, U0 = f["P"], f["ref"], f["U0"]
    assert np.all(rel_l2(P, got - ref, ref) <= STATE_TOL[precision])
    inc = rel_l2(P, got - ref, ref - U0)
    assert np.all(inc <= INC_TOL[precision]), inc
