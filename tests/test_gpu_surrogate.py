"""The load surrogate trained on trajectories the DG solver generates.

* 24 small VIV cases (seeded O-grids, p = 2..4, U* in [3, 8], Re in
  [100, 150], m* = 10, zeta = 1e-3) advance together in a batch for 120 steps
  from perturbed starts; their per-step histories give windows of
  (y, y', C_L, C_D) with the next-step change of (C_L, C_D) as target.
* The network is trained on 18 cases and judged on the other 6: its
  one-step-ahead lift and drag must beat the lagged load that the weakly
  coupled scheme uses without it (persistence: no change over the step),
  and its lift (the load of the transverse Newmark step), learnt as a
  correction to linear extrapolation, must also beat linear extrapolation.
* In the coupled loop on a held-out case the predicted end-of-step lift
  drives the Newmark step; the DG forces of every step judge it.
"""
import numpy as np
import pytest

import dg_inputs
from dg_inputs.states import to_kcn

pytestmark = pytest.mark.gpu
GAMMA, MACH = 1.4, 0.2
P_INF = 1.0 / (GAMMA * MACH * MACH)
FAR = dict(rho_inf=1.0, u_inf=1.0, v_inf=0.0, p_inf=P_INF)
NSTEPS, NCASES, NTRAIN = 120, 24, 18


@pytest.fixture(scope="module")
def dg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_17917_gb300 import build
    build.build()
    import paper_2508_17917_gb300 as dg
    return dg


def structure(ustar, mstar=10.0, zeta=1e-3):
    fn = 1.0 / ustar
    return dict(M_r=1.0, C_r=4 * np.pi * fn * zeta, K_r=(1 + 1 / mstar) * (2 * np.pi * fn) ** 2,
                mass=mstar * np.pi / 4.0)


def start_state(x, y, seed):
    r = np.hypot(x, y)
    U = to_kcn(dg_inputs.free_stream(x.shape, rho=1.0, u=1.0, v=0.0, p=P_INF))
    damp = np.tanh(4.0 * (r - 0.5))
    U[:, 1] *= damp
    U[:, 2] = 0.05 * damp * np.sin(np.arctan2(y, x))
    U[:, 3] = P_INF / (GAMMA - 1) + 0.5 * (U[:, 1] ** 2 + U[:, 2] ** 2) / U[:, 0]
    return dg_inputs.perturb(U, seed=seed, amp=2e-3)


def case_list():
    rng = np.random.default_rng(42)
    out = []
    for i in range(NCASES):
        ustar, re = rng.uniform(3, 8), rng.uniform(100, 150)
        mesh = dg_inputs.ogrid_cylinder(int(rng.integers(16, 33)), int(rng.integers(4, 9)), 0.5,
                                        float(rng.uniform(3, 5)), seed=int(rng.integers(0, 1000)))
        out.append(dict(mesh=mesh, p=2 + i % 3, mu=1.0 / re, y0=float(rng.uniform(-0.05, 0.05)),
                        ustar=ustar, re=re, **structure(ustar)))
    return out


@pytest.fixture(scope="module")
def data(dg):
    import torch
    from paper_2508_17917_gb300.surrogate import make_windows
    cases = case_list()
    b = dg.BatchSolver([{k: c[k] for k in ("mesh", "p", "mu", "M_r", "C_r", "K_r", "mass", "y0")}
                        for c in cases], **FAR)
    states = []
    for i in range(len(cases)):
        x, y = b.node_coords(i)
        states.append(start_state(x, y, seed=200 + i))
        b.set_state(i, states[-1])
    hist = torch.zeros((NSTEPS, len(cases), 8), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    b.reset_history()
    b.run(0.3, NSTEPS, use_graph=True, hist=hist)
    h = hist.cpu().numpy()
    per_case = [make_windows(h[:, i, :], c["ustar"], 10.0, c["re"]) for i, c in enumerate(cases)]
    return cases, states, per_case


def test_surrogate_beats_the_lagged_load(dg, data):
    from paper_2508_17917_gb300.surrogate import LoadSurrogate
    cases, _, per_case = data
    Xtr = np.concatenate([p[0] for p in per_case[:NTRAIN]])
    Ttr = np.concatenate([p[1] for p in per_case[:NTRAIN]])
    Xte = np.concatenate([p[0] for p in per_case[NTRAIN:]])
    Tte = np.concatenate([p[1] for p in per_case[NTRAIN:]])
    Ste = np.concatenate([p[2] for p in per_case[NTRAIN:]])
    sur = LoadSurrogate(seed=1)
    loss = sur.fit(Xtr, Ttr, steps=1500, lr=2e-3)
    assert loss[-1] < 0.5 * loss[0]
    err = (sur.predict(Xte) - Tte) * Ste                # absolute one-step errors of (C_L, C_D)
    rmse = np.sqrt(np.mean(err ** 2, axis=0))
    lag = np.sqrt(np.mean((Tte * Ste) ** 2, axis=0))    # lagged load: no change over the step
    # last increment repeated (linear extrapolation), for the record
    lin = np.sqrt(np.mean(((Tte - Xte[:, [46, 62]]) * Ste) ** 2, axis=0))
    print("surrogate rmse", rmse, "lagged", lag, "linear extrapolation", lin)
    assert np.all(rmse < 0.3 * lag), (rmse, lag, lin)
    # the lift (the load of the transverse Newmark step) beats linear extrapolation;
    # the drag correction is left at most 2x worse than it
    assert rmse[0] <= lin[0] and rmse[1] <= 2.0 * lin[1], (rmse, lin)


def test_coupled_loop_with_surrogate_and_dg_judge(dg, data):
    import torch
    from paper_2508_17917_gb300.surrogate import LoadSurrogate, coupled_run
    cases, states, per_case = data
    sur = LoadSurrogate(seed=2)
    sur.fit(np.concatenate([p[0] for p in per_case[:NTRAIN]]),
            np.concatenate([p[1] for p in per_case[:NTRAIN]]), steps=1500, lr=2e-3)
    i = NTRAIN
    c = cases[i]
    s = dg.Solver(c["mesh"], c["p"], "mixed", stream=torch.cuda.current_stream().cuda_stream, mu=c["mu"], **FAR)
    s.set_state(states[i])
    rec = coupled_run(s, sur, (c["M_r"], c["C_r"], c["K_r"]), c["mass"], c["ustar"], 10.0, c["re"], 60,
                      state0=(c["y0"], 0.0, 0.0))
    used = rec[:, 8] > 0
    assert used.sum() >= 30                                   # predictions drove most steps
    lift, pred = rec[:, 6], rec[:, 7]
    have = np.isfinite(pred)
    miss = np.abs(pred[have] - lift[have])
    lagerr = np.abs(lift[1:] - lift[:-1])[have[1:]]
    assert np.mean(miss) < 0.3 * np.mean(lagerr), (np.mean(miss), np.mean(lagerr))
    assert np.all(np.isfinite(rec[:, :7]))
