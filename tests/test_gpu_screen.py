"""A reduced-velocity sweep over physical time, the load surrogate trained on
it, and the surrogate as a screen of the sweep (Sec. 3.3 set-up; the
surrogate is not in the paper).

Sweep: 12 elastically mounted cylinders, U* = 3..8, m* = 10, zeta = 1e-3,
Re = 100, M = 0.2, each on a seeded 32 x 12 O-grid (768 triangles, far field
at 8 D), p = 3, advanced together as one batch at a fixed step (CFL 4 of the
first step's bound) from a smoothed free-stream start to t = 120, sampled
every 0.05.  The DG histories show vortex shedding (St ~ 0.17 away from
lock-in) and a lock-in range where the cylinder oscillates at its natural
frequency with A / D ~ 0.45.

Surrogate: windows of 16 samples of (y, y', C_L, C_D) plus (U*, m*, Re) ->
next (C_L, C_D), trained on 8 cases with the library's MLP kernels; 4 cases
(U* = 3.9, 5.3, 6.6, 7.5) are held out and judge it.

Screen: every case runs DG to t = 40 only; the surrogate then predicts the
loads and drives the Newmark step alone to t = 120.  Its amplitude over
t = 80..120 is compared with the full DG run for every case: the lock-in
classification (A / D > 0.1) agrees for every case whose DG amplitude is
clear of the threshold (more than 10 % away from it), the held-out cases
are within 25 % and the training cases within 15 %.
"""
import numpy as np
import pytest

import dg_inputs
from dg_inputs.states import to_kcn

pytestmark = pytest.mark.gpu
GAMMA, MACH, RE, MSTAR, ZETA = 1.4, 0.2, 100.0, 10.0, 1e-3
P_INF = 1.0 / (GAMMA * MACH * MACH)
T_END, SAMPLE, T_PREFIX, WINDOW = 120.0, 0.05, 40.0, 16
USTARS = np.linspace(3.0, 8.0, 12)
HELD_OUT = [2, 5, 8, 10]
TRAIN = [i for i in range(12) if i not in HELD_OUT]


@pytest.fixture(scope="module")
def sweep():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_17917_gb300 import build
    build.build()
    import paper_2508_17917_gb300 as dg
    from paper_2508_17917_gb300 import surrogate as sg
    cases, coeffs, masses, params = [], [], [], []
    for i, us in enumerate(USTARS):
        fn = 1.0 / us
        c = dict(M_r=1.0, C_r=4 * np.pi * fn * ZETA, K_r=(1 + 1 / MSTAR) * (2 * np.pi * fn) ** 2,
                 mass=MSTAR * np.pi / 4.0)
        cases.append(dict(mesh=dg_inputs.ogrid_cylinder(32, 12, 0.5, 8.0, seed=i), p=3, mu=1.0 / RE, **c))
        coeffs.append((c["M_r"], c["C_r"], c["K_r"]))
        masses.append(c["mass"])
        params.append((us, MSTAR, RE))
    b = dg.BatchSolver(cases, rho_inf=1.0, u_inf=1.0, v_inf=0.0, p_inf=P_INF)
    for i in range(len(cases)):
        x, y = b.node_coords(i)
        U = to_kcn(dg_inputs.free_stream(x.shape, rho=1.0, u=1.0, v=0.0, p=P_INF))
        U[:, 1] *= np.tanh(4.0 * (np.hypot(x, y) - 0.5))
        U[:, 3] = P_INF / (GAMMA - 1) + 0.5 * U[:, 1] ** 2 / U[:, 0]
        b.set_state(i, dg_inputs.perturb(U, seed=i, amp=1e-3))
    b.run(4.0, 1, use_graph=False)
    dt = float(b.rigid()[:, 1].min())
    dt = SAMPLE / np.ceil(SAMPLE / dt)            # a whole number of steps per sample
    H = sg.sweep_histories(b, dt, T_END, SAMPLE)
    assert not np.any(b.rigid()[:, 9]) and np.all(np.isfinite(H))
    Xs, Ts = [], []
    for i in TRAIN:
        X, T, _, _ = sg.make_windows(H[:, i], *params[i], WINDOW, mode="values")
        Xs.append(X)
        Ts.append(T)
    X, T = np.concatenate(Xs), np.concatenate(Ts)
    sel = np.random.default_rng(0).choice(len(X), size=8192, replace=False)
    sur = sg.LoadSurrogate(window=WINDOW, seed=0, max_batch=8192, mode="values")
    loss = sur.fit(X[sel], T[sel], steps=4000, lr=2e-3)
    return dict(sg=sg, H=H, sur=sur, loss=loss, coeffs=coeffs, masses=masses, params=params)


def late(H, col, t0=80.0):
    return H[H[:, 0, 0] >= t0][:, :, col]


def test_sweep_sheds_and_locks_in(sweep):
    sg, H = sweep["sg"], sweep["H"]
    y = late(H, 2)
    amp = np.array([sg.amplitude(y[:, i]) for i in range(12)])
    # lock-in: large oscillation at the natural frequency for U* ~ 5.3..6.6
    lock = (USTARS > 5.0) & (USTARS < 6.8)
    assert amp[lock].min() > 0.3, amp
    assert amp[USTARS < 4.5].max() < 0.05, amp
    import bench
    t = late(H, 0)[:, 0]
    for i in np.where(lock)[0]:
        f_y = bench.strouhal(t, y[:, i] - y[:, i].mean())
        assert 0.9 < f_y * USTARS[i] < 1.15, (USTARS[i], f_y)
    # away from lock-in the lift oscillates at the shedding frequency
    cl = late(H, 6) / 0.5
    st = bench.strouhal(t, cl[:, 0])
    assert 0.14 < st < 0.2, st


def test_surrogate_one_step_gain(sweep):
    """On the held-out cases the surrogate's next-sample lift beats the
    lagged load (the previous sample's lift) by at least 4x."""
    sg, H, sur = sweep["sg"], sweep["H"], sweep["sur"]
    assert sweep["loss"][-1] < 0.01 * sweep["loss"][0]
    err_net, err_lag = [], []
    for i in HELD_OUT:
        X, T, _, _ = sg.make_windows(H[:, i], *sweep["params"][i], WINDOW, mode="values")
        pred = sur.predict(X)
        err_net.append(pred[:, 0] - T[:, 0])
        err_lag.append(X[:, sur.last[0]] - T[:, 0])
    rms = lambda e: float(np.sqrt(np.mean(np.concatenate(e) ** 2)))  # noqa: E731
    assert rms(err_net) < 0.25 * rms(err_lag), (rms(err_net), rms(err_lag))


def test_screen_matches_dg(sweep):
    sg, H, sur = sweep["sg"], sweep["H"], sweep["sur"]
    nP = int(round(T_PREFIX / SAMPLE))
    roll = sg.screen_rollout(sur, H[:nP + 1], sweep["coeffs"], sweep["masses"], sweep["params"],
                             H.shape[0] - 1 - nP)
    t = roll[:, 0, 0]
    a_screen = np.array([sg.amplitude(roll[t >= 80.0, i, 2]) for i in range(12)])
    a_dg = np.array([sg.amplitude(late(H, 2)[:, i]) for i in range(12)])
    # lock-in (A / D > 0.1) is classified alike wherever the DG amplitude is
    # clear of the threshold: a case within 10 % of it (U* = 7.5 sits at
    # A / D = 0.096 to 0.10 depending on the FP32 rounding of its history to
    # t = 120) has no defined class, and its amplitude is held below instead
    clear = np.abs(a_dg - 0.1) > 0.01
    assert np.array_equal((a_screen > 0.1)[clear], (a_dg > 0.1)[clear]), (a_screen, a_dg)
    rel = np.abs(a_screen - a_dg) / a_dg
    assert rel[HELD_OUT].max() <= 0.25, rel
    assert rel[TRAIN].max() <= 0.15, rel
