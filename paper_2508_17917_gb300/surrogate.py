"""Load surrogate for the weakly coupled rigid-body step (Algorithm 3).

A small network (include/dg_mlp.h) maps a window of the last `window` steps
of (y, dy/dt, C_L, C_D) plus (U*, m*, Re) to the change of (C_L, C_D) over
the next step, both in units of the window's own increments.  In the
coupled loop its prediction of the end-of-step lift replaces the lagged
lift of the previous step in the Newmark equation; the
DG solve still runs every step, judges the prediction against the force it
computes and takes over (lagged lift) whenever the prediction misses by more
than a tolerance.

Data preparation (windows, feature scaling) is host bookkeeping in numpy;
training and inference run in the library's kernels.
"""
from __future__ import annotations

import numpy as np

from .binding import Mlp, dg_rigid_step

Q_REF = 0.5          # 1/2 rho_inf |v_inf|^2 D with rho_inf = |v_inf| = D = 1


def make_windows(rows, ustar, mstar, re, window=16, q=Q_REF, mode="increments"):
    """Samples from one trajectory.

    mode "values": the four series (y, y', C_L, C_D) enter as `window` values
    each, followed by (U*, m*, Re); T [n][2] is the next (C_L, C_D), S = 1 and
    C = 0.  For trajectories sampled at a fixed step over physical time
    (sweep_histories), where the series have their physical sizes.

    mode "increments" (scale-free form, for per-step DG histories whose time
    steps differ between cases by orders of magnitude):

    rows: [nsteps][>= 7] per-step records (t, dt, y, y', v_b, Fx, Fy, ...), as
    written by dg_batch_run's history.  For each of the four series
    (y, y', C_L, C_D) a window of `window` values gives window - 1 increments;
    they are divided by their root mean square s and followed by log10(s), so
    cases whose time steps (and hence increments) differ by orders of
    magnitude look alike.  Returns X [n][4 window + 3] (the four scaled
    increment windows, then U*, m*, Re), T [n][2] (the next increment of
    (C_L, C_D) divided by the same s), S [n][2] (those scales) and C [n][2]
    (the last (C_L, C_D) of each window): the prediction is C + T S."""
    rows = np.asarray(rows, dtype=np.float64)
    feat = np.stack([rows[:, 2], rows[:, 3], rows[:, 6] / q, rows[:, 5] / q], axis=1)
    X, T, S, C = [], [], [], []
    if mode == "values":
        for n in range(window - 1, rows.shape[0] - 1):
            X.append(np.concatenate([feat[n - window + 1:n + 1].T.ravel(), [ustar, mstar, re]]))
            T.append(feat[n + 1, [2, 3]])
            S.append([1.0, 1.0])
            C.append([0.0, 0.0])
        return np.array(X), np.array(T), np.array(S), np.array(C)
    for n in range(window - 1, rows.shape[0] - 1):
        w = feat[n - window + 1:n + 1]
        d = np.diff(w, axis=0)                                    # [window - 1][4]
        sc = np.sqrt(np.mean(d * d, axis=0)) + 1e-300
        x = np.concatenate([np.concatenate([d[:, j] / sc[j], [np.log10(sc[j])]]) for j in range(4)])
        X.append(np.concatenate([x, [ustar, mstar, re]]))
        S.append(sc[[2, 3]])
        C.append(feat[n, [2, 3]])
        T.append((feat[n + 1, [2, 3]] - feat[n, [2, 3]]) / sc[[2, 3]])
    return np.array(X), np.array(T), np.array(S), np.array(C)


class LoadSurrogate:
    """The network plus the feature and target scaling fitted on its data.

    The network learns a correction: in "increments" mode its target is the
    scaled next increment minus the last scaled increment of the window (a
    network that outputs zero reproduces linear extrapolation); in "values"
    mode the next value minus the last one (zero output: the lagged load)."""

    def __init__(self, window=16, width=128, depth=3, seed=0, max_batch=8192, mode="increments"):
        self.window = window
        self.mode = mode
        self.n_in = 4 * window + 3
        if mode == "values":
            self.last = [3 * window - 1, 4 * window - 1]                  # last C_L, C_D values
        else:
            self.last = [2 * window + window - 2, 3 * window + window - 2]    # last C_L, C_D increments
        self.net = Mlp(self.n_in, width, depth, 2, max_batch=max_batch, seed=seed)
        self.mu_x = self.sd_x = self.mu_t = self.sd_t = None

    def _scale_x(self, X):
        return ((np.asarray(X) - self.mu_x) / self.sd_x).astype(np.float32)

    def fit(self, X, T, steps=2000, lr=2e-3):
        """Full-batch Adam on (X, T); returns the loss history (scaled units)."""
        import torch
        X, T = np.asarray(X, dtype=np.float64), np.asarray(T, dtype=np.float64)
        R = T - X[:, self.last]
        self.mu_x, self.sd_x = X.mean(axis=0), X.std(axis=0) + 1e-12
        self.mu_t, self.sd_t = R.mean(axis=0), R.std(axis=0) + 1e-30
        xs = torch.from_numpy(self._scale_x(X)).cuda()
        ts = torch.from_numpy(((R - self.mu_t) / self.sd_t).astype(np.float32)).cuda()
        return self.net.train(xs, ts, steps, lr).cpu().numpy()

    def predict(self, X):
        """Predicted scaled next increment of (C_L, C_D), [n][2] (multiply by
        the window scales S of make_windows)."""
        import torch
        X = np.atleast_2d(np.asarray(X, dtype=np.float64))
        y = self.net.forward(torch.from_numpy(self._scale_x(X)).cuda()).cpu().numpy()
        return X[:, self.last] + y.astype(np.float64) * self.sd_t + self.mu_t


def coupled_run(solver, surrogate, coeff, mass, ustar, mstar, re, nsteps, cfl=0.3, tol=0.05,
                state0=(0.0, 0.0, 0.0), q=Q_REF, dt_fixed=None):
    """Algorithm 3 on one case with the surrogate as the load predictor.

    Each step: dt from the CFL bound (or dt_fixed when given); the Newmark step takes the predicted
    end-of-step lift when the window is full and the previous prediction
    passed the judge, else the lagged DG lift; the DG step runs with
    v_w = (0, v_b); its forces judge the prediction (relative miss measured
    against |C_L| + |dC_L|).  Returns per-step records
    (t, dt, y, y', v_b, Fx, Fy, predicted lift or nan, used prediction)."""
    st = np.array(state0, dtype=np.float64)
    F = solver.wall_forces()
    vb, t = 0.0, 0.0
    rows, out = [], []
    trusted = True
    for _ in range(nsteps):
        dt = solver.dt(cfl, (0.0, vb)) if dt_fixed is None else float(dt_fixed)
        pred = np.nan
        if len(rows) >= surrogate.window:
            X, _, S, C = make_windows(np.array(rows[-surrogate.window:] + [rows[-1]]), ustar, mstar, re,
                                      surrogate.window, q, surrogate.mode)
            dC = surrogate.predict(X[:1])[0] * S[0]
            pred = (C[0, 0] + dC[0]) * q
        use = trusted and np.isfinite(pred)
        F_r = (pred if use else F[1]) / mass
        st, vb = dg_rigid_step(coeff, F_r, dt, st)
        solver.step(t, dt, (0.0, vb))
        t += dt
        F = solver.wall_forces()
        if np.isfinite(pred):
            scale = abs(F[1]) + abs(F[1] - rows[-1][6]) + 1e-300
            trusted = abs(pred - F[1]) <= tol * scale
        rows.append([t, dt, st[0], st[1], vb, F[0], F[1], 0.0])
        out.append(rows[-1][:7] + [pred, float(use)])
    return np.array(out)


# ---- reduced-velocity sweeps over physical time, and the screen ------------

def rigid_to_rows(r):
    """dg_batch_rigid rows (t, dt, y, y', y'', v_b, Fx, Fy, Mz, frozen) ->
    history rows (t, dt, y, y', v_b, Fx, Fy, 0) as make_windows reads them."""
    r = np.asarray(r, dtype=np.float64)
    out = np.zeros(r.shape[:-1] + (8,))
    out[..., [0, 1, 2, 3, 4, 5, 6]] = r[..., [0, 1, 2, 3, 5, 6, 7]]
    return out


def sweep_histories(batch, dt, t_end, sample_dt, cfl=1.0):
    """Advance every case of a BatchSolver at the fixed step dt up to t_end,
    sampling the rigid-body state and the loads every sample_dt (a whole
    number of steps; dg_batch_run between samples, one synchronising read per
    sample).  Returns H [nsamples + 1][ncases][8] in the history-row format,
    starting with the state at t = 0."""
    batch.set_fixed_dt(dt)
    every = max(1, int(round(sample_dt / dt)))
    rows = [rigid_to_rows(batch.rigid())]
    n = int(np.ceil(t_end / (every * dt)))
    for _ in range(n):
        batch.run(cfl, every, use_graph=True)
        rows.append(rigid_to_rows(batch.rigid()))
    return np.array(rows)


def amplitude(y):
    """Half the range of a displacement history."""
    y = np.asarray(y)
    return 0.5 * float(y.max() - y.min()) if y.size else 0.0


def screen_rollout(surrogate, prefix, coeffs, masses, params, nsteps, q=Q_REF):
    """The screen's continuation of several cases at once.  prefix: DG rows
    [n][ncases][8] (history format, uniformly spaced in time); coeffs[i] =
    (M_r, C_r, K_r), masses[i], params[i] = (U*, m*, Re).  Every step the
    surrogate predicts the next (C_L, C_D) of every case from its last window,
    and the Newmark step (Eq. 1dof_oscillator, step = the prefix's sample
    spacing) takes the predicted lift; nsteps steps.  Returns the continued
    rows [nsteps][ncases][8]."""
    P = np.asarray(prefix, dtype=np.float64)
    nc = P.shape[1]
    h = P[-1, 0, 0] - P[-2, 0, 0]
    w = surrogate.window
    hist = [list(P[max(0, P.shape[0] - w):, i]) for i in range(nc)]
    hist = [[list(r) for r in rows] for rows in hist]
    states = []
    for i in range(nc):
        r = hist[i][-1]
        c = coeffs[i]
        states.append(np.array([r[2], r[3], (r[6] / masses[i] - c[1] * r[3] - c[2] * r[2]) / c[0]]))
    out = np.zeros((nsteps, nc, 8))
    for n in range(nsteps):
        Xs, Ss, Cs = [], [], []
        for i in range(nc):
            X, _, S, C = make_windows(np.array(hist[i][-w:] + [hist[i][-1]]), *params[i], w, q,
                                      surrogate.mode)
            Xs.append(X[0]); Ss.append(S[0]); Cs.append(C[0])
        dC = surrogate.predict(np.array(Xs)) * np.array(Ss)
        for i in range(nc):
            cl, cd = Cs[i][0] + dC[i, 0], Cs[i][1] + dC[i, 1]
            states[i], vb = dg_rigid_step(coeffs[i], cl * q / masses[i], h, states[i])
            row = [hist[i][-1][0] + h, h, states[i][0], states[i][1], vb, cd * q, cl * q, 0.0]
            hist[i].append(row)
            hist[i] = hist[i][-w:]
            out[n, i] = row
    return out
