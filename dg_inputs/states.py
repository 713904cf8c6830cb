"""Seeded initial states, evaluated at node coordinates the caller supplies.

State layout everywhere: ``U[k, c, i]`` with element ``k``, conserved field
``c`` in (rho, rho*v1, rho*v2, E) and element-local node ``i``; E is the total
energy per unit volume.
"""
from __future__ import annotations

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def shu_vortex_params(gamma=1.4, mach=0.3, beta=5.0, center=(5.0, 5.0), L=10.0):
    """Free stream rho=1, p=1, velocity (M sqrt(gamma), 0); vortex strength beta."""
    return dict(gamma=gamma, mach=mach, beta=beta, center=center, L=L,
                rho_inf=1.0, p_inf=1.0, u_inf=mach * np.sqrt(gamma), v_inf=0.0)


def isentropic_vortex(x, y, t=0.0, gamma=1.4, mach=0.3, beta=5.0,
                      center=(5.0, 5.0), L=10.0, periodic=True):
    """Isentropic (Shu) vortex advected by the free stream; returns (..., 4).

    Temperature T = 1 - (gamma-1) beta^2 exp(1-r^2) / (8 gamma pi^2),
    velocity perturbation beta/(2 pi) exp((1-r^2)/2) (-(y-yc), x-xc),
    rho = T^(1/(gamma-1)), p = rho T.  On a periodic square the vortex centre
    is the nearest periodic image of the advected centre.
    """
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    u0 = mach * np.sqrt(gamma)
    xc = center[0] + u0 * t
    yc = center[1]
    dx = x - xc
    dy = y - yc
    if periodic:
        dx = dx - L * np.round(dx / L)
        dy = dy - L * np.round(dy / L)
    r2 = dx * dx + dy * dy
    T = 1.0 - (gamma - 1.0) * beta ** 2 * np.exp(1.0 - r2) / (8.0 * gamma * np.pi ** 2)
    du = -beta / (2.0 * np.pi) * np.exp(0.5 * (1.0 - r2)) * dy
    dv = beta / (2.0 * np.pi) * np.exp(0.5 * (1.0 - r2)) * dx
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho * T
    u = u0 + du
    v = dv
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    return np.stack([rho, rho * u, rho * v, E], axis=-1)


def free_stream(shape, rho=1.0, u=1.0, v=0.0, p=1.0, gamma=1.4):
    """Uniform state broadcast to ``shape + (4,)``."""
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    out = np.empty(tuple(shape) + (4,), dtype=np.float64)
    out[..., 0] = rho
    out[..., 1] = rho * u
    out[..., 2] = rho * v
    out[..., 3] = E
    return out


def splitmix64_uniform(seed: int, index) -> np.ndarray:
    """Uniform variates in [-1, 1) from SplitMix64 keyed by (seed, index).

    z = seed + (index + 1) * 0x9E3779B97F4A7C15, followed by the SplitMix64
    finaliser; the top 53 bits map to [0, 1) and then to [-1, 1).  Keyed by a
    global index, so the value of a degree of freedom does not depend on the
    order in which it is generated.
    """
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (np.uint64(seed) + (idx + np.uint64(1)) * np.uint64(0x9E3779B97F4A7C15)) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        z = z ^ (z >> np.uint64(31))
    u01 = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return 2.0 * u01 - 1.0


def perturb(U, seed: int, amp: float = 1e-3) -> np.ndarray:
    """U * (1 + amp * xi) with xi from SplitMix64 keyed by the flat index of U[k, c, i]."""
    U = np.asarray(U, dtype=np.float64)
    xi = splitmix64_uniform(seed, np.arange(U.size, dtype=np.uint64)).reshape(U.shape)
    return U * (1.0 + amp * xi)


def to_kcn(U_nodes_last):
    """(K, Np, 4) -> (K, 4, Np) contiguous."""
    return np.ascontiguousarray(np.transpose(U_nodes_last, (0, 2, 1)))
