"""Seeded case lists for batches of independent cylinder / VIV cases.

Each entry describes one case by its synthetic mesh (seeded O-grid sizes and
diagonal seed), polynomial degree and flow / structure parameters (reduced
velocity U*, Reynolds number, mass ratio, damping ratio).  Turning these into
solver coefficients is the caller's business; nothing here evaluates the
method.
"""
import numpy as np

from .meshes import ogrid_cylinder


def viv_sweep(n_cases=64, k_min=10_000, k_max=60_000, degrees=(3, 4, 5, 6), seed=0,
              r1=30.0, ustar=(3.0, 8.0), re=(100.0, 150.0), mstar=10.0, zeta=1e-3):
    """Case list of a reduced-velocity sweep: triangle counts uniform in
    [k_min, k_max] (O-grids of n_theta x n_r cells, 2 triangles each), degree
    cycling through `degrees`, U* and Re uniform in their ranges."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_cases):
        k = int(rng.integers(k_min, k_max + 1))
        n_theta = int(rng.choice([64, 80, 96, 112, 128]))
        n_r = max(2, int(round(k / (2 * n_theta))))
        out.append(dict(n_theta=n_theta, n_r=n_r, r1=r1, mesh_seed=int(rng.integers(0, 2**31 - 1)),
                        p=int(degrees[i % len(degrees)]), ustar=float(rng.uniform(*ustar)),
                        re=float(rng.uniform(*re)), mstar=float(mstar), zeta=float(zeta)))
    return out


def sweep_mesh(case):
    """The O-grid of one case of `viv_sweep` (wall r = 0.5, far field r1)."""
    return ogrid_cylinder(case["n_theta"], case["n_r"], 0.5, case["r1"], seed=case["mesh_seed"])
