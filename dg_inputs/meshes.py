"""Seeded synthetic triangle meshes.

Conventions (shared by every consumer of these arrays):

* ``EToV[k] = (v0, v1, v2)`` lists the vertices of element ``k`` counter-
  clockwise (positive signed area).
* Face ``f`` of element ``k`` joins ``EToV[k, f]`` and ``EToV[k, (f+1) % 3]``:
  face 0 = (v0, v1), face 1 = (v1, v2), face 2 = (v2, v0).
* ``EToE[k, f]`` / ``EToF[k, f]`` name the neighbouring element and its face.
  A boundary face points at itself (``EToE[k, f] == k``, ``EToF[k, f] == f``).
* ``bc[k, f]``: 0 interior or periodic face, 1 solid wall, 2 far field.

Periodic meshes keep duplicated vertex coordinates on the wrapped edges so
that every element is a plain affine triangle; the pairing across the period
lives only in ``EToE`` / ``EToF``.
"""
from __future__ import annotations

import dataclasses
import numpy as np

BC_INTERIOR, BC_WALL, BC_FARFIELD = 0, 1, 2


@dataclasses.dataclass
class Mesh:
    vx: np.ndarray          # (Nv,) float64
    vy: np.ndarray          # (Nv,) float64
    EToV: np.ndarray        # (K, 3) int32, counter-clockwise
    EToE: np.ndarray        # (K, 3) int32
    EToF: np.ndarray        # (K, 3) int32
    bc: np.ndarray          # (K, 3) int32
    period: tuple | None    # (Lx, Ly) for periodic squares, else None
    name: str = ""

    @property
    def K(self) -> int:
        return int(self.EToV.shape[0])

    @property
    def Nv(self) -> int:
        return int(self.vx.shape[0])


def _orient_ccw(vx, vy, EToV):
    x = vx[EToV]
    y = vy[EToV]
    area2 = (x[:, 1] - x[:, 0]) * (y[:, 2] - y[:, 0]) - (x[:, 2] - x[:, 0]) * (y[:, 1] - y[:, 0])
    flip = area2 < 0
    out = EToV.copy()
    out[flip, 1], out[flip, 2] = EToV[flip, 2], EToV[flip, 1]
    return out


def _connect(EToV, canon):
    """Pair faces that join the same two canonical vertices.

    ``canon[v]`` identifies vertices that coincide (directly or through a
    period).  Every canonical edge must be shared by exactly one or two faces;
    returns EToE, EToF and a dict {(a, b): (k, f)} of the unpaired faces.
    """
    K = EToV.shape[0]
    EToE = np.tile(np.arange(K, dtype=np.int32)[:, None], (1, 3))
    EToF = np.tile(np.arange(3, dtype=np.int32)[None, :], (K, 1))
    a = canon[EToV].astype(np.int64)                     # (K, 3)
    b = canon[np.roll(EToV, -1, axis=1)].astype(np.int64)
    lo, hi = np.minimum(a, b).ravel(), np.maximum(a, b).ravel()
    order = np.lexsort((hi, lo))
    lo_s, hi_s = lo[order], hi[order]
    same = (lo_s[1:] == lo_s[:-1]) & (hi_s[1:] == hi_s[:-1])
    if np.any(same[1:] & same[:-1]):
        raise RuntimeError("an edge is shared by more than two faces")
    first = np.nonzero(same)[0]
    f1, f2 = order[first], order[first + 1]
    k1, j1, k2, j2 = f1 // 3, f1 % 3, f2 // 3, f2 % 3
    EToE[k1, j1], EToF[k1, j1] = k2, j2
    EToE[k2, j2], EToF[k2, j2] = k1, j1
    paired = np.zeros(3 * K, dtype=bool)
    paired[f1] = True
    paired[f2] = True
    owner = {}
    for g in np.nonzero(~paired)[0]:
        owner[(int(lo[g]), int(hi[g]))] = (int(g // 3), int(g % 3))
    return EToE, EToF, owner


def periodic_square(n: int, L: float = 10.0, diagonal: str = "swne") -> Mesh:
    """[0, L]^2, n x n quads, each split into two triangles; fully periodic.

    ``diagonal='swne'`` splits every quad along its south-west -> north-east
    diagonal.  K = 2 n^2.  n must be at least 3 so that periodic edges are
    unambiguous.
    """
    if n < 3:
        raise ValueError("periodic_square needs n >= 3")
    h = L / n
    idx = lambda i, j: j * (n + 1) + i  # noqa: E731
    I, J = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="xy")
    vx = (I.ravel() * h).astype(np.float64)
    vy = (J.ravel() * h).astype(np.float64)
    tris = []
    for j in range(n):
        for i in range(n):
            a, b, c, d = idx(i, j), idx(i + 1, j), idx(i + 1, j + 1), idx(i, j + 1)
            if diagonal == "swne":
                tris += [(a, b, c), (a, c, d)]
            else:
                tris += [(a, b, d), (b, c, d)]
    EToV = _orient_ccw(vx, vy, np.array(tris, dtype=np.int32))
    canon = np.array([(v % (n + 1)) % n + ((v // (n + 1)) % n) * n
                      for v in range(vx.size)], dtype=np.int64)
    EToE, EToF, unpaired = _connect(EToV, canon)
    if unpaired:
        raise RuntimeError("periodic square left unpaired faces")
    bc = np.zeros_like(EToE)
    return Mesh(vx, vy, EToV, EToE, EToF, bc, (L, L), f"periodic_square_{n}")


def geometric_ratio(h1: float, n: int, length: float) -> float:
    """Ratio q with h1 * (q^n - 1) / (q - 1) == length, by bisection."""
    lo, hi = 1.0 + 1e-12, 2.0
    f = lambda q: h1 * (q ** n - 1.0) / (q - 1.0) - length  # noqa: E731
    if f(lo) > 0:
        raise ValueError("first cell too large for a stretched grid")
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(mid) > 0:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


def ogrid_cylinder(n_theta: int = 120, n_r: int = 170, r0: float = 0.5,
                   r1: float = 30.0, seed: int = 0) -> Mesh:
    """O-grid around a cylinder of radius r0 out to a far-field radius r1.

    Radial spacing is geometric with first cell equal to the wall arc length
    2 pi r0 / n_theta; each quad is split along a diagonal picked by a seeded
    generator.  The wall (r = r0) carries bc 1, the outer ring bc 2.
    K = 2 n_theta n_r.
    """
    h1 = 2.0 * np.pi * r0 / n_theta
    q = geometric_ratio(h1, n_r, r1 - r0)
    radii = np.empty(n_r + 1)
    radii[0] = r0
    for k in range(n_r):
        radii[k + 1] = radii[k] + h1 * q ** k
    radii[-1] = r1
    theta = 2.0 * np.pi * np.arange(n_theta) / n_theta
    vid = lambda i, k: k * n_theta + (i % n_theta)  # noqa: E731
    R, T = np.meshgrid(radii, theta, indexing="ij")
    vx = (R * np.cos(T)).ravel().astype(np.float64)
    vy = (R * np.sin(T)).ravel().astype(np.float64)
    rng = np.random.default_rng(seed)
    flips = rng.integers(0, 2, size=(n_r, n_theta))
    kk, ii = np.meshgrid(np.arange(n_r), np.arange(n_theta), indexing="ij")
    a, b = vid(ii, kk), vid(ii + 1, kk)
    c, d = vid(ii + 1, kk + 1), vid(ii, kk + 1)
    f = flips[..., None].astype(bool)
    t1 = np.where(f, np.stack([a, b, c], -1), np.stack([a, b, d], -1))
    t2 = np.where(f, np.stack([a, c, d], -1), np.stack([b, c, d], -1))
    tris = np.stack([t1, t2], axis=2).reshape(-1, 3)      # (k, i, two triangles) order
    EToV = _orient_ccw(vx, vy, tris.astype(np.int32))
    canon = np.arange(vx.size, dtype=np.int64)
    EToE, EToF, unpaired = _connect(EToV, canon)
    bc = np.zeros_like(EToE)
    rr = np.hypot(vx, vy)
    for (a, b), (k, f) in unpaired.items():
        ra, rb = rr[a], rr[b]
        if abs(ra - r0) < 1e-9 * r1 and abs(rb - r0) < 1e-9 * r1:
            bc[k, f] = BC_WALL
        elif abs(ra - r1) < 1e-9 * r1 and abs(rb - r1) < 1e-9 * r1:
            bc[k, f] = BC_FARFIELD
        else:
            raise RuntimeError("O-grid has an unpaired face off both boundaries")
    return Mesh(vx, vy, EToV, EToE, EToF, bc, None,
                f"ogrid_{n_theta}x{n_r}_seed{seed}")
