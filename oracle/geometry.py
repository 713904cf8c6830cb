"""Affine element geometry and face-node matching for the CPU oracle.

Oracle header: test infrastructure only (see oracle/refelem.py).

For the affine map T_K (Sec. 2.2) from K^ with vertices (v1, v2, v3):
x(r, s) = (-(r+s) v1 + (1+r) v2 + (1+s) v3) / 2, whose Jacobian matrix is
constant, so rx, ry, sx, sy and J are one number per element.  Outward unit
normals and sJ = |e|/2 come straight from the counter-clockwise edge vectors.
The neighbour node of every face node (the map behind E^e, Sec. 2.2) is found
by matching physical coordinates after removing the translation between the
two faces (zero for interior faces, one period for periodic ones).
"""
from __future__ import annotations

import numpy as np


def element_geometry(vx, vy, EToV, r, s):
    """Node coordinates and metric terms of every element."""
    X = vx[EToV]
    Y = vy[EToV]
    x = 0.5 * (-(r + s)[None, :] * X[:, 0:1] + (1 + r)[None, :] * X[:, 1:2] + (1 + s)[None, :] * X[:, 2:3])
    y = 0.5 * (-(r + s)[None, :] * Y[:, 0:1] + (1 + r)[None, :] * Y[:, 1:2] + (1 + s)[None, :] * Y[:, 2:3])
    xr = 0.5 * (X[:, 1] - X[:, 0])
    xs = 0.5 * (X[:, 2] - X[:, 0])
    yr = 0.5 * (Y[:, 1] - Y[:, 0])
    ys = 0.5 * (Y[:, 2] - Y[:, 0])
    J = xr * ys - xs * yr
    if np.any(J <= 0):
        raise ValueError("element with non-positive Jacobian (not counter-clockwise)")
    rx = ys / J
    ry = -xs / J
    sx = -yr / J
    sy = xr / J
    nx = np.empty((EToV.shape[0], 3))
    ny = np.empty_like(nx)
    sJ = np.empty_like(nx)
    for f in range(3):
        a, b = f, (f + 1) % 3
        tx = X[:, b] - X[:, a]
        ty = Y[:, b] - Y[:, a]
        ln = np.hypot(tx, ty)
        nx[:, f] = ty / ln
        ny[:, f] = -tx / ln
        sJ[:, f] = 0.5 * ln
    return dict(x=x, y=y, rx=rx, ry=ry, sx=sx, sy=sy, J=J, nx=nx, ny=ny, sJ=sJ)


def match_face_nodes(x, y, Fmask, EToE, EToF, bc):
    """mapP[k, f, i]: node index, inside element EToE[k,f], that coincides with
    face node i of face f of element k (up to the face-to-face translation)."""
    K = x.shape[0]
    Nfp = Fmask.shape[1]
    mapP = np.broadcast_to(Fmask[None, :, :], (K, 3, Nfp)).copy()
    kk, ff = np.nonzero(bc == 0)
    if kk.size == 0:
        return mapP, 0.0
    k2 = EToE[kk, ff]
    f2 = EToF[kk, ff]
    own = Fmask[ff]                     # (F, Nfp)
    nbr = Fmask[f2]                     # (F, Nfp)
    pa = np.stack([x[kk[:, None], own], y[kk[:, None], own]], axis=2)
    pb = np.stack([x[k2[:, None], nbr], y[k2[:, None], nbr]], axis=2)
    pb = pb + (pa.mean(axis=1, keepdims=True) - pb.mean(axis=1, keepdims=True))
    d = np.linalg.norm(pa[:, :, None, :] - pb[:, None, :, :], axis=3)   # (F, Nfp, Nfp)
    j = np.argmin(d, axis=2)
    worst = float(np.take_along_axis(d, j[:, :, None], axis=2).max())
    if np.any(np.sort(j, axis=1) != np.arange(Nfp)[None, :]):
        raise ValueError("face nodes do not match one to one")
    mapP[kk, ff] = np.take_along_axis(nbr, j, axis=1)
    return mapP, worst
