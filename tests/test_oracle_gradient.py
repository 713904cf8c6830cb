"""Pins for the oracle's broken gradient (Sec. 2.2: grad_h U on each element
through the metric terms and Dr, Ds).

Polynomial fields of degree <= p are differentiated exactly on any affine
element: a linear field's gradient is its constant slope at every node, a
quadratic field's gradient (p >= 2) its linear derivative, on a periodic
square and on the O-grid; and the gradient is linear in U."""
import numpy as np
import pytest

import dg_inputs
import oracle


def meshes():
    return [dg_inputs.periodic_square(4), dg_inputs.ogrid_cylinder(16, 4, 0.5, 3.0, seed=1)]


@pytest.mark.parametrize("p", [1, 3, 6])
def test_linear_fields_exact(p):
    rng = np.random.default_rng(p)
    for mesh in meshes():
        P = oracle.Problem(mesh, p)
        a, b, d = rng.normal(size=(3, 4))
        U = a[None, :, None] + b[None, :, None] * P.x[:, None, :] + d[None, :, None] * P.y[:, None, :]
        Ux, Uy = P.broken_gradient(U)
        assert np.abs(Ux - b[None, :, None]).max() < 1e-11 * (1 + np.abs(b).max())
        assert np.abs(Uy - d[None, :, None]).max() < 1e-11 * (1 + np.abs(d).max())


@pytest.mark.parametrize("p", [2, 4])
def test_quadratic_fields_exact(p):
    for mesh in meshes():
        P = oracle.Problem(mesh, p)
        x, y = P.x, P.y
        U = np.stack([x * x, x * y, y * y, 3 * x * x - 2 * x * y + 1], axis=1)
        Ux, Uy = P.broken_gradient(U)
        want_x = np.stack([2 * x, y, 0 * x, 6 * x - 2 * y], axis=1)
        want_y = np.stack([0 * x, x, 2 * y, -2 * x], axis=1)
        scale = 1 + np.abs(x).max() + np.abs(y).max()
        assert np.abs(Ux - want_x).max() < 1e-10 * scale
        assert np.abs(Uy - want_y).max() < 1e-10 * scale


def test_gradient_is_linear():
    P = oracle.Problem(dg_inputs.periodic_square(3), 3)
    rng = np.random.default_rng(7)
    U, V = rng.normal(size=(2, P.K, 4, P.Np))
    gu, gv, guv = P.broken_gradient(U), P.broken_gradient(V), P.broken_gradient(2 * U - V)
    for c in range(2):
        assert np.allclose(guv[c], 2 * gu[c] - gv[c], atol=1e-12 * np.abs(guv[c]).max())
