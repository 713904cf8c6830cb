"""Pins of the surrogate MLP oracle (oracle/mlp.py) against facts that do not
depend on it: bfloat16 rounding of exactly representable neighbours, GELU
identities, central differences of the loss, the first Adam step, and the
bf16 mode reducing to the FP64 mode on bf16-representable data."""
import numpy as np
import pytest

from oracle import mlp


def test_bf16_round_ties_to_even_and_specials():
    u = 2.0 ** -7                                   # bf16 ulp at 1
    vals = np.array([1.0, 1 + u / 2, 1 + 1.5 * u, 1 + 0.5001 * u, -(1 + 1.5 * u), 3.0, 0.0, np.inf])
    want = np.array([1.0, 1.0, 1 + 2 * u, 1 + u, -(1 + 2 * u), 3.0, 0.0, np.inf])
    assert np.array_equal(mlp.bf16_round(vals), want)
    assert np.isnan(mlp.bf16_round(np.array([np.nan]))[0])
    x = np.random.default_rng(0).normal(size=1000)
    r = mlp.bf16_round(x)
    assert np.all(np.abs(r - x) <= 2.0 ** -8 * np.abs(x))     # half an ulp: at most 2^-8 relative
    assert np.array_equal(mlp.bf16_round(r), r)


def test_gelu_identities():
    z = np.linspace(-6, 6, 241)
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert np.allclose(mlp.gelu(z) - mlp.gelu(-z), z, atol=1e-15)          # Phi(z) + Phi(-z) = 1
    h = 1e-5
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.allclose(mlp.gelu_grad(z), fd, atol=1e-9)
    assert abs(mlp.gelu(np.array([8.0]))[0] - 8.0) < 1e-12


@pytest.mark.parametrize("depth", [0, 1, 3])
def test_gradient_by_central_differences(depth):
    rng = np.random.default_rng(depth)
    sizes = mlp.layer_sizes(5, 7, depth, 3)
    params = mlp.init_params(sizes, seed=depth) + 0.1 * rng.normal(size=mlp.param_count(sizes))
    x, t = rng.normal(size=(9, 5)), rng.normal(size=(9, 3))
    loss, g = mlp.loss_and_grad(params, sizes, x, t)
    h = 1e-6
    fd = np.empty_like(params)
    for i in range(params.size):
        e = np.zeros_like(params)
        e[i] = h
        fd[i] = (mlp.loss_and_grad(params + e, sizes, x, t)[0] - mlp.loss_and_grad(params - e, sizes, x, t)[0]) / (2 * h)
    assert np.abs(g - fd).max() <= 1e-7 * max(1.0, np.abs(fd).max())


def test_bias_gradient_vanishes_at_the_mean():
    sizes = mlp.layer_sizes(4, 6, 0, 2)
    rng = np.random.default_rng(1)
    x, t = rng.normal(size=(11, 4)), rng.normal(size=(11, 2))
    params = np.concatenate([np.zeros(8), t.mean(axis=0)])
    _, g = mlp.loss_and_grad(params, sizes, x, t)
    assert np.abs(g[8:]).max() < 1e-15


def test_first_adam_step_is_lr_times_sign():
    g = np.array([3.0, -0.2, 1e-3, -50.0])
    p, m, v = mlp.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    assert np.allclose(p, -0.01 * np.sign(g), rtol=1e-4)
    p2, _, _ = mlp.adam_step(p, g, m, v, 2, lr=0.01)
    assert np.allclose(p2, -0.02 * np.sign(g), rtol=1e-4)


def test_bf16_mode_equals_fp64_on_representable_data():
    sizes = mlp.layer_sizes(4, 8, 2, 2)
    rng = np.random.default_rng(2)
    params = rng.integers(-4, 5, size=mlp.param_count(sizes)) / 8.0
    Ws, bs = mlp.unpack(params, sizes)
    x = rng.integers(-3, 4, size=(6, 4)).astype(float)
    # one linear layer: exact products of bf16-representable numbers
    lin = mlp.layer_sizes(4, 8, 0, 2)
    pl = rng.integers(-4, 5, size=mlp.param_count(lin)) / 8.0
    assert np.array_equal(mlp.forward(pl, lin, x, bf16=True)[0], mlp.forward(pl, lin, x)[0])
    # deeper nets differ only through the rounding of the hidden activations
    y64 = mlp.forward(params, sizes, x)[0]
    y16 = mlp.forward(params, sizes, x, bf16=True)[0]
    assert np.abs(y16 - y64).max() <= 0.05 * max(1.0, np.abs(y64).max())
