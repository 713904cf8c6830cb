"""Plain FP64 reference of the load-surrogate MLP (test infrastructure).

Oracle header: only tests, the smoke check and the benchmark's CPU-baseline
leg may import this module; the CUDA library never uses it and it uses
nothing from the library.

The network (a multilayer perceptron; not part of the paper, it predicts the
next-step lift and drag coefficients from a window of the rigid-body state
and force history):
    h_0 = x,  z_l = h_{l-1} W_l^T + b_l,  h_l = GELU(z_l)  (l = 1..L-1),
    y = z_L = h_{L-1} W_L^T + b_L,
    GELU(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2,
loss = mean over the batch and the outputs of (y - t)^2, gradients by the
chain rule written out layer by layer, and the Adam update (Kingma & Ba,
2015) with bias correction.

With bf16=True every matrix-product input (x, the hidden activations h_l,
the back-propagated dz_l and the weights) is first rounded to bfloat16
(round to nearest, ties to even, from the float32 value), as the GPU kernels
do; products and sums stay FP64 here.

Parameter layout (shared with the C ABI): for l = 1..L, W_l row-major
[n_out][n_in] followed by b_l [n_out], all concatenated.
"""
import numpy as np
from scipy.special import erf

SQRT2 = np.sqrt(2.0)


def bf16_round(a):
    """float32 -> bfloat16 -> float64, round to nearest, ties to even."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    nan = np.isnan(f)
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / SQRT2))


def gelu_grad(z):
    """d GELU / dz = Phi(z) + z phi(z)."""
    return 0.5 * (1.0 + erf(z / SQRT2)) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def layer_sizes(n_in, width, depth, n_out):
    """(n_in, n_out) of every layer: depth hidden layers of `width`."""
    dims = [n_in] + [width] * depth + [n_out]
    return list(zip(dims[:-1], dims[1:]))


def unpack(params, sizes):
    Ws, bs, o = [], [], 0
    for ni, no in sizes:
        Ws.append(np.asarray(params[o:o + ni * no], dtype=np.float64).reshape(no, ni))
        o += ni * no
        bs.append(np.asarray(params[o:o + no], dtype=np.float64))
        o += no
    assert o == len(params)
    return Ws, bs


def pack(Ws, bs):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in zip(Ws, bs)])


def param_count(sizes):
    return sum(ni * no + no for ni, no in sizes)


def forward(params, sizes, x, bf16=False):
    """Returns y and the per-layer (input, pre-activation) pairs."""
    q = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    Ws, bs = unpack(params, sizes)
    h = np.asarray(x, dtype=np.float64)
    cache = []
    for l, (W, b) in enumerate(zip(Ws, bs)):
        hin = q(h)
        z = hin @ q(W).T + b
        cache.append((hin, z))
        h = gelu(z) if l < len(Ws) - 1 else z
    return h, cache


def loss_and_grad(params, sizes, x, t, bf16=False):
    """Mean squared error and its gradient with respect to every parameter."""
    q = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    Ws, bs = unpack(params, sizes)
    y, cache = forward(params, sizes, x, bf16)
    t = np.asarray(t, dtype=np.float64)
    n = y.size
    loss = np.sum((y - t) ** 2) / n
    dz = 2.0 * (y - t) / n                       # d loss / d z_L
    gW, gb = [None] * len(Ws), [None] * len(Ws)
    for l in range(len(Ws) - 1, -1, -1):
        hin, z = cache[l]
        dzq = q(dz)
        gW[l] = dzq.T @ hin                      # sum over the batch
        gb[l] = dz.sum(axis=0)
        if l > 0:
            dh = dzq @ q(Ws[l])                  # d loss / d h_{l-1}
            dz = dh * gelu_grad(cache[l - 1][1])
    return loss, pack(gW, gb)


def adam_step(params, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new params, m, v."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return params - lr * mhat / (np.sqrt(vhat) + eps), m, v


def init_params(sizes, seed=0):
    """Seeded uniform init in +-sqrt(6 / (n_in + n_out)) for W, zero biases."""
    rng = np.random.default_rng(seed)
    Ws, bs = [], []
    for ni, no in sizes:
        a = np.sqrt(6.0 / (ni + no))
        Ws.append(rng.uniform(-a, a, size=(no, ni)))
        bs.append(np.zeros(no))
    return pack(Ws, bs).astype(np.float32).astype(np.float64)
