"""The eigenvalue step of the paired penalty norm (pair2.cuh).

The mixed-precision kernels take the largest eigenvalue of a symmetric 3x3
matrix by the trigonometric solution of its characteristic cubic, q + 2 p
cos(acos(r) / 3), and evaluate cos(acos(r) / 3) as a polynomial of degree 7
in w = sqrt((1 + r) / 2) = cos(acos(r) / 2), since cos(acos(r) / 3) =
cos(2/3 acos(w)) and that is analytic on w in [0, 1].  These CPU checks read
the coefficients from the kernel source and hold the polynomial, evaluated
by FP32 Horner steps as the kernel does, to the closed form over the whole
range of r, and the resulting eigenvalue to numpy's on random symmetric
matrices.
"""
import os
import re

import numpy as np

SRC = os.path.join(os.path.dirname(__file__), "..", "paper_2508_17917_gb300", "csrc", "pair2.cuh")


def coefficients():
    """The Horner coefficients, highest degree first, as FP32."""
    text = open(SRC).read()
    body = text[text.index("pf2 c = fma2("):text.index("const pf2 l = fma2(")]
    vals = re.findall(r"sp\((-?[0-9.]+(?:e-?[0-9]+)?)f\)", body)
    assert len(vals) == 8, vals
    return [np.float32(v) for v in vals]


def poly32(w):
    c = coefficients()
    w = w.astype(np.float32)
    acc = np.full_like(w, c[0])
    for a in c[1:]:
        acc = (acc * w + a).astype(np.float32)      # FMA rounding differs from this by at most one step
    return acc


def test_polynomial_matches_the_closed_form():
    r = np.linspace(-1.0, 1.0, 200001)
    w = np.sqrt((1.0 + r) / 2.0)
    exact = np.cos(np.arccos(r) / 3.0)
    got = poly32(w).astype(np.float64)
    assert np.abs(got - exact).max() < 2e-7
    # the end points: r = 1 (three equal roots scaled: cos 0), r = -1 (cos(pi/3))
    assert abs(poly32(np.array([1.0]))[0] - 1.0) < 2e-7
    assert abs(poly32(np.array([0.0]))[0] - 0.5) < 2e-7


def test_largest_eigenvalue_of_random_symmetric_matrices():
    rng = np.random.default_rng(3)
    worst = 0.0
    for _ in range(2000):
        a = rng.normal(size=(3, 3)) * rng.choice([1e-3, 1.0, 1e3])
        A = a @ a.T + np.diag(rng.uniform(0, 1, 3))      # symmetric positive, as B B^T is
        q = np.trace(A) / 3.0
        Bm = A - q * np.eye(3)
        p = np.sqrt((Bm * Bm).sum() / 6.0)
        r = np.clip(np.linalg.det(Bm / p) / 2.0, -1.0, 1.0)
        lam = q + 2.0 * p * poly32(np.array([np.sqrt((1.0 + r) / 2.0)]))[0]
        ref = np.linalg.eigvalsh(A)[-1]
        worst = max(worst, abs(lam - ref) / ref)
    assert worst < 1e-6, worst
