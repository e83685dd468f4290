"""Pins of the FP64 reference perceptron: central finite differences of the
loss on a small batch agree with the written-out backward pass; GELU is the
tanh form of Hendrycks & Gimpel (its distance to the exact x Phi(x), its
symmetry, limits and derivative by differences)."""
import math

import numpy as np

from oracle import mlp


def test_gelu_tanh_form_and_derivative():
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    z = np.linspace(-8.0, 8.0, 3201)
    exact = np.array([0.5 * x * (1 + math.erf(x / math.sqrt(2))) for x in z])
    # the tanh form stays within 5e-4 of x Phi(x) everywhere (the approximation's known accuracy)
    assert np.max(np.abs(mlp.gelu(z) - exact)) < 5e-4
    # Phi(x) + Phi(-x) = 1 holds for the form too: gelu(z) - gelu(-z) = z
    assert np.allclose(mlp.gelu(z) - mlp.gelu(-z), z, rtol=0, atol=1e-14)
    assert abs(mlp.gelu(np.array([30.0]))[0] - 30.0) < 1e-12 and abs(mlp.gelu(np.array([-30.0]))[0]) < 1e-12
    h = 1e-6
    zz = np.array([1.0, -2.0, 3.5, -0.3, 0.0])
    num = (mlp.gelu(zz + h) - mlp.gelu(zz - h)) / (2 * h)
    assert np.allclose(mlp.gelu_grad(zz), num, rtol=1e-8, atol=1e-10)


def test_backward_matches_central_differences():
    rng = np.random.default_rng(0)
    p = rng.normal(0, 0.15, mlp.n_params())
    X = rng.normal(0, 1, (8, mlp.IN))
    t = rng.normal(0, 1, 8)
    loss, g = mlp.loss_and_grad(p, X, t)
    idx = rng.choice(mlp.n_params(), 60, replace=False)
    idx = np.concatenate([idx, [mlp.n_params() - 1, mlp.n_params() - 2, 0, 32 * 256]])  # head, first W and b
    h = 1e-5
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        num = (mlp.loss_and_grad(pp, X, t)[0] - mlp.loss_and_grad(pm, X, t)[0]) / (2 * h)
        assert abs(num - g[i]) <= 1e-6 * max(1.0, abs(num)), (i, num, g[i])


def test_bf16_rounding():
    # BF16 keeps 7 fraction bits: the spacing at 1 is 2^-7
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -9, 3.14159265])
    r = mlp.bf16(x)
    assert r[0] == 1.0 and r[3] == 1.0
    assert r[1] == 1.0 and r[2] == 1.0 + 2 ** -6                    # halfway cases go to the even neighbour
    assert abs(r[4] - x[4]) <= 2 ** -8 * x[4]
