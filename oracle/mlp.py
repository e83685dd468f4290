"""FP64 CPU reference of the surrogate perceptron (TEST INFRASTRUCTURE).

Only tests/ may import this.  The network: 32 -> 256 -> 256 -> 256 -> 256 -> 1
with GELU in its tanh form (Hendrycks & Gimpel, "Gaussian Error Linear Units",
2016: x Phi(x) ~ x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))) / 2), flat
parameters W1 [32][256], b1, W2, b2, W3, b3, W4, b4
(each W row-major [in][out]), w5 [256], b5 [1]; loss = mean squared error.
Backward pass written out by the chain rule.

``bf16=True`` evaluates the same definition with BF16 storage where the GPU
stores BF16 -- the inputs (each feature as an exact hi + lo pair of BF16
values, which the first layer reads against the same weights), the four
weight matrices, the activations the matrix products read (the head reads
the last hidden layer unrounded) and the back-propagated pre-activation
gradients that feed the matrix products -- and FP64 everywhere else, so the two differ only by FP32 accumulation order
and rare BF16 rounding flips.  Pinned against central finite differences.
"""
from __future__ import annotations

import math

import numpy as np

IN, H = 32, 256
_C = math.sqrt(2.0 / math.pi)   # the tanh form's scale
_K = 0.044715                   # and its cubic coefficient


def dims():
    return [(IN, H), (H, H), (H, H), (H, H)]


def n_params():
    return sum(i * o + o for i, o in dims()) + H + 1


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, o = [], 0
    for i, j in dims():
        W = p[o:o + i * j].reshape(i, j)
        o += i * j
        b = p[o:o + j]
        o += j
        out.append((W, b))
    w5 = p[o:o + H]
    b5 = p[o + H]
    return out, w5, b5


def bf16(x):
    """Round to the nearest BF16 value (ties to even), returned as FP64."""
    a = np.ascontiguousarray(x, dtype=np.float32).copy()
    u = a.view(np.uint32)
    u += 0x7FFF + ((u >> 16) & 1)
    u &= 0xFFFF0000
    return a.astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(_C * (z + _K * z ** 3)))


def gelu_grad(z):
    t = np.tanh(_C * (z + _K * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * _C * (1.0 + 3.0 * _K * z * z)


def forward(p, X, bf16_storage=False):
    layers, w5, b5 = unpack(p)
    r = bf16 if bf16_storage else (lambda x: np.asarray(x, dtype=np.float64))
    X = np.asarray(X, dtype=np.float64)
    A = bf16(X) + bf16(X - bf16(X)) if bf16_storage else X
    Zs, As = [], [A]
    for li, (W, b) in enumerate(layers):
        Z = A @ r(W) + b
        A = gelu(Z) if li == len(layers) - 1 else r(gelu(Z))
        Zs.append(Z)
        As.append(A)
    y = A @ w5 + b5
    return y, Zs, As


def loss_and_grad(p, X, t, bf16_storage=False):
    """Mean squared error and its gradient in the flat layout."""
    layers, w5, b5 = unpack(p)
    r = bf16 if bf16_storage else (lambda x: np.asarray(x, dtype=np.float64))
    y, Zs, As = forward(p, X, bf16_storage)
    n = len(t)
    e = y - t
    loss = float(np.mean(e * e))
    dy = 2.0 * e / n
    g_w5 = As[4].T @ dy
    g_b5 = dy.sum()
    dZ = np.outer(dy, w5) * gelu_grad(Zs[3])
    grads = [None] * 4
    for l in range(3, -1, -1):
        W, _ = layers[l]
        dZr = r(dZ)
        gW = As[l].T @ dZr
        gb = dZ.sum(axis=0)
        grads[l] = (gW, gb)
        if l > 0:
            dZ = (dZr @ r(W).T) * gelu_grad(Zs[l - 1])
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads] + [g_w5, [g_b5]])
    return loss, flat
