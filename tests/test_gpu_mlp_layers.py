"""Layer-by-layer parity of the surrogate network's kernels against the FP64
reference network (oracle/mlp.py), each layer fed the GPU's own BF16 inputs.

``rsv_mlp_trace`` returns every layer's FP32 pre-activations and the BF16
values the GPU stored for the next product (and, for the training kernels,
the backward pass).  For layer l the reference takes the BF16 activations the
GPU stored for layer l-1 and the BF16 weights, so only these differences are
left, and each is bounded per element:

* FP32 accumulation of exact BF16 x BF16 products over K terms (K = 64 hi + lo
  feature halves, 256 hidden units, or the n rows of a weight gradient), plus
  the bias add: |z - z_ref| <= (K + 2) 2^-23 sum_k |a_k w_k| (2^-23 allows an
  accumulator that truncates rather than rounds).
* GELU in its tanh form through the hardware tanh.approx (relative error below
  2^-10.9): |gelu - gelu_ref| <= |z| |t| 2^-10.9 / 2 + a few FP32 roundings,
  and for gelu' the same error through its derivative with respect to t.
* The BF16 store of an activation: half an ulp (2^-8 relative) of the value
  it rounds.

A bias column off by a fraction of its size already breaks these bounds by
orders of magnitude; the test plants such an error in the reference and checks
that the comparison catches it.
"""
import math

import numpy as np
import pytest
import torch

from oracle import mlp as ref
from paper_1401_1757_gb300 import rsv

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -23        # FP32 accumulation, per addition (truncation allowed)
U24 = 2.0 ** -24        # FP32 rounding to nearest
TANH_REL = 2.0 ** -10.9
BF16_HALF_ULP = 2.0 ** -8
C, K3 = math.sqrt(2.0 / math.pi), 0.044715
N = 256


@pytest.fixture
def ctx():
    h = rsv.rsv_create(0, torch.cuda.current_stream())
    yield h
    rsv.rsv_destroy(h)


def params(seed):
    rng = np.random.default_rng(seed)
    p = np.zeros(ref.n_params())
    o = 0
    for i, j in ref.dims():
        p[o:o + i * j] = rng.normal(0, math.sqrt(2.0 / i), i * j)
        o += i * j
        p[o:o + j] = rng.normal(0, 0.05, j)
        o += j
    p[o:o + 256] = rng.normal(0, 1 / 16, 256)
    p[o + 256] = 0.1
    return p.astype(np.float32).astype(np.float64)


def gelu_err(z):
    """Bound on |gelu_hw(z) - gelu(z)| (tanh.approx plus FP32 roundings)."""
    u = C * (z + K3 * z ** 3)
    t = np.tanh(u)
    return 0.5 * np.abs(z) * (TANH_REL * np.abs(t) + 4 * U24 * (1 + np.abs(u))) + 4 * U24 * np.abs(z)


def gelu_grad_err(z):
    """Bound on |gelu'_hw(z) - gelu'(z)|: the tanh error through d gelu' / d t."""
    u = C * (z + K3 * z ** 3)
    t = np.tanh(u)
    dgdt = np.abs(0.5 - z * t * C * (1.0 + 3.0 * K3 * z * z))
    g = ref.gelu_grad(z)
    return dgdt * (TANH_REL * np.abs(t) + 4 * U24 * (1 + np.abs(u))) + 8 * U24 * (np.abs(g) + 1.0)


def worst(err, bound):
    return float(np.max(np.abs(err) / (bound + 1e-300)))


def forward_report(p, tr, tc, bias_shift=None):
    """Worst |error| / bound of each forward check; ``bias_shift`` = (layer,
    column, delta) plants a bias error in the reference."""
    layers, w5, b5 = ref.unpack(p)
    out = {}
    Xb = tr["Xb"]                        # [n][64]: hi halves then lo halves
    A_prev = Xb
    for l in range(4):
        W, b = layers[l]
        b = b.copy()
        if bias_shift and bias_shift[0] == l:
            b[bias_shift[1]] += bias_shift[2]
        Wb = ref.bf16(W)
        Wk = np.vstack([Wb, Wb]) if l == 0 else Wb          # the tied first layer reads [W1; W1]
        K = Wk.shape[0]
        z_ref = A_prev @ Wk + b
        z_abs = np.abs(A_prev) @ np.abs(Wk) + np.abs(b)
        Z = tr["Z"][l]
        out[f"z{l + 1}"] = worst(Z - z_ref, (K + 2) * U32 * z_abs)
        g_ref = ref.gelu(Z)
        eg = gelu_err(Z)
        if l < 3 or not tc:
            A = tr["A"][l] / (2.0 if tc else 1.0)             # tcgen05 stores 2 gelu
            out[f"a{l + 1}"] = worst(A - g_ref, eg + BF16_HALF_ULP * (np.abs(g_ref) + eg))
            A_prev = A
    Z4 = tr["Z"][3]
    y_ref = ref.gelu(Z4) @ w5 + b5
    y_bound = gelu_err(Z4) @ np.abs(w5) + (N + 2) * U32 * (np.abs(ref.gelu(Z4)) @ np.abs(w5) + abs(b5))
    out["y"] = worst(tr["y"] - y_ref, y_bound)
    return out


def backward_report(p, tr, t):
    layers, w5, b5 = ref.unpack(p)
    n = len(t)
    g = tr["grads"]
    o_w = [0]
    for i, j in ref.dims():
        o_w.append(o_w[-1] + i * j + j)
    out = {}
    dy = 2.0 * (tr["y"] - t) / n
    Z4 = tr["Z"][3]
    d4_ref = np.outer(dy, w5) * ref.gelu_grad(Z4)
    d4_bound = np.abs(np.outer(dy, w5)) * gelu_grad_err(Z4) + 8 * U24 * np.abs(d4_ref) + 1e-30
    out["dz4"] = worst(tr["dZ"][3] - d4_ref, d4_bound)
    for l in range(3, -1, -1):
        W, _ = layers[l]
        Wb = ref.bf16(W)
        dZb = tr["dZb"][l]
        assert np.array_equal(dZb, ref.bf16(tr["dZ"][l]))        # the products read the BF16 of the FP32 dZ
        A_prev = tr["Xb"] if l == 0 else tr["A"][l - 1]
        dW = A_prev.T @ dZb
        dW_abs = np.abs(A_prev).T @ np.abs(dZb)
        if l == 0:                                                   # tied weights: the hi and lo rows add up
            dW, dW_abs = dW[:32] + dW[32:], dW_abs[:32] + dW_abs[32:]
        i, j = W.shape
        gW = g[o_w[l]:o_w[l] + i * j].reshape(i, j)
        out[f"dW{l + 1}"] = worst(gW - dW, (n + 3) * U32 * dW_abs)
        db = tr["dZ"][l].sum(axis=0)
        gb = g[o_w[l] + i * j:o_w[l + 1]]
        out[f"db{l + 1}"] = worst(gb - db, (n + 2) * U32 * np.abs(tr["dZ"][l]).sum(axis=0))
        if l > 0:
            P = dZb @ Wb.T
            P_abs = np.abs(dZb) @ np.abs(Wb.T)
            Zp = tr["Z"][l - 1]
            d_ref = P * ref.gelu_grad(Zp)
            bound = (N + 2) * U32 * P_abs * np.abs(ref.gelu_grad(Zp)) + np.abs(P) * gelu_grad_err(Zp) + 1e-30
            out[f"dz{l}"] = worst(tr["dZ"][l - 1] - d_ref, bound)
    o5 = o_w[4]
    A4 = ref.gelu(Z4)
    out["dw5"] = worst(g[o5:o5 + 256] - A4.T @ dy,
                       np.abs(dy) @ gelu_err(Z4) + (n + 2) * U32 * (np.abs(A4).T @ np.abs(dy)))
    out["db5"] = worst(g[o5 + 256] - dy.sum(), (n + 2) * U32 * np.abs(dy).sum())
    return out


@pytest.mark.parametrize("backend", [rsv.RSV_MLP_MMA_SYNC, rsv.RSV_MLP_TCGEN05])
def test_forward_layer_by_layer(ctx, backend):
    """Each layer's FP32 pre-activations within the FP32-accumulation bound of
    the reference on the GPU's own BF16 inputs, each activation within the
    hardware-tanh bound plus half a BF16 ulp, the head likewise; for both the
    training kernels (mma.sync) and the inference kernel (tcgen05, TMEM)."""
    p = params(21)
    rng = np.random.default_rng(22)
    X = rng.normal(0, 1, (N, 32)).astype(np.float32)
    X[:, 20:] = 0.0                                   # padded feature slots, as in the surrogate
    rsv.rsv_mlp_set_params(ctx, p)
    tr = rsv.rsv_mlp_trace(ctx, X, backend=backend)
    tc = backend == rsv.RSV_MLP_TCGEN05
    rep = forward_report(p, tr, tc)
    print(("tcgen05" if tc else "mma.sync"), {k: round(v, 3) for k, v in rep.items()})
    assert max(rep.values()) <= 1.0, rep
    # a bias column off by 1% of the largest bias in the reference is caught
    layers, _, _ = ref.unpack(p)
    for l in range(4):
        shift = 0.01 * float(np.max(np.abs(layers[l][1])))
        bad = forward_report(p, tr, tc, bias_shift=(l, 97, shift))
        assert bad[f"z{l + 1}"] > 1.0, (l, bad)


def test_backward_layer_by_layer(ctx):
    """The training kernels' backward pass, layer by layer against the
    reference on the GPU's own BF16 operands: dW_l = A_{l-1}^T dZ_l, the bias
    gradients, dZ_{l-1} = (dZ_l W_l^T) gelu'(z_{l-1}) and the head's."""
    p = params(23)
    rng = np.random.default_rng(24)
    X = rng.normal(0, 1, (N, 32)).astype(np.float32)
    X[:, 20:] = 0.0
    t = rng.normal(0, 1, N).astype(np.float32)
    rsv.rsv_mlp_set_params(ctx, p)
    tr = rsv.rsv_mlp_trace(ctx, X, backend=rsv.RSV_MLP_MMA_SYNC, target=t)
    fw = forward_report(p, tr, False)
    bw = backward_report(p, tr, t.astype(np.float64))
    print("backward", {k: round(v, 3) for k, v in bw.items()})
    assert max(fw.values()) <= 1.0, fw
    assert max(bw.values()) <= 1.0, bw
    # the same gradients as rsv_mlp_gradient
    g, _ = rsv.rsv_mlp_gradient(ctx, X, t)
    assert np.array_equal(g.astype(np.float64), tr["grads"])
