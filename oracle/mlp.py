"""FP64 reference of the sweep surrogate MLP (4 -> 64 -> 64 -> 3, GELU).

TEST INFRASTRUCTURE ONLY: the independent checker of the tensor-core MLP
kernels of the CUDA library (plain numpy, no code shared with them).  Only
tests/, __graft_entry__.smoke() and bench.py's CPU legs may use it.

Parameters are packed as W1[64][4] b1[64] W2[64][64] b2[64] W3[3][64] b3[3].
Inputs are normalised as (x - in_mean) / in_scale; the network's output o is
mapped to y = out_mean + out_scale * o; the loss is the mean over all B x 3
entries of (o - (t - out_mean) / out_scale)^2.  GELU is the exact form
0.5 z (1 + erf(z / sqrt 2)).

``operands="bf16"`` follows the arithmetic contract of the tensor-core
kernels instead of exact arithmetic: each matrix contraction takes BF16
operands (the normalised inputs, the activations H1 and H2 and the output
gradient of the forward and backward products that run on the tensor cores,
and dZ2) and sums them exactly, while the 3- and 4-wide gradient reductions
(dW3 = dY^T H2, dW1 = dZ1^T Xn and the biases) take their FP32 operands as
they are.  With the weights already rounded to BF16 it differs from the
kernels only by their FP32 accumulation and FP32 GELU.
"""
from __future__ import annotations

import math

import numpy as np

NI, NH, NO = 4, 64, 3
SHAPES = [("W1", (NH, NI)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("W3", (NO, NH)), ("b3", (NO,))]
NP = sum(int(np.prod(s)) for _, s in SHAPES)

_erf = np.vectorize(math.erf)


def unpack(p):
    out, o = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = np.asarray(p[o:o + k], dtype=np.float64).reshape(shape)
        o += k
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_d(z):
    return 0.5 * (1.0 + _erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def bf16(x):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    a = np.asarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _operand(operands):
    if operands is None:
        return lambda a: a
    assert operands == "bf16", operands
    return bf16


def forward(p, X, norm, operands=None):
    """Outputs y [B, 3] and the intermediates needed by backward."""
    r = _operand(operands)
    w = unpack(p)
    xn = (np.asarray(X, np.float64) - norm["in_mean"]) / norm["in_scale"]
    z1 = r(xn) @ w["W1"].T + w["b1"]
    h1 = gelu(z1)
    z2 = r(h1) @ w["W2"].T + w["b2"]
    h2 = gelu(z2)
    o = r(h2) @ w["W3"].T + w["b3"]
    y = norm["out_mean"] + norm["out_scale"] * o
    return y, dict(xn=xn, z1=z1, h1=h1, z2=z2, h2=h2, o=o)


def loss_and_grad(p, X, T, norm, operands=None):
    """Mean squared error on normalised outputs and its gradient (packed)."""
    r = _operand(operands)
    w = unpack(p)
    y, c = forward(p, X, norm, operands)
    tn = (np.asarray(T, np.float64) - norm["out_mean"]) / norm["out_scale"]
    e = c["o"] - tn
    B = e.shape[0]
    loss = float((e * e).sum() / (B * NO))
    do = 2.0 * e / (B * NO)
    g = {}
    g["W3"] = do.T @ c["h2"]
    g["b3"] = do.sum(0)
    dz2 = (r(do) @ w["W3"]) * gelu_d(c["z2"])
    g["W2"] = r(dz2).T @ r(c["h1"])
    g["b2"] = dz2.sum(0)
    dz1 = (r(dz2) @ w["W2"]) * gelu_d(c["z1"])
    g["W1"] = dz1.T @ c["xn"]
    g["b1"] = dz1.sum(0)
    return loss, pack(g)


def bf16_operands(p, X, T, norm):
    """Every value ``operands="bf16"`` rounds to BF16 (flattened), for
    checking how far each lies from a BF16 rounding boundary."""
    w = unpack(p)
    _, c = forward(p, X, norm, "bf16")
    tn = (np.asarray(T, np.float64) - norm["out_mean"]) / norm["out_scale"]
    do = 2.0 * (c["o"] - tn) / (c["o"].shape[0] * NO)
    dz2 = (bf16(do) @ w["W3"]) * gelu_d(c["z2"])
    return np.concatenate([a.ravel() for a in (c["xn"], c["h1"], c["h2"], do, dz2)])


def init_params(seed=0):
    """He-style random initial parameters (the same for the CUDA network and this reference)."""
    rng = np.random.default_rng(seed)
    d = {"W1": rng.normal(0, math.sqrt(2.0 / NI), (NH, NI)), "b1": np.zeros(NH),
         "W2": rng.normal(0, math.sqrt(2.0 / NH), (NH, NH)), "b2": np.zeros(NH),
         "W3": rng.normal(0, math.sqrt(1.0 / NH), (NO, NH)), "b3": np.zeros(NO)}
    return pack(d)


def weight_mask():
    """1 on the entries of W1, W2, W3 (decayed), 0 on the biases."""
    return pack({k: np.full(s, 1.0 if k.startswith("W") else 0.0) for k, s in SHAPES})


def adam_step(p, m, v, g, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0):
    """One Adam step (Kingma & Ba, bias-corrected moments; t counts from 1) with
    decoupled weight decay on the weight matrices (Loshchilov & Hutter).
    Returns the new (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    p = p - lr * (mhat / (np.sqrt(vhat) + eps) + weight_decay * weight_mask() * p)
    return p, m, v
