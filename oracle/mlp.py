"""Plain float64 CPU reference of the learned remap's network.

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline may use this module; the library never does.

The network is 16 -> 64 -> 64 -> 64 -> 27: affine layers with the Gaussian
error linear unit GELU(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2 on the
hidden layers, a softmax on the output, and the cross-entropy loss
L = -1/n sum_rows sum_o Y_o log P_o against target distributions Y.  The
input is normalised first, x_n = (x - mean) * scale.  Parameters are one
flat float vector in the layout of include/bt.h (W_l row-major [out][in]).

The backward pass is the chain rule written out: dL/dz_out = (P - Y)/n,
dW = dZ^T H_prev, db = sum_rows dZ, dH_prev = dZ W, dZ_prev = dH_prev *
GELU'(z_prev) with GELU'(z) = Phi(z) + z phi(z).  It is pinned by central
finite differences in tests/test_surrogate_cpu.py.

``operand_round`` emulates the tensor-core path's operand precision: when
given (e.g. ``bf16``), the MMA operands -- normalised inputs, weights and
hidden activations -- are rounded by it while every sum stays float64.
"""
from __future__ import annotations

import math

import numpy as np

N_IN, N_H, N_OUT = 16, 64, 27
SHAPES = [("W1", (N_H, N_IN)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)),
          ("W3", (N_H, N_H)), ("b3", (N_H,)), ("W4", (N_OUT, N_H)), ("b4", (N_OUT,)),
          ("mean", (N_IN,)), ("scale", (N_IN,))]
N_PARAM = sum(int(np.prod(s)) for _, s in SHAPES)   # 11195


def unpack(p):
    """Flat parameter vector -> dict of float64 arrays (views into a copy)."""
    p = np.asarray(p, dtype=np.float64).copy()
    out, o = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = p[o:o + k].reshape(shape)
        o += k
    assert o == N_PARAM
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], np.float64).reshape(-1) for name, _ in SHAPES])


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    x = np.asarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)


_erf = np.vectorize(math.erf, otypes=[np.float64])


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_d(z):
    return 0.5 * (1.0 + _erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def softmax(z):
    m = z.max(axis=-1, keepdims=True)
    e = np.exp(z - m)
    return e / e.sum(axis=-1, keepdims=True)


def forward(p, X, operand_round=None, keep=False):
    """P [n][27] for inputs X [n][16]; with keep=True also the activations."""
    q = unpack(p)
    r = operand_round if operand_round is not None else (lambda a: a)
    x = (np.asarray(X, np.float64) - q["mean"]) * q["scale"]
    if operand_round is not None:
        x = r(np.asarray(x, np.float32))   # the device normalises in float32
    hs, zs = [x], []
    h = x
    for l in (1, 2, 3):
        z = r(h) @ r(q["W%d" % l]).T + q["b%d" % l]
        zs.append(z)
        h = gelu(z)
        hs.append(h)
    zo = r(h) @ r(q["W4"]).T + q["b4"]
    P = softmax(zo)
    if keep:
        return P, hs, zs, zo
    return P


def loss_and_grad(p, X, Y):
    """Mean cross entropy over the rows and its gradient (flat, normaliser
    entries zero), all float64."""
    q = unpack(p)
    P, hs, zs, zo = forward(p, X, keep=True)
    Y = np.asarray(Y, np.float64)
    n = len(X)
    logP = zo - zo.max(axis=1, keepdims=True)
    logP = logP - np.log(np.exp(logP).sum(axis=1, keepdims=True))
    L = -(Y * logP).sum() / n
    g = {name: np.zeros(shape) for name, shape in SHAPES}
    dz = (P - Y) / n
    g["W4"] = dz.T @ hs[3]
    g["b4"] = dz.sum(axis=0)
    dh = dz @ q["W4"]
    for l in (3, 2, 1):
        dz = dh * gelu_d(zs[l - 1])
        g["W%d" % l] = dz.T @ hs[l - 1]
        g["b%d" % l] = dz.sum(axis=0)
        dh = dz @ q["W%d" % l]
    return L, pack(g)


def init_params(seed, mean=None, scale=None):
    """He-uniform weights, zero biases, identity normaliser unless given
    (a seeded input generator: both sides receive the same vector)."""
    rng = np.random.default_rng(seed)
    d = {}
    for l, (o, i) in enumerate([(N_H, N_IN), (N_H, N_H), (N_H, N_H), (N_OUT, N_H)], start=1):
        lim = math.sqrt(6.0 / i)
        d["W%d" % l] = rng.uniform(-lim, lim, (o, i))
        d["b%d" % l] = np.zeros(o)
    d["mean"] = np.zeros(N_IN) if mean is None else np.asarray(mean, np.float64)
    d["scale"] = np.ones(N_IN) if scale is None else np.asarray(scale, np.float64)
    return pack(d)
