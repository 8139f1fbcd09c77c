"""Pins of the CPU float64 network reference (oracle/mlp.py) against what
mathematics fixes: central finite differences of the loss for the gradient,
GELU identities, softmax normalisation, bfloat16 rounding of known values,
and the parameter count of include/bt.h."""
import math
import os
import re

import numpy as np
import pytest

from oracle import mlp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_parameter_count_matches_header():
    src = open(os.path.join(ROOT, "include", "bt.h")).read()
    n = int(re.search(r"#define BT_SUR_NPARAM (\d+)", src).group(1))
    assert n == mlp.N_PARAM == 64 * 16 + 64 + 2 * (64 * 64 + 64) + 27 * 64 + 27 + 32


def test_gelu_identities():
    z = np.linspace(-6, 6, 101)
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert mlp.gelu_d(np.array([0.0]))[0] == 0.5
    # GELU(z) - GELU(-z) = z (Phi(z) + Phi(-z)) = z
    assert np.allclose(mlp.gelu(z) - mlp.gelu(-z), z, atol=1e-14)
    # derivative by central differences
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.allclose(mlp.gelu_d(z), fd, atol=1e-8)
    # large |z|: GELU -> relu
    assert abs(mlp.gelu(np.array([10.0]))[0] - 10.0) < 1e-12


def test_softmax_rows_sum_to_one_and_shift_invariance():
    rng = np.random.default_rng(0)
    z = rng.normal(0, 5, (20, 27))
    p = mlp.softmax(z)
    assert np.allclose(p.sum(axis=1), 1.0, atol=1e-15)
    assert np.allclose(mlp.softmax(z + 123.0), p, atol=1e-15)


def test_bf16_rounding_known_values():
    v = mlp.bf16(np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, -2.5, 1.0 + 2.0 ** -7 + 2.0 ** -8, 0.0]))
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties to even -> 1
    # 1 + 2^-7 + 2^-8 is halfway between 1 + 2^-7 (odd) and 1 + 2^-6: -> 1 + 2^-6
    assert list(v) == [1.0, 1.0, 1.0 + 2.0 ** -7, -2.5, 1.0 + 2.0 ** -6, 0.0]


def _problem(seed, n=7):
    rng = np.random.default_rng(seed)
    p = mlp.init_params(seed)
    q = mlp.unpack(p)
    for l in (1, 2, 3):
        q["b%d" % l][:] = rng.normal(0, 0.3, q["b%d" % l].shape)
    q["b4"][:] = rng.normal(0, 0.3, 27)
    q["mean"][:] = rng.normal(0, 0.1, 16)
    q["scale"][:] = rng.uniform(0.5, 2.0, 16)
    p = mlp.pack(q)
    X = rng.normal(0, 1, (n, 16))
    Y = rng.dirichlet(np.ones(27), n)
    return p, X, Y


@pytest.mark.parametrize("seed", [1, 2])
def test_gradient_by_central_differences(seed):
    p, X, Y = _problem(seed)
    L, g = mlp.loss_and_grad(p, X, Y)
    rng = np.random.default_rng(100 + seed)
    # entries of every trained block, and the normaliser (gradient 0 by design)
    offs, o = [], 0
    for name, shape in mlp.SHAPES:
        k = int(np.prod(shape))
        offs.append((name, o, k))
        o += k
    idx = []
    for name, o, k in offs:
        if name in ("mean", "scale"):
            continue
        idx += list(o + rng.choice(k, 8, replace=False))
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (mlp.loss_and_grad(pp, X, Y)[0] - mlp.loss_and_grad(pm, X, Y)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(fd)), (i, fd, g[i])
    o_mean = [o for name, o, k in offs if name == "mean"][0]
    assert not np.any(g[o_mean:])


def test_loss_is_cross_entropy_of_softmax():
    p, X, Y = _problem(3, n=5)
    P = mlp.forward(p, X)
    L, _ = mlp.loss_and_grad(p, X, Y)
    assert math.isclose(L, -(Y * np.log(P)).sum() / 5, rel_tol=1e-13)
    # a one-hot target equal to argmax does not give zero loss unless P is one-hot
    assert L > 0


def test_operand_rounding_only_changes_operands():
    p, X, Y = _problem(4, n=9)
    P64 = mlp.forward(p, X)
    P16 = mlp.forward(p, X, operand_round=mlp.bf16)
    # bf16 operands move the output by well under a percent, not more
    assert np.abs(P16 - P64).max() < 2e-2
    assert np.abs(P16 - P64).max() > 0
