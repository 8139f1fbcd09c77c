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


# ---------------------------------------------------------------------------
# Rows of the exact remap (oracle orc_sur_sample): features and targets
# ---------------------------------------------------------------------------
def _column(v1, phi1, n_mu=6, n_phi=4, n_e=5):
    from paper_2003_02845_gb300 import workloads as W
    p = W.random_column(21, n_r=6, n_e=n_e, n_mu=n_mu, n_phi=n_phi, n_s=1)
    b0, b1 = p.backgrounds
    for bg in (b0, b1):
        bg.v[:] = 0.0
        bg.alpha[:] = 1.0
        bg.phi[:] = 1.0
    b1.v[:] = v1
    b1.phi[:] = phi1
    return p


def _oracle_rows(p, idx):
    import oracle
    o = oracle.Oracle(p)
    o.set_background(p.backgrounds[0])
    o.set_background(p.backgrounds[1])
    return o.sur_samples(idx)


def _unpack_offsets(y):
    """27 weights -> (energy, mu, Phi) marginals over offsets -1, 0, 1"""
    w = y.reshape(3, 3, 3)
    return w.sum(axis=(1, 2)), w.sum(axis=(0, 2)), w.sum(axis=(0, 1))


def test_time_row_of_a_static_background_is_the_identity():
    p = _column(0.0, 1.0)
    idx = [(z, 0, a) for z in range(p.n_zone) for a in range(p.n_ang)]
    X, Y, v = _oracle_rows(p, idx)
    assert np.all(v == 1)
    one = np.zeros(27)
    one[13] = 1.0
    assert np.allclose(Y, one, atol=1e-15)
    assert np.allclose(np.linalg.norm(X[:, :3], axis=1), 1.0, atol=1e-15)
    assert not np.any(X[:, 3:])


def test_time_row_conformal_kick_shifts_energy_only():
    # phi_src / phi_dst = sqrt(1.05): the time kick scales the energy by 1.05
    # (phi^2 p conserved) and leaves the direction alone
    p = _column(0.0, 1.0 / math.sqrt(1.05))
    R = (p.eps_edges[2] / p.eps_edges[1])
    idx = [(2, 0, a) for a in range(p.n_ang)]
    X, Y, v = _oracle_rows(p, idx)
    assert np.all(v == 1)
    we = (1.05 - 1.0) / (R - 1.0)                  # linear weight of the upper group
    for y in Y:
        e, m, f = _unpack_offsets(y)
        assert np.allclose(e, [0.0, 1.0 - we, we], atol=1e-13)
        assert np.allclose(m, [0, 1, 0], atol=1e-13) and np.allclose(f, [0, 1, 0], atol=1e-13)
    assert np.allclose(X[:, 15], math.log(1.05), atol=1e-15)


def test_time_row_radial_boost_is_doppler_and_aberration():
    # previous background at rest, current one moving with beta along r:
    # comoving energy ratio gamma (1 - beta mu) and mu* = (mu - beta)/(1 - beta mu)
    beta = 0.1
    p = _column(np.array([beta, 0.0, 0.0]), 1.0, n_mu=8, n_phi=4)
    import oracle
    mu_nodes, _ = oracle.gauss_legendre(p.n_mu)
    R = p.eps_edges[2] / p.eps_edges[1]
    g = 1.0 / math.sqrt(1.0 - beta * beta)
    idx = [(3, 0, a) for a in range(p.n_ang)]
    X, Y, v = _oracle_rows(p, idx)
    for a, (x, y, ok) in enumerate(zip(X, Y, v)):
        j = a // p.n_phi
        mu = mu_nodes[j]
        rho = g * (1.0 - beta * mu)
        mus = (mu - beta) / (1.0 - beta * mu)
        m = math.floor(math.log(rho) / math.log(R))
        we = (rho / R ** m - 1.0) / (R - 1.0)
        jl = max(k for k in range(p.n_mu - 1) if mu_nodes[k] <= mus) if mus > mu_nodes[0] else 0
        wm = 0.0 if mus <= mu_nodes[0] else (mus - mu_nodes[jl]) / (mu_nodes[jl + 1] - mu_nodes[jl])
        if ok != 1:
            # only an energy shift of more than one group, or a mu shift of
            # more than one node, is unrepresentable
            assert m < -1 or m > 0 or jl - j < -1 or jl + 1 - j > 1
            continue
        e, mm, f = _unpack_offsets(y)
        assert math.isclose(float(e @ [-1, 0, 1]), m + we, abs_tol=1e-12)
        assert math.isclose(float(mm @ [-1, 0, 1]), (jl - j) + wm, abs_tol=1e-12)
        assert np.allclose(f, [0, 1, 0], atol=1e-12)      # a radial boost keeps Phi
        assert np.allclose(x[3:6], 0.0) and np.allclose(x[6:9], [beta, 0, 0])


def test_face_rows_are_normalised_and_frames_consistent():
    from paper_2003_02845_gb300 import workloads as W
    p = W.random_2d(22, n_r=7, n_theta=4, n_e=4, n_mu=4, n_phi=6, n_s=1)
    rng = np.random.default_rng(1)
    idx = np.stack([rng.integers(0, p.n_zone, 3000), rng.integers(1, 31, 3000), rng.integers(0, p.n_ang, 3000)], 1)
    X, Y, v = _oracle_rows(p, idx)
    ok = v == 1
    assert ok.sum() > 1000
    assert np.allclose(Y[ok].sum(axis=1), 1.0, atol=1e-13)
    assert np.all(Y >= 0.0)
    assert not np.any(Y[v != 1]) and not np.any(X[v == 0])
    # the kick-axis feature sits on the face's axis only: radial faces (kinds
    # 1..12) on component 12, polar faces (13..24) on 13, azimuthal on 14
    kind = idx[:, 1]
    for lo, hi, comp in ((1, 13, 12), (13, 25, 13), (25, 31, 14)):
        sel = ok & (kind >= lo) & (kind < hi)
        others = [c for c in (12, 13, 14) if c != comp]
        assert not np.any(X[sel][:, others])
    # cell P remapped into its outer radial face (kind 1 + 6 + 1) and the face
    # remapped back into P (kind 1 + 6 + 4) see opposite rotations
    z, a = 10, 5
    Xa, _, va = _oracle_rows(p, [(z, 1 + 6 * 1 + 1, a), (z, 1 + 6 * 1 + 4, a)])
    assert list(va) == [1, 1]
    assert np.allclose(Xa[0, 9:12], -Xa[1, 9:12], atol=1e-15)
