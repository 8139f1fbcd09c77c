"""Data set and training run of the learned remap (the network of
include/bt.h, bt_sur_*).

Rows of the exact remap are drawn uniformly over (zone, remap kind, source
angle) from seeded background pairs and evaluated by the library's own
generator (bt_sur_samples, float64 on the GPU); rows whose exact weights fall
outside the 27 offsets are dropped.  Training runs in the library
(bt_sur_train: tensor-core forward and backward, Adam).  This module only
orders those calls and moves tensors.
"""
from __future__ import annotations

import numpy as np

from . import bt, workloads as W


def training_set(prob, pairs, n_rows: int, seed: int, stream=None):
    """Up to n_rows usable rows from the background pairs (B_prev, B_cur) of
    `pairs`, shuffled: device tensors X [n][16], Y [n][27]."""
    import torch
    t = bt.Transport(prob, "mixed", stream=stream)
    per = -(-n_rows // len(pairs))
    Xs, Ys = [], []
    for k, (b0, b1) in enumerate(pairs):
        t.set_background(b0)
        t.set_background(b1)
        # draw a little more than needed: some rows have no remap
        idx = W.sur_rows(prob.n_zone, prob.n_ang, int(per * 1.35), seed + k)
        X, Y, v = t.sur_samples(idx)
        keep = v == 1
        Xs.append(X[keep][:per])
        Ys.append(Y[keep][:per])
    t.close()
    X, Y = torch.cat(Xs), torch.cat(Ys)
    g = torch.Generator().manual_seed(seed)
    perm = torch.randperm(X.shape[0], generator=g)[:n_rows].to(X.device)
    return X[perm].contiguous(), Y[perm].contiguous()


def train(X, Y, epochs=10, batch=4096, lr=2e-3, lr_final=5e-5, seed=0, stream=None):
    """A fresh network (seeded He-uniform weights, normaliser fitted to X)
    trained on (X, Y); returns (network, per-epoch mean loss)."""
    s = bt.Surrogate(stream=stream)
    s.set_params(init_params(seed))
    s.fit_normalizer(X)
    log = s.train(X, Y, epochs=epochs, batch=batch, lr=lr, lr_final=lr_final)
    return s, log


def init_params(seed: int) -> np.ndarray:
    """He-uniform weights, zero biases, identity normaliser (float32)."""
    rng = np.random.default_rng(seed)
    parts = []
    for o, i in ((64, 16), (64, 64), (64, 64), (27, 64)):
        lim = np.sqrt(6.0 / i)
        parts += [rng.uniform(-lim, lim, o * i), np.zeros(o)]
    parts += [np.zeros(16), np.ones(16)]
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == bt.SUR_NPARAM
    return p
