"""The allocation-free totals entry point (bt_weighted_totals_noalloc).

It serves callers that cannot allocate device memory -- a host code whose
own allocator owns the GPU's memory, or a loop that must never allocate --
by keeping its partial sums in a fixed device array inside the library.
Here it is called through the C ABI and checked against the handle-based
bt_totals on two consecutive calls, in both precisions.  This file is
collected last so that a stop at the first failure has run every other test.
"""
import math

import numpy as np
import pytest

from paper_2003_02845_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _weights(orc, prob, bg):
    # number weights of bt_totals: w_za[z][b] = dV phi^6 u^0 dOmega, w_e = dGamma
    g = orc.Oracle(prob).grid()
    mu, dmu = g["mu"], g["dmu"]
    nph = prob.n_phi
    ph = (np.arange(nph) + 0.5) * 2 * math.pi / nph
    s = np.sqrt(1 - mu ** 2)
    n = np.stack([np.repeat(mu, nph), np.outer(s, np.cos(ph)).ravel(), np.outer(s, np.sin(ph)).ravel()], 1)
    dom = np.repeat(dmu, nph) * 2 * math.pi / nph
    gam = 1 / np.sqrt(1 - (bg.v ** 2).sum(1))
    u0 = gam[:, None] * (1 + bg.v @ n.T)
    w_za = g["vol"][:, None] * bg.phi[:, None] ** 6 * u0 * dom[None, :]
    return np.ascontiguousarray(w_za), np.ascontiguousarray(g["dgam"])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_totals_match_bt_totals(orc, precision):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2003_02845_gb300 import build, bt
    build.build()
    p = W.random_2d(21, n_r=9, n_theta=5, n_e=4, n_mu=4, n_phi=6, n_s=2)
    bg = p.backgrounds[0]
    t = bt.Transport(p, precision)
    t.set_background(bg)
    t.set_f(p.f0)
    dt = t.max_dt(0.5)
    w_za, w_e = _weights(orc, p, bg)
    w_za_d = torch.as_tensor(w_za).cuda()
    w_e_d = torch.as_tensor(w_e).cuda()
    dtype = torch.float32 if precision == "mixed" else torch.float64
    for call in range(2):
        t.step(dt)                      # the two calls see different distributions
        f_d = torch.empty(t.shape, dtype=dtype, device="cuda")
        t.get_f(f_d)
        ref = t.totals()[0]
        out = torch.full((p.n_species,), float("nan"), dtype=torch.float64, device="cuda")
        bt.weighted_totals_noalloc(f_d, w_za_d, w_e_d, precision, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.allclose(got, ref, rtol=1e-12, atol=0), (call, got, ref)
