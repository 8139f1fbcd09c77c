"""Batched graph step and autotuned launch shapes (GPU).

A batch advances independent problems of uneven size with one CUDA-graph
launch per step; every member must equal the same problem run alone (same
kernels, same inputs) and the FP64 oracle.  The launch shape the autotuner
picks must not change the FP64 results at all.
"""
import numpy as np
import pytest

from paper_2003_02845_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2003_02845_gb300 import build, bt
    build.build()
    return bt


def _probs():
    return [W.random_2d(31, n_r=9, n_theta=5, n_e=4, n_mu=4, n_phi=6, n_s=2),
            W.random_column(32, n_r=13, n_e=6, n_mu=6, n_phi=4, n_s=3),
            W.random_2d(33, n_r=6, n_theta=4, n_e=3, n_mu=5, n_phi=7, n_s=1, r_min=0.0)]


def _run_batch(bt, probs, precision, n_steps, dts):
    b = bt.Batch(probs, precision)
    for m, p in zip(b.members, probs):
        m.set_background(p.backgrounds[0])
        m.set_f(p.f0)
    for k in range(n_steps):
        for m, p in zip(b.members, probs):
            m.set_background(p.backgrounds[(k + 1) % 2])
        b.step(dts)
    return b


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_equals_members_run_alone(gpu, precision):
    probs = _probs()
    dts = [0.01, 0.02, 0.015]
    b = _run_batch(gpu, probs, precision, 6, dts)
    assert b.graph_launches == 6
    for m, p, dt in zip(b.members, probs, dts):
        t, _ = gpu.run(p, precision, n_steps=6, dt=dt)
        assert np.array_equal(m.get_f(), t.get_f())
        for a, c in zip(m.moments(), t.moments()):
            assert np.array_equal(a, c)


def test_batch_fp64_matches_oracle(orc, gpu):
    probs = _probs()
    dts = [0.01, 0.02, 0.015]
    b = _run_batch(gpu, probs, "fp64", 5, dts)
    for m, p, dt in zip(b.members, probs, dts):
        o, _ = orc.run(p, n_steps=5, dt=dt)
        fo = o.get_f()
        e = np.abs(m.get_f() - fo).sum() / np.abs(fo).sum()
        assert e <= 1e-12, e


def test_launch_shapes_give_identical_fp64_results(gpu):
    p = W.random_2d(34, n_r=8, n_theta=5, n_e=4, n_mu=4, n_phi=6, n_s=2)
    ref = None
    for nt in (128, 256, 512):
        t = gpu.Transport(p, "fp64")
        t.set_launch_shape(nt)
        assert t.launch_shape == nt
        t.set_background(p.backgrounds[0])
        t.set_f(p.f0)
        for k in range(4):
            t.set_background(p.backgrounds[(k + 1) % 2])
            t.step(0.01)
        f = t.get_f()
        if ref is None:
            ref = f
        else:
            assert np.array_equal(f, ref)


def test_mixed_launch_shapes_agree(gpu):
    p = W.random_2d(35, n_r=8, n_theta=5, n_e=4, n_mu=4, n_phi=6, n_s=2)
    out = []
    for nt in (128, 256, 512):
        t = gpu.Transport(p, "mixed")
        t.set_launch_shape(nt)
        t.set_background(p.backgrounds[0])
        t.set_f(p.f0)
        for k in range(4):
            t.set_background(p.backgrounds[(k + 1) % 2])
            t.step(0.01)
        out.append(t.get_f().astype(np.float64))
    for f in out[1:]:
        assert np.abs(f - out[0]).sum() / np.abs(out[0]).sum() < 1e-6


def test_autotune_and_cache(gpu, tmp_path, monkeypatch):
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("BT_TUNE_CACHE", str(cache))
    p = W.random_2d(36, n_r=10, n_theta=6, n_e=4, n_mu=4, n_phi=6, n_s=2)
    t = gpu.Transport(p, "mixed")
    t.set_background(p.backgrounds[0])
    t.set_f(p.f0)
    f0 = t.get_f()
    nt = t.autotune(0.01)
    assert nt in (128, 256, 512, gpu.SHAPE_SPLIT | 256, gpu.SHAPE_SPLIT | 512)
    assert t.launch_shape == nt
    assert np.array_equal(t.get_f(), f0)          # tuning leaves f untouched
    assert cache.exists() and str(nt) in cache.read_text()
    t2 = gpu.Transport(p, "mixed")                 # picks the cached shape
    assert t2.launch_shape == nt
