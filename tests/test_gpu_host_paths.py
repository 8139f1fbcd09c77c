"""Host-side paths of the library on the GPU: the J/H/K diagnostic against
the oracle, the batch graph cache after the buffers it captured were freed
and replaced, the autotuner leaving the last step's moments alone, and the
choice of a launch shape at creation when the fused form does not fit."""
import copy

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


def rel_l1(a, b):
    return np.abs(np.asarray(a, np.float64) - b).sum() / max(np.abs(b).sum(), 1e-300)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-4)])
def test_jhk_matches_oracle(orc, gpu, precision, tol):
    # comoving angular moments per (species, zone, group) (Sec. 4.1)
    p = W.random_2d(41, n_r=8, n_theta=5, n_e=4, n_mu=5, n_phi=6, n_s=2)
    o, dt = orc.run(p, n_steps=4)
    t, _ = gpu.run(p, precision, n_steps=4, dt=dt)
    for a, b in zip(t.jhk(), o.jhk()):
        assert a.shape == b.shape
        assert rel_l1(a, b) <= tol


def test_batch_graph_after_split_buffers_replaced(gpu):
    # a batch step captures the split form's deposit buffers; a shape change
    # frees them and the next split shape allocates new ones.  The next batch
    # step must not replay the graph that holds the freed buffers.
    probs = [W.random_2d(42, n_r=8, n_theta=5, n_e=4, n_mu=4, n_phi=6, n_s=2),
             W.random_column(43, n_r=10, n_e=5, n_mu=6, n_phi=4, n_s=2)]
    split = gpu.SHAPE_SPLIT | 256
    b = gpu.Batch(probs, "mixed")
    for m, p in zip(b.members, probs):
        m.set_launch_shape(split)
        m.set_background(p.backgrounds[0])
        m.set_f(p.f0)
    dts = [0.01, 0.02]
    b.step(dts)
    b.members[0].set_launch_shape(256)     # frees the deposit rows
    b.members[0].set_launch_shape(split)   # allocates new ones
    b.step(dts)
    assert b.graph_launches == 2
    for m, p, dt in zip(b.members, probs, dts):
        t = gpu.Transport(p, "mixed")
        t.set_launch_shape(split)
        t.set_background(p.backgrounds[0])
        t.set_f(p.f0)
        t.step(dt)
        t.step(dt)
        assert np.array_equal(m.get_f(), t.get_f())


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_autotune_keeps_last_step_moments(gpu, precision):
    p = W.random_2d(44, n_r=8, n_theta=5, n_e=4, n_mu=4, n_phi=6, n_s=2)
    t = gpu.Transport(p, precision)
    t.set_background(p.backgrounds[0])
    t.set_f(p.f0)
    dt = t.max_dt(0.5)
    t.step(dt)
    before = [a.copy() for a in t.moments()]
    f_before = t.get_f()
    tot_before = t.totals()
    t.autotune(dt)
    for a, b in zip(t.moments(), before):
        assert np.array_equal(a, b)
    assert np.array_equal(t.get_f(), f_before)
    for a, b in zip(t.totals(), tot_before):
        assert np.array_equal(a, b)


def test_create_picks_a_shape_that_fits(orc, gpu):
    # 6 species, 20 groups, 192 angles in mixed precision: the fused kernel
    # needs about 286 KB of shared memory per CTA, above the opt-in limit;
    # the split form's passes need about 175 KB.  Creation takes split/256.
    p = W.random_2d(45, n_r=4, n_theta=3, n_e=20, n_mu=16, n_phi=12, n_s=6)
    t = gpu.Transport(p, "mixed")
    assert t.launch_shape == gpu.SHAPE_SPLIT | 256
    with pytest.raises(gpu.BtError) as e:
        t.set_launch_shape(256)
    assert e.value.code == -1
    o, dt = orc.run(p, n_steps=2)
    t.set_background(p.backgrounds[0])
    t.set_f(p.f0)
    for k in range(2):
        t.set_background(p.backgrounds[(k + 1) % 2])
        t.step(dt)
    assert rel_l1(t.get_f(), o.get_f()) <= 1e-4


def test_background_checks(gpu):
    # host backgrounds are checked before anything is copied: a NaN or a
    # negative opacity is refused (BT_ERR_BACKGROUND); the opacities here are
    # large enough (4 species x 65536 zones x 20 groups) for the check to be
    # split over host threads
    p = W.cc2d(512, 128, 20, 2, 2, (1.0, 0.5, 0.2, 0.2), W.BASE_SEED + 97, "checks")
    t = gpu.Transport(p, "mixed")
    t.set_background(p.backgrounds[0])
    for field, idx, val in (("kappa_a", (3, 60000, 19), -1.0), ("kappa_s", (2, 123, 4), float("nan")),
                            ("f_eq", (1, 65535, 0), float("inf"))):
        bad = copy.deepcopy(p.backgrounds[1])
        getattr(bad, field)[idx] = val
        with pytest.raises(gpu.BtError) as e:
            t.set_background(bad)
        assert e.value.code == -2
    t.set_background(p.backgrounds[1])   # a valid one is still taken
    t.set_f(p.f0)
    t.step(t.max_dt(0.5))
