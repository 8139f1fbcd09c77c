"""Local time stepping on the GPU (bt_lts_levels, bt_step_lts) against the
oracle's (reading R-19): the same levels, FP64 f, moments and totals to
1e-12, mixed to 1e-4, and one level equal to the split global step to the
bit."""
import math

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


def _cases():
    col = W.random_column(111, n_r=20, n_e=4, n_mu=6, n_phi=4, n_s=2, r_min=0.5, r_max=12.0)
    d2 = W.random_2d(112, n_r=14, n_theta=6, n_e=3, n_mu=4, n_phi=6, n_s=2, r_min=0.5, r_max=12.0)
    lob = W.random_2d(113, n_r=12, n_theta=5, n_e=3, n_mu=5, n_phi=6, n_s=1, r_min=0.5, r_max=10.0)
    lob.mu_quadrature = "lobatto"
    return {"column": col, "2d": d2, "2d_lobatto": lob}


@pytest.mark.parametrize("case", ["column", "2d", "2d_lobatto"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-4)])
def test_lts_matches_oracle(orc, gpu, case, precision, tol):
    p = _cases()[case]
    o = orc.Oracle(p)
    o.set_background(p.backgrounds[0])
    o.set_f(p.f0)
    dt0, lev = o.lts_levels(0.5, 3)
    t = gpu.Transport(p, precision)
    t.set_background(p.backgrounds[0])
    t.set_f(p.f0)
    dt0g, levg = t.lts_levels(0.5, 3)
    assert np.array_equal(levg, lev) and lev.max() == 2
    assert math.isclose(dt0g, dt0, rel_tol=1e-12)
    for k in range(4):
        o.set_background(p.backgrounds[(k + 1) % 2])
        t.set_background(p.backgrounds[(k + 1) % 2])
        o.step_lts(dt0, lev, 3)
        t.step_lts(dt0)
    fo = o.get_f()
    assert rel_l1(t.get_f(), fo) <= tol
    No, Ng = o.totals(), t.totals()
    for a, b in zip(Ng, No):
        assert np.allclose(a, b, rtol=tol if precision == "fp64" else 1e-6, atol=0)
    if precision == "fp64":
        for a, b in zip(t.moments(), o.moments()):
            assert rel_l1(a, b) <= 1e-10


def test_one_level_equals_the_split_step(gpu):
    p = _cases()["2d"]
    a = gpu.Transport(p, "fp64")
    a.set_launch_shape(gpu.SHAPE_SPLIT | 256)
    b = gpu.Transport(p, "fp64")
    for t in (a, b):
        t.set_background(p.backgrounds[0])
        t.set_f(p.f0)
    dt = a.max_dt(0.5)
    b.set_levels(np.zeros(p.n_zone, dtype=np.int32), 1)
    for k in range(3):
        for t in (a, b):
            t.set_background(p.backgrounds[(k + 1) % 2])
        a.step(dt)
        b.step_lts(dt)
    assert np.array_equal(a.get_f(), b.get_f())
    for x, y in zip(a.moments(), b.moments()):
        assert np.array_equal(x, y)
    for x, y in zip(a.totals(), b.totals()):
        assert np.array_equal(x, y)


def test_lts_argument_checks(gpu):
    p = _cases()["column"]
    t = gpu.Transport(p, "fp64")
    t.set_background(p.backgrounds[0])
    with pytest.raises(gpu.BtError) as e:
        t.step_lts(0.01)                       # no levels yet
    assert e.value.code == -6
    with pytest.raises(gpu.BtError) as e:
        t.set_levels(np.full(p.n_zone, 3, dtype=np.int32), 3)
    assert e.value.code == -1
