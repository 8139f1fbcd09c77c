"""Local time stepping (Sec. 5: larger steps for the larger outer zones;
reading R-19) in the oracle.  Pins: one level is the global step to the
bit; number is conserved face by face whatever the levels; the levels keep
every zone within its own Courant limit with neighbours at most one level
apart; and over the same time the local steps follow the global steps to
the accuracy of the time discretisation.  No GPU."""
import math

import numpy as np
import pytest

from paper_2003_02845_gb300 import workloads as W


def _start(orc, p, bg=0):
    o = orc.Oracle(p)
    o.set_background(p.backgrounds[bg])
    o.set_f(p.f0)
    return o


def test_one_level_is_the_global_step(orc):
    p = W.random_2d(101, n_r=7, n_theta=4, n_e=3, n_mu=4, n_phi=6, n_s=2)
    a, b = _start(orc, p), _start(orc, p)
    dt = a.max_dt(0.5)
    for k in range(3):
        a.set_background(p.backgrounds[(k + 1) % 2])
        b.set_background(p.backgrounds[(k + 1) % 2])
        a.step(dt)
        b.step_lts(dt, np.zeros(p.n_zone, dtype=np.int32), 1)
    assert np.array_equal(a.get_f(), b.get_f())
    for x, y in zip(a.moments(), b.moments()):
        assert np.array_equal(x, y)
    for x, y in zip(a.totals(), b.totals()):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("geom", ["column", "2d"])
def test_levels_respect_each_zones_limit(orc, geom):
    if geom == "column":
        p = W.random_column(102, n_r=24, n_e=3, n_mu=4, n_phi=4, n_s=1, r_min=0.5, r_max=20.0)
    else:
        p = W.random_2d(103, n_r=16, n_theta=6, n_e=3, n_mu=4, n_phi=6, n_s=1, r_min=0.5, r_max=20.0)
    o = _start(orc, p)
    dt0, lev = o.lts_levels(0.5, 4)
    rate = o.zone_rates()
    assert math.isclose(dt0, 0.5 / rate.max(), rel_tol=1e-15)
    assert np.all(dt0 * 2.0 ** lev * rate <= 0.5 * (1 + 1e-12))      # within its own limit
    assert lev.max() >= 2 and lev.min() == 0                           # the levels are used
    L2 = lev.reshape(p.n_theta, p.n_r)
    assert np.all(np.abs(np.diff(L2, axis=1)) <= 1)
    assert np.all(np.abs(np.diff(L2, axis=0)) <= 1)


@pytest.mark.parametrize("geom", ["column", "2d"])
def test_local_steps_conserve_number(orc, geom):
    # moving curved backgrounds alternating every macro step (time remap
    # included), no absorption: content + outflow is conserved to round-off
    if geom == "column":
        p = W.random_column(104, n_r=20, n_e=3, n_mu=4, n_phi=4, n_s=2, r_min=0.5, r_max=12.0)
    else:
        p = W.random_2d(105, n_r=12, n_theta=5, n_e=3, n_mu=4, n_phi=6, n_s=1, r_min=0.5, r_max=12.0)
    for bg in p.backgrounds:
        bg.kappa_a[:] = 0.0
    o = _start(orc, p)
    N0 = o.totals()[0]
    dt0, lev = o.lts_levels(0.5, 3)
    assert lev.max() == 2
    for k in range(4):
        o.set_background(p.backgrounds[(k + 1) % 2])
        o.step_lts(dt0, lev, 3)
        N, _, No, _ = o.totals()
        assert np.allclose(N + No, N0, rtol=1e-13, atol=0)


def test_local_steps_follow_the_global_steps(orc):
    # the radiating sphere (Sec. 4.1 setup) on a log grid: the inner zones
    # step 4x more often than the outer ones.  After the same time the local
    # steps differ from the global steps by the time-discretisation error:
    # no more than 3x the difference that doubling the global step makes
    p = W.homogeneous_sphere(n_r=40, kappa=4.0, n_e=1, n_mu=8, n_phi=4, dang=0.25)
    p.r_edges = np.geomspace(0.1, 4.0, 41)
    a, b, c = _start(orc, p), _start(orc, p), _start(orc, p)
    dt0, lev = b.lts_levels(0.5, 3)
    assert lev.max() == 2 and lev.min() == 0
    for _ in range(60):
        b.step_lts(dt0, lev, 3)
    for _ in range(60 * 4):
        a.step(dt0)
    for _ in range(60 * 2):
        c.step(2 * dt0)
    fa, fb, fc = a.get_f(), b.get_f(), c.get_f()
    scale = np.abs(fa - fc).sum() / np.abs(fa).sum()
    assert 0 < np.abs(fa - fb).sum() / np.abs(fa).sum() < 3 * scale
    # fewer zone updates for the same time
    assert sum(2 ** (2 - lv) for lv in lev) < 0.5 * 4 * p.n_zone
