"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the
same seeded inputs.  FP64 path: relative L1 <= 1e-12 (the bar the transport
step is held to); mixed path: relative L1 <= 1e-4 after 100 steps."""
import math

import numpy as np
import pytest

from paper_2003_02845_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL_MIXED = 1e-4


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


def compare_run(orc, bt, prob, n_steps, precision="fp64", tol=TOL64, cfl=0.5):
    o, dt = orc.run(prob, n_steps=n_steps, cfl=cfl)
    t, _ = bt.run(prob, precision, n_steps=n_steps, dt=dt)
    fo, fg = o.get_f(), t.get_f()
    e = rel_l1(fg, fo)
    assert e <= tol, "rel-L1(f) = %.3e > %.1e" % (e, tol)
    # element-wise: FP64 every bin within 50 tol of the largest value of its
    # (species, zone, group) row; mixed, of its (species, zone) block -- the
    # float32 remap mixes groups of very different size (spectral tails), so
    # its rounding is relative to the zone's magnitude
    # mixed: also an absolute floor of 1e-6 of the species' largest value (a
    # float32 flux from a bright zone into a dim one carries an absolute error
    # relative to the bright zone)
    # FP64: the row scale is floored at 1e-6 of the (species, zone) block's
    # largest value -- the energy remap feeds each group from its neighbours,
    # and in the diffusion region a spectral tail's rows lie 40 or more
    # orders of magnitude below the zone's bulk, so their rounding is
    # relative to the bulk, not to themselves
    axes = (-1,) if precision == "fp64" else (-2, -1)
    scale = np.maximum(np.abs(fo).max(axis=axes, keepdims=True), 1e-300)
    if precision == "fp64":
        scale = np.maximum(scale, 1e-6 * np.abs(fo).max(axis=(-2, -1), keepdims=True))
    else:
        gmax = np.abs(fo).max(axis=(1, 2, 3), keepdims=True)
        scale = np.maximum(scale, 1e-6 / (50 * tol) * gmax)
    assert np.max(np.abs(fg - fo) / scale) <= 50 * tol
    return o, t, dt


# ---------------------------------------------------------------------------
# FP64 path: element-wise parity on small cases spanning every face type
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed", [1, 2])
def test_fp64_column_moving_gr(orc, gpu, seed):
    p = W.random_column(seed, n_r=11, n_e=5, n_mu=6, n_phi=4, n_s=2)
    o, t, dt = compare_run(orc, gpu, p, 12)
    # moments and totals
    mo, mg = o.moments(), t.moments()
    for a, b in zip(mg, mo):
        assert rel_l1(a, b) <= 1e-11
    No, Ng = o.totals(), t.totals()
    for a, b in zip(Ng, No):
        assert np.allclose(a, b, rtol=1e-12, atol=1e-300)


def test_fp64_column_origin(orc, gpu):
    # r_edges[0] == 0: zero-area inner face, pyramid zone at the centre
    p = W.homogeneous_sphere(n_r=13, n_e=3, n_mu=6, n_phi=4, dang=0.25)
    p.f0 = np.random.default_rng(3).uniform(0, 1, p.f0.shape)
    compare_run(orc, gpu, p, 10)


@pytest.mark.parametrize("seed", [4, 5])
def test_fp64_2d(orc, gpu, seed):
    p = W.random_2d(seed, n_r=9, n_theta=5, n_e=4, n_mu=4, n_phi=6, n_s=2)
    o, t, dt = compare_run(orc, gpu, p, 8)
    assert math.isclose(t.max_dt(0.5), o.max_dt(0.5), rel_tol=1e-12)
    No, Ng = o.totals(), t.totals()
    for a, b in zip(Ng, No):
        assert np.allclose(a, b, rtol=1e-12, atol=1e-300)


def test_fp64_2d_origin_and_ragged(orc, gpu):
    # origin pyramids, poles, odd mu count, angles not a multiple of 32
    p = W.random_2d(6, n_r=7, n_theta=3, n_e=3, n_mu=5, n_phi=7, n_s=1, r_min=0.0)
    compare_run(orc, gpu, p, 6)


def test_fp64_slab(orc, gpu):
    p = W.slab_diffusion(kappa_s=30.0, dz=0.02, z_max=0.3, n_mu=6)
    p.f0 = p.f0 * np.random.default_rng(8).uniform(0.5, 1.5, p.f0.shape)
    compare_run(orc, gpu, p, 20)


def test_fp64_config1_100_steps(orc, gpu):
    # the homogeneous-sphere configuration at its full size, 100 steps
    compare_run(orc, gpu, W.config1(), 100)


def test_fp64_single_group_single_phi(orc, gpu):
    p = W.random_column(9, n_r=6, n_e=1, n_mu=4, n_phi=1, n_s=1)
    compare_run(orc, gpu, p, 5)


def narrow_groups(p, ratio=1.06):
    """Regrid p's energy groups to a ratio close to 1: the Doppler and lapse
    shifts of the moving backgrounds then move content by several groups
    (about one row in nine of the remaps cannot be written with offsets of
    one), so the energy pass's general rows and its clamped edge rows with
    several terms run, not only the sub-group shifts."""
    ne = len(p.eps_edges) - 1
    p.eps_edges = np.geomspace(1.0, ratio ** ne, ne + 1)
    return p


@pytest.mark.parametrize("precision,tol", [("fp64", TOL64), ("mixed", TOL_MIXED)])
def test_shifts_of_several_groups(orc, gpu, precision, tol):
    p = narrow_groups(W.random_column(14, n_r=10, n_e=8, n_mu=6, n_phi=4, n_s=2))
    compare_run(orc, gpu, p, 10, precision=precision, tol=tol)


def test_fp64_2d_shifts_of_several_groups(orc, gpu):
    p = narrow_groups(W.random_2d(15, n_r=7, n_theta=4, n_e=6, n_mu=4, n_phi=6, n_s=1))
    compare_run(orc, gpu, p, 6)


# ---------------------------------------------------------------------------
# Gauss-Lobatto mu cells (Sec. 3.1): pole nodes mu = +-1, content moved into
# them spread evenly over their Phi cells
# ---------------------------------------------------------------------------
def lobatto(p):
    p.mu_quadrature = "lobatto"
    return p


@pytest.mark.parametrize("precision,tol", [("fp64", TOL64), ("mixed", TOL_MIXED)])
def test_lobatto_column_moving_gr(orc, gpu, precision, tol):
    p = lobatto(W.random_column(21, n_r=11, n_e=5, n_mu=6, n_phi=4, n_s=2))
    o, t, dt = compare_run(orc, gpu, p, 12, precision=precision, tol=tol)
    if precision == "fp64":
        for a, b in zip(t.moments(), o.moments()):
            assert rel_l1(a, b) <= 1e-11
        # the pole nodes' cells stay one value (every deposit spreads evenly)
        f = t.get_f().reshape(p.n_species, p.n_zone, p.n_eps, p.n_mu, p.n_phi)
        for j in (0, p.n_mu - 1):
            assert np.allclose(f[..., j, :], f[..., j, :1], rtol=1e-13, atol=0)


@pytest.mark.parametrize("precision,tol", [("fp64", TOL64), ("mixed", TOL_MIXED)])
def test_lobatto_2d(orc, gpu, precision, tol):
    p = lobatto(W.random_2d(22, n_r=9, n_theta=5, n_e=4, n_mu=5, n_phi=6, n_s=2))
    compare_run(orc, gpu, p, 8, precision=precision, tol=tol)


def test_lobatto_2d_origin_ragged(orc, gpu):
    p = lobatto(W.random_2d(23, n_r=7, n_theta=3, n_e=3, n_mu=7, n_phi=7, n_s=1, r_min=0.0))
    compare_run(orc, gpu, p, 6)


def test_lobatto_config1_100_steps(orc, gpu):
    compare_run(orc, gpu, lobatto(W.config1()), 100)


@pytest.mark.parametrize("precision,tol", [("fp64", TOL64), ("mixed", TOL_MIXED)])
def test_lobatto_config2(orc, gpu, precision, tol):
    compare_run(orc, gpu, lobatto(W.config2()), 10, precision=precision, tol=tol)


# ---------------------------------------------------------------------------
# Mixed precision path
# ---------------------------------------------------------------------------
def test_mixed_config1_100_steps(orc, gpu):
    compare_run(orc, gpu, W.config1(), 100, precision="mixed", tol=TOL_MIXED)


def test_mixed_column_moving(orc, gpu):
    p = W.random_column(11, n_r=10, n_e=5, n_mu=6, n_phi=4, n_s=2)
    compare_run(orc, gpu, p, 20, precision="mixed", tol=TOL_MIXED)


def test_mixed_2d(orc, gpu):
    p = W.random_2d(12, n_r=8, n_theta=5, n_e=4, n_mu=4, n_phi=6, n_s=2)
    compare_run(orc, gpu, p, 10, precision="mixed", tol=TOL_MIXED)


# ---------------------------------------------------------------------------
# Conservation, determinism, degenerate inputs, errors
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("mixed", 1e-6)])
def test_gpu_conservation_static(gpu, precision, tol):
    p = W.random_2d(13, n_r=8, n_theta=4, n_e=3, n_mu=4, n_phi=6, n_s=1)
    rng = np.random.default_rng(0)
    for bg in p.backgrounds:
        bg.v[:] = 0.0
        bg.alpha[:] = 1.0
        bg.phi[:] = 1.0
        bg.kappa_a[:] = 0.0
        bg.kappa_s[:] = rng.uniform(0, 3, bg.kappa_s.shape)
    t = gpu.Transport(p, precision)
    t.set_background(p.backgrounds[0])
    t.set_f(p.f0)
    N0, E0, _, _ = t.totals()
    dt = t.max_dt(0.5)
    for _ in range(30):
        t.step(dt)
    N, E, No, Eo = t.totals()
    assert np.allclose(N + No, N0, rtol=tol, atol=0)
    assert np.allclose(E + Eo, E0, rtol=tol, atol=0)


def test_gpu_deterministic(gpu):
    p = W.random_2d(14, n_r=8, n_theta=4, n_e=3, n_mu=4, n_phi=6, n_s=2)
    a, _ = gpu.run(p, "fp64", n_steps=4, dt=0.01)
    b, _ = gpu.run(p, "fp64", n_steps=4, dt=0.01)
    assert np.array_equal(a.get_f(), b.get_f())


def test_gpu_zero_state_stays_zero(gpu):
    p = W.random_column(15, n_r=6, n_e=3, n_mu=4, n_phi=4, n_s=1)
    for bg in p.backgrounds:
        bg.kappa_a[:] = 0.0
    p.f0[:] = 0.0
    t, _ = gpu.run(p, "fp64", n_steps=3, dt=0.01)
    assert not np.any(t.get_f())


def test_gpu_errors(gpu):
    p = W.random_column(16, n_r=4, n_e=2, n_mu=2, n_phi=2, n_s=1)
    t = gpu.Transport(p, "fp64")
    with pytest.raises(gpu.BtError) as e:
        t.step(0.1)                              # no background yet
    assert e.value.code == -6
    t.set_background(p.backgrounds[0])
    with pytest.raises(gpu.BtError) as e:
        t.step(-1.0)
    assert e.value.code == -3
    bad = p.backgrounds[0]
    bad.alpha = bad.alpha.copy()
    bad.alpha[1] = float("nan")
    with pytest.raises(gpu.BtError) as e:
        t.set_background(bad)
    assert e.value.code == -2
    q = W.random_column(16, n_r=4, n_e=3, n_mu=2, n_phi=2, n_s=1)
    q.eps_edges = np.array([1.0, 2.0, 3.0, 5.0])
    with pytest.raises(gpu.BtError) as e:
        gpu.Transport(q, "fp64")
    assert e.value.code == -1


# ---------------------------------------------------------------------------
# Full-size workloads: sampled zones against the oracle's subset step
# ---------------------------------------------------------------------------
def sampled_parity(orc, bt, prob, precision, tol, zones):
    o = orc.Oracle(prob)
    o.set_background(prob.backgrounds[0])
    o.set_f(prob.f0)
    dt = o.max_dt(prob.cfl)
    o.set_background(prob.backgrounds[1])
    ref = o.step_zones(dt, zones)[:, zones]
    t = bt.Transport(prob, precision)
    t.set_background(prob.backgrounds[0])
    t.set_f(prob.f0)
    assert math.isclose(t.max_dt(prob.cfl), dt, rel_tol=1e-12)
    t.set_background(prob.backgrounds[1])
    t.step(dt)
    got = t.get_f()[:, zones]
    e = rel_l1(got, ref)
    assert e <= tol, "sampled rel-L1 %.3e" % e


def _sample_zones(prob, n, seed):
    rng = np.random.default_rng(seed)
    z = set(rng.choice(prob.n_zone, n, replace=False).tolist())
    # boundaries and poles
    z |= {0, prob.n_r - 1, prob.n_zone - 1, prob.n_zone - prob.n_r}
    return sorted(z)


@pytest.mark.parametrize("precision,tol", [("fp64", TOL64), ("mixed", TOL_MIXED)])
def test_config3_sampled(orc, gpu, precision, tol):
    p = W.config3()
    sampled_parity(orc, gpu, p, precision, tol, _sample_zones(p, 24, 1))


@pytest.mark.parametrize("precision,tol", [("fp64", TOL64), ("mixed", TOL_MIXED)])
def test_config2_full(orc, gpu, precision, tol):
    # the moving-background diffusion column at its full size, 100 steps
    p = W.config2()
    compare_run(orc, gpu, p, 100, precision=precision, tol=tol)


@pytest.fixture(scope="module")
def config3_oracle_10(orc):
    p = W.config3()
    o, dt = orc.run(p, n_steps=10)
    return p, o, dt


@pytest.mark.slow
@pytest.mark.parametrize("precision,tol", [("fp64", TOL64), ("mixed", TOL_MIXED)])
def test_config3_ten_full_steps(config3_oracle_10, gpu, precision, tol):
    # the 2D core-collapse-like problem at its full size (256 x 64 zones,
    # 12 groups, 80 angles, 3 species), ten whole steps with the backgrounds
    # alternating (time remap every step); totals too
    p, o, dt = config3_oracle_10
    t, _ = gpu.run(p, precision, n_steps=10, dt=dt)
    fo = o.get_f()
    e = rel_l1(t.get_f(), fo)
    assert e <= tol, "rel-L1(f) = %.3e > %.1e" % (e, tol)
    # totals: FP64 to 1e-10; the mixed path stores f in float32 (its
    # number conservation is tested on its own, not against the oracle here)
    No, Ng = o.totals(), t.totals()
    for a, b in zip(Ng[:2], No[:2]):
        assert np.allclose(a, b, rtol=1e-10 if precision == "fp64" else 1e-6, atol=0), (a, b)
    # collision source terms: in these optically thick zones (kappa dt up to
    # 1e7) the increment is a small difference of nearly equal contents, so
    # its error is measured against the zones' number content per dt
    # (sum_i 4pi J_i / eps_i over dt), the size of the terms it is formed from
    J = o.jhk()[0]
    eps_c = o.grid()["eps_c"]
    content_rate = np.abs(4 * np.pi * J / eps_c[None, None, :]).sum(axis=2) / dt     # [s][zone]
    dNo, dNg = o.moments()[0], t.moments()[0]
    err = np.abs(dNg - dNo).sum() / content_rate.sum()
    assert err <= (1e-11 if precision == "fp64" else 1e-5), err


@pytest.mark.slow
def test_config5_largest_member_sampled(orc, gpu):
    # the largest problem of the batched workload: 512 x 128 zones, 20
    # groups, 128 angles (16 mu x 8 Phi), 6 species, face pass at 512
    # threads per CTA (five rows per list walk) and, in float32, at 384 (the
    # benchmark's shape: seven rows per walk, the grid fixed at compile
    # time), one step from the time remap on, sampled zones against the
    # oracle's subset step
    p = W.config5_problems()[2]
    zones = _sample_zones(p, 16, 3)
    o = orc.Oracle(p)
    o.set_background(p.backgrounds[0])
    o.set_f(p.f0)
    dt = o.max_dt(p.cfl)
    o.set_background(p.backgrounds[1])
    ref = o.step_zones(dt, zones)[:, zones]
    for precision, tol, nt in (("fp64", TOL64, 512), ("mixed", TOL_MIXED, 512), ("mixed", TOL_MIXED, 384)):
        t = gpu.Transport(p, precision)
        t.set_launch_shape(gpu.SHAPE_SPLIT | nt)
        t.set_background(p.backgrounds[0])
        t.set_f(p.f0)
        assert math.isclose(t.max_dt(p.cfl), dt, rel_tol=1e-12)
        t.set_background(p.backgrounds[1])
        t.step(dt)
        got = t.get_f()[:, zones]
        e = rel_l1(got, ref)
        assert e <= tol, "%s sampled rel-L1 %.3e" % (precision, e)
        del t


def test_gpu_size_limits(gpu):
    # more angles than the kernels hold, and rows too long for shared memory,
    # are refused at creation with an argument error (nothing is launched)
    p = W.random_column(17, n_r=4, n_e=2, n_mu=17, n_phi=16, n_s=1)   # 272 angles > 256
    with pytest.raises(gpu.BtError) as e:
        gpu.Transport(p, "fp64")
    assert e.value.code == -1
    q = W.random_column(18, n_r=4, n_e=64, n_mu=16, n_phi=16, n_s=1)  # 16384 bins per row
    with pytest.raises(gpu.BtError) as e:
        gpu.Transport(q, "fp64")
    assert e.value.code == -1 and "shared memory" in str(e.value)


def test_launch_shapes_cover_every_angle(orc, gpu):
    # 192 angles: a 128-thread CTA would leave angles without a thread, so
    # that shape is refused and the autotuner does not consider it
    p = W.random_column(19, n_r=6, n_e=3, n_mu=16, n_phi=12, n_s=1)
    t = gpu.Transport(p, "fp64")
    with pytest.raises(gpu.BtError) as e:
        t.set_launch_shape(128)
    assert e.value.code == -1
    t.set_launch_shape(256)
    t.set_background(p.backgrounds[0])
    t.set_f(p.f0)
    assert t.autotune(0.01) & 0xffff >= 192
    o, t2, dt = compare_run(orc, gpu, p, 4)


# ---------------------------------------------------------------------------
# Axisymmetric tests of Sec. 4.5 at oracle sizes: the 2D radiating sphere and
# the radiating disk's open face at theta = pi/2 (imposed inflow)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("precision,tol", [("fp64", TOL64), ("mixed", TOL_MIXED)])
def test_radiating_sphere_2d_parity(orc, gpu, precision, tol):
    p = W.radiating_sphere_2d(n_r=10, n_theta=6, n_mu=6, n_phi=6)
    compare_run(orc, gpu, p, 40, precision=precision, tol=tol)


@pytest.mark.parametrize("precision,tol", [("fp64", TOL64), ("mixed", TOL_MIXED)])
@pytest.mark.parametrize("shape", [256, 0x10000 | 256])
def test_radiating_disk_parity(orc, gpu, precision, tol, shape):
    p = W.radiating_disk(n_r=10, n_theta=5, n_mu=6, n_phi=6, r_min=0.2, r_max=2.0)
    o, dt = orc.run(p, n_steps=30)
    t = gpu.Transport(p, precision)
    t.set_launch_shape(shape)
    t.set_background(p.backgrounds[0])
    t.set_f(p.f0)
    assert math.isclose(t.max_dt(0.5), dt, rel_tol=1e-12)
    for _ in range(30):
        t.step(dt)
    fo = o.get_f()
    assert rel_l1(t.get_f(), fo) <= tol
    No, Ng = o.totals(), t.totals()
    for a, b in zip(Ng, No):
        assert np.allclose(a, b, rtol=1e-12 if precision == "fp64" else 1e-5, atol=0)


def test_open_face_needs_a_2d_grid(gpu):
    p = W.random_column(91, n_r=4, n_e=2, n_mu=2, n_phi=2, n_s=1)
    t = gpu.Transport(p, "fp64")
    with pytest.raises(gpu.BtError) as e:
        t.set_boundary(np.zeros((1, 4, 2)))
    assert e.value.code == -1
    q = W.random_column(92, n_r=4, n_e=2, n_mu=2, n_phi=2, n_s=1)
    q.theta_max = 1.0
    with pytest.raises(gpu.BtError) as e:
        gpu.Transport(q, "fp64")
    assert e.value.code == -1
