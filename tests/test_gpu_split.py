"""The split flux step (face pass + zone pass, every face computed once)
against the fused one and against the oracle.  The split form gathers each
zone's deposits in the fused form's order, so the two must agree bit for
bit in both precisions."""
import numpy as np
import pytest

from paper_2003_02845_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SPLIT = 0x10000


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2003_02845_gb300 import build, bt
    build.build()
    return bt


def _cases():
    sphere = W.homogeneous_sphere(n_r=13, n_e=3, n_mu=6, n_phi=4, dang=0.25)
    sphere.f0 = np.random.default_rng(3).uniform(0, 1, sphere.f0.shape)
    slab = W.slab_diffusion(kappa_s=30.0, dz=0.02, z_max=0.3, n_mu=6)
    slab.f0 = slab.f0 * np.random.default_rng(8).uniform(0.5, 1.5, slab.f0.shape)
    narrow = W.random_2d(15, n_r=7, n_theta=4, n_e=6, n_mu=4, n_phi=6, n_s=2)
    narrow.eps_edges = np.geomspace(1.0, 1.06 ** 6, 7)
    return {
        "column": W.random_column(1, n_r=11, n_e=5, n_mu=6, n_phi=4, n_s=2),
        "origin": sphere,
        "2d": W.random_2d(4, n_r=9, n_theta=5, n_e=4, n_mu=4, n_phi=6, n_s=2),
        "2d_origin_ragged": W.random_2d(6, n_r=7, n_theta=3, n_e=3, n_mu=5, n_phi=7, n_s=1, r_min=0.0),
        "slab": slab,
        # shifts of several energy groups (the energy pass's general rows)
        "2d_narrow_groups": narrow,
        # Gauss-Lobatto mu cells: pole nodes spread in both passes
        "2d_lobatto": _lob(W.random_2d(16, n_r=8, n_theta=5, n_e=4, n_mu=5, n_phi=6, n_s=2)),
        "origin_lobatto": _lob(W.random_2d(17, n_r=6, n_theta=4, n_e=3, n_mu=6, n_phi=7, n_s=1, r_min=0.0)),
    }


def _lob(p):
    p.mu_quadrature = "lobatto"
    return p


def _run(gpu, p, precision, shape, steps, dt):
    t = gpu.Transport(p, precision)
    t.set_launch_shape(shape)
    assert t.launch_shape == shape
    t.set_background(p.backgrounds[0])
    t.set_f(p.f0)
    for k in range(steps):
        if p.alternate and len(p.backgrounds) > 1:
            t.set_background(p.backgrounds[(k + 1) % 2])
        t.step(dt)
    return t


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["column", "origin", "2d", "2d_origin_ragged", "slab", "2d_narrow_groups",
                                  "2d_lobatto", "origin_lobatto"])
def test_split_equals_fused(gpu, case, precision):
    p = _cases()[case]
    a = _run(gpu, p, precision, 256, 6, 0.004)
    # (the 384-thread face pass exists in the mixed precision only)
    shapes = (SPLIT | 256, SPLIT | 512) if precision == "fp64" else (SPLIT | 256, SPLIT | 384, SPLIT | 512)
    for shape in shapes:
        b = _run(gpu, p, precision, shape, 6, 0.004)
        assert np.array_equal(a.get_f(), b.get_f())
        for x, y in zip(a.moments(), b.moments()):
            assert np.array_equal(x, y)
        for x, y in zip(a.totals(), b.totals()):
            assert np.array_equal(x, y)


def test_split_fp64_matches_oracle(orc, gpu):
    p = W.random_2d(5, n_r=9, n_theta=5, n_e=4, n_mu=4, n_phi=6, n_s=2)
    o, dt = orc.run(p, n_steps=8)
    t = _run(gpu, p, "fp64", SPLIT | 256, 8, dt)
    fo = o.get_f()
    assert np.abs(t.get_f() - fo).sum() / np.abs(fo).sum() <= 1e-12


def test_autotune_considers_split(gpu, tmp_path, monkeypatch):
    monkeypatch.setenv("BT_TUNE_CACHE", str(tmp_path / "tune.txt"))
    p = W.random_2d(7, n_r=12, n_theta=6, n_e=4, n_mu=4, n_phi=6, n_s=2)
    t = gpu.Transport(p, "mixed")
    t.set_background(p.backgrounds[0])
    t.set_f(p.f0)
    nt = t.autotune(0.01)
    assert nt in (128, 256, 512, SPLIT | 256, SPLIT | 512)
    t.step(0.01)   # the chosen shape runs


# The face and zone passes have instantiations for the benchmark
# configurations' grids (groups, mu cells and Phi cells fixed at compile
# time, float32; the zone pass's with paired loads).  On small spatial grids
# with those momentum grids, the specialised passes must give bit for bit
# what the generic fused kernel gives.
@pytest.mark.parametrize("n_e,n_mu,n_phi,shape", [(20, 16, 8, SPLIT | 512), (20, 16, 8, SPLIT | 384),
                                                  (12, 8, 10, SPLIT | 256), (8, 6, 8, SPLIT | 256)])
def test_specialised_grids_equal_fused(gpu, n_e, n_mu, n_phi, shape):
    # opacities scaled down: the fluxes and remaps, not the collision, decide f
    p = W.cc2d(12, 6, n_e, n_mu, n_phi, (1.0, 0.2), W.BASE_SEED + 90 + n_e, "spec_%d_%d_%d" % (n_e, n_mu, n_phi),
               opacity_scale=1e-4)
    t = gpu.Transport(p, "mixed")
    t.set_background(p.backgrounds[0])
    dt = t.max_dt(0.5)
    del t
    a = _run(gpu, p, "mixed", 256, 4, dt)
    b = _run(gpu, p, "mixed", shape, 4, dt)
    assert np.array_equal(a.get_f(), b.get_f())
    for x, y in zip(a.moments(), b.moments()):
        assert np.array_equal(x, y)


def test_split_384_is_mixed_only(gpu):
    p = W.cc2d(8, 4, 20, 16, 8, (1.0,), W.BASE_SEED + 95, "spec_fp64_384")
    t = gpu.Transport(p, "fp64")
    with pytest.raises(gpu.BtError):
        t.set_launch_shape(SPLIT | 384)
