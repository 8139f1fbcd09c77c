"""Physics of the axisymmetric tests of Sec. 4.5 at resolutions the oracle
cannot reach in a test run, on the GPU (whose parity with the oracle is
established at oracle sizes in test_gpu_parity.py):

- the homogeneous radiating sphere on the 2D grid (Sec. 4.5.1): every polar
  row against the analytic H/J and K/J of Sec. 4.1, and mirror symmetry
  about the equator;
- the radiating disk (Sec. 4.5.2): the steady mean intensity above an
  optically thick, geometrically thin disk against the integral of the
  equilibrium distribution over the disk's projected surface.

Angular resolution is 16 Gauss-Lobatto mu x 16 Phi cells (the kernels hold
at most 256 angles per location; the paper uses 17 x 32), so the bounds are
ours and looser than the paper's plots.
"""
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


def sphere_exact(r, R=1.0, ka=4.0, n=4000):
    """H/J and K/J of f(r, mu) = 1 - exp(-ka s(r, mu)) (Sec. 4.1), with s the
    path length through the sphere along the backward ray."""
    mu = np.linspace(-1.0, 1.0, n)
    b2 = r * r * (1 - mu * mu)
    inside = b2 < R * R
    root = np.sqrt(np.maximum(R * R - b2, 0.0))
    s = np.where(inside & (r * mu + root > 0), np.where(r < R, r * mu + root, 2 * root), 0.0)
    f = 1 - np.exp(-ka * s)
    trap = lambda y: float(np.sum(0.5 * (y[1:] + y[:-1]) * np.diff(mu)))
    return trap(mu * f) / trap(f), trap(mu * mu * f) / trap(f)


def disk_J(x, z, r0, r1):
    """Mean intensity (Sec. 4.5.2) at cylindrical radius x and height z of an
    isotropic f = 1 annulus r0 < r < r1 in the plane z = 0: the solid angle it
    subtends over 4 pi."""
    from scipy import integrate
    f = lambda ph, r: r * z / ((x - r * math.cos(ph)) ** 2 + z ** 2 + (r * math.sin(ph)) ** 2) ** 1.5
    v, _ = integrate.dblquad(f, r0, r1, 0.0, 2 * math.pi, epsabs=1e-10, epsrel=1e-8)
    return v / (4 * math.pi)


def test_radiating_sphere_2d_rows(gpu):
    p = W.radiating_sphere_2d(n_r=60, n_theta=16, n_mu=16, n_phi=16, tau=4.0)
    t = gpu.Transport(p, "fp64")
    t.set_background(p.backgrounds[0])
    t.set_f(p.f0)
    dt = t.max_dt(0.5)
    for _ in range(int(5.0 / dt)):
        t.step(dt)
    J, H, K = (x[0, :, 0].reshape(p.n_theta, p.n_r) for x in t.jhk())
    assert np.allclose(J, J[::-1], rtol=1e-12, atol=0)   # equatorial mirror symmetry
    rc = 0.5 * (p.r_edges[1:] + p.r_edges[:-1])
    m = (rc > 1.0) & (rc < 2.0)
    ex = np.array([sphere_exact(r) for r in rc[m]])
    for b in range(p.n_theta):
        assert np.sqrt(np.mean((H[b, m] / J[b, m] - ex[:, 0]) ** 2)) < 0.03
        assert np.sqrt(np.mean((K[b, m] / J[b, m] - ex[:, 1]) ** 2)) < 0.03


def test_radiating_disk_mean_intensity(gpu):
    p = W.radiating_disk(n_r=60, n_theta=16, n_mu=16, n_phi=16, r_min=0.1, r_max=3.0)
    t = gpu.Transport(p, "mixed")
    t.set_background(p.backgrounds[0])
    t.set_f(p.f0)
    dt = t.max_dt(0.5)
    for _ in range(int(5.0 / dt)):
        t.step(dt)
    J = t.jhk()[0][0, :, 0].reshape(p.n_theta, p.n_r)
    e_lo, e_hi = p.eps_edges
    J = J / (0.75 * (e_hi ** 4 - e_lo ** 4) / (e_hi ** 3 - e_lo ** 3) * (e_hi ** 3 - e_lo ** 3) / 3)
    rc = 0.5 * (p.r_edges[1:] + p.r_edges[:-1])
    th_e = np.linspace(0, 0.5 * np.pi, p.n_theta + 1)
    thc = 0.5 * (th_e[1:] + th_e[:-1])
    r1 = p.r_edges[np.nonzero(rc < 1.0)[0][-1] + 1]      # outer edge of the imposed disk
    errs = []
    # away from the polar axis (the paper's own artefact there covers the
    # three rows next to the pole) and from the disk surface
    for b in range(3, p.n_theta):
        for a in range(0, p.n_r, 2):
            x, z = rc[a] * math.sin(thc[b]), rc[a] * math.cos(thc[b])
            if z < 0.2 or rc[a] > 2.0:
                continue
            errs.append(J[b, a] / disk_J(x, z, p.r_edges[0], r1) - 1.0)
    errs = np.abs(np.array(errs))
    assert len(errs) > 100
    assert np.median(errs) < 0.10, np.median(errs)
    assert np.quantile(errs, 0.9) < 0.35, np.quantile(errs, 0.9)
