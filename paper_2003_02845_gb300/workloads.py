"""Seeded synthetic workloads for the discrete-ordinate transport step.

This module builds INPUTS only: grids, fluid backgrounds, opacities and
initial distributions, each from a fixed recipe and a numpy
``default_rng(seed)``.  It holds none of the transport method's arithmetic
(no group centres, no remap, no fluxes, no collision solve): both the CUDA
library and the CPU oracle consume what it returns, and each of them derives
every method quantity on its own.

The recipes stand in for the paper's test problems and its core-collapse
setting (Sec. 4); the paper uses no external dataset.  Units: c = 1, lengths
in cm (or code units for the dimensionless tests), energies in MeV,
velocities in units of c, opacities per unit length.

Opacities and equilibrium occupations are evaluated at the geometric mean of
each energy group's edges, ``sqrt(e_i e_{i+1})`` -- an input-recipe choice
that is independent of how either implementation places its group centres.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

G_CGS = 6.674e-8
C_CGS = 2.99792458e10
MSUN_CGS = 1.989e33

GEOM_SPHERICAL = 0
GEOM_SLAB = 1

NUE, NUEBAR, NUX = 0, 1, 2

BASE_SEED = 20240303


@dataclasses.dataclass
class Background:
    """Per-zone fluid/metric state plus per-(species, zone, group) opacities.

    Arrays are zone-major with zone = b * n_r + a (a radial, b polar).
    ``v`` holds (v_r, v_theta, v_phi) in the zone's local orthonormal triad.
    """
    rho: np.ndarray
    T: np.ndarray
    Ye: np.ndarray
    v: np.ndarray        # [n_zone, 3]
    alpha: np.ndarray    # [n_zone]
    phi: np.ndarray      # [n_zone] conformal factor
    shift: np.ndarray    # [n_zone, 3] (must be zero)
    kappa_a: np.ndarray  # [n_s, n_zone, n_e]
    kappa_s: np.ndarray  # [n_s, n_zone, n_e]
    f_eq: np.ndarray     # [n_s, n_zone, n_e]


@dataclasses.dataclass
class Problem:
    name: str
    geom: int
    r_edges: np.ndarray          # n_r + 1 (z edges for a slab)
    n_theta: int
    theta_periodic: bool         # True: 1D column (n_theta == 1)
    dtheta_column: float         # column only
    dphi: float                  # azimuthal wedge
    species_kind: List[int]
    eps_edges: np.ndarray        # n_e + 1
    n_mu: int
    n_phi: int
    backgrounds: List[Background]
    f0: np.ndarray               # [n_s, n_zone, n_e, n_mu * n_phi]
    cfl: float = 0.5
    n_steps: int = 100
    alternate: bool = False      # alternate backgrounds[0]/[1] every step
    mu_quadrature: str = "legendre"   # mu cells: "legendre" or "lobatto" (nodes at mu = +-1)
    theta_max: float = 0.0       # 2D polar range [0, theta_max] (0: pi); below pi the face at theta_max is open
    f_boundary: Optional[np.ndarray] = None   # [n_s, n_r, n_e] imposed on that face's incoming bins

    @property
    def n_r(self) -> int:
        return len(self.r_edges) - 1

    @property
    def n_zone(self) -> int:
        return self.n_r * self.n_theta

    @property
    def n_species(self) -> int:
        return len(self.species_kind)

    @property
    def n_eps(self) -> int:
        return len(self.eps_edges) - 1

    @property
    def n_ang(self) -> int:
        return self.n_mu * self.n_phi

    @property
    def n_bins(self) -> int:
        return self.n_species * self.n_zone * self.n_eps * self.n_ang


def _eps_mid(eps_edges: np.ndarray) -> np.ndarray:
    return np.sqrt(eps_edges[:-1] * eps_edges[1:])


def _fermi(eps: np.ndarray, T: np.ndarray) -> np.ndarray:
    x = np.clip(eps[None, :] / T[:, None], None, 700.0)
    return 1.0 / (np.exp(x) + 1.0)


def _flat_background(n_zone: int, n_s: int, n_e: int) -> Background:
    z = np.zeros(n_zone)
    return Background(
        rho=z.copy(), T=np.ones(n_zone), Ye=np.full(n_zone, 0.5),
        v=np.zeros((n_zone, 3)), alpha=np.ones(n_zone), phi=np.ones(n_zone),
        shift=np.zeros((n_zone, 3)),
        kappa_a=np.zeros((n_s, n_zone, n_e)), kappa_s=np.zeros((n_s, n_zone, n_e)),
        f_eq=np.zeros((n_s, n_zone, n_e)))


# ---------------------------------------------------------------------------
# Homogeneous radiating sphere (Sec. 4.1), 1D column
# ---------------------------------------------------------------------------
def homogeneous_sphere(n_r: int = 64, r_max: float = 2.0, radius: float = 1.0,
                       kappa: float = 4.0, n_e: int = 8, n_mu: int = 16,
                       n_phi: int = 4, dang: float = 0.125, n_steps: int = 100,
                       name: str = "sphere1d") -> Problem:
    """Static flat background; kappa_a = kappa inside r < radius, 0 outside;
    f_eq Fermi-Dirac with T = 1, zero chemical potential; f = 0 initially."""
    r_edges = np.linspace(0.0, r_max, n_r + 1)
    eps_edges = 2.0 ** (5.0 * np.arange(n_e + 1) / n_e)   # [1, 32]
    rc = 0.5 * (r_edges[:-1] + r_edges[1:])
    bg = _flat_background(n_r, 1, n_e)
    inside = rc < radius
    bg.kappa_a[0, inside, :] = kappa
    feq = 1.0 / (np.exp(_eps_mid(eps_edges)) + 1.0)
    bg.f_eq[0, :, :] = feq[None, :]
    f0 = np.zeros((1, n_r, n_e, n_mu * n_phi))
    return Problem(name, GEOM_SPHERICAL, r_edges, 1, True, dang, dang, [NUE],
                   eps_edges, n_mu, n_phi, [bg], f0, 0.5, n_steps)


def config1() -> Problem:
    """64 zones on [0, 2R], kappa_a = 4/R inside, 8 groups on [1, 32],
    16 Gauss-Legendre mu x 4 Phi, CFL 0.5, 100 steps, one species."""
    return homogeneous_sphere(name="config1_sphere1d_fp64")


# ---------------------------------------------------------------------------
# Core-collapse-like recipes (configs 2, 3, 5)
# ---------------------------------------------------------------------------
def _rho_powerlaw(r: np.ndarray) -> np.ndarray:
    return 1e14 * (r / 1e6) ** -3


def _temperature(rho: np.ndarray) -> np.ndarray:
    return 10.0 * (rho / 1e14) ** (1.0 / 3.0)


def _opacities(rho, T, eps_edges, scales):
    em = _eps_mid(eps_edges)
    ks1 = (rho / 1e10)[:, None] * (em[None, :] / 10.0) ** 2
    feq = _fermi(em, T)
    n_s = len(scales)
    ks = np.stack([s * ks1 for s in scales])
    ka = 0.1 * ks
    fe = np.broadcast_to(feq, (n_s,) + feq.shape).copy()
    return ka, ks, fe


def config2(seed: Optional[int] = None, n_r: int = 256, n_e: int = 16,
            n_mu: int = 32, n_phi: int = 4) -> Problem:
    """1D moving-background diffusion column: r log-spaced on [1e6, 1e8] cm,
    rho = 1e14 (r/1e6)^-3 with 1% lognormal noise, kappa_s = rho/1e10 (e/10)^2,
    kappa_a = 0.1 kappa_s, homologous v = 0.1 r/r_max, 16 groups on [2, 200]
    MeV, 32 mu x 4 Phi, a Gaussian pulse on f_eq; backgrounds alternate
    between v and 1.001 v so the time remap runs every step."""
    rng = np.random.default_rng(BASE_SEED + 1 if seed is None else seed)
    r_edges = np.geomspace(1e6, 1e8, n_r + 1)
    eps_edges = np.geomspace(2.0, 200.0, n_e + 1)
    rc = 0.5 * (r_edges[:-1] + r_edges[1:])
    rho = _rho_powerlaw(rc) * np.exp(0.01 * rng.standard_normal(n_r))
    T = _temperature(rho)
    ka, ks, fe = _opacities(rho, T, eps_edges, [1.0])
    bgs = []
    for vs in (1.0, 1.001):
        v = np.zeros((n_r, 3))
        v[:, 0] = 0.1 * rc / r_edges[-1] * vs
        bgs.append(Background(rho, T, np.full(n_r, 0.3), v, np.ones(n_r),
                              np.ones(n_r), np.zeros((n_r, 3)), ka, ks, fe))
    pulse = 1.0 + 0.2 * np.exp(-((np.log(rc) - np.log(1e7)) / 0.3) ** 2)
    f0 = (fe[0] * pulse[:, None])[None, :, :, None] * np.ones(n_mu * n_phi)
    dang = np.log(r_edges[-1] / r_edges[0]) / n_r
    return Problem("config2_diffusion1d", GEOM_SPHERICAL, r_edges, 1, True, dang, dang,
                   [NUE], eps_edges, n_mu, n_phi, bgs, f0, 0.5, 100, True)


def _legendre_perturbation(theta_c: np.ndarray, rng) -> np.ndarray:
    c = rng.standard_normal(5)
    c[0] = 0.0
    d = np.polynomial.legendre.legval(np.cos(theta_c), c)
    return d / np.max(np.abs(d))


def cc_background_pair(r_edges, n_theta, eps_edges, scales, seed,
                       r_shock=1.5e7, v_infall=0.2, m_core=1.4):
    """Two backgrounds B0, B1 of the 2D core-collapse-like recipe:
    power-law rho with a x10 drop outside r_shock, infall
    -v_infall (r/r_shock)^-1/2 outside, seeded l <= 4 perturbations of 5%,
    lapse sqrt(1 - 2GM(r)/rc^2) from an enclosed mass (m_core solar masses
    plus the angle-averaged density), conformal factor alpha^-1/2.
    B1 = B0 with v x 1.001 and the enclosed mass x 1.0005."""
    rng = np.random.default_rng(seed)
    n_r = len(r_edges) - 1
    rc = 0.5 * (r_edges[:-1] + r_edges[1:])
    th_e = np.linspace(0.0, np.pi, n_theta + 1)
    thc = 0.5 * (th_e[:-1] + th_e[1:])
    d1 = _legendre_perturbation(thc, rng)
    d2 = _legendre_perturbation(thc, rng)
    rho_r = _rho_powerlaw(rc) * np.where(rc > r_shock, 0.1, 1.0)
    vr_r = np.where(rc > r_shock, -v_infall * (rc / r_shock) ** -0.5, 0.0)
    # zone = b * n_r + a
    rho = (rho_r[None, :] * (1.0 + 0.05 * d1[:, None])).reshape(-1)
    vr = (vr_r[None, :] * (1.0 + 0.05 * d1[:, None])).reshape(-1)
    vth = (0.05 * np.abs(vr_r)[None, :] * d2[:, None]).reshape(-1)
    dr = np.diff(r_edges)
    m_enc = m_core * MSUN_CGS + np.cumsum(4.0 * np.pi * rc ** 2 * rho_r * dr)
    T = _temperature(rho)
    ka, ks, fe = _opacities(rho, T, eps_edges, scales)
    n_zone = n_r * n_theta
    out = []
    for vs, ms in ((1.0, 1.0), (1.001, 1.0005)):
        alpha_r = np.sqrt(1.0 - 2.0 * G_CGS * m_enc * ms / (rc * C_CGS ** 2))
        alpha = np.tile(alpha_r, n_theta)
        v = np.zeros((n_zone, 3))
        v[:, 0] = vr * vs
        v[:, 1] = vth * vs
        out.append(Background(rho, T, np.full(n_zone, 0.3), v, alpha, alpha ** -0.5,
                              np.zeros((n_zone, 3)), ka, ks, fe))
    return out


def cc2d(n_r=256, n_theta=64, n_e=12, n_mu=8, n_phi=10, scales=(1.0, 0.5, 0.2),
         seed=None, name="cc2d", n_steps=100, opacity_scale=1.0) -> Problem:
    seed = BASE_SEED + 2 if seed is None else seed
    r_edges = np.geomspace(1e6, 1e8, n_r + 1)
    eps_edges = np.geomspace(2.0, 200.0, n_e + 1)
    bgs = cc_background_pair(r_edges, n_theta, eps_edges, list(scales), seed)
    if opacity_scale != 1.0:
        for bg in bgs:
            bg.kappa_a = bg.kappa_a * opacity_scale
            bg.kappa_s = bg.kappa_s * opacity_scale
    fe = bgs[0].f_eq
    f0 = fe[:, :, :, None] * np.ones(n_mu * n_phi)
    kinds = [NUE, NUEBAR, NUX, NUX, NUX, NUX][:len(scales)]
    return Problem(name, GEOM_SPHERICAL, r_edges, n_theta, False, 0.0, np.pi / 64,
                   kinds, eps_edges, n_mu, n_phi, bgs, f0, 0.5, n_steps, True)


def config3(seed=None) -> Problem:
    """2D axisymmetric 256 r x 64 theta, 12 groups on [2, 200] MeV,
    80 angles (8 mu x 10 Phi), 3 species with opacity scales 1, 0.5, 0.2."""
    return cc2d(seed=seed, name="config3_cc2d_256x64x12x80x3")


def config3_transport(seed=None) -> Problem:
    """Config 3's grid, backgrounds and initial f with every opacity scaled by
    1e-6: at the Courant step (about 1e3 cm) kappa dt is below 1 in most
    zones and groups (it reaches 1e7 in the innermost core of config 3), so
    the step's result is decided by the fluxes and remaps rather than reset
    to f_eq by the collision -- the case an accuracy measure of the remap
    and fluxes needs."""
    return cc2d(seed=seed, name="config3_transport_cc2d_256x64x12x80x3_kappa1e-6", opacity_scale=1e-6)


def config5_problems(seed=None) -> List[Problem]:
    """Three uneven 2D problems x 6 species (batched step)."""
    base = BASE_SEED + 5 if seed is None else seed
    sc = (1.0, 0.5, 0.2, 0.2, 0.2, 0.2)
    return [cc2d(128, 32, 8, 6, 8, sc, base, "config5_p0_128x32x8x48x6"),
            cc2d(256, 64, 12, 8, 10, sc, base + 1, "config5_p1_256x64x12x80x6"),
            cc2d(512, 128, 20, 16, 8, sc, base + 2, "config5_p2_512x128x20x128x6")]


def config4_backgrounds(k: int, n_r=256, n_theta=64, n_e=12, scales=(1.0, 0.5, 0.2)):
    """Background pair k of the learned remap's data: k = 0..15 make the
    training set, k >= 16 are held out.  The config-3 recipe with its own
    perturbation seed, shock radius uniform in [1e7, 3e7] cm and infall
    amplitude uniform in [0.1, 0.3] (both drawn from the pair's seed)."""
    rng = np.random.default_rng(BASE_SEED + 400 + k)
    r_shock = rng.uniform(1e7, 3e7)
    v_infall = rng.uniform(0.1, 0.3)
    r_edges = np.geomspace(1e6, 1e8, n_r + 1)
    eps_edges = np.geomspace(2.0, 200.0, n_e + 1)
    return cc_background_pair(r_edges, n_theta, eps_edges, list(scales), BASE_SEED + 500 + k,
                              r_shock=r_shock, v_infall=v_infall)


def sur_rows(n_zone: int, n_ang: int, n: int, seed: int) -> np.ndarray:
    """n remap rows (zone, kind, source angle), uniform over zones, the 31
    remap kinds of a zone and the source angles: [n][3] int32."""
    rng = np.random.default_rng(seed)
    return np.stack([rng.integers(0, n_zone, n), rng.integers(0, 31, n), rng.integers(0, n_ang, n)],
                    axis=1).astype(np.int32)


# ---------------------------------------------------------------------------
# Small cases (oracle physics pins and GPU parity at oracle-friendly sizes)
# ---------------------------------------------------------------------------
def slab_diffusion(kappa_s=100.0, dz=0.01, z_max=1.0, t0=1.0, n_mu=8) -> Problem:
    """Planar diffusion wave (Sec. 4.3): kappa_s = 100, dz = 0.01, isotropic
    f initialised from E = sqrt(kappa_s/t0) exp(-3 kappa_s z^2 / 4 t0)."""
    n = int(round(2 * z_max / dz))
    z_edges = np.linspace(-z_max, z_max, n + 1)
    zc = 0.5 * (z_edges[:-1] + z_edges[1:])
    bg = _flat_background(n, 1, 1)
    bg.kappa_s[:] = kappa_s
    E = np.sqrt(kappa_s / t0) * np.exp(-3.0 * kappa_s * zc ** 2 / (4.0 * t0))
    f0 = E[None, :, None, None] * np.ones((1, n, 1, n_mu))
    return Problem("slab_diffusion", GEOM_SLAB, z_edges, 1, True, 0.0, 0.0, [NUE],
                   np.array([1.0, 2.0]), n_mu, 1, [bg], f0, 0.5, 0)


def random_column(seed: int, n_r=12, n_e=4, n_mu=4, n_phi=4, n_s=2,
                  r_min=1.0, r_max=3.0, moving=True, gr=True, kappa_scale=1.0,
                  name="random_column") -> Problem:
    """Small 1D column with seeded smooth random backgrounds (tests)."""
    rng = np.random.default_rng(seed)
    r_edges = np.geomspace(r_min, r_max, n_r + 1) if r_min > 0 else np.linspace(0, r_max, n_r + 1)
    eps_edges = np.geomspace(1.0, 1.0 * 1.6 ** n_e, n_e + 1)
    n_zone = n_r
    rc = 0.5 * (r_edges[:-1] + r_edges[1:])
    bgs = []
    base_v = 0.1 * rng.standard_normal(3) if moving else np.zeros(3)
    for k in range(2):
        v = np.zeros((n_zone, 3))
        if moving:
            ph = rng.uniform(0, 2 * np.pi)
            v[:, 0] = base_v[0] + 0.15 * np.sin(2 * rc + ph)
            v[:, 1] = 0.05 * np.cos(3 * rc + ph)
            v[:, 2] = 0.03 * np.sin(rc - ph)
        alpha = 1.0 - (0.2 / rc if gr else 0 * rc) * (1.0 + 0.01 * k)
        phi = alpha ** -0.5
        ka = kappa_scale * rng.uniform(0.0, 2.0, (n_s, n_zone, n_e))
        ks = kappa_scale * rng.uniform(0.0, 3.0, (n_s, n_zone, n_e))
        fe = rng.uniform(0.05, 0.9, (n_s, n_zone, n_e))
        bgs.append(Background(np.ones(n_zone), np.ones(n_zone), np.full(n_zone, 0.5), v, alpha, phi,
                              np.zeros((n_zone, 3)), ka, ks, fe))
    f0 = rng.uniform(0.0, 1.0, (n_s, n_zone, n_e, n_mu * n_phi))
    kinds = [NUE, NUEBAR, NUX, NUX, NUX, NUX][:n_s]
    dang = 0.3
    return Problem(name, GEOM_SPHERICAL, r_edges, 1, True, dang, dang, kinds, eps_edges,
                   n_mu, n_phi, bgs, f0, 0.5, 10, True)


def random_2d(seed: int, n_r=10, n_theta=6, n_e=4, n_mu=4, n_phi=6, n_s=2,
              r_min=1.0, r_max=4.0, dphi=0.2, name="random_2d") -> Problem:
    """Small 2D axisymmetric problem with seeded smooth random backgrounds."""
    rng = np.random.default_rng(seed)
    r_edges = np.geomspace(r_min, r_max, n_r + 1) if r_min > 0 else np.linspace(0, r_max, n_r + 1)
    eps_edges = np.geomspace(1.0, 1.0 * 1.5 ** n_e, n_e + 1)
    th_e = np.linspace(0, np.pi, n_theta + 1)
    thc = 0.5 * (th_e[:-1] + th_e[1:])
    rc = 0.5 * (r_edges[:-1] + r_edges[1:])
    R, TH = np.meshgrid(rc, thc)            # [b, a]
    R = R.reshape(-1)
    TH = TH.reshape(-1)
    n_zone = n_r * n_theta
    bgs = []
    ph = rng.uniform(0, 2 * np.pi, 4)
    for k in range(2):
        s = 1.0 + 0.002 * k
        v = np.zeros((n_zone, 3))
        v[:, 0] = s * (-0.2 * np.exp(-R / r_max) + 0.05 * np.cos(2 * TH + ph[0]))
        v[:, 1] = s * 0.08 * np.sin(TH) * np.cos(R + ph[1])
        v[:, 2] = s * 0.02 * np.sin(2 * TH) * np.sin(R + ph[2])
        alpha = 1.0 - 0.25 * r_min / R * (1.0 + 0.003 * k) * (1.0 + 0.05 * np.cos(TH + ph[3]))
        phi = alpha ** -0.5
        ka = rng.uniform(0.0, 2.0, (n_s, n_zone, n_e))
        ks = rng.uniform(0.0, 3.0, (n_s, n_zone, n_e))
        fe = rng.uniform(0.05, 0.9, (n_s, n_zone, n_e))
        bgs.append(Background(np.ones(n_zone), np.ones(n_zone), np.full(n_zone, 0.5), v,
                              alpha, phi, np.zeros((n_zone, 3)), ka, ks, fe))
    f0 = rng.uniform(0.0, 1.0, (n_s, n_zone, n_e, n_mu * n_phi))
    kinds = [NUE, NUEBAR, NUX, NUX, NUX, NUX][:n_s]
    return Problem(name, GEOM_SPHERICAL, r_edges, n_theta, False, 0.0, dphi, kinds, eps_edges,
                   n_mu, n_phi, bgs, f0, 0.5, 10, True)


def radiating_disk(n_r=40, n_theta=16, n_mu=8, n_phi=8, r_min=0.05, r_max=3.0, disk_radius=1.0, dphi=0.3,
                   quadrature="lobatto") -> Problem:
    """The radiating disk of Sec. 4.5.2: vacuum everywhere on 0 < theta < pi/2,
    and an isotropic f = 1 imposed on the incoming bins of the theta = pi/2
    face for the radial zones whose centre lies inside disk_radius (an
    optically thick, geometrically thin disk).  r log-spaced from r_min
    (a reflecting wall) to r_max; one group; f = 0 initially."""
    r_edges = np.geomspace(r_min, r_max, n_r + 1)
    rc = 0.5 * (r_edges[:-1] + r_edges[1:])
    bg = _flat_background(n_r * n_theta, 1, 1)
    fbc = np.zeros((1, n_r, 1))
    fbc[0, rc < disk_radius, 0] = 1.0
    f0 = np.zeros((1, n_r * n_theta, 1, n_mu * n_phi))
    p = Problem("radiating_disk", GEOM_SPHERICAL, r_edges, n_theta, False, 0.0, dphi, [NUE],
                np.array([1.0, 2.0]), n_mu, n_phi, [bg], f0, 0.5, 0)
    p.theta_max = 0.5 * np.pi
    p.f_boundary = fbc
    p.mu_quadrature = quadrature
    return p


def radiating_sphere_2d(n_r=24, n_theta=8, n_mu=12, n_phi=8, tau=4.0, r_min=0.2, r_max=2.0, dphi=0.3,
                        quadrature="lobatto") -> Problem:
    """The homogeneous radiating sphere (Sec. 4.1) on the 2D grid (Sec. 4.5.1):
    kappa_a = tau inside r < 1, vacuum outside, f_eq = 1, f = 0 initially;
    r log-spaced from r_min (a reflecting wall deep inside the sphere) to
    r_max, theta on [0, pi]."""
    r_edges = np.geomspace(r_min, r_max, n_r + 1)
    rc = 0.5 * (r_edges[:-1] + r_edges[1:])
    nz = n_r * n_theta
    bg = _flat_background(nz, 1, 1)
    bg.kappa_a[0, np.tile(rc, n_theta) < 1.0, 0] = tau
    bg.f_eq[0, :, 0] = 1.0
    f0 = np.zeros((1, nz, 1, n_mu * n_phi))
    p = Problem("radiating_sphere_2d", GEOM_SPHERICAL, r_edges, n_theta, False, 0.0, dphi, [NUE],
                np.array([1.0, 2.0]), n_mu, n_phi, [bg], f0, 0.5, 0)
    p.mu_quadrature = quadrature
    return p


def by_name(name: str) -> Problem:
    table = {"config1": config1, "config2": config2, "config3": config3, "config3_transport": config3_transport}
    return table[name]()
