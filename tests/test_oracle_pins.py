"""Pins of oracle parts that the transport pins do not reach: the collision
source terms of Eq. hydrosource (scale, energy weight, momentum direction and
the lepton-number sign), the clamped energy edges of the remap (reading R-7)
and the diffusion-limit identity of the Lax-Wendroff interface state
(Appendix A).  Each is checked against a value derived here by another route
(a closed form of the implicit solve on inputs that make the advection
vanish, or a moment identity), not by re-running the oracle's formula.  No GPU.
"""
import math

import numpy as np
import pytest

from paper_2003_02845_gb300 import workloads as W


def _uniform_slab(n_z=8, n_e=3, n_mu=4, n_phi=4, ka=2.0, ks=3.0, feq=(0.2, 0.5, 0.7), kinds=(W.NUE,)):
    """A slab of identical zones at rest: every interior face carries the
    same flux, so an interior zone's advective change is exactly zero and its
    step is the local implicit solve alone (Sec. 3.5)."""
    n_s = len(kinds)
    z_edges = np.linspace(0.0, 0.1 * n_z, n_z + 1)
    eps_edges = np.geomspace(1.0, 1.5 ** n_e, n_e + 1)
    bg = W._flat_background(n_z, n_s, n_e)
    bg.kappa_a[:] = ka
    bg.kappa_s[:] = ks
    bg.f_eq[:] = np.asarray(feq)[None, None, :]
    f0 = np.zeros((n_s, n_z, n_e, n_mu * n_phi))
    return W.Problem("uniform_slab", W.GEOM_SLAB, z_edges, 1, True, 0.0, 0.0, list(kinds), eps_edges,
                     n_mu, n_phi, [bg], f0, 0.5, 1)


def _step_once(orc, p, phase_norm=1.0):
    o = orc.Oracle(p, phase_norm=phase_norm)
    o.set_background(p.backgrounds[0])
    o.set_f(p.f0)
    dt = o.max_dt(0.5)
    o.step(dt)
    return o, dt


def test_moments_isotropic_closed_form(orc):
    # isotropic f_i in every zone: scattering leaves it isotropic, so the
    # implicit solve gives f' = (f + dt ka feq) / (1 + ka dt) per group, and
    # the number and energy gains per unit volume and time are
    #   dN = 4pi sum_i dGamma_i ka (feq_i - f_i) / (1 + ka dt),  dE with eps_i
    # (the sum of dOmega over the sphere is 4pi); the momentum gain vanishes.
    ka, feq = 2.0, np.array([0.2, 0.5, 0.7])
    p = _uniform_slab(ka=ka, feq=feq)
    fi = np.array([0.9, 0.1, 0.4])
    p.f0[:] = fi[None, None, :, None]
    o, dt = _step_once(orc, p)
    g = o.grid()
    dN, dE, dP, _ = o.moments()
    rate = 4 * math.pi * g["dgam"] * ka * (feq - fi) / (1 + ka * dt)
    for z in range(2, p.n_r - 2):   # untouched by the open ends in one step
        assert math.isclose(dN[0, z], rate.sum(), rel_tol=1e-12)
        assert math.isclose(dE[0, z], (rate * g["eps_c"]).sum(), rel_tol=1e-12)
        assert np.all(np.abs(dP[0, z]) <= 1e-12 * abs(dE[0, z]))
    f = o.get_f()
    ref = (fi + dt * ka * feq) / (1 + ka * dt)
    assert np.allclose(f[0, 2:-2], ref[None, :, None], rtol=1e-13, atol=0)


def test_moments_beam_direction(orc):
    # a beam in the outermost mu node (all Phi cells), pure absorption with
    # f_eq = 0: each bin decays as f / (1 + ka dt) on its own.  The momentum
    # the neutrinos lose is along the beam: dP = mu_top dE in the stepping
    # direction (component 0), nothing across it, and negative.
    ka = 5.0
    p = _uniform_slab(ka=ka, ks=0.0, feq=(0.0, 0.0, 0.0), n_mu=6, n_phi=4)
    beam = np.zeros(p.n_ang)
    beam[(p.n_mu - 1) * p.n_phi:] = 1.0
    amp = np.array([0.3, 0.6, 0.2])
    p.f0[:] = amp[None, None, :, None] * beam[None, None, None, :]
    o, dt = _step_once(orc, p)
    g = o.grid()
    mu_top, dmu_top = g["mu"][-1], g["dmu"][-1]
    dN, dE, dP, _ = o.moments()
    # number lost per unit volume and time: the top node's solid angle
    # (dmu_top 2pi) times sum_i dGamma_i f_i ka / (1 + ka dt)
    loss = 2 * math.pi * dmu_top * g["dgam"] * amp * ka / (1 + ka * dt)
    for z in range(2, p.n_r - 2):
        assert math.isclose(dN[0, z], -loss.sum(), rel_tol=1e-12)
        assert math.isclose(dE[0, z], -(loss * g["eps_c"]).sum(), rel_tol=1e-12)
        assert dP[0, z, 0] < 0
        assert math.isclose(dP[0, z, 0], mu_top * dE[0, z], rel_tol=1e-12)
        assert abs(dP[0, z, 1]) <= 1e-12 * abs(dP[0, z, 0])
        assert abs(dP[0, z, 2]) <= 1e-12 * abs(dP[0, z, 0])


@pytest.mark.parametrize("kind,sign", [(W.NUE, -1.0), (W.NUEBAR, +1.0), (W.NUX, 0.0)])
def test_lepton_source_sign(orc, kind, sign):
    # Eq. hydrosource: Q_Ye = -(1/h^3) (integral of C_nue - C_nuebar).  An
    # emitter (f = 0, f_eq > 0) of electron neutrinos only takes electron
    # fraction from the fluid (Q_Ye < 0), one of electron antineutrinos
    # gives it (Q_Ye > 0), heavy-lepton neutrinos leave it alone; the 1/h^3
    # factor is phase_norm.
    p = _uniform_slab(ka=1.5, ks=0.0, kinds=(kind,))
    o, dt = _step_once(orc, p, phase_norm=2.5)
    dN, _, _, qye = o.moments()
    for z in range(2, p.n_r - 2):
        assert dN[0, z] > 0
        assert math.isclose(qye[z], sign * 2.5 * dN[0, z], rel_tol=1e-13, abs_tol=0.0)


def test_lepton_source_of_mixed_species(orc):
    # nue and nuebar together: Q_Ye = -(dN_nue - dN_nuebar) phase_norm, each
    # species' dN from its own closed form
    p = _uniform_slab(ka=1.5, ks=0.5, kinds=(W.NUE, W.NUEBAR, W.NUX))
    fi = np.array([[0.1, 0.1, 0.1], [0.6, 0.9, 0.95], [0.0, 0.0, 0.0]])
    p.f0[:] = fi[:, None, :, None]
    o, dt = _step_once(orc, p, phase_norm=0.75)
    g = o.grid()
    feq = np.array([0.2, 0.5, 0.7])
    dN, _, _, qye = o.moments()
    rate = [(4 * math.pi * g["dgam"] * 1.5 * (feq - fi[s]) / (1 + 1.5 * dt)).sum() for s in range(3)]
    for z in range(2, p.n_r - 2):
        assert math.isclose(qye[z], -0.75 * (rate[0] - rate[1]), rel_tol=1e-12)


def test_energy_edge_clamp_keeps_number(orc):
    # [R-7] content in the first and last groups, moved by boosts of 0.3c
    # that alternate in direction every step: many energy targets fall past
    # the end groups.  They must pile into the end group (number kept), not
    # vanish: with no absorption, content + cumulative outflow is conserved.
    p = W.random_column(61, n_r=8, n_e=5, n_mu=6, n_phi=4, n_s=1, moving=False, gr=False)
    for k, bg in enumerate(p.backgrounds):
        bg.v[:, 0] = 0.3 if k == 0 else -0.3
        bg.v[:, 1] = 0.1
        bg.kappa_a[:] = 0.0
    p.f0[:] = 0.0
    rng = np.random.default_rng(5)
    p.f0[:, :, 0, :] = rng.uniform(0.2, 1.0, p.f0[:, :, 0, :].shape)
    p.f0[:, :, -1, :] = rng.uniform(0.2, 1.0, p.f0[:, :, -1, :].shape)
    o = orc.Oracle(p)
    o.set_background(p.backgrounds[0])
    o.set_f(p.f0)
    N0 = o.totals()[0][0]
    dt = 0.5 * o.max_dt(0.5)
    for k in range(6):
        o.set_background(p.backgrounds[(k + 1) % 2])
        o.step(dt)
        N, _, No, _ = o.totals()
        assert math.isclose(N[0] + No[0], N0, rel_tol=1e-13)
    n_e_clamp, _ = o.clamp_counts()
    assert n_e_clamp > 1000


def test_mu_edge_clamp_counted(orc):
    # [R-7] a Gauss-Legendre grid has no node at mu = +-1: a boost takes
    # some targets past the outermost node, where all their weight goes to
    # that node.  The count is the diagnostic the remap keeps for it.
    p = W.random_column(62, n_r=6, n_e=3, n_mu=4, n_phi=4, n_s=1, moving=True, gr=False)
    o, _ = orc.run(p, n_steps=2)
    assert o.clamp_counts()[1] > 0


def test_appendix_diffusion_identity(orc):
    # Appendix A: at an interface between isotropic cells i, i+1 of a slab,
    # the Lax-Wendroff half step with the implicit collision at dt/2 gives,
    # after multiplying by mu and summing over directions,
    #   (K_{i+1} - K_i)/dz = -(ka + ks + 2/dt) H_{i+1/2},
    # which tends to the diffusion law -(ka + ks) H for dt (ka + ks)/2 >> 1.
    # H is read off the face's flux (slab at rest: u^0 = 1, normal velocity
    # mu, phi = 1): sum_b F_b = dt dA dGamma 4pi H.  With kappa dz = 1000 the
    # flux-switch weight exp(-kappa dz) is 0, so the interface state is the
    # Lax-Wendroff one.
    n_z, dz, ks, ka = 6, 0.01, 8e4, 2e4
    z_edges = np.arange(n_z + 1) * dz
    bg = W._flat_background(n_z, 1, 1)
    bg.kappa_s[:] = ks
    bg.kappa_a[:] = ka
    bg.f_eq[:] = 0.4
    J = np.array([1.0, 1.3, 0.7, 2.0, 1.1, 0.5])
    n_mu = 8
    f0 = J[None, :, None, None] * np.ones((1, n_z, 1, n_mu))
    p = W.Problem("slab_identity", W.GEOM_SLAB, z_edges, 1, True, 0.0, 0.0, [W.NUE],
                  np.array([1.0, 2.0]), n_mu, 1, [bg], f0, 0.5, 0)
    o = orc.Oracle(p)
    o.set_background(bg)
    o.set_f(f0)
    dt = o.max_dt(0.5)
    g = o.grid()
    K = J / 3.0          # (1/4pi) sum dOmega mu^2 J for an isotropic cell
    for q in range(1, n_z):   # interior faces: face q lies between zones q-1 and q
        flux, area = o.face_flux(q, 0, dt)
        H = flux.sum() / (dt * area * g["dgam"][0] * 4 * math.pi)
        lhs = (K[q] - K[q - 1]) / dz
        assert math.isclose(lhs, -(ka + ks + 2.0 / dt) * H, rel_tol=1e-9)
        assert math.isclose(lhs, -(ka + ks) * H, rel_tol=2.0 / (dt * (ka + ks)) * 1.01)


def test_oracle_threads_do_not_change_results(orc):
    # the parallel face blocks are summed in face-list order: one thread and
    # many give the same bits (f, moments, totals, time remap included)
    p = W.random_2d(63, n_r=7, n_theta=5, n_e=3, n_mu=4, n_phi=6, n_s=2)
    out = []
    n0 = orc.threads()
    try:
        for n in (1, 3, max(n0, 2)):
            orc.set_threads(n)
            o, _ = orc.run(p, n_steps=3)
            out.append((o.get_f(), o.moments(), o.totals()))
    finally:
        orc.set_threads(n0)
    for f, m, t in out[1:]:
        assert np.array_equal(f, out[0][0])
        for a, b in zip(m, out[0][1]):
            assert np.array_equal(a, b)
        for a, b in zip(t, out[0][2]):
            assert np.array_equal(a, b)
