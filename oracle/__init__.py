"""CPU oracle of the transport step (plain FP64 C, loaded through ctypes).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the
benchmark's CPU-baseline leg are the only callers.  The product library never
imports this package, and this package imports nothing from the product
library; both consume the seeded inputs of ``paper_2003_02845_gb300.workloads``.

``build()`` compiles ``bt_oracle.c`` with gcc (OpenMP) into ``oracle/_build``;
``set_threads`` picks the number of threads, which does not change results.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bt_oracle.c")
_OUT = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT, "liborc.so")
_lib = None

KICK_R, KICK_TH, KICK_PH, KICK_TIME, KICK_NONE = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    os.makedirs(_OUT, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        d, i, p = C.c_double, C.c_int, C.c_void_p
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        L.orc_create.restype = p
        L.orc_create.argtypes = [i, i, i, dp, i, d, d, i, ip, i, dp, i, i, d, i, d]
        L.orc_set_boundary.argtypes = [p, dp]
        L.orc_destroy.argtypes = [p]
        L.orc_set_background.argtypes = [p, dp, dp, dp, dp, dp, dp]
        L.orc_set_f.argtypes = [p, dp]
        L.orc_get_f.argtypes = [p, dp]
        L.orc_step.argtypes = [p, d]
        L.orc_step_zones.argtypes = [p, d, ip, dp]
        L.orc_max_dt.restype = d
        L.orc_max_dt.argtypes = [p, d]
        L.orc_zone_rates.argtypes = [p, dp]
        L.orc_lts_levels.restype = d
        L.orc_lts_levels.argtypes = [p, d, i, ip]
        L.orc_step_lts.restype = i
        L.orc_step_lts.argtypes = [p, d, ip, i]
        L.orc_moments.argtypes = [p, dp, dp, dp, dp]
        L.orc_totals.argtypes = [p, dp, dp, dp, dp]
        L.orc_jhk.argtypes = [p, dp, dp, dp]
        L.orc_grid.argtypes = [p, dp, dp, dp, dp, dp]
        L.orc_tir_count.restype = i
        L.orc_tir_count.argtypes = [p]
        L.orc_clamp_counts.argtypes = [p, C.POINTER(C.c_long)]
        L.orc_set_threads.argtypes = [i]
        L.orc_threads.restype = i
        L.orc_face_flux.restype = i
        L.orc_face_flux.argtypes = [p, i, i, d, dp, dp]
        L.orc_gauss_legendre.argtypes = [i, dp, dp]
        L.orc_gauss_lobatto.argtypes = [i, dp, dp]
        L.orc_triad.argtypes = [d, d, dp]
        L.orc_rotation.argtypes = [d, d, d, d, dp]
        L.orc_boost.argtypes = [dp, i, dp, dp]
        L.orc_kick.restype = i
        L.orc_kick.argtypes = [i, d, d, d, d, dp, dp]
        L.orc_chain.restype = i
        L.orc_chain.argtypes = [dp, d, d, dp, d, d, dp, i, dp, dp, dp, dp]
        L.orc_weights_eps.argtypes = [d, d, ip, dp]
        L.orc_weights_mu.argtypes = [d, i, dp, ip, dp]
        L.orc_weights_phi.argtypes = [d, i, ip, dp]
        L.orc_collision_row.argtypes = [i, dp, dp, d, d, dp, dp]
        L.orc_mc.restype = d
        L.orc_mc.argtypes = [d, d]
        for fn in ("orc_face_area_r", "orc_face_area_th"):
            getattr(L, fn).restype = d
            getattr(L, fn).argtypes = [d, d, d, d]
        L.orc_face_area_ph.restype = d
        L.orc_face_area_ph.argtypes = [d, d, d, d, d]
        L.orc_cell_volume.restype = d
        L.orc_cell_volume.argtypes = [d, d, d, d, d]
        L.orc_sur_sample.restype = i
        L.orc_sur_sample.argtypes = [p, i, i, i, dp, dp]
        L.orc_sur_samples.argtypes = [p, C.c_long, ip, dp, dp, ip]
        _lib = L
    return _lib


def set_threads(n: int):
    """Threads of the oracle's parallel loops (its results do not depend on
    the number)."""
    lib().orc_set_threads(int(n))


def threads() -> int:
    return int(lib().orc_threads())


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


# ---------------------------------------------------------------------------
# Unit-level entry points (pinned by tests/test_oracle_*.py)
# ---------------------------------------------------------------------------
def gauss_legendre(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    lib().orc_gauss_legendre(n, _dp(x), _dp(w))
    return x, w


def gauss_lobatto(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    lib().orc_gauss_lobatto(n, _dp(x), _dp(w))
    return x, w


def triad(th, ph):
    E = np.zeros(9)
    lib().orc_triad(th, ph, _dp(E))
    return E.reshape(3, 3)


def rotation(th_s, ph_s, th_d, ph_d):
    G = np.zeros(9)
    lib().orc_rotation(th_s, ph_s, th_d, ph_d, _dp(G))
    return G.reshape(3, 3)


def boost(v, sign, u):
    v = _f64(v)
    u = _f64(u)
    out = np.zeros(4)
    lib().orc_boost(_dp(v), sign, _dp(u), _dp(out))
    return out


def kick(axis, a_src, p_src, a_dst, p_dst, u):
    u = _f64(u)
    out = np.zeros(4)
    tir = lib().orc_kick(axis, a_src, p_src, a_dst, p_dst, _dp(u), _dp(out))
    return out, tir


def chain(v_src, a_src, p_src, v_dst, a_dst, p_dst, G, axis, n):
    v_src, v_dst, G, n = _f64(v_src), _f64(v_dst), _f64(np.asarray(G).reshape(-1)), _f64(n)
    rho, mu, ph = C.c_double(), C.c_double(), C.c_double()
    tir = lib().orc_chain(_dp(v_src), a_src, p_src, _dp(v_dst), a_dst, p_dst, _dp(G), axis,
                          _dp(n), C.byref(rho), C.byref(mu), C.byref(ph))
    return rho.value, mu.value, ph.value, tir


def weights_eps(rho, R):
    m = C.c_int()
    w = C.c_double()
    lib().orc_weights_eps(rho, R, C.byref(m), C.byref(w))
    return m.value, w.value


def weights_mu(mus, mu_nodes):
    mu_nodes = _f64(mu_nodes)
    j = C.c_int()
    w = C.c_double()
    lib().orc_weights_mu(mus, len(mu_nodes), _dp(mu_nodes), C.byref(j), C.byref(w))
    return j.value, w.value


def weights_phi(phis, n_phi):
    k = C.c_int()
    w = C.c_double()
    lib().orc_weights_phi(phis, n_phi, C.byref(k), C.byref(w))
    return k.value, w.value


def collision_row(r, tau, ka, ks, dOm):
    r, tau, dOm = _f64(r), _f64(tau), _f64(dOm)
    f = np.zeros_like(r)
    lib().orc_collision_row(len(r), _dp(r), _dp(tau), ka, ks, _dp(dOm), _dp(f))
    return f


def mc(a, b):
    return lib().orc_mc(a, b)


def face_area_r(r, th0, th1, dphi):
    return lib().orc_face_area_r(r, th0, th1, dphi)


def face_area_th(r0, r1, th, dphi):
    return lib().orc_face_area_th(r0, r1, th, dphi)


def face_area_ph(r0, r1, th0, th1, ph):
    return lib().orc_face_area_ph(r0, r1, th0, th1, ph)


def cell_volume(r0, r1, th0, th1, dphi):
    return lib().orc_cell_volume(r0, r1, th0, th1, dphi)


# ---------------------------------------------------------------------------
# Whole-problem oracle
# ---------------------------------------------------------------------------
class Oracle:
    """Plain FP64 transport state built from a ``workloads.Problem``."""

    def __init__(self, prob, phase_norm: float = 1.0):
        L = lib()
        self.prob = prob
        self._keep = []
        r_e = _f64(prob.r_edges)
        e_e = _f64(prob.eps_edges)
        kinds = np.ascontiguousarray(np.asarray(prob.species_kind, dtype=np.int32))
        self._keep += [r_e, e_e, kinds]
        self.h = L.orc_create(prob.geom, prob.n_r, prob.n_theta, _dp(r_e), int(prob.theta_periodic),
                              float(prob.dtheta_column), float(prob.dphi), prob.n_species, _ip(kinds),
                              prob.n_eps, _dp(e_e), prob.n_mu, prob.n_phi, phase_norm,
                              1 if getattr(prob, "mu_quadrature", "legendre") == "lobatto" else 0,
                              float(getattr(prob, "theta_max", 0.0) or 0.0))
        fbc = getattr(prob, "f_boundary", None)
        if fbc is not None:
            self.set_boundary(fbc)
        self.shape = (prob.n_species, prob.n_zone, prob.n_eps, prob.n_ang)

    def close(self):
        if self.h:
            lib().orc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_background(self, bg):
        a = [_f64(bg.v), _f64(bg.alpha), _f64(bg.phi), _f64(bg.kappa_a), _f64(bg.kappa_s), _f64(bg.f_eq)]
        lib().orc_set_background(self.h, *[_dp(x) for x in a])

    def set_boundary(self, fbc):
        """Distribution imposed on the incoming bins of the open face at
        theta_max, [species][radial zone][group]."""
        fbc = _f64(fbc).reshape(self.prob.n_species, self.prob.n_r, self.prob.n_eps)
        lib().orc_set_boundary(self.h, _dp(fbc))

    def set_f(self, f):
        f = _f64(f).reshape(self.shape)
        lib().orc_set_f(self.h, _dp(f))

    def get_f(self) -> np.ndarray:
        f = np.zeros(self.shape)
        lib().orc_get_f(self.h, _dp(f))
        return f

    def step(self, dt: float):
        lib().orc_step(self.h, float(dt))

    def step_zones(self, dt: float, zones) -> np.ndarray:
        sel = np.zeros(self.prob.n_zone, dtype=np.int32)
        sel[np.asarray(zones)] = 1
        out = np.zeros(self.shape)
        lib().orc_step_zones(self.h, float(dt), _ip(sel), _dp(out))
        return out

    def max_dt(self, cfl: float) -> float:
        return lib().orc_max_dt(self.h, float(cfl))

    def zone_rates(self) -> np.ndarray:
        """Per-zone Courant rate (max over bins of the outflow rate)."""
        out = np.zeros(self.prob.n_zone)
        lib().orc_zone_rates(self.h, _dp(out))
        return out

    def lts_levels(self, cfl: float, max_levels: int):
        """(dt0, levels [zone]) of the local time stepping (reading R-19)."""
        lev = np.zeros(self.prob.n_zone, dtype=np.int32)
        dt0 = lib().orc_lts_levels(self.h, float(cfl), int(max_levels), _ip(lev))
        return dt0, lev

    def step_lts(self, dt0: float, levels, n_levels: int):
        """One local-time-stepping macro step of dt0 2^(n_levels-1): zone z
        steps with dt0 2^levels[z]."""
        lev = np.ascontiguousarray(np.asarray(levels, dtype=np.int32))
        if lib().orc_step_lts(self.h, float(dt0), _ip(lev), int(n_levels)) != 0:
            raise ValueError("levels out of range")

    def moments(self):
        S, Z = self.prob.n_species, self.prob.n_zone
        dN, dE, dP, q = np.zeros((S, Z)), np.zeros((S, Z)), np.zeros((S, Z, 3)), np.zeros(Z)
        lib().orc_moments(self.h, _dp(dN), _dp(dE), _dp(dP), _dp(q))
        return dN, dE, dP, q

    def totals(self):
        S = self.prob.n_species
        N, E, No, Eo = np.zeros(S), np.zeros(S), np.zeros(S), np.zeros(S)
        lib().orc_totals(self.h, _dp(N), _dp(E), _dp(No), _dp(Eo))
        return N, E, No, Eo

    def jhk(self):
        sh = (self.prob.n_species, self.prob.n_zone, self.prob.n_eps)
        J, H, K = np.zeros(sh), np.zeros(sh), np.zeros(sh)
        lib().orc_jhk(self.h, _dp(J), _dp(H), _dp(K))
        return J, H, K

    def grid(self):
        p = self.prob
        ec, dg, mu, dmu, vol = np.zeros(p.n_eps), np.zeros(p.n_eps), np.zeros(p.n_mu), np.zeros(p.n_mu), np.zeros(p.n_zone)
        lib().orc_grid(self.h, _dp(ec), _dp(dg), _dp(mu), _dp(dmu), _dp(vol))
        return dict(eps_c=ec, dgam=dg, mu=mu, dmu=dmu, vol=vol)

    def tir_count(self) -> int:
        return lib().orc_tir_count(self.h)

    def clamp_counts(self):
        """(energy, mu) clamps of the remaps so far: deposits whose energy
        target lay past the end groups, source bins whose mu target lay past
        the outermost node (reading R-7)."""
        c = (C.c_long * 2)()
        lib().orc_clamp_counts(self.h, c)
        return int(c[0]), int(c[1])

    def face_flux(self, q: int, s: int, dt: float):
        """Flux content [group][angle] of face q of the step's face list for
        species s over dt, from the current f, and the face area."""
        out = np.zeros((self.prob.n_eps, self.prob.n_ang))
        area = C.c_double()
        if not lib().orc_face_flux(self.h, int(q), int(s), float(dt), _dp(out), C.byref(area)):
            raise IndexError("face %d" % q)
        return out, area.value

    def sur_samples(self, idx):
        """Learned-remap rows idx [n][3] = (zone, kind, source angle):
        features [n][16], exact targets [n][27], validity [n] (see
        orc_sur_sample)."""
        idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int32).reshape(-1, 3))
        n = len(idx)
        X, Y = np.zeros((n, 16)), np.zeros((n, 27))
        v = np.zeros(n, dtype=np.int32)
        lib().orc_sur_samples(self.h, n, _ip(idx), _dp(X), _dp(Y), _ip(v))
        return X, Y, v


def run(prob, n_steps=None, dt=None, cfl=None):
    """Run a problem through the oracle: background 0 (alternating with 1 if
    prob.alternate), f0, n_steps steps at dt (default: cfl * Courant limit of
    background 0).  Returns (oracle, dt)."""
    o = Oracle(prob)
    o.set_background(prob.backgrounds[0])
    o.set_f(prob.f0)
    if dt is None:
        dt = o.max_dt(prob.cfl if cfl is None else cfl)
    n = prob.n_steps if n_steps is None else n_steps
    for k in range(n):
        if prob.alternate and len(prob.backgrounds) > 1:
            o.set_background(prob.backgrounds[(k + 1) % 2])
        o.step(dt)
    return o, dt
