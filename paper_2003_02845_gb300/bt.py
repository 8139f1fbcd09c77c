"""Python binding of the C ABI in include/bt.h (argument marshalling only).

Every step of the transport update runs in the CUDA kernels of
``_build/libbt.so``; this module only converts arguments.  PyTorch provides
the device workspace and the stream.  If the library is missing the import
of ``lib()`` raises: there is no CPU path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

BT_OK = 0
BT_GEOM_SPHERICAL, BT_GEOM_SLAB = 0, 1
BT_FP64, BT_MIXED = 0, 1
BT_MEM_HOST, BT_MEM_DEVICE = 0, 1
BT_GAUSS_LEGENDRE, BT_GAUSS_LOBATTO = 0, 1
SHAPE_SPLIT = 0x10000   # launch-shape flag of the split flux step

_lib = None


class BtConfig(C.Structure):
    _fields_ = [
        ("geom", C.c_int32), ("n_r", C.c_int32), ("n_theta", C.c_int32),
        ("r_edges", C.POINTER(C.c_double)),
        ("theta_periodic", C.c_int32), ("dtheta_column", C.c_double), ("dphi_wedge", C.c_double),
        ("n_species", C.c_int32), ("species_kind", C.POINTER(C.c_int32)),
        ("n_eps", C.c_int32), ("eps_edges", C.POINTER(C.c_double)),
        ("n_mu", C.c_int32), ("n_phi", C.c_int32), ("precision", C.c_int32),
        ("phase_norm", C.c_double), ("stream", C.c_void_p),
        ("mu_quadrature", C.c_int32), ("theta_max", C.c_double),
    ]


class BtTrainCfg(C.Structure):
    _fields_ = [("epochs", C.c_int32), ("batch", C.c_int32), ("lr", C.c_float), ("lr_final", C.c_float),
                ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float)]


SUR_NIN, SUR_NOUT, SUR_NPARAM = 16, 27, 11195


class BtError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("bt error %d: %s" % (code, msg))
        self.code = code


def lib():
    """Load libbt.so (built in-tree by ``build.build()``)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError("CUDA transport library not built: %s (run __graft_entry__.build())" % path)
        L = C.CDLL(path)
        vp, dp, i32 = C.c_void_p, C.c_void_p, C.c_int
        L.bt_last_error.restype = C.c_char_p
        L.bt_workspace_bytes.restype = C.c_size_t
        L.bt_workspace_bytes.argtypes = [C.POINTER(BtConfig)]
        L.bt_create.argtypes = [C.POINTER(BtConfig), vp, C.POINTER(vp)]
        L.bt_destroy.argtypes = [vp]
        L.bt_set_background.argtypes = [vp, i32] + [dp] * 10
        L.bt_set_f.argtypes = [vp, i32, vp]
        L.bt_set_boundary.argtypes = [vp, i32, vp]
        L.bt_set_levels.argtypes = [vp, vp, i32]
        L.bt_lts_levels.argtypes = [vp, C.c_double, i32, C.POINTER(C.c_double), vp]
        L.bt_n_levels.argtypes = [vp]
        L.bt_step_lts.argtypes = [vp, C.c_double]
        L.bt_get_f.argtypes = [vp, i32, vp]
        L.bt_max_dt.argtypes = [vp, C.c_double, C.POINTER(C.c_double)]
        L.bt_step.argtypes = [vp, C.c_double]
        L.bt_moments.argtypes = [vp, i32, dp, dp, dp, dp]
        L.bt_totals.argtypes = [vp, dp, dp, dp, dp]
        L.bt_jhk.argtypes = [vp, i32, dp, dp, dp]
        L.bt_launch_count.restype = C.c_int64
        L.bt_launch_count.argtypes = [vp]
        L.bt_weighted_totals_noalloc.argtypes = [vp, i32, i32, i32, i32, i32, vp, vp, vp, vp]
        L.bt_autotune.argtypes = [vp, C.c_double, C.POINTER(C.c_int)]
        L.bt_launch_shape.argtypes = [vp, C.POINTER(C.c_int)]
        L.bt_set_launch_shape.argtypes = [vp, i32]
        L.bt_batch_create.argtypes = [C.POINTER(BtConfig), i32, vp, C.POINTER(vp)]
        L.bt_batch_member.argtypes = [vp, i32, C.POINTER(vp)]
        L.bt_batch_step.argtypes = [vp, C.POINTER(C.c_double)]
        L.bt_batch_launch_count.restype = C.c_int64
        L.bt_batch_launch_count.argtypes = [vp]
        L.bt_batch_graph_launches.restype = C.c_int64
        L.bt_batch_graph_launches.argtypes = [vp]
        L.bt_batch_destroy.argtypes = [vp]
        L.bt_profile.argtypes = [vp, i32]
        L.bt_profile_read.argtypes = [vp, i32, C.POINTER(C.c_double), C.POINTER(C.c_int64)]
        L.bt_peak_fma.argtypes = [i32, C.POINTER(C.c_double), vp]
        L.bt_sur_samples.argtypes = [vp, vp, C.c_int64, vp, vp, vp]
        L.bt_set_surrogate.argtypes = [vp, vp, C.c_double]
        L.bt_sur_stats.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        L.bt_sur_create.argtypes = [vp, C.POINTER(vp)]
        L.bt_sur_destroy.argtypes = [vp]
        L.bt_sur_set_params.argtypes = [vp, i32, vp]
        L.bt_sur_get_params.argtypes = [vp, i32, vp]
        L.bt_sur_fit_normalizer.argtypes = [vp, vp, C.c_int64]
        L.bt_sur_forward.argtypes = [vp, vp, C.c_int64, vp]
        L.bt_sur_grad.argtypes = [vp, vp, vp, C.c_int64, vp, vp]
        L.bt_sur_train.argtypes = [vp, vp, vp, C.c_int64, C.POINTER(BtTrainCfg), vp]
        _lib = L
    return _lib


def _check(rc):
    if rc != BT_OK:
        raise BtError(rc, lib().bt_last_error().decode())


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()          # torch tensor


def _host64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def make_config(prob, precision: str, stream_handle: int, phase_norm: float = 1.0, keep=None):
    """bt_config for a workloads.Problem; host arrays are appended to `keep`."""
    r = _host64(prob.r_edges)
    e = _host64(prob.eps_edges)
    k = np.ascontiguousarray(np.asarray(prob.species_kind, dtype=np.int32))
    if keep is not None:
        keep += [r, e, k]
    cfg = BtConfig()
    cfg.geom = prob.geom
    cfg.n_r = prob.n_r
    cfg.n_theta = prob.n_theta
    cfg.r_edges = r.ctypes.data_as(C.POINTER(C.c_double))
    cfg.theta_periodic = int(prob.theta_periodic)
    cfg.dtheta_column = float(prob.dtheta_column)
    cfg.dphi_wedge = float(prob.dphi)
    cfg.n_species = prob.n_species
    cfg.species_kind = k.ctypes.data_as(C.POINTER(C.c_int32))
    cfg.n_eps = prob.n_eps
    cfg.eps_edges = e.ctypes.data_as(C.POINTER(C.c_double))
    cfg.n_mu = prob.n_mu
    cfg.n_phi = prob.n_phi
    cfg.precision = BT_MIXED if precision == "mixed" else BT_FP64
    cfg.phase_norm = phase_norm
    cfg.stream = stream_handle
    cfg.mu_quadrature = BT_GAUSS_LOBATTO if getattr(prob, "mu_quadrature", "legendre") == "lobatto" \
        else BT_GAUSS_LEGENDRE
    cfg.theta_max = float(getattr(prob, "theta_max", 0.0) or 0.0)
    return cfg


class Transport:
    """One transport problem on the current CUDA device.

    prob: a ``workloads.Problem`` (geometry, grids, species).
    precision: "fp64" or "mixed".
    """

    def __init__(self, prob, precision: str = "fp64", stream=None, phase_norm: float = 1.0, _handle=None):
        import torch
        L = lib()
        self.prob = prob
        self.mixed = precision == "mixed"
        self.fdtype = np.float32 if self.mixed else np.float64
        self.torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.shape = (prob.n_species, prob.n_zone, prob.n_eps, prob.n_ang)
        if _handle is not None:          # a batch member: owned by the batch
            self.h = _handle
            self.owned = False
            return
        self._keep = []
        cfg = make_config(prob, precision, self.stream.cuda_stream, phase_norm, self._keep)
        self.cfg = cfg
        nbytes = L.bt_workspace_bytes(C.byref(cfg))
        if nbytes == 0:
            raise BtError(-1, L.bt_last_error().decode())
        # workspace from PyTorch's allocator, kept alive by this object
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = self.workspace.data_ptr()
        aligned = (base + 255) & ~255
        h = C.c_void_p()
        _check(L.bt_create(C.byref(cfg), C.c_void_p(aligned), C.byref(h)))
        self.h = h
        self.owned = True
        if getattr(prob, "f_boundary", None) is not None:
            self.set_boundary(prob.f_boundary)

    def close(self):
        if getattr(self, "h", None) and getattr(self, "owned", False):
            lib().bt_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- inputs -------------------------------------------------------------
    def set_background(self, bg):
        """Host (numpy) background: copied host -> device on the stream."""
        arrs = [_host64(bg.rho), _host64(bg.T), _host64(bg.Ye), _host64(bg.v), _host64(bg.alpha),
                _host64(bg.phi), _host64(bg.shift), _host64(bg.kappa_a), _host64(bg.kappa_s), _host64(bg.f_eq)]
        _check(lib().bt_set_background(self.h, BT_MEM_HOST, *[_ptr(a) for a in arrs]))
        self._keep_bg = arrs

    def set_background_device(self, v, alpha, phi, kappa_a, kappa_s, f_eq):
        """Device (torch float64, contiguous) background."""
        _check(lib().bt_set_background(self.h, BT_MEM_DEVICE, None, None, None, _ptr(v), _ptr(alpha), _ptr(phi),
                                       None, _ptr(kappa_a), _ptr(kappa_s), _ptr(f_eq)))

    def set_boundary(self, fbc):
        """Distribution imposed on the incoming bins of the open face at
        theta_max, [species][radial zone][group] (host numpy)."""
        a = _host64(fbc).reshape(self.prob.n_species, self.prob.n_r, self.prob.n_eps)
        self._keep_bc = np.ascontiguousarray(a)
        _check(lib().bt_set_boundary(self.h, BT_MEM_HOST, _ptr(self._keep_bc)))

    def set_f(self, f):
        if isinstance(f, np.ndarray):
            a = np.ascontiguousarray(f.astype(self.fdtype, copy=False).reshape(self.shape))
            _check(lib().bt_set_f(self.h, BT_MEM_HOST, _ptr(a)))
            self.torch.cuda.synchronize()
        else:
            _check(lib().bt_set_f(self.h, BT_MEM_DEVICE, _ptr(f)))

    # -- step ---------------------------------------------------------------
    def max_dt(self, cfl: float) -> float:
        out = C.c_double()
        _check(lib().bt_max_dt(self.h, float(cfl), C.byref(out)))
        return out.value

    def step(self, dt: float):
        _check(lib().bt_step(self.h, float(dt)))

    # -- local time stepping ------------------------------------------------
    def lts_levels(self, cfl: float, max_levels: int):
        """Levels from the current background (bt_lts_levels): (dt0, levels)."""
        dt0 = C.c_double()
        lev = np.zeros(self.prob.n_zone, dtype=np.int32)
        _check(lib().bt_lts_levels(self.h, float(cfl), int(max_levels), C.byref(dt0), lev.ctypes.data))
        return dt0.value, lev

    def set_levels(self, levels, n_levels: int):
        lev = np.ascontiguousarray(np.asarray(levels, dtype=np.int32))
        _check(lib().bt_set_levels(self.h, lev.ctypes.data, int(n_levels)))

    @property
    def n_levels(self) -> int:
        return int(lib().bt_n_levels(self.h))

    def step_lts(self, dt0: float):
        _check(lib().bt_step_lts(self.h, float(dt0)))

    # -- outputs ------------------------------------------------------------
    def get_f(self, out=None) -> np.ndarray:
        if out is not None:
            _check(lib().bt_get_f(self.h, BT_MEM_DEVICE if not isinstance(out, np.ndarray) else BT_MEM_HOST, _ptr(out)))
            return out
        a = np.empty(self.shape, dtype=self.fdtype)
        _check(lib().bt_get_f(self.h, BT_MEM_HOST, _ptr(a)))
        return a

    def moments(self, out=None):
        S, Z = self.prob.n_species, self.prob.n_zone
        if out is None:
            out = (np.empty((S, Z)), np.empty((S, Z)), np.empty((S, Z, 3)), np.empty(Z))
        mem = BT_MEM_HOST if isinstance(out[0], np.ndarray) else BT_MEM_DEVICE
        _check(lib().bt_moments(self.h, mem, *[_ptr(a) for a in out]))
        return out

    def totals(self):
        S = self.prob.n_species
        N, E, No, Eo = np.empty(S), np.empty(S), np.empty(S), np.empty(S)
        _check(lib().bt_totals(self.h, _ptr(N), _ptr(E), _ptr(No), _ptr(Eo)))
        return N, E, No, Eo

    def jhk(self):
        sh = (self.prob.n_species, self.prob.n_zone, self.prob.n_eps)
        J, H, K = np.empty(sh), np.empty(sh), np.empty(sh)
        _check(lib().bt_jhk(self.h, BT_MEM_HOST, _ptr(J), _ptr(H), _ptr(K)))
        return J, H, K

    @property
    def launch_count(self) -> int:
        return int(lib().bt_launch_count(self.h))

    def autotune(self, dt: float) -> int:
        nt = C.c_int()
        _check(lib().bt_autotune(self.h, float(dt), C.byref(nt)))
        return nt.value

    @property
    def launch_shape(self) -> int:
        nt = C.c_int()
        _check(lib().bt_launch_shape(self.h, C.byref(nt)))
        return nt.value

    def set_launch_shape(self, nt: int):
        _check(lib().bt_set_launch_shape(self.h, int(nt)))

    def sur_samples(self, idx):
        """Learned-remap rows idx [n][3] (zone, kind, source angle) -> device
        tensors X [n][16], Y [n][27], valid [n] (bt_sur_samples)."""
        import torch
        idx = torch.as_tensor(np.ascontiguousarray(np.asarray(idx, dtype=np.int32).reshape(-1, 3))).cuda()
        n = idx.shape[0]
        X = torch.empty((n, SUR_NIN), dtype=torch.float32, device="cuda")
        Y = torch.empty((n, SUR_NOUT), dtype=torch.float32, device="cuda")
        v = torch.empty(n, dtype=torch.int32, device="cuda")
        _check(lib().bt_sur_samples(self.h, idx.data_ptr(), n, X.data_ptr(), Y.data_ptr(), v.data_ptr()))
        return X, Y, v

    def set_surrogate(self, sur, tol: float):
        """Learned remap weights in every step (sur = None: exact weights)."""
        self._sur = sur
        _check(lib().bt_set_surrogate(self.h, sur.h if sur is not None else None, float(tol)))

    def sur_stats(self):
        a, b = C.c_int64(), C.c_int64()
        _check(lib().bt_sur_stats(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def profile(self, enable: bool):
        _check(lib().bt_profile(self.h, int(enable)))

    def profile_read(self, kernel: int):
        ms, n = C.c_double(), C.c_int64()
        _check(lib().bt_profile_read(self.h, int(kernel), C.byref(ms), C.byref(n)))
        return ms.value, n.value


K_TIME_REMAP, K_FLUX, K_OUTFLOW, K_SUR_TABLE, K_ZONE = 0, 1, 2, 3, 4


class Batch:
    """Several independent problems advanced by one CUDA-graph launch per
    step (bt_batch_* in include/bt.h).  ``members[i]`` is a Transport view of
    problem i for backgrounds, f and outputs."""

    def __init__(self, probs, precision="mixed", stream=None):
        import torch
        L = lib()
        self.probs = list(probs)
        # the step is captured into a CUDA graph, which the legacy default
        # stream does not allow: without a stream, the batch makes its own
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self._keep = []
        n = len(self.probs)
        cfgs = (BtConfig * n)()
        for i, p in enumerate(self.probs):
            cfgs[i] = make_config(p, precision, self.stream.cuda_stream, 1.0, self._keep)
        h = C.c_void_p()
        _check(L.bt_batch_create(cfgs, n, self.stream.cuda_stream, C.byref(h)))
        self.h = h
        self.members = []
        for i, p in enumerate(self.probs):
            mh = C.c_void_p()
            _check(L.bt_batch_member(h, i, C.byref(mh)))
            self.members.append(Transport(p, precision, stream=self.stream, _handle=mh))

    def step(self, dts):
        arr = (C.c_double * len(self.members))(*[float(x) for x in dts])
        _check(lib().bt_batch_step(self.h, arr))

    @property
    def launch_count(self) -> int:
        return int(lib().bt_batch_launch_count(self.h))

    @property
    def graph_launches(self) -> int:
        return int(lib().bt_batch_graph_launches(self.h))

    def close(self):
        if getattr(self, "h", None):
            for m in self.members:
                m.h = None
            lib().bt_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def weighted_totals_noalloc(f, w_za, w_e, precision: str, out, stream=None):
    """Allocation-free weighted totals (see bt_weighted_totals_noalloc in
    include/bt.h).  f, w_za, w_e, out: contiguous CUDA tensors (f float64 or
    float32 as `precision` says, weights and out float64)."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    n_s, n_zone, n_e, n_ang = f.shape
    rc = lib().bt_weighted_totals_noalloc(f.data_ptr(), BT_MIXED if precision == "mixed" else BT_FP64,
                                          n_s, n_zone, n_e, n_ang, w_za.data_ptr(), w_e.data_ptr(),
                                          out.data_ptr(), s.cuda_stream)
    if rc != BT_OK:
        raise BtError(rc, "bt_weighted_totals_noalloc failed")
    return out


def run(prob, precision="fp64", n_steps=None, dt=None, cfl=None):
    """Same protocol as the oracle's ``run``: background 0 (alternating with
    background 1 every step if prob.alternate), f0, n_steps steps."""
    t = Transport(prob, precision)
    t.set_background(prob.backgrounds[0])
    t.set_f(prob.f0)
    if dt is None:
        dt = t.max_dt(prob.cfl if cfl is None else cfl)
    n = prob.n_steps if n_steps is None else n_steps
    for k in range(n):
        if prob.alternate and len(prob.backgrounds) > 1:
            t.set_background(prob.backgrounds[(k + 1) % 2])
        t.step(dt)
    return t, dt


class Surrogate:
    """The learned remap's network (bt_sur_* in include/bt.h).  Inputs and
    outputs are contiguous float32 CUDA tensors; parameters go in and out as
    host numpy float32 vectors of SUR_NPARAM entries."""

    def __init__(self, stream=None):
        import torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        _check(lib().bt_sur_create(self.stream.cuda_stream, C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().bt_sur_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, p):
        p = np.ascontiguousarray(np.asarray(p, dtype=np.float32))
        assert p.size == SUR_NPARAM
        _check(lib().bt_sur_set_params(self.h, BT_MEM_HOST, p.ctypes.data))

    def get_params(self) -> np.ndarray:
        p = np.empty(SUR_NPARAM, dtype=np.float32)
        _check(lib().bt_sur_get_params(self.h, BT_MEM_HOST, p.ctypes.data))
        return p

    def fit_normalizer(self, X):
        _check(lib().bt_sur_fit_normalizer(self.h, X.data_ptr(), X.shape[0]))

    def forward(self, X, out=None):
        import torch
        n = X.shape[0]
        if out is None:
            out = torch.empty((n, SUR_NOUT), dtype=torch.float32, device=X.device)
        _check(lib().bt_sur_forward(self.h, X.data_ptr(), n, out.data_ptr()))
        return out

    def grad(self, X, Y):
        import torch
        g = torch.empty(SUR_NPARAM, dtype=torch.float32, device=X.device)
        loss = torch.empty(1, dtype=torch.float32, device=X.device)
        _check(lib().bt_sur_grad(self.h, X.data_ptr(), Y.data_ptr(), X.shape[0], g.data_ptr(), loss.data_ptr()))
        return g, float(loss.item())

    def train(self, X, Y, epochs, batch=4096, lr=2e-3, lr_final=5e-5, beta1=0.9, beta2=0.999, eps=1e-8):
        cfg = BtTrainCfg(int(epochs), int(batch), lr, lr_final, beta1, beta2, eps)
        log = np.zeros(int(epochs), dtype=np.float32)
        _check(lib().bt_sur_train(self.h, X.data_ptr(), Y.data_ptr(), X.shape[0], C.byref(cfg), log.ctypes.data))
        return log


def peak_fma(precision: str, stream=None) -> float:
    """Measured FMA rate (flop/s) of the current GPU in float64 ("fp64") or
    float32 ("mixed"), see bt_peak_fma."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    out = C.c_double()
    rc = lib().bt_peak_fma(BT_MIXED if precision == "mixed" else BT_FP64, C.byref(out), s.cuda_stream)
    if rc != BT_OK:
        raise BtError(rc, "bt_peak_fma failed")
    return out.value


def shape_name(nt: int) -> str:
    """Readable launch shape: 'fused/256' or 'split/512'."""
    return ("split/%d" if nt & SHAPE_SPLIT else "fused/%d") % (nt & 0xFFFF)
