"""Benchmark of the transport step on GB300.

One "step" = the whole hot path on one synthetic background: the time remap
to a new background (backgrounds B0/B1 alternate every step), the face
fluxes + collision kernels, and the outflow/moment reductions.  The metric is
zone-group-angle updates per second (species included) of a full step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload config5]
                  [--precision mixed|fp64] [--impl ours|reference]

The default workload, config5, is the batched form: three independent 2D
problems of uneven size (128x32, 256x64, 512x128 zones; 8, 12, 20 groups;
48, 80, 128 angles; 6 species) advanced by one CUDA-graph launch per step;
its units are the bins of all three problems.  The line carries the same
batch in plain FP64 on the same GPU (vs_fp64_gpu), the accuracy of the
mixed form against it (f, its increment and the source terms), the accuracy
on a transport-dominated variant of config 3 (opacities x 1e-6), and a short
config-3 measurement under "extra".  --workload config3 times the single 2D
problem (and, with the learned remap on, trains and times the network).

--impl reference times the FP64 CPU oracle (all host cores) on a bounded
sample of zones of the same workload.  Under torchrun (N > 1) every rank runs
an independent replica; rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "zone·group·angle updates/sec per full step vs plain FP64 GPU path at ≤1e-4 rel L1"
UNIT = "zone·group·angle·species updates/s"


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            return d, "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def hbm_peak(d):
    for k in ("hbm_gbs", "hbm_GBs", "hbm_copy_gbs", "copy_gbs"):
        if k in d:
            v = d[k]
            if isinstance(v, dict):
                v = v.get("value", v.get("burst", None))
            if v:
                return float(v)
    return 6800.0


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm = [float(r[0]) for r in self.rows if len(r) >= 8 and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) >= 8 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) < 8:
                continue
            for n, v in zip(names, r[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def max_over_ranks(x: float) -> float:
    """The largest x over the ranks of the process group (the job's time is
    its slowest rank's)."""
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank: float, world: int, ms_per_step: float) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return world * units_per_rank / (ms_per_step * 1e-3)


def dist_init(n_gpus):
    import torch
    rank, world = 0, 1
    if n_gpus > 1 or "RANK" in os.environ:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        rank, world = dist.get_rank(), dist.get_world_size()
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", rank)))
    else:
        torch.cuda.set_device(0)
    return rank, world


def alu_peaks():
    """Measured FMA rates of this GPU (flop/s) in float32 and float64 and its SM
    count, read from the device (bt_peak_fma: independent FMA chains on every
    SM, CUDA events)."""
    import torch
    from paper_2003_02845_gb300 import bt
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    return {"fp32_tflops": bt.peak_fma("mixed") / 1e12, "fp64_tflops": bt.peak_fma("fp64") / 1e12,
            "sms": props.multi_processor_count, "source": "measured: bt_peak_fma (FMA chains, CUDA events)"}


def host_cpu():
    """Host cores and CPU model (the oracle's machine)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return os.cpu_count(), model


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one flux
# step from an ncu capture of the profiling driver's run, keyed by
# workload, precision and launch shape, and valid only for the kernel code
# it was taken on (a fingerprint of bt_kernels.cu without its comments and
# blank lines): changed kernel code reports null until re-captured.
# For the split form the figure is the face pass plus the zone pass: f read
# and written once plus the deposit rows (six per zone) written and read.
TRAFFIC = {
    ("config3_cc2d_256x64x12x80x3", "mixed", "split/256"):
        (217.14e6 + 1348.28e6 + 1352.18e6 + 429.01e6, "fcbeb618733754eb056abaf54f31788e79c44b4b5a28914a5d730eb6b61319ee"),
    # captured on the same problem at 128 x 32 zones (python -m
    # paper_2003_02845_gb300.profiling config5_largest_128x32 mixed split/384 3)
    # and scaled by the 16x zones of the full 512 x 128 grid (the traffic of
    # both passes is per zone)
    ("config5_p2_512x128x20x128x6", "mixed", "split/384"):
        (16 * (483.69e6 + 1458.76e6 + 2011.14e6 + 509.15e6), "fcbeb618733754eb056abaf54f31788e79c44b4b5a28914a5d730eb6b61319ee"),
}


def kernel_fingerprint(path=None):
    """sha256 of the kernel source with comments, blank lines and trailing
    spaces removed (a comment-only edit keeps it)."""
    import hashlib
    import re
    path = path or os.path.join(ROOT, "paper_2003_02845_gb300", "csrc", "bt_kernels.cu")
    src = open(path).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    lines = [re.sub(r"//.*$", "", ln).rstrip() for ln in src.splitlines()]
    return hashlib.sha256("\n".join(ln for ln in lines if ln).encode()).hexdigest()


def measured_traffic(workload, precision, nt):
    rec = TRAFFIC.get((workload, precision, nt))
    if rec is None:
        return None
    return rec[0] if kernel_fingerprint() == rec[1] else None


def algorithmic_flops_per_bin(prob):
    """Arithmetic the method needs per zone-group-angle-species bin and step,
    counted on unique faces (3 per zone in spherical geometry, 1 in a slab):
    per face six remaps (four stencil cells into the face frame, the flux
    back into both neighbours), each a trilinear split costing 6 FMA per bin;
    about 28 flops for the Lax-Wendroff half step, MC upwind, blend and flux;
    the weight chain (~150 flops per remap and angle) shared by all groups and
    species; and ~20 flops for the implicit collision."""
    faces = 1 if prob.geom == 1 else 3
    per_face = 6 * 12 + 28 + 6 * 150.0 / (prob.n_eps * prob.n_species)
    return faces * per_face + 20.0


def algorithmic_bytes_per_bin(prob, mixed):
    """Bytes that one full step must move per zone-group-angle-species bin:
    read f^n and write f^{n+1}, plus the opacities (3 float64 per zone, group
    and species, amortised over the angles) and the per-zone background (7
    float64, amortised over groups, angles and species)."""
    fb = 4 if mixed else 8
    return 2 * fb + 24.0 / prob.n_ang + 56.0 / (prob.n_ang * prob.n_eps * prob.n_species)


def _device_backgrounds(prob):
    import torch
    return [[torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64)).cuda()
             for x in (bg.v, bg.alpha, bg.phi, bg.kappa_a, bg.kappa_s, bg.f_eq)] for bg in prob.backgrounds]


def _pinned_backgrounds(prob):
    import torch
    return [[torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64)).pin_memory()
             for x in (bg.rho, bg.T, bg.Ye, bg.v, bg.alpha, bg.phi, bg.shift,
                       bg.kappa_a, bg.kappa_s, bg.f_eq)] for bg in prob.backgrounds]


def _roofline(prob, mixed, kernel, flux_avg_ms, face_avg_ms, zone_avg_ms, remap_avg_ms, alu, traffic):
    """Roofline of the flux step (face pass + zone pass, or the fused kernel):
    ALU bound (the arithmetic of the remaps runs in shared memory), with the
    HBM fraction of the algorithmic bytes and of the ncu-measured traffic
    beside it."""
    peaks, peak_src = load_peaks()
    hbm = hbm_peak(peaks)
    bins = prob.n_bins
    bpb = algorithmic_bytes_per_bin(prob, mixed)
    fpb = algorithmic_flops_per_bin(prob)
    s = flux_avg_ms * 1e-3
    achieved_tf = bins * fpb / s / 1e12
    peak_tf = alu["fp32_tflops"] if mixed else alu["fp64_tflops"]
    achieved_gbs = bins * bpb / s / 1e9
    out = {
        "kernel": kernel,
        "bound": "alu",
        "achieved": achieved_tf,
        "peak": peak_tf,
        "peak_source": "%s; %s FMA rate (%d SMs)" % (alu["source"], "float32" if mixed else "float64", alu["sms"]),
        "unit": "TFLOP/s",
        "frac": achieved_tf / peak_tf,
        "traffic": traffic,
        "traffic_unit": "bytes per launch (ncu dram read + write)",
        "algorithmic_flops_per_bin": fpb,
        "avg_launch_ms": flux_avg_ms,
        "face_pass_avg_ms": face_avg_ms,
        "zone_pass_avg_ms": zone_avg_ms,
        "time_remap_avg_ms": remap_avg_ms,
        "hbm": {"achieved": achieved_gbs, "peak": hbm, "peak_source": peak_src + " (MEASURED_PEAKS.json copy)",
                "unit": "GB/s", "frac": achieved_gbs / hbm, "algorithmic_bytes_per_bin": bpb,
                "traffic_gbs": traffic / s / 1e9 if traffic else None,
                "traffic_frac": traffic / s / 1e9 / hbm if traffic else None},
    }
    if remap_avg_ms:
        # the time remap alone: one read and one write of f
        gbs = bins * 2 * (4 if mixed else 8) / (remap_avg_ms * 1e-3) / 1e9
        out["time_remap_hbm"] = {"achieved": gbs, "frac": gbs / hbm, "unit": "GB/s",
                                 "algorithmic_bytes_per_bin": 2 * (4 if mixed else 8)}
    return out


def run_ours(args):
    import torch
    from paper_2003_02845_gb300 import build, bt, workloads as W
    rank, world = dist_init(args.gpus)
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    build.build()
    if args.workload == "config5":
        return run_batch(args, rank, world)
    prob = W.by_name(args.workload)
    res, t = single_problem(prob, args, world)
    if args.precision == "mixed" and not args.no_fp64_compare:
        ms64 = time_fp64_path(prob, t.dev)
        res["vs_fp64_gpu"] = {"value": prob.n_bins / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64,
                              "speedup": ms64 / res["ms_per_step"],
                              "what": "the same step in plain FP64 on this GPU (same kernels, T = double, "
                                      "autotuned launch shape)"}
    shape = t.launch_shape
    t.close()
    if args.precision == "mixed" and args.accuracy_steps > 0:
        res["accuracy"] = accuracy_single(prob, args.accuracy_steps)
        res["accuracy_transport"] = accuracy_single(W.config3_transport(), args.accuracy_steps)
        if args.learned_remap:
            try:
                res["learned_remap"] = learned_remap_block(prob, args, res["ms_per_step"], shape)
            except Exception as e:   # report, do not lose the line
                res["learned_remap"] = {"error": repr(e)}
    if rank == 0 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(prob, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def single_problem(prob, args, world, steps=None, e2e=True):
    """Time one problem's full step (device-resident backgrounds alternating),
    its kernels, and the same step end to end through the C ABI with host
    buffers.  Returns (result dict, the Transport, which keeps .dev)."""
    import torch
    from paper_2003_02845_gb300 import bt
    steps = args.steps if steps is None else steps
    mixed = args.precision == "mixed"
    stream = torch.cuda.Stream()
    t = bt.Transport(prob, args.precision, stream=stream)
    t.dev = _device_backgrounds(prob)
    torch.cuda.synchronize()
    t.set_background(prob.backgrounds[0])
    t.set_f(prob.f0)
    dt = t.max_dt(prob.cfl)
    if args.shape:
        t.set_launch_shape(parse_shape(args.shape))
    elif args.autotune:
        t.autotune(dt)
    bins = prob.n_bins

    def one_step(k):
        t.set_background_device(*t.dev[(k + 1) % 2])
        t.step(dt)

    for k in range(args.warmup):
        one_step(k)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    l0 = t.launch_count
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for k in range(steps):
            one_step(args.warmup + k)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / steps
    launches = t.launch_count - l0
    if world > 1:
        ms = max_over_ranks(ms)
        torch.distributed.barrier()

    # per-kernel durations with CUDA events on the transport stream
    t.profile(True)
    for k in range(steps):
        one_step(args.warmup + steps + k)
    flux_ms, flux_n = t.profile_read(bt.K_FLUX)
    zone_ms, zone_n = t.profile_read(bt.K_ZONE)
    remap_ms, remap_n = t.profile_read(bt.K_TIME_REMAP)
    t.profile(False)
    split = bool(t.launch_shape & bt.SHAPE_SPLIT)
    face_avg = flux_ms / max(flux_n, 1)
    zone_avg = zone_ms / max(zone_n, 1) if split else None
    flux_avg = face_avg + (zone_avg or 0.0)

    e2e_block = None
    if e2e:
        # end to end through the C ABI with host buffers: pinned host
        # background in, source terms out, every step
        pinned = _pinned_backgrounds(prob)
        S, Z = prob.n_species, prob.n_zone
        outs = [torch.empty(sh, dtype=torch.float64).pin_memory() for sh in ((S, Z), (S, Z), (S, Z, 3), (Z,))]
        h2d = sum(x.numel() * 8 for x in pinned[0][3:6] + pinned[0][7:10])
        d2h = sum(x.numel() * 8 for x in outs)
        L = bt.lib()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(steps):
            pm = pinned[(k + 1) % 2]
            bt._check(L.bt_set_background(t.h, bt.BT_MEM_HOST, *[x.data_ptr() for x in pm]))
            t.step(dt)
            bt._check(L.bt_moments(t.h, bt.BT_MEM_HOST, *[x.data_ptr() for x in outs]))
        e2e_s = (time.perf_counter() - t0) / steps
        if world > 1:
            e2e_s = max_over_ranks(e2e_s)
        e2e_block = {"value": world * bins / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                     "d2h_bytes_per_step": d2h}

    alu = alu_peaks()
    shape = bt.shape_name(t.launch_shape)
    res = {
        "metric": METRIC,
        "value": job_value(bins, world, ms),
        "unit": UNIT,
        "n_gpus": world,
        "steps": steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if mixed else "f64",
        "data": "synthetic",
        "config": {
            "workload": prob.name,
            "precision": args.precision + (" (f32 f/fluxes/remap; collision and sums in double-float/f64)"
                                           if mixed else ""),
            "zones": prob.n_zone, "groups": prob.n_eps, "angles": prob.n_ang, "species": prob.n_species,
            "bins_per_step": bins,
            "updates_per_s_without_species": world * prob.n_zone * prob.n_eps * prob.n_ang / (ms * 1e-3),
            "l2": "inputs larger than L2 (f is %.0f MB per buffer)" % (bins * (4 if mixed else 8) / 1e6),
            "parallelism": "replicas" if world > 1 else "single GPU",
            "backgrounds": "B0/B1 alternate every step (time remap active)",
            "launch_shape": shape,
        },
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "e2e": e2e_block,
        "roofline": _roofline(prob, mixed, kernel_name(mixed, split), flux_avg, face_avg if split else None,
                              zone_avg, remap_ms / max(remap_n, 1), alu,
                              measured_traffic(prob.name, args.precision, shape)),
    }
    return res, t


def parse_shape(name):
    """'fused/256' or 'split/512' -> the library's launch-shape code"""
    from paper_2003_02845_gb300 import bt
    form, nt = name.split("/")
    return (bt.SHAPE_SPLIT if form == "split" else 0) | int(nt)


def kernel_name(mixed, split):
    tn = "float" if mixed else "double"
    if split:
        return "k_flux_faces<%s> + k_zone_collide<%s> (split flux step)" % (tn, tn)
    return "k_flux_collide<%s>" % tn


def rel_l1(a, b):
    return float((a.double() - b.double()).abs().sum() / b.double().abs().sum())


def run_steps(prob, precision, steps, sur=None, tol=0.0, stream=None, shape=None):
    """State after `steps` steps from f0 with the backgrounds alternating as in
    the timed run, dt from the Courant limit of B0: f (device tensor),
    moments and totals (host)."""
    import torch
    from paper_2003_02845_gb300 import bt
    stream = stream if stream is not None else torch.cuda.Stream()
    dev = _device_backgrounds(prob)
    t = bt.Transport(prob, precision, stream=stream)
    if shape is not None:
        t.set_launch_shape(shape)
    if sur is not None:
        t.set_surrogate(sur, tol)
    t.set_background(prob.backgrounds[0])
    t.set_f(prob.f0)
    dt = t.max_dt(prob.cfl)
    for k in range(steps):
        t.set_background_device(*dev[(k + 1) % 2])
        t.step(dt)
    f = torch.empty(prob.f0.shape, dtype=torch.float32 if precision == "mixed" else torch.float64, device="cuda")
    t.get_f(out=f)
    out = {"f": f, "moments": t.moments(), "totals": t.totals(), "dt": dt}
    if sur is not None:
        out["sur_stats"] = t.sur_stats()
    t.close()
    return out


def compare_states(a, b, f0):
    """Accuracy of state a against the reference b (both from f0 [device]):
    rel-L1 of f, of the increment f - f0, of the number source dN, and the
    relative difference of the totals (number, energy at infinity) with
    their outflows."""
    inc = float((a["f"].double() - b["f"].double()).abs().sum() / (b["f"].double() - f0).abs().sum())
    dNa, dNb = a["moments"][0], b["moments"][0]
    dEa, dEb = a["moments"][1], b["moments"][1]
    Na = a["totals"][0] + a["totals"][2]
    Nb = b["totals"][0] + b["totals"][2]
    Ea = a["totals"][1] + a["totals"][3]
    Eb = b["totals"][1] + b["totals"][3]
    return {"rel_l1_f": rel_l1(a["f"], b["f"]),
            "rel_l1_increment": inc,
            "rel_l1_dN": float(np.abs(dNa - dNb).sum() / max(np.abs(dNb).sum(), 1e-300)),
            "rel_l1_dE": float(np.abs(dEa - dEb).sum() / max(np.abs(dEb).sum(), 1e-300)),
            "rel_N_plus_outflow": float(np.max(np.abs(Na - Nb) / np.abs(Nb))),
            "rel_E_plus_outflow": float(np.max(np.abs(Ea - Eb) / np.abs(Eb)))}


def accuracy_single(prob, steps):
    """The mixed path against the plain FP64 GPU path (which matches the FP64
    oracle to 1e-12) after `steps` steps from the same f0, same backgrounds
    and dt."""
    import torch
    f64 = run_steps(prob, "fp64", steps)
    mix = run_steps(prob, "mixed", steps)
    f0 = torch.as_tensor(np.ascontiguousarray(prob.f0, dtype=np.float64)).cuda()
    out = {"workload": prob.name, "steps": steps,
           "what": "mixed path vs the plain FP64 GPU path (itself within 1e-12 of the FP64 oracle)"}
    out.update(compare_states(mix, f64, f0))
    return out


def learned_remap_block(prob, args, ms_exact, shape):
    """Train the network on rows of the exact remap from 16 seeded background
    pairs (the workload's own backgrounds are held out), then time the step
    with it and measure its error at a few trip tolerances, on the workload
    and on its transport-dominated variant (opacities x 1e-6)."""
    import torch
    from paper_2003_02845_gb300 import bt, learned_remap as LR, workloads as W
    stream = torch.cuda.Stream()      # network, data and steps share it
    t0 = time.perf_counter()
    pairs = [W.config4_backgrounds(k) for k in range(16)]
    with torch.cuda.stream(stream):
        X, Y = LR.training_set(prob, pairs, args.sur_samples, seed=777, stream=stream)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    net, log = LR.train(X, Y, epochs=args.sur_epochs, batch=4096, stream=stream)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    n_rows = int(X.shape[0])
    del X, Y
    thin = W.config3_transport()
    ref = {name: run_steps(p, "fp64", args.accuracy_steps) for name, p in (("thick", prob), ("transport", thin))}
    exact_thin = run_steps(thin, "mixed", args.accuracy_steps, stream=stream, shape=shape)
    f0 = {name: torch.as_tensor(np.ascontiguousarray(p.f0, dtype=np.float64)).cuda()
          for name, p in (("thick", prob), ("transport", thin))}
    out = {"samples": n_rows, "epochs": args.sur_epochs, "batch": 4096, "launch_shape": bt.shape_name(shape),
           "loss_per_epoch": [float(x) for x in log],
           "data_seconds": t1 - t0, "train_seconds": t2 - t1,
           "exact_mixed_transport": compare_states(exact_thin, ref["transport"], f0["transport"]),
           "runs": []}
    dev = _device_backgrounds(prob)
    for tol in args.sur_tols:
        t = bt.Transport(prob, "mixed", stream=stream)
        t.set_launch_shape(shape)            # the exact run's launch shape
        t.set_surrogate(net, tol)
        t.set_background(prob.backgrounds[0])
        t.set_f(prob.f0)
        dt = t.max_dt(prob.cfl)
        for k in range(3):
            t.set_background_device(*dev[(k + 1) % 2])
            t.step(dt)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        for k in range(args.steps):
            t.set_background_device(*dev[(k + 4) % 2])
            t.step(dt)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms_sur = ev0.elapsed_time(ev1) / args.steps
        t.profile(True)
        for k in range(3):
            t.set_background_device(*dev[(k + 1) % 2])
            t.step(dt)
        tab_ms, tab_n = t.profile_read(bt.K_SUR_TABLE)
        t.profile(False)
        t.close()
        run = {"tol_bins": tol, "ms_per_step": ms_sur, "value": prob.n_bins / (ms_sur * 1e-3),
               "speed_vs_exact_mixed": ms_exact / ms_sur, "table_kernel_ms": tab_ms / max(tab_n, 1)}
        for name, p in (("thick", prob), ("transport", thin)):
            st = run_steps(p, "mixed", args.accuracy_steps, sur=net, tol=tol, stream=stream, shape=shape)
            n_eval, n_trip = st["sur_stats"]
            run[name] = compare_states(st, ref[name], f0[name])
            run[name]["trip_fraction"] = n_trip / max(n_eval, 1)
            del st
        out["runs"].append(run)
    net.close()
    return out


def time_fp64_path(prob, dev, steps=5, warmup=3):
    """ms per step of the plain FP64 path on the same workload and device
    backgrounds (events on its own stream)."""
    import torch
    from paper_2003_02845_gb300 import bt
    stream = torch.cuda.Stream()
    t = bt.Transport(prob, "fp64", stream=stream)
    t.set_background(prob.backgrounds[0])
    t.set_f(prob.f0)
    dt = t.max_dt(prob.cfl)
    t.autotune(dt)          # its own best launch shape, as the timed path has
    for k in range(warmup):
        t.set_background_device(*dev[(k + 1) % 2])
        t.step(dt)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for k in range(steps):
        t.set_background_device(*dev[(warmup + k + 1) % 2])
        t.step(dt)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / steps
    t.close()
    return ms


def lts_block(prob, levels=4, macro_steps=3):
    """Local time stepping (Sec. 5) on one problem, mixed precision: the
    background changes once per hydro step of 2^(levels-1) finest steps dt0
    (time remap once), then either 2^(levels-1) global steps of dt0 or one
    local-time-stepping macro step.  Reports both times per hydro step, the
    ratio, the share of zone updates the levels leave, and the rel-L1
    difference of f after the same simulated time (the two are different
    time integrations: that difference is the time-discretisation one)."""
    import torch
    from paper_2003_02845_gb300 import bt
    K = 1 << (levels - 1)
    dev = _device_backgrounds(prob)
    out = {"levels": levels, "hydro_steps": macro_steps}
    res = {}
    for mode in ("global", "lts"):
        stream = torch.cuda.Stream()
        t = bt.Transport(prob, "mixed", stream=stream)
        t.set_launch_shape(bt.SHAPE_SPLIT | 256)
        t.set_background(prob.backgrounds[0])
        t.set_f(prob.f0)
        dt0, lev = t.lts_levels(prob.cfl, levels)

        def hydro_step(k):
            t.set_background_device(*dev[(k + 1) % 2])
            if mode == "lts":
                t.step_lts(dt0)
            else:
                for _ in range(K):
                    t.step(dt0)

        hydro_step(0)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for k in range(macro_steps):
            hydro_step(1 + k)
        ev1.record(stream)
        torch.cuda.synchronize()
        f = torch.empty(prob.f0.shape, dtype=torch.float32, device="cuda")
        t.get_f(out=f)
        res[mode] = {"ms_per_hydro_step": ev0.elapsed_time(ev1) / macro_steps, "f": f}
        if mode == "lts":
            cnt = np.bincount(lev, minlength=levels)
            out["zones_per_level"] = cnt.tolist()
            out["zone_update_share"] = float(sum(cnt[l] * 2 ** (levels - 1 - l) for l in range(levels))
                                             / (prob.n_zone * K))
        t.close()
    out["ms_per_hydro_step_global"] = res["global"]["ms_per_hydro_step"]
    out["ms_per_hydro_step_lts"] = res["lts"]["ms_per_hydro_step"]
    out["speedup"] = out["ms_per_hydro_step_global"] / out["ms_per_hydro_step_lts"]
    out["rel_l1_vs_global_steps"] = rel_l1(res["lts"]["f"], res["global"]["f"])
    out["workload"] = prob.name
    return out


class BatchRun:
    """A batch of the config-5 problems in one precision, backgrounds on the
    device, launch shapes autotuned (or fixed)."""

    def __init__(self, probs, precision, shapes=None, autotune=True):
        import torch
        from paper_2003_02845_gb300 import bt
        self.probs = probs
        self.stream = torch.cuda.Stream()
        self.b = bt.Batch(probs, precision, stream=self.stream)
        self.dev, self.dts, self.shapes = [], [], []
        for i, (m, p) in enumerate(zip(self.b.members, probs)):
            self.dev.append(_device_backgrounds(p))
            m.set_background(p.backgrounds[0])
            m.set_f(p.f0)
            dt = m.max_dt(p.cfl)
            self.dts.append(dt)
            if shapes:
                m.set_launch_shape(parse_shape(shapes[min(i, len(shapes) - 1)]))
            elif autotune:
                m.autotune(dt)
            self.shapes.append(bt.shape_name(m.launch_shape))
        torch.cuda.synchronize()

    def step(self, k):
        for m, d in zip(self.b.members, self.dev):
            m.set_background_device(*d[(k + 1) % 2])
        self.b.step(self.dts)

    def time(self, steps, warmup, k0=0, clock=False):
        import torch
        for k in range(warmup):
            self.step(k0 + k)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        clk = ClockSampler(torch.cuda.current_device()) if clock else None
        if clk:
            clk.__enter__()
        torch.cuda.synchronize()
        ev0.record(self.stream)
        for k in range(steps):
            self.step(k0 + warmup + k)
        ev1.record(self.stream)
        torch.cuda.synchronize()
        if clk:
            clk.__exit__(None, None, None)
        return ev0.elapsed_time(ev1) / steps, clk

    def state(self):
        """Per-member f (device), moments and totals (host)."""
        import torch
        out = []
        for m, p in zip(self.b.members, self.probs):
            f = torch.empty(p.f0.shape, dtype=torch.float32 if m.mixed else torch.float64, device="cuda")
            m.get_f(out=f)
            out.append({"f": f, "moments": m.moments(), "totals": m.totals()})
        return out

    def close(self):
        self.b.close()


def accuracy_batch(probs, steps, shapes32, shapes64):
    """The mixed batch against the same batch in plain FP64 after `steps`
    steps from f0: per member and over all members (bins-weighted sums)."""
    import torch
    states = {}
    for prec, shapes in (("fp64", shapes64), ("mixed", shapes32)):
        r = BatchRun(probs, prec, shapes=shapes, autotune=False)
        for k in range(steps):
            r.step(k)
        torch.cuda.synchronize()
        states[prec] = r.state()
        r.close()
        del r
    members = []
    num = {"f": 0.0, "inc": 0.0, "dN": 0.0}
    den = {"f": 0.0, "inc": 0.0, "dN": 0.0}
    for p, a, b in zip(probs, states["mixed"], states["fp64"]):
        f0 = torch.as_tensor(np.ascontiguousarray(p.f0, dtype=np.float64)).cuda()
        c = compare_states(a, b, f0)
        c["problem"] = p.name
        members.append(c)
        num["f"] += float((a["f"].double() - b["f"]).abs().sum())
        den["f"] += float(b["f"].abs().sum())
        num["inc"] += float((a["f"].double() - b["f"]).abs().sum())
        den["inc"] += float((b["f"] - f0).abs().sum())
        num["dN"] += float(np.abs(a["moments"][0] - b["moments"][0]).sum())
        den["dN"] += float(np.abs(b["moments"][0]).sum())
        del f0
    return {"steps": steps, "what": "mixed batch vs the same batch in plain FP64 on this GPU",
            "rel_l1_f": num["f"] / den["f"], "rel_l1_increment": num["inc"] / den["inc"],
            "rel_l1_dN": num["dN"] / den["dN"], "members": members}


def run_batch(args, rank, world):
    """The batched form: every member's step in one CUDA-graph launch."""
    import torch
    from paper_2003_02845_gb300 import bt, workloads as W
    probs = W.config5_problems()
    mixed = args.precision == "mixed"
    fixed = args.shape.split(",") if args.shape else None
    run = BatchRun(probs, args.precision, shapes=fixed, autotune=args.autotune)
    b = run.b
    bins = sum(p.n_bins for p in probs)
    for k in range(args.warmup):
        run.step(k)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    l0, g0 = b.launch_count, b.graph_launches
    ms, clk = run.time(args.steps, 0, k0=args.warmup, clock=True)
    launches, graphs = b.launch_count - l0, b.graph_launches - g0
    if world > 1:
        ms = max_over_ranks(ms)
        torch.distributed.barrier()

    # end to end: pinned host backgrounds in, every member's source terms out
    L = bt.lib()
    pinned, outs = [], []
    for p in probs:
        pinned.append(_pinned_backgrounds(p))
        S, Z = p.n_species, p.n_zone
        outs.append([torch.empty(sh, dtype=torch.float64).pin_memory() for sh in ((S, Z), (S, Z), (S, Z, 3), (Z,))])
    h2d = sum(x.numel() * 8 for pm in pinned for x in pm[0][3:6] + pm[0][7:10])
    d2h = sum(x.numel() * 8 for o in outs for x in o)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        for m, pm in zip(b.members, pinned):
            bt._check(L.bt_set_background(m.h, bt.BT_MEM_HOST, *[x.data_ptr() for x in pm[(k + 1) % 2]]))
        b.step(run.dts)
        for m, o in zip(b.members, outs):
            bt._check(L.bt_moments(m.h, bt.BT_MEM_HOST, *[x.data_ptr() for x in o]))
    e2e_s = (time.perf_counter() - t0) / args.steps
    if world > 1:
        e2e_s = max_over_ranks(e2e_s)
    del pinned, outs

    # the dominant kernels: the largest member's, timed alone with events
    big = max(range(len(probs)), key=lambda i: probs[i].n_bins)
    m, p = b.members[big], probs[big]
    m.profile(True)
    for k in range(args.steps):
        m.set_background_device(*run.dev[big][(k + 1) % 2])
        m.step(run.dts[big])
    flux_ms, flux_n = m.profile_read(bt.K_FLUX)
    zone_ms, zone_n = m.profile_read(bt.K_ZONE)
    remap_ms, remap_n = m.profile_read(bt.K_TIME_REMAP)
    m.profile(False)
    split = bool(m.launch_shape & bt.SHAPE_SPLIT)
    face_avg = flux_ms / max(flux_n, 1)
    zone_avg = zone_ms / max(zone_n, 1) if split else None
    flux_avg = face_avg + (zone_avg or 0.0)
    shapes32 = list(run.shapes)
    alu = alu_peaks()
    run.close()
    del run, b
    torch.cuda.synchronize()

    res = {
        "metric": METRIC,
        "value": job_value(bins, world, ms),
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if mixed else "f64",
        "data": "synthetic",
        "config": {
            "workload": "config5_batched_3x2d_6species",
            "problems": [q.name for q in probs],
            "precision": args.precision + (" (f32 f/fluxes/remap; collision and sums in double-float/f64)"
                                           if mixed else ""),
            "bins_per_step": bins,
            "updates_per_s_without_species": world * sum(q.n_zone * q.n_eps * q.n_ang for q in probs) / (ms * 1e-3),
            "launch_shapes": shapes32,
            "graph_launches_per_step": graphs / args.steps,
            "l2": "inputs larger than L2 (f is %.0f MB per buffer)" % (bins * (4 if mixed else 8) / 1e6),
            "parallelism": "replicas" if world > 1 else "single GPU",
            "backgrounds": "B0/B1 alternate every step (time remap active)",
        },
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "e2e": {"value": world * bins / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "roofline": _roofline(p, mixed, "%s of %s" % (kernel_name(mixed, split), p.name), flux_avg,
                              face_avg if split else None, zone_avg, remap_ms / max(remap_n, 1), alu,
                              measured_traffic(p.name, args.precision, shapes32[big])),
    }
    if mixed and not args.no_fp64_compare:
        # the same batch in plain FP64 (float64 f, remaps, fluxes and solve)
        r64 = BatchRun(probs, "fp64", autotune=args.autotune)
        ms64, _ = r64.time(args.fp64_steps, 2)
        shapes64 = list(r64.shapes)
        r64.close()
        del r64
        res["vs_fp64_gpu"] = {"value": bins / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64,
                              "speedup": ms64 / ms, "launch_shapes": shapes64,
                              "what": "the same batched step in plain FP64 on this GPU (same kernels, T = double, "
                                      "autotuned launch shapes)"}
        if args.accuracy_steps_batch > 0:
            res["accuracy"] = accuracy_batch(probs, args.accuracy_steps_batch, shapes32, shapes64)
    if mixed and args.accuracy_steps > 0:
        res["accuracy_transport"] = accuracy_single(W.config3_transport(), args.accuracy_steps)
    if mixed and not args.no_extra:
        # the single 2D problem of config 3 (one per line is the batch's)
        a3 = argparse.Namespace(**vars(args))
        a3.shape = None
        r3, t3 = single_problem(W.config3(), a3, world, steps=min(args.steps, 10), e2e=False)
        t3.close()
        try:
            lts3 = lts_block(W.config3())
        except Exception as e:   # report, do not lose the line
            lts3 = {"error": repr(e)}
        res["extra"] = {"config3": {k: r3[k] for k in ("value", "ms_per_step")},
                        "config3_local_time_stepping": lts3,
                        "config3_launch_shape": r3["config"]["launch_shape"],
                        "config3_roofline": {k: r3["roofline"][k] for k in
                                             ("avg_launch_ms", "face_pass_avg_ms", "zone_pass_avg_ms",
                                              "time_remap_avg_ms", "frac")},
                        "config3_time_remap_hbm": r3["roofline"].get("time_remap_hbm")}
    if rank == 0 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline_multi(probs, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def cpu_baseline_multi(probs, budget_s, threads=None):
    """The oracle on a sample of every problem of a batch, budget split by
    bins; value = sampled bins / seconds."""
    tot = sum(p.n_bins for p in probs)
    done, spent, parts, cores = 0.0, 0.0, [], None
    for p in probs:
        r = cpu_baseline(p, max(1.0, budget_s * p.n_bins / tot), threads=threads)
        done += r["bins"]
        spent += r["seconds"]
        parts.append(r["sample"])
        cores = r["cores"]
    ncpu, model = host_cpu()
    return {"value": done / spent, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": model,
            "host_cpus": ncpu, "sample": "; ".join(parts)}


def cpu_baseline(prob, budget_s=15.0, threads=None):
    """The FP64 oracle (OpenMP over the host's cores unless `threads` says
    otherwise; its results do not depend on the thread count) on a bounded
    sample of zones of the same workload: one subset step, static background
    (the time remap is not in the sample)."""
    import oracle
    oracle.build()
    if threads:
        oracle.set_threads(threads)
    cores = oracle.threads()
    o = oracle.Oracle(prob)
    o.set_background(prob.backgrounds[0])
    o.set_f(prob.f0)
    dt = o.max_dt(prob.cfl)
    rng = np.random.default_rng(0)
    n = 64
    spent, done_bins = 0.0, 0
    per_zone = None
    while spent < budget_s:
        if per_zone is not None:
            # size the next chunk to the time left
            n = int(min(2 * n, prob.n_zone, max(1, (budget_s - spent) / per_zone)))
        zones = rng.choice(prob.n_zone, min(n, prob.n_zone), replace=False)
        t0 = time.perf_counter()
        o.step_zones(dt, zones)
        el = time.perf_counter() - t0
        spent += el
        done_bins += len(zones) * prob.n_species * prob.n_eps * prob.n_ang
        per_zone = el / len(zones) if el > 0.05 else None
        if per_zone is None:
            n = min(n * 2, prob.n_zone)
    ncpu, model = host_cpu()
    return {"value": done_bins / spent, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": model,
            "host_cpus": ncpu, "seconds": spent, "bins": done_bins,
            "sample": "%d zone updates (all species, groups, angles) of %s by the FP64 oracle on %d threads "
                      "in %.1f s, static background (time remap not in the sample)"
                      % (done_bins // (prob.n_species * prob.n_eps * prob.n_ang), prob.name, cores, spent)}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2003_02845_gb300 import workloads as W
    if args.workload == "config5":
        return run_reference_multi(args, W.config5_problems())
    prob = W.by_name(args.workload)
    per_step = max(2.0, 60.0 / max(args.steps + args.warmup, 1))
    for _ in range(args.warmup):
        cpu_baseline(prob, 1.0)
    vals = [cpu_baseline(prob, per_step) for _ in range(args.steps)]
    v = statistics.median(x["value"] for x in vals)
    cb = dict(vals[-1])
    cb["value"] = v
    res = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": prob.n_bins / v * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": prob.name, "precision": "fp64 oracle (CPU)"},
           "cpu_baseline": cb,
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(res), flush=True)


def run_reference_multi(args, probs):
    per_step = max(3.0, 60.0 / max(args.steps + args.warmup, 1))
    bins = sum(p.n_bins for p in probs)
    for _ in range(args.warmup):
        cpu_baseline_multi(probs, 3.0)
    vals = [cpu_baseline_multi(probs, per_step) for _ in range(args.steps)]
    v = statistics.median(x["value"] for x in vals)
    cb = dict(vals[-1])
    cb["value"] = v
    res = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": bins / v * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": "config5_batched_3x2d_6species", "precision": "fp64 oracle (CPU)"},
           "cpu_baseline": cb,
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(res), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="config5")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--accuracy-steps", type=int, default=100,
                    help="steps of the single-problem accuracy comparisons against the FP64 path (0: skip)")
    ap.add_argument("--accuracy-steps-batch", type=int, default=10,
                    help="steps of the batched workload's accuracy comparison against its FP64 batch (0: skip)")
    ap.add_argument("--fp64-steps", type=int, default=4, help="timed steps of the FP64 batch")
    ap.add_argument("--no-extra", action="store_true", help="skip the config-3 measurement of the batched line")
    ap.add_argument("--no-learned-remap", dest="learned_remap", action="store_false")
    ap.add_argument("--sur-samples", type=int, default=2_000_000)
    ap.add_argument("--sur-epochs", type=int, default=10)
    ap.add_argument("--sur-tols", type=float, nargs="+", default=[0.01, 0.05, 0.25])
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="keep the default launch shape instead of timing the candidates")
    ap.add_argument("--shape", default=None,
                    help="fixed launch shape, e.g. split/256 or fused/256 (no autotuning); for the batched "
                         "workload a comma-separated list, one per problem")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
