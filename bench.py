"""Benchmark of the transport step on GB300.

One "step" = the whole hot path on one synthetic background: the time remap
to a new background (backgrounds B0/B1 alternate every step), the fused face
fluxes + collision kernel, and the outflow/moment reductions.  The metric is
zone-group-angle updates per second (species included) of a full step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload config3]
                  [--precision mixed|fp64] [--impl ours|reference]

--workload config5 runs the batched form: three independent 2D problems of
uneven size (128x32, 256x64, 512x128 zones; 8, 12, 20 groups; 48, 80, 128
angles; 6 species) advanced by one CUDA-graph launch per step; its units are
the bins of all three problems.

--impl reference times the FP64 CPU oracle (single thread) on a bounded
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


# GB300 unit counts and clock (nominal): 152 SMs, 128 FP32 lanes per SM,
# float64 at 1/64 of the float32 rate, maximum SM clock 2070 MHz.  A fused
# multiply-add counts as two flops.
GB300_SMS, GB300_FP32_LANES, GB300_SM_GHZ = 152, 128, 2.07
FP32_PEAK_TFLOPS = GB300_SMS * GB300_FP32_LANES * 2 * GB300_SM_GHZ / 1e3
FP64_PEAK_TFLOPS = FP32_PEAK_TFLOPS / 64


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one flux
# launch from an ncu capture of this bench's small invocation, keyed by
# workload, precision and launch shape, and valid only for the kernel code
# it was taken on (a fingerprint of bt_kernels.cu without its comments and
# blank lines): changed kernel code reports null until re-captured.
# For the split form the figure is the face pass plus the zone pass: f read
# and written once plus the deposit rows (six per zone) written and read.
TRAFFIC = {
    ("config3_cc2d_256x64x12x80x3", "mixed", "split/256"):
        (208.30e6 + 1079.68e6 + 1343.23e6 + 213.29e6,
         "66e714065ec8e1e4aea82c38d28894f52b7261fc94a6273a118ebec40c77eb44"),
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
    mixed = args.precision == "mixed"
    stream = torch.cuda.Stream()
    t = bt.Transport(prob, args.precision, stream=stream)
    B = prob.backgrounds
    # device-resident copies of both backgrounds
    dev = []
    for bg in B:
        dev.append([torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64)).cuda()
                    for x in (bg.v, bg.alpha, bg.phi, bg.kappa_a, bg.kappa_s, bg.f_eq)])
    torch.cuda.synchronize()
    t.set_background(B[0])
    t.set_f(prob.f0)
    dt = t.max_dt(prob.cfl)
    if args.shape:
        t.set_launch_shape(parse_shape(args.shape))
    elif args.autotune:
        t.autotune(dt)
    shape = t.launch_shape
    bins = prob.n_bins
    units_per_step = bins

    def one_step(k):
        d = dev[(k + 1) % 2]
        t.set_background_device(*d)
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
        for k in range(args.steps):
            one_step(args.warmup + k)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    launches = t.launch_count - l0
    if world > 1:
        ms = max_over_ranks(ms)
        torch.distributed.barrier()

    # per-kernel durations with CUDA events on the transport stream
    t.profile(True)
    for k in range(args.steps):
        one_step(args.warmup + args.steps + k)
    flux_ms, flux_n = t.profile_read(bt.K_FLUX)
    zone_ms, zone_n = t.profile_read(bt.K_ZONE)
    remap_ms, remap_n = t.profile_read(bt.K_TIME_REMAP)
    t.profile(False)
    split = bool(t.launch_shape & bt.SHAPE_SPLIT)
    face_avg_ms = flux_ms / max(flux_n, 1)
    if split:
        # the split flux step: face pass + zone pass make one unit of work
        flux_ms, flux_n = flux_ms + zone_ms, flux_n

    # end to end through the C ABI with host buffers: pinned host background in,
    # source terms out, every step
    pinned = []
    for bg in B:
        pinned.append([torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64)).pin_memory()
                       for x in (bg.rho, bg.T, bg.Ye, bg.v, bg.alpha, bg.phi, bg.shift,
                                 bg.kappa_a, bg.kappa_s, bg.f_eq)])
    S, Z = prob.n_species, prob.n_zone
    outs = [torch.empty(s, dtype=torch.float64).pin_memory() for s in ((S, Z), (S, Z), (S, Z, 3), (Z,))]
    h2d = sum(x.numel() * 8 for x in pinned[0][3:6] + pinned[0][7:10])
    d2h = sum(x.numel() * 8 for x in outs)
    L = bt.lib()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        p = pinned[(k + 1) % 2]
        bt._check(L.bt_set_background(t.h, bt.BT_MEM_HOST, *[x.data_ptr() for x in p]))
        t.step(dt)
        bt._check(L.bt_moments(t.h, bt.BT_MEM_HOST, *[x.data_ptr() for x in outs]))
    e2e_s = (time.perf_counter() - t0) / args.steps
    if world > 1:
        e2e_s = max_over_ranks(e2e_s)

    peaks, peak_src = load_peaks()
    bpb = algorithmic_bytes_per_bin(prob, mixed)
    fpb = algorithmic_flops_per_bin(prob)
    flux_avg_ms = flux_ms / max(flux_n, 1)
    achieved_gbs = bins * bpb / (flux_avg_ms * 1e-3) / 1e9
    achieved_tf = bins * fpb / (flux_avg_ms * 1e-3) / 1e12
    peak_tf = FP32_PEAK_TFLOPS if mixed else FP64_PEAK_TFLOPS
    peak = hbm_peak(peaks)
    res = {
        "metric": METRIC,
        "value": job_value(units_per_step, world, ms),
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
            "workload": prob.name,
            "precision": args.precision + (" (f32 f/fluxes/remap, f64 collision and sums)" if mixed else ""),
            "zones": prob.n_zone, "groups": prob.n_eps, "angles": prob.n_ang, "species": prob.n_species,
            "bins_per_step": bins,
            "updates_per_s_without_species": world * prob.n_zone * prob.n_eps * prob.n_ang / (ms * 1e-3),
            "l2": "inputs larger than L2 (f is %.0f MB per buffer)" % (bins * (4 if mixed else 8) / 1e6),
            "parallelism": "replicas" if world > 1 else "single GPU",
            "backgrounds": "B0/B1 alternate every step (time remap active)",
            "launch_shape": bt.shape_name(t.launch_shape),
        },
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "e2e": {"value": world * units_per_step / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "roofline": {
            "kernel": kernel_name(mixed, split),
            "bound": "alu",
            "achieved": achieved_tf,
            "peak": peak_tf,
            "peak_source": "derived: %d SMs x %d FP32 lanes x 2 x %.2f GHz%s" % (
                GB300_SMS, GB300_FP32_LANES, GB300_SM_GHZ, "" if mixed else " / 64 (float64)"),
            "unit": "TFLOP/s",
            "frac": achieved_tf / peak_tf,
            "traffic": measured_traffic(prob.name, args.precision, bt.shape_name(t.launch_shape)),
            "traffic_unit": "bytes per launch (ncu dram read + write)",
            "algorithmic_flops_per_bin": fpb,
            "avg_launch_ms": flux_avg_ms,
            "face_pass_avg_ms": face_avg_ms if split else None,
            "zone_pass_avg_ms": zone_ms / max(zone_n, 1) if split else None,
            "time_remap_avg_ms": remap_ms / max(remap_n, 1),
            "hbm": {"achieved": achieved_gbs, "peak": peak, "peak_source": peak_src, "unit": "GB/s",
                    "frac": achieved_gbs / peak, "algorithmic_bytes_per_bin": bpb},
        },
    }
    if mixed and not args.no_fp64_compare:
        t.close()
        del t
        ms64 = time_fp64_path(prob, dev)
        res["vs_fp64_gpu"] = {"value": units_per_step / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64,
                              "speedup": ms64 / ms,
                              "what": "the same step in plain FP64 on this GPU (same kernels, T = double, "
                                      "autotuned launch shape)"}
    if mixed and args.accuracy_steps > 0:
        f64 = run_steps(prob, dev, "fp64", args.accuracy_steps)
        res["accuracy"] = {"steps": args.accuracy_steps,
                           "what": "rel-L1 of f against the plain FP64 GPU path (which matches the FP64 oracle to "
                                   "1e-12) after the given steps, same backgrounds and dt",
                           "mixed_rel_l1": rel_l1(run_steps(prob, dev, "mixed", args.accuracy_steps), f64)}
        if args.learned_remap:
            try:
                res["learned_remap"] = learned_remap_block(prob, dev, args, ms, f64, shape)
            except Exception as e:   # report, do not lose the line
                res["learned_remap"] = {"error": repr(e)}
        del f64
    if rank == 0 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(prob, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


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


def run_steps(prob, dev, precision, steps, sur=None, tol=0.0, stream=None, shape=None):
    """f (device tensor) after `steps` steps from f0 with the backgrounds
    alternating as in the timed run, dt from the Courant limit of B0."""
    import torch
    from paper_2003_02845_gb300 import bt
    stream = stream if stream is not None else torch.cuda.Stream()
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
    stats = t.sur_stats() if sur is not None else None
    t.close()
    return (f, stats) if sur is not None else f


def learned_remap_block(prob, dev, args, ms_exact, f64, shape):
    """Train the network on rows of the exact remap from 16 seeded background
    pairs (the workload's own backgrounds are held out), then time the step
    with it and measure its error at a few trip tolerances."""
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
    out = {"samples": n_rows, "epochs": args.sur_epochs, "batch": 4096, "launch_shape": bt.shape_name(shape),
           "loss_per_epoch": [float(x) for x in log],
           "data_seconds": t1 - t0, "train_seconds": t2 - t1, "runs": []}
    for tol in args.sur_tols:
        t = bt.Transport(prob, "mixed", stream=stream)
        t.set_launch_shape(shape)            # the exact run's launch shape
        net_s = net
        t.set_surrogate(net_s, tol)
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
        fs, (n_eval, n_trip) = run_steps(prob, dev, "mixed", args.accuracy_steps, sur=net_s, tol=tol, stream=stream,
                                         shape=shape)
        out["runs"].append({"tol_bins": tol, "ms_per_step": ms_sur, "value": prob.n_bins / (ms_sur * 1e-3),
                            "speed_vs_exact_mixed": ms_exact / ms_sur,
                            "table_kernel_ms": tab_ms / max(tab_n, 1),
                            "trip_fraction": n_trip / max(n_eval, 1),
                            "rel_l1_vs_fp64": rel_l1(fs, f64)})
        del fs
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


def run_batch(args, rank, world):
    """The batched form: every member's step in one CUDA-graph launch."""
    import torch
    from paper_2003_02845_gb300 import bt, workloads as W
    probs = W.config5_problems()
    mixed = args.precision == "mixed"
    stream = torch.cuda.Stream()
    b = bt.Batch(probs, args.precision, stream=stream)
    dev, dts = [], []
    for m, p in zip(b.members, probs):
        dev.append([[torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64)).cuda()
                     for x in (bg.v, bg.alpha, bg.phi, bg.kappa_a, bg.kappa_s, bg.f_eq)] for bg in p.backgrounds])
        m.set_background(p.backgrounds[0])
        m.set_f(p.f0)
        dts.append(m.max_dt(p.cfl))
    shapes = []
    fixed = args.shape.split(",") if args.shape else None
    for i, (m, d, dt) in enumerate(zip(b.members, dev, dts)):
        if fixed:
            m.set_launch_shape(parse_shape(fixed[min(i, len(fixed) - 1)]))
        elif args.autotune:
            m.autotune(dt)
        shapes.append(bt.shape_name(m.launch_shape))
    torch.cuda.synchronize()
    bins = sum(p.n_bins for p in probs)

    def one_step(k):
        for m, d in zip(b.members, dev):
            m.set_background_device(*d[(k + 1) % 2])
        b.step(dts)

    for k in range(args.warmup):
        one_step(k)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    l0, g0 = b.launch_count, b.graph_launches
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for k in range(args.steps):
            one_step(args.warmup + k)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    launches, graphs = b.launch_count - l0, b.graph_launches - g0
    if world > 1:
        ms = max_over_ranks(ms)
        torch.distributed.barrier()

    # end to end: pinned host backgrounds in, every member's source terms out
    L = bt.lib()
    pinned, outs = [], []
    for p in probs:
        pinned.append([[torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64)).pin_memory()
                        for x in (bg.rho, bg.T, bg.Ye, bg.v, bg.alpha, bg.phi, bg.shift,
                                  bg.kappa_a, bg.kappa_s, bg.f_eq)] for bg in p.backgrounds])
        S, Z = p.n_species, p.n_zone
        outs.append([torch.empty(sh, dtype=torch.float64).pin_memory() for sh in ((S, Z), (S, Z), (S, Z, 3), (Z,))])
    h2d = sum(x.numel() * 8 for pm in pinned for x in pm[0][3:6] + pm[0][7:10])
    d2h = sum(x.numel() * 8 for o in outs for x in o)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        for m, pm in zip(b.members, pinned):
            bt._check(L.bt_set_background(m.h, bt.BT_MEM_HOST, *[x.data_ptr() for x in pm[(k + 1) % 2]]))
        b.step(dts)
        for m, o in zip(b.members, outs):
            bt._check(L.bt_moments(m.h, bt.BT_MEM_HOST, *[x.data_ptr() for x in o]))
    e2e_s = (time.perf_counter() - t0) / args.steps
    if world > 1:
        e2e_s = max_over_ranks(e2e_s)

    # the dominant kernel: the flux kernel of the largest member, timed alone
    big = max(range(len(probs)), key=lambda i: probs[i].n_bins)
    m, p = b.members[big], probs[big]
    m.profile(True)
    for k in range(args.steps):
        m.set_background_device(*dev[big][(k + 1) % 2])
        m.step(dts[big])
    flux_ms, flux_n = m.profile_read(bt.K_FLUX)
    zone_ms, zone_n = m.profile_read(bt.K_ZONE)
    m.profile(False)
    split = bool(m.launch_shape & bt.SHAPE_SPLIT)
    face_avg_ms = flux_ms / max(flux_n, 1)
    flux_avg_ms = (flux_ms + (zone_ms if split else 0.0)) / max(flux_n, 1)
    fpb = algorithmic_flops_per_bin(p)
    bpb = algorithmic_bytes_per_bin(p, mixed)
    achieved_tf = p.n_bins * fpb / (flux_avg_ms * 1e-3) / 1e12
    achieved_gbs = p.n_bins * bpb / (flux_avg_ms * 1e-3) / 1e9
    peak_tf = FP32_PEAK_TFLOPS if mixed else FP64_PEAK_TFLOPS
    peaks, peak_src = load_peaks()
    peak = hbm_peak(peaks)
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
            "problems": [p.name for p in probs],
            "precision": args.precision + (" (f32 f/fluxes/remap, f64 collision and sums)" if mixed else ""),
            "bins_per_step": bins,
            "launch_shapes": shapes,
            "graph_launches_per_step": graphs / args.steps,
            "l2": "inputs larger than L2 (f is %.0f MB per buffer)" % (bins * (4 if mixed else 8) / 1e6),
            "parallelism": "replicas" if world > 1 else "single GPU",
            "backgrounds": "B0/B1 alternate every step (time remap active)",
        },
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "e2e": {"value": world * bins / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "roofline": {
            "kernel": "%s of %s" % (kernel_name(mixed, split), p.name),
            "bound": "alu",
            "achieved": achieved_tf,
            "peak": peak_tf,
            "peak_source": "derived: %d SMs x %d FP32 lanes x 2 x %.2f GHz%s" % (
                GB300_SMS, GB300_FP32_LANES, GB300_SM_GHZ, "" if mixed else " / 64 (float64)"),
            "unit": "TFLOP/s",
            "frac": achieved_tf / peak_tf,
            "traffic": None,
            "algorithmic_flops_per_bin": fpb,
            "avg_launch_ms": flux_avg_ms,
            "face_pass_avg_ms": face_avg_ms if split else None,
            "zone_pass_avg_ms": zone_ms / max(zone_n, 1) if split else None,
            "hbm": {"achieved": achieved_gbs, "peak": peak, "peak_source": peak_src, "unit": "GB/s",
                    "frac": achieved_gbs / peak, "algorithmic_bytes_per_bin": bpb},
        },
    }
    if rank == 0 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline_multi(probs, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(res), flush=True)
    b.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def cpu_baseline_multi(probs, budget_s):
    """The oracle on a sample of every problem of a batch, budget split by
    bins; value = sampled bins / seconds."""
    tot = sum(p.n_bins for p in probs)
    done, spent, parts = 0.0, 0.0, []
    for p in probs:
        r = cpu_baseline(p, max(1.0, budget_s * p.n_bins / tot))
        done += r["bins"]
        spent += r["seconds"]
        parts.append(r["sample"])
    return {"value": done / spent, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": "; ".join(parts)}


def cpu_baseline(prob, budget_s=15.0, steps=1):
    """The FP64 oracle, single thread, on a bounded sample of zones of the
    same workload (one subset step after the time remap has been applied)."""
    import oracle
    oracle.build()
    o = oracle.Oracle(prob)
    o.set_background(prob.backgrounds[0])
    o.set_f(prob.f0)
    dt = o.max_dt(prob.cfl)
    rng = np.random.default_rng(0)
    n = 4
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
    return {"value": done_bins / spent, "unit": UNIT, "cores": 1, "kind": "oracle",
            "seconds": spent, "bins": done_bins,
            "sample": "%d zone updates (all species, groups, angles) of %s by the single-threaded FP64 "
                      "oracle in %.1f s, static background (time remap not in the sample)"
                      % (done_bins // (prob.n_species * prob.n_eps * prob.n_ang), prob.name, spent)}


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
    ap.add_argument("--workload", default="config3")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--accuracy-steps", type=int, default=100,
                    help="steps of the accuracy comparison against the FP64 path (0: skip)")
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
