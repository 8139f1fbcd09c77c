"""A few transport steps of one workload at a fixed launch shape, for ncu
captures of single kernels (the benchmark's own runs autotune and time many
launches, which a capture should not replay):

  python -m paper_2003_02845_gb300.profiling WORKLOAD PRECISION SHAPE STEPS

WORKLOAD: config2, config3, config3_transport, or config5_largest_NRxNT (the
largest problem of the batched workload -- 20 groups, 16 x 8 angles, 6
species -- on NR x NT zones; config5_largest_512x128 is the full member, a
smaller grid keeps a capture within a few GB).  PRECISION: mixed or fp64.
SHAPE: fused/256, split/256, split/512, ...  The backgrounds alternate every
step, so the time remap runs in each.
"""
from __future__ import annotations

import sys


def problem(name: str):
    from . import workloads as W
    if name.startswith("config5_largest_"):
        nr, nt = (int(x) for x in name[len("config5_largest_"):].split("x"))
        return W.cc2d(nr, nt, 20, 16, 8, (1.0, 0.5, 0.2, 0.2, 0.2, 0.2), W.BASE_SEED + 7,
                      "config5_p2_512x128x20x128x6" if (nr, nt) == (512, 128) else name)
    return W.by_name(name)


def main(argv):
    import torch
    from . import build, bt
    build.build()
    name, precision, shape, steps = argv[0], argv[1], argv[2], int(argv[3])
    p = problem(name)
    t = bt.Transport(p, precision)
    form, nt = shape.split("/")
    t.set_launch_shape((bt.SHAPE_SPLIT if form == "split" else 0) | int(nt))
    t.set_background(p.backgrounds[0])
    t.set_f(p.f0)
    dt = t.max_dt(p.cfl)
    for k in range(steps):
        t.set_background(p.backgrounds[(k + 1) % 2])
        t.step(dt)
    torch.cuda.synchronize()
    print("%s %s %s: %d steps, %d launches, %d bins" % (p.name, precision, shape, steps, t.launch_count, p.n_bins))


if __name__ == "__main__":
    main(sys.argv[1:])
