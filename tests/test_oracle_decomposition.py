"""Zone decomposition of the step over ranks, the form a partitioned
multi-GPU run takes: each rank owns a band of polar rows, keeps a halo of
rows on either side, advances only its own zones, and the ranks exchange
their zones after every step (here with the CPU oracle and two gloo ranks).
The face stencil reaches two zones into the neighbour (cells P-1, P, Q,
Q+1, Sec. 3.3), so with a halo of two rows the decomposed run must equal the
undecomposed one bit for bit, and with a halo of one row it must not."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N_STEPS = 4


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    from paper_2003_02845_gb300 import workloads as W
    return W.random_2d(21, n_r=6, n_theta=8, n_e=3, n_mu=4, n_phi=4, n_s=2)


def _zones(p, rows):
    return np.array([b * p.n_r + a for b in rows for a in range(p.n_r)], dtype=np.int64)


def _rank(rank, world, port, halo, out):
    import sys
    sys.path.insert(0, ROOT)
    import oracle as orc
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = _problem()
        band = p.n_theta // world
        own_rows = list(range(rank * band, (rank + 1) * band))
        keep_rows = list(range(max(0, own_rows[0] - halo), min(p.n_theta, own_rows[-1] + 1 + halo)))
        own, keep = _zones(p, own_rows), _zones(p, keep_rows)
        o = orc.Oracle(p)
        o.set_background(p.backgrounds[0])
        dt = o.max_dt(p.cfl)               # backgrounds only: the same on every rank
        f = np.zeros(p.f0.shape)
        f[:, keep] = p.f0[:, keep]         # the rest of the grid is not held
        o.set_f(f)
        for k in range(N_STEPS):
            o.set_background(p.backgrounds[(k + 1) % 2])
            new = o.step_zones(dt, own)
            # exchange: every rank's own zones to every rank, then each keeps
            # its band and halo
            mine = torch.from_numpy(np.ascontiguousarray(new[:, own]))
            parts = [torch.empty_like(mine) for _ in range(world)]
            dist.all_gather(parts, mine)
            full = np.zeros(p.f0.shape)
            for r, part in enumerate(parts):
                full[:, _zones(p, range(r * band, (r + 1) * band))] = part.numpy()
            f = np.zeros(p.f0.shape)
            f[:, keep] = full[:, keep]
            o.set_f(f)
        out[rank] = o.get_f()[:, own]
    finally:
        dist.destroy_process_group()


def _decomposed(halo, world=2):
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        ps = [ctx.Process(target=_rank, args=(r, world, port, halo, out)) for r in range(world)]
        for q in ps:
            q.start()
        for q in ps:
            q.join(300)
            assert q.exitcode == 0
        res = dict(out)
    p = _problem()
    band = p.n_theta // world
    f = np.zeros(p.f0.shape)
    for r in range(world):
        f[:, _zones(p, range(r * band, (r + 1) * band))] = res[r]
    return f


def _whole():
    import oracle as orc
    p = _problem()
    o = orc.Oracle(p)
    o.set_background(p.backgrounds[0])
    dt = o.max_dt(p.cfl)
    o.set_f(p.f0)
    for k in range(N_STEPS):
        o.set_background(p.backgrounds[(k + 1) % 2])
        o.step(dt)
    return o.get_f()


def test_two_ranks_with_a_two_row_halo_equal_the_whole_grid():
    assert np.array_equal(_decomposed(halo=2), _whole())


def test_a_one_row_halo_is_too_thin():
    assert not np.array_equal(_decomposed(halo=1), _whole())
