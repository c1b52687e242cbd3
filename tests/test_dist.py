"""Multi-rank host logic on CPU with gloo, world_size 2: strip partition,
map all-reduce and timing max; a strip-sharded map (oracle per rank, summed
over ranks) equals the single-process map."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2211_00354_gb300 import dist as ldist
from paper_2211_00354_gb300 import synth


def test_row_strips_cover_exactly_once():
    for ny in (1, 7, 100, 3493):
        for world in (1, 2, 3, 8):
            s = ldist.row_strips(ny, world)
            assert len(s) == world
            covered = [r for r0, n in s for r in range(r0, r0 + n)]
            assert covered == list(range(ny))
            sizes = [n for _, n in s]
            assert max(sizes) - min(sizes) <= 1


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        f = synth.config_uniform(seed=3, n=300, kappa_star=0.4, kappa_s=0.05, gamma=0.2)
        grid = synth.Grid(x0=-3.0, y0=-3.0, h=0.05, nx=120, ny=120)
        box = (-1.0, 1.0, -1.0, 1.0)
        r0, n = ldist.row_strips(grid.ny, world)[rank]
        g = ldist.strip_grid(grid, r0, n)
        y = oracle.deflect(f.stars, f.masses, f.kappa_s, f.gamma, g.corners().reshape(-1, 2))
        mp_, st = oracle.ipm_map(y.reshape(g.ny + 1, g.nx + 1, 2), g.h, box, 30, 30)
        t = torch.tensor(mp_)
        ldist.allreduce_map(t)
        led = ldist.allreduce_ledger(st, ("area_total", "area_in_map", "area_outside"), "cpu")
        tmax = ldist.max_over_ranks(1.0 + rank, "cpu")
        if rank == 0:
            q.put((t.numpy(), led, tmax))
    finally:
        dist.destroy_process_group()


def test_strip_sharded_map_equals_single_map():
    import oracle
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = q.get(timeout=300)
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    mp_sum, led, tmax = got
    f = synth.config_uniform(seed=3, n=300, kappa_star=0.4, kappa_s=0.05, gamma=0.2)
    grid = synth.Grid(x0=-3.0, y0=-3.0, h=0.05, nx=120, ny=120)
    y = oracle.deflect(f.stars, f.masses, f.kappa_s, f.gamma, grid.corners().reshape(-1, 2))
    ref, st = oracle.ipm_map(y.reshape(grid.ny + 1, grid.nx + 1, 2), grid.h,
                             (-1.0, 1.0, -1.0, 1.0), 30, 30)
    np.testing.assert_allclose(mp_sum, ref, rtol=1e-12, atol=1e-12)
    assert led["area_total"] == pytest.approx(st["area_total"], rel=1e-12)
    assert led["area_in_map"] == pytest.approx(st["area_in_map"], rel=1e-10)
    assert tmax == 2.0
