"""The slab decomposition of one domain (paper_1902_08933_gb300/slab.py) on CPU.

Every slab is advanced by the FP64 oracle standing in for its GPU; the ghost-row
exchange (which rows, when, into which rows of which neighbour) is the same code
the GPU path runs. The slabs' own rows must equal the undivided oracle run bit
for bit: the decomposition changes which process computes a cell, never the
arithmetic on it. Walled bubble (the benchmark's boundaries) and periodic
droplet, 2 and 3 slabs, an exchange every step (3 ghost rows) or every second
step (6), single process and world-size-2/3 gloo ranks.
"""
import multiprocessing as mp
import os
import socket
import time

import numpy as np
import pytest

from paper_1902_08933_gb300 import slab
from paper_1902_08933_gb300 import workloads as wl

STEPS = 11


class OracleSlab:
    """Backend for SlabRun: one slab's oracle state (FP64), rows packed as the
    planes h (9), g (9), phi u (2), p (1), each slab row contiguous."""

    def __init__(self, orc, cfg, phi0):
        self.orc = orc
        self.P = orc.params(cfg)
        self.st = orc.init(self.P, phi0)
        self.nx = cfg["nx"]
        self.stepper = self

    def step(self, n):
        self.orc.step(self.P, self.st, n)

    def _arrays(self):
        return [self.st["h"], self.st["g"], self.st["phiu_prev"], self.st["p_prev"][None]]

    def empty(self, nrows):
        import torch
        return torch.empty(21 * nrows * self.nx, dtype=torch.float64)

    def pack(self, y, nrows):
        import torch
        return torch.from_numpy(np.concatenate([a[:, y:y + nrows, :].ravel() for a in self._arrays()]))

    def unpack(self, y, nrows, t):
        flat, off = t.numpy(), 0
        for a in self._arrays():
            n = a.shape[0] * nrows * a.shape[2]
            a[:, y:y + nrows, :] = flat[off:off + n].reshape(a.shape[0], nrows, a.shape[2])
            off += n


def _case(name):
    if name == "bubble":   # walls in y, as the 1024 x 4096 benchmark
        cfg = wl.rising_bubble(nx=20, ny=44, R=6.0, cy=15.0, W=4.0, Re=5.0)
    else:                  # periodic in y
        cfg = wl.static_droplet(n=30, R=8.0)
    rng = np.random.default_rng(5)
    phi0 = np.clip(wl.initial_phi(cfg) + 0.01 * rng.standard_normal((cfg["ny"], cfg["nx"])), 0, 1)
    return cfg, phi0


def _reference(orc, cfg, phi0, n):
    P = orc.params(cfg)
    st = orc.init(P, phi0)
    orc.step(P, st, n)
    return st


def _own(st, s):
    return {k: np.ascontiguousarray(st[k][..., s.lo:s.lo + s.own, :]) for k in ("h", "g", "phiu_prev", "p_prev")}


def test_plan_geometry():
    s = slab.plan(4096, 4, 6, periodic=False)
    assert [(x.y0, x.y1, x.lo, x.hi) for x in s] == [(0, 1024, 0, 6), (1024, 2048, 6, 6),
                                                     (2048, 3072, 6, 6), (3072, 4096, 6, 0)]
    s = slab.plan(10, 3, 3, periodic=True)
    assert [(x.y0, x.y1, x.lo, x.hi) for x in s] == [(0, 4, 3, 3), (4, 7, 3, 3), (7, 10, 3, 3)]
    assert list(slab.local_rows(s[0], 10)) == [7, 8, 9, 0, 1, 2, 3, 4, 5, 6]
    one = slab.plan(50, 1, 3, periodic=True)[0]
    assert (one.lo, one.hi, one.ny_local) == (0, 0, 50)
    assert slab.steps_between_exchanges(9) == 3
    with pytest.raises(ValueError):
        slab.plan(10, 4, 3, periodic=False)    # 2- and 3-row slabs thinner than 3 ghost rows
    with pytest.raises(ValueError):
        slab.plan(100, 2, 4, periodic=False)   # not a multiple of the 3-row reach


def test_ghosts_must_cover_the_reach(orc):
    # Planted mistake: with only 2 ghost rows refreshed every step (one row
    # short of the 3-row reach of a step), the slabs' own rows drift from the
    # undivided run -- the tests below would catch a geometry off by one.
    cfg, phi0 = _case("bubble")
    ref = _reference(orc, cfg, phi0, STEPS)
    slabs = slab.plan(cfg["ny"], 2, 3, periodic=False)
    short = [slab.Slab(x.rank, x.y0, x.y1, min(x.lo, 2), min(x.hi, 2)) for x in slabs]
    backends = {x.rank: OracleSlab(orc, slab.local_config(cfg, x, 2), slab.local_field(phi0, x)) for x in short}
    run = slab.SlabRun(short, 3, backends, periodic=False)
    run.ghost = 2
    run.start()
    run.advance(STEPS)
    diff = max(np.max(np.abs(_own(backends[x.rank].st, x)["h"] - ref["h"][:, x.y0:x.y1, :])) for x in short)
    assert diff > 0


@pytest.mark.parametrize("case", ["bubble", "droplet"])
@pytest.mark.parametrize("world,ghost", [(2, 3), (3, 6), (2, 6)])
def test_local_slabs_equal_undivided_run(orc, case, world, ghost):
    cfg, phi0 = _case(case)
    periodic = not cfg["walls_y"]
    ref = _reference(orc, cfg, phi0, STEPS)
    slabs = slab.plan(cfg["ny"], world, ghost, periodic)
    backends = {x.rank: OracleSlab(orc, slab.local_config(cfg, x, world), slab.local_field(phi0, x))
                for x in slabs}
    run = slab.SlabRun(slabs, ghost, backends, periodic)
    run.start()
    run.advance(4)
    run.advance(STEPS - 4)     # a call that starts between two exchanges
    for x in slabs:
        got = _own(backends[x.rank].st, x)
        for k in got:
            assert np.array_equal(got[k], ref[k][..., x.y0:x.y1, :]), (case, world, ghost, x.rank, k)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir, case, ghost):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), OMP_NUM_THREADS="1")
    import datetime
    import torch.distributed as dist
    from oracle import oracle as orc
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=30))
    try:
        cfg, phi0 = _case(case)
        periodic = not cfg["walls_y"]
        slabs = slab.plan(cfg["ny"], world, ghost, periodic)
        me = slabs[rank]
        b = OracleSlab(orc, slab.local_config(cfg, me, world), slab.local_field(phi0, me))
        run = slab.SlabRun(slabs, ghost, {rank: b}, periodic, group=dist.group.WORLD)
        run.start()
        run.advance(STEPS)
        np.savez(os.path.join(outdir, "rank%d.npz" % rank), **_own(b.st, me))
    finally:
        dist.destroy_process_group()


def _launch(world, outdir, case, ghost, timeout=120):
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, str(outdir), case, ghost))
             for r in range(world)]
    for p in procs:
        p.start()
    deadline = time.time() + timeout
    for p in procs:
        p.join(max(1.0, deadline - time.time()))
    alive = [p for p in procs if p.is_alive()]
    for p in alive:
        p.kill()
        p.join()
    assert not alive, "a rank did not finish in time"
    return [p.exitcode for p in procs]


@pytest.mark.parametrize("case,world,ghost", [("bubble", 2, 3), ("droplet", 2, 6), ("bubble", 3, 6)])
def test_gloo_ranks_equal_undivided_run(orc, tmp_path, case, world, ghost):
    assert _launch(world, tmp_path, case, ghost) == [0] * world
    cfg, phi0 = _case(case)
    ref = _reference(orc, cfg, phi0, STEPS)
    for x in slab.plan(cfg["ny"], world, ghost, not cfg["walls_y"]):
        got = np.load(tmp_path / ("rank%d.npz" % x.rank))
        for k in ("h", "g", "phiu_prev", "p_prev"):
            assert np.array_equal(got[k], ref[k][..., x.y0:x.y1, :]), (case, x.rank, k)
