"""One domain over several GPUs: a decomposition into horizontal slabs (rows of
y) with ghost rows, for the single large grid (the 1024 x 4096 rising bubble).

Why ghost rows of the whole state. One time step of a cell reads the state up to
three rows away: phi = sum h (Eq. 18) at distance two feeds mu (Eqs. 8, 30b) at
distance one, whose gradient and Laplacian (Eq. 30) feed the collision of the
neighbour, which streams into the cell (Eqs. 10, 24); the pressure of the
previous step enters through its gradient (one row). So a slab that holds
G = 3k rows of its neighbours' state on each inner side (ghost rows) advances
its own rows exactly -- the same arithmetic on the same values as the undivided
grid -- for k steps, whatever happens at its outer edge meanwhile. The step
kernels are used unchanged: every slab is an ordinary walled instance whose
inner edges lie inside the ghost bands (the wall treatment there only spoils
ghost rows, 3 rows a step). After k steps each slab sends its first and last G
own rows to its neighbours, which overwrite their ghost rows with them
(lbm_pack_rows / lbm_unpack_rows move every stored plane of those rows); then
the next k steps. One exchange every k steps of 2 x G rows of state per inner
boundary (21 words a cell, FP32: 3 k x 1024 x 84 bytes a message on the
1024-wide grid), in exchange for 2 G rows of redundant computation per slab.

Transports: all slabs in one process (several instances of one context on one
GPU, exchanged with device-to-device copies: the single-GPU check of the
decomposition) or one slab per rank with torch.distributed point-to-point
messages (NCCL between GPUs; gloo on CPU for the tests). Each rank posts its
sends and receives in the same order (to the lower neighbour, to the upper, from
the upper, from the lower), so pairs of ranks match messages in order even where
both neighbours are one rank (two ranks with periodic y).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Dict, List, Optional, Sequence

import numpy as np

# rows one time step reaches: h two rows out (phi for mu), mu one row (stencil
# of the collision), then streaming one row
REACH = 3


@dataclass(frozen=True)
class Slab:
    """Rows [y0, y1) of the global grid owned by one rank, plus `lo` ghost rows
    below and `hi` above in its local grid (local row j = global y0 - lo + j,
    wrapped for periodic y)."""
    rank: int
    y0: int
    y1: int
    lo: int
    hi: int

    @property
    def own(self) -> int:
        return self.y1 - self.y0

    @property
    def ny_local(self) -> int:
        return self.lo + self.own + self.hi


def plan(ny: int, world: int, ghost: int, periodic: bool) -> List[Slab]:
    """Even split of ny rows over `world` slabs (the first ny % world get one row
    more), with `ghost` rows (a multiple of REACH) on every inner side."""
    if world < 1 or ny < 1:
        raise ValueError("need ny >= 1 and world >= 1")
    if ghost < REACH or ghost % REACH:
        raise ValueError("ghost rows must be a positive multiple of %d" % REACH)
    base, extra = divmod(ny, world)
    out, y = [], 0
    for r in range(world):
        own = base + (1 if r < extra else 0)
        inner_lo = world > 1 and (periodic or r > 0)
        inner_hi = world > 1 and (periodic or r < world - 1)
        if world > 1 and own < ghost:
            raise ValueError("slab of %d rows is thinner than its %d ghost rows" % (own, ghost))
        out.append(Slab(r, y, y + own, ghost if inner_lo else 0, ghost if inner_hi else 0))
        y += own
    return out


def steps_between_exchanges(ghost: int) -> int:
    return ghost // REACH


def local_config(cfg: dict, slab: Slab, world: int) -> dict:
    """Parameters of one slab's local grid: the global ones with ny of the slab;
    walls in y unless the undivided periodic grid is kept whole (world 1)."""
    c = dict(cfg)
    c["ny"] = slab.ny_local
    if world > 1:
        c["walls_y"] = 1
    c["name"] = "%s_slab%d" % (cfg.get("name", "grid"), slab.rank)
    return c


def local_rows(slab: Slab, ny: int) -> np.ndarray:
    """Global row of each local row."""
    return (slab.y0 - slab.lo + np.arange(slab.ny_local)) % ny


def local_field(field: np.ndarray, slab: Slab) -> np.ndarray:
    """Rows of a global (ny, nx) field for one slab's local grid."""
    return np.ascontiguousarray(field[local_rows(slab, field.shape[0])])


class SlabRun:
    """Advances the slabs this process holds and keeps their ghost rows fresh.

    backends: {rank: backend} for the slabs held here (all of them for a local
    run, this rank's for a distributed one). A backend has pack(y, nrows) ->
    tensor, unpack(y, nrows, tensor), empty(nrows) -> a receive buffer, and
    `stepper`, the object whose step(n) advances it (slabs sharing one context
    share one stepper, stepped once a round); rows are local rows.
    group: torch.distributed group for slabs held elsewhere (None: all slabs
    are local)."""

    def __init__(self, slabs: Sequence[Slab], ghost: int, backends: Dict[int, object], periodic: bool,
                 group=None):
        self.slabs = list(slabs)
        self.world = len(self.slabs)
        self.ghost = ghost
        self.k = steps_between_exchanges(ghost)
        self.backends = backends
        self.periodic = periodic
        self.group = group
        self.steps_since = 0

    def _down(self, r: int) -> Optional[int]:
        if r > 0:
            return r - 1
        return self.world - 1 if self.periodic and self.world > 1 else None

    def _up(self, r: int) -> Optional[int]:
        if r < self.world - 1:
            return r + 1
        return 0 if self.periodic and self.world > 1 else None

    def exchange(self):
        """Every slab's first and last `ghost` own rows into its neighbours'
        ghost rows."""
        if self.world == 1:
            return
        G = self.ghost
        outgoing = {}   # (from, to, direction) -> tensor
        for r, b in self.backends.items():
            s = self.slabs[r]
            if self._down(r) is not None:
                outgoing[(r, self._down(r), "down")] = b.pack(s.lo, G)
            if self._up(r) is not None:
                outgoing[(r, self._up(r), "up")] = b.pack(s.lo + s.own - G, G)
        incoming = {}
        remote = [key for key in outgoing if key[1] not in self.backends]
        needs = []   # (to, from, direction) this process receives from elsewhere
        for r in self.backends:
            up, dn = self._up(r), self._down(r)
            if up is not None and up not in self.backends:
                needs.append((r, up, "down"))   # the upper neighbour's message going down
            if dn is not None and dn not in self.backends:
                needs.append((r, dn, "up"))
        if remote or needs:
            incoming = self._transfer(outgoing, needs)
        for r, b in self.backends.items():
            s = self.slabs[r]
            up, dn = self._up(r), self._down(r)
            if up is not None:   # top ghost rows from the upper neighbour's lowest own rows
                t = outgoing.get((up, r, "down")) if up in self.backends else incoming[(r, up, "down")]
                b.unpack(s.lo + s.own, G, t)
            if dn is not None:   # bottom ghost rows from the lower neighbour's highest own rows
                t = outgoing.get((dn, r, "up")) if dn in self.backends else incoming[(r, dn, "up")]
                b.unpack(0, G, t)

    def _transfer(self, outgoing, needs):
        import torch.distributed as dist
        ops, incoming = [], {}
        tag = {"down": 0, "up": 1}
        for r in self.backends:   # one slab per rank in a distributed run
            dn, up = self._down(r), self._up(r)
            for peer, d in ((dn, "down"), (up, "up")):
                if peer is not None and peer not in self.backends:
                    ops.append(dist.P2POp(dist.isend, outgoing[(r, peer, d)], peer, self.group, tag[d]))
            for peer, d in ((up, "down"), (dn, "up")):
                if peer is not None and (r, peer, d) in needs:
                    buf = self.backends[r].empty(self.ghost)
                    incoming[(r, peer, d)] = buf
                    ops.append(dist.P2POp(dist.irecv, buf, peer, self.group, tag[d]))
        for w in dist.batch_isend_irecv(ops):
            w.wait()
        return incoming

    def start(self):
        """Fills the ghost rows once after initialisation (the outermost ghost row
        of a fresh slab was initialised next to its local wall)."""
        self.exchange()
        self.steps_since = 0

    def advance(self, nsteps: int):
        while nsteps > 0:
            j = min(self.k - self.steps_since, nsteps)
            steppers = []
            for b in self.backends.values():
                if not any(b.stepper is t for t in steppers):
                    steppers.append(b.stepper)
            for t in steppers:
                t.step(j)
            self.steps_since += j
            nsteps -= j
            if self.steps_since == self.k:
                self.exchange()
                self.steps_since = 0

    def own_rows(self, r: int, local: np.ndarray) -> np.ndarray:
        """The own rows of slab r of a local array whose second-to-last axis is y."""
        s = self.slabs[r]
        return local[..., s.lo:s.lo + s.own, :]


class GpuSlab:
    """Backend: instance `instance` of a liblbm Simulation (several slabs may be
    instances of one context on one GPU; the Simulation is then their common
    stepper). Pack and unpack run on the context's stream."""

    def __init__(self, lbm, sim, instance: int):
        import torch
        self.lbm, self.sim, self.k = lbm, sim, instance
        self.stepper = sim
        self.row_bytes = lbm.lbm_row_bytes(sim.ctx, instance)
        self.device = torch.device("cuda", torch.cuda.current_device())

    def empty(self, nrows: int):
        import torch
        return torch.empty(nrows * self.row_bytes, dtype=torch.uint8, device=self.device)

    def pack(self, y: int, nrows: int):
        buf = self.empty(nrows)
        self.lbm.lbm_pack_rows(self.sim.ctx, self.k, y, nrows, buf.data_ptr(), buf.numel())
        return buf

    def unpack(self, y: int, nrows: int, buf):
        self.lbm.lbm_unpack_rows(self.sim.ctx, self.k, y, nrows, buf.data_ptr(), buf.numel())
