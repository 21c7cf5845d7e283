"""One grid split into z-slabs (domain decomposition).

L(u) of Eq. 2 at a cell reads the r neighbouring cells along each axis
(Sec. 1, after Eq. 2), and the global Lax-Friedrichs speeds of Sec. 1.2 are
maxima over the whole grid.  So a grid cut into z-slabs advances exactly like
the whole grid if, before every RK stage, each slab's r ghost planes per side
hold the neighbouring slab's planes of that stage's input (or the boundary
rule's values at the two ends), and every speed slot is max-reduced over the
slabs after the stage that fills it.  That is one halo exchange and one
3-double max-reduce per RK stage.

A slab is a ``Hydro`` handle made with ``bc[2] = BC_HALO`` (any object with
the same six methods -- halo_doubles, halo_pack, halo_unpack,
halo_fill_outflow, stage, speed_slot -- works, which is how the protocol is
tested on CPU).  Two exchanges implement the protocol:

* ``LocalExchange``: several slabs driven by this process (one GPU, or CPU
  stand-ins); packs go through staging buffers, the max is taken here.
* ``DistExchange``: one slab per rank of a ``torch.distributed`` group;
  packs travel by point-to-point send/recv to the two z-neighbours and the
  speeds by an all-reduce(MAX).  Buffers live where the backend wants them
  (CUDA for NCCL, host for gloo).

``SlabDomain`` drives the stage protocol for either.
"""
import numpy as np

from ._binding import BC_HALO, BC_OUTFLOW, BC_PERIODIC, Hydro

STENCIL_HALF_WIDTH = {5: 3, 7: 4, 2: 2}


def slab_bounds(nz, nslabs, min_planes=1):
    """Contiguous, balanced z ranges [(z0, z1), ...] covering 0..nz."""
    if nslabs < 1 or nz < nslabs * min_planes:
        raise ValueError("cannot cut %d planes into %d slabs of >= %d planes" % (nz, nslabs, min_planes))
    q, r = divmod(nz, nslabs)
    out, z = [], 0
    for i in range(nslabs):
        k = q + (1 if i < r else 0)
        out.append((z, z + k))
        z += k
    return out


def make_slab(g, z0, z1, stream=None):
    """A halo handle for planes z0..z1 of the workloads.Grid g (same x/y,
    dx, scheme, splitting and charges; origin shifted to the slab)."""
    origin = (g.origin[0], g.origin[1], g.origin[2] + z0 * g.dx[2])
    return Hydro((g.n[0], g.n[1], z1 - z0), g.dx, scheme=g.scheme, bc=(g.bc[0], g.bc[1], BC_HALO), cs2=g.cs2,
                 cfl=g.cfl, eps=g.eps, origin=origin, dt_fixed=getattr(g, "dt_fixed", 0.0),
                 split=getattr(g, "split", 0), nq=getattr(g, "nq", 1), limiter=getattr(g, "limiter", 0),
                 musta_stages=getattr(g, "musta_stages", 2), charwise=getattr(g, "charwise", 0),
                 eos_mass=getattr(g, "mass", 0.0), stream=stream)


def _zeros(n, device):
    if device is None:
        return np.zeros(n)
    import torch
    return torch.zeros(n, dtype=torch.float64, device=device)


class LocalExchange:
    """Exchange among slabs that this process drives, listed bottom to top.

    zbc: the whole grid's z rule (BC_OUTFLOW or BC_PERIODIC).
    device: None for host staging buffers, else a torch device."""

    def __init__(self, slabs, zbc, device=None):
        if zbc not in (BC_OUTFLOW, BC_PERIODIC):
            raise ValueError("zbc must be BC_OUTFLOW or BC_PERIODIC")
        self.slabs, self.zbc, self.device = list(slabs), zbc, device
        self.lo = [_zeros(s.halo_doubles(), device) for s in self.slabs]
        self.hi = [_zeros(s.halo_doubles(), device) for s in self.slabs]
        self.spd = [_zeros(3, device) for _ in self.slabs]

    def exchange(self, level):
        S, n = self.slabs, len(self.slabs)
        for i, s in enumerate(S):
            s.halo_pack(level, 0, self.lo[i])
            s.halo_pack(level, 1, self.hi[i])
        for i, s in enumerate(S):
            if i > 0 or self.zbc == BC_PERIODIC:
                s.halo_unpack(level, 0, self.hi[(i - 1) % n])
            else:
                s.halo_fill_outflow(level, 0)
            if i < n - 1 or self.zbc == BC_PERIODIC:
                s.halo_unpack(level, 1, self.lo[(i + 1) % n])
            else:
                s.halo_fill_outflow(level, 1)

    def reduce_speeds(self, slot):
        for s, b in zip(self.slabs, self.spd):
            s.speed_slot(slot, b)
        if self.device is None:
            m = np.max(np.stack(self.spd), axis=0)
        else:
            import torch
            m = torch.amax(torch.stack(self.spd), dim=0).contiguous()
        for s in self.slabs:
            s.speed_slot(slot, m, write=True)


class DistExchange:
    """Exchange for one slab per rank: rank k holds the k-th slab from the
    bottom of the grid.  dist is an initialised torch.distributed; device is
    where the message buffers live (a CUDA device for NCCL, None for host).

    With device buffers the slab must run on torch's current stream (make it
    with stream=None): packs and unpacks are queued on that stream, and the
    NCCL send/recv and all-reduce order themselves after it and make it wait
    for their results.  Host buffers synchronise inside pack/read."""

    TAG_DOWN, TAG_UP = 1, 2

    def __init__(self, slab, rank, world, zbc, dist, device=None):
        if zbc not in (BC_OUTFLOW, BC_PERIODIC):
            raise ValueError("zbc must be BC_OUTFLOW or BC_PERIODIC")
        import torch
        self.torch, self.dist = torch, dist
        self.slab, self.rank, self.world, self.zbc = slab, rank, world, zbc
        dev = device if device is not None else "cpu"
        n = slab.halo_doubles()
        mk = lambda k: torch.zeros(k, dtype=torch.float64, device=dev)  # noqa: E731
        self.send_lo, self.send_hi, self.recv_lo, self.recv_hi = mk(n), mk(n), mk(n), mk(n)
        self.spd = mk(3)
        per = zbc == BC_PERIODIC
        self.down = (rank - 1) % world if (rank > 0 or per) else None
        self.up = (rank + 1) % world if (rank < world - 1 or per) else None

    def exchange(self, level):
        s, P2P = self.slab, self.dist.P2POp
        s.halo_pack(level, 0, self.send_lo)
        s.halo_pack(level, 1, self.send_hi)
        if self.world == 1:                 # periodic grid held by one slab
            if self.down is not None:
                s.halo_unpack(level, 0, self.send_hi)
                s.halo_unpack(level, 1, self.send_lo)
            else:
                s.halo_fill_outflow(level, 0)
                s.halo_fill_outflow(level, 1)
            return
        ops = []
        # same order on every rank: send down, send up, receive from up, from down
        if self.down is not None:
            ops.append(P2P(self.dist.isend, self.send_lo, self.down, tag=self.TAG_DOWN))
        if self.up is not None:
            ops.append(P2P(self.dist.isend, self.send_hi, self.up, tag=self.TAG_UP))
        if self.up is not None:
            ops.append(P2P(self.dist.irecv, self.recv_hi, self.up, tag=self.TAG_DOWN))
        if self.down is not None:
            ops.append(P2P(self.dist.irecv, self.recv_lo, self.down, tag=self.TAG_UP))
        for r in self.dist.batch_isend_irecv(ops):
            r.wait()
        if self.down is not None:
            s.halo_unpack(level, 0, self.recv_lo)
        else:
            s.halo_fill_outflow(level, 0)
        if self.up is not None:
            s.halo_unpack(level, 1, self.recv_hi)
        else:
            s.halo_fill_outflow(level, 1)

    def reduce_speeds(self, slot):
        self.slab.speed_slot(slot, self.spd)
        if self.world > 1:
            self.dist.all_reduce(self.spd, op=self.dist.ReduceOp.MAX)
        self.slab.speed_slot(slot, self.spd, write=True)


class SlabDomain:
    """Drive the slabs of an exchange through RK3 steps, stage by stage."""

    def __init__(self, exchange):
        self.ex = exchange
        self.slabs = exchange.slabs if hasattr(exchange, "slabs") else [exchange.slab]

    def loaded(self):
        """Call once after every slab's state is set: slot 0 becomes global."""
        self.ex.reduce_speeds(0)

    def step(self, nsteps=1, t_end=-1.0):
        for _ in range(int(nsteps)):
            for s in self.slabs:
                s.stage(0, t_end)
            for st in (1, 2, 3):
                self.ex.exchange(st - 1)
                for s in self.slabs:
                    s.stage(st)
                self.ex.reduce_speeds(st)
            for s in self.slabs:
                s.stage(4)


def split_grid(g, nslabs, stream=None):
    """Slab handles and their z ranges for the workloads.Grid g cut into
    nslabs z-slabs (each at least the stencil half-width thick)."""
    G = STENCIL_HALF_WIDTH[g.scheme]
    bounds = slab_bounds(g.n[2], nslabs, G)
    return [make_slab(g, z0, z1, stream) for z0, z1 in bounds], bounds
