"""The z-slab protocol of paper_1604_03360_gb300.domain on CPU.

Each slab is a CPU stand-in for a halo handle: it keeps its nz interior
planes plus G ghost planes per side for the three RK levels and applies the
oracle's L(u) (Eq. 2) to the padded slab, so its interior cells see exactly
the cells the whole grid would give them once the ghost planes are filled.
Driven by the same exchange code as the GPU slabs -- in one process
(LocalExchange) and as world-size-2 gloo ranks (DistExchange) -- the slabs
must reproduce the oracle's whole-grid run bit for bit."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import workloads as W
from paper_1604_03360_gb300.domain import (STENCIL_HALF_WIDTH, DistExchange, LocalExchange, SlabDomain,
                                           slab_bounds)


def _np(buf):
    return buf.numpy() if isinstance(buf, torch.Tensor) else buf


class OracleSlab:
    """Planes z0..z1 of grid g, with the six methods of a halo handle."""

    def __init__(self, g, z0, z1):
        self.g, self.G, self.nz = g, STENCIL_HALF_WIDTH[g.scheme], z1 - z0
        nx, ny = g.n[0], g.n[1]
        self.nf = 4 + g.nq
        mk = lambda nz: oracle.make_cfg((nx, ny, nz), g.dx, cs2=g.cs2, scheme=g.scheme,  # noqa: E731
                                        bc=(g.bc[0], g.bc[1], 0), cfl=g.cfl, eps=g.eps)
        self.c_ext, self.c_int = mk(self.nz + 2 * self.G), mk(self.nz)
        self.U = [np.zeros((self.nf, self.nz + 2 * self.G, ny, nx)) for _ in range(3)]
        self.slots = np.zeros((4, 3))
        self.dt, self.t, self.steps = 0.0, 0.0, 0

    def interior(self, level=0):
        return self.U[level][:, self.G:self.G + self.nz]

    def set_primitive(self, w, t=0.0):
        self.interior()[...] = oracle.prim2con(np.ascontiguousarray(w), self.g.cs2)
        self.slots[0] = oracle.alpha(self.c_int, np.ascontiguousarray(self.interior()))
        self.t, self.steps = t, 0

    def halo_doubles(self):
        return self.nf * self.G * self.g.n[0] * self.g.n[1]

    def halo_pack(self, level, side, buf):
        z = self.nz if side else self.G
        _np(buf)[:] = self.U[level][:, z:z + self.G].reshape(-1)

    def halo_unpack(self, level, side, buf):
        z = self.G + self.nz if side else 0
        self.U[level][:, z:z + self.G] = _np(buf).reshape(self.nf, self.G, self.g.n[1], self.g.n[0])

    def halo_fill_outflow(self, level, side):
        src = self.G + self.nz - 1 if side else self.G
        z = self.G + self.nz if side else 0
        self.U[level][:, z:z + self.G] = self.U[level][:, src:src + 1]

    def stage(self, which, t_end=-1.0):
        if which == 0:
            # dt from the speeds of u^n: CFL x min dx over the active axes / max speed
            act = [d for d in range(3) if self.g.n[d] > 1]
            dt = self.g.cfl * min(self.g.dx[d] for d in act) / max(self.slots[0][d] for d in act)
            if t_end >= 0 and self.t + dt > t_end:
                dt = t_end - self.t
            self.dt = dt if dt > 0 else 0.0
            self.slots[1:] = 0.0
        elif which in (1, 2, 3):
            if not self.dt > 0:
                return
            us = self.U[which - 1]
            Lu = oracle.L(self.c_ext, us, self.slots[which - 1])
            G, nz = self.G, self.nz
            s = us[:, G:G + nz] + self.dt * Lu[:, G:G + nz]
            un = self.interior(0)
            a, b = ((0.0, 1.0), (0.75, 0.25), (1.0 / 3.0, 2.0 / 3.0))[which - 1]
            out = s if a == 0.0 else a * un + b * s
            self.interior(which % 3)[...] = out
            self.slots[which] = oracle.alpha(self.c_int, np.ascontiguousarray(out))
        elif which == 4 and self.dt > 0:
            self.slots[0] = self.slots[3]
            self.t += self.dt
            self.steps += 1

    def speed_slot(self, slot, buf, write=False):
        if write:
            self.slots[slot] = _np(buf)[:3]
        else:
            _np(buf)[:3] = self.slots[slot]
        return buf


def _grid(zbc):
    if zbc == 1:
        return W.smooth_periodic(n=(9, 8, 14), amp=0.3, vamp=0.5, seed=6, scheme=5)
    g, w = W.lumpy(n=(9, 8, 14), seed=12, scheme=5)
    x, y, z = g.centres()
    w[3] = np.broadcast_to(0.2 * np.sin(z / 2.0) * np.ones_like(x * y), w[3].shape)
    return g, w


def _whole(g, w, nsteps, t_end=-1.0):
    c = oracle.make_cfg(g.n, g.dx, cs2=g.cs2, scheme=g.scheme, bc=g.bc, cfl=g.cfl, eps=g.eps)
    return oracle.run(c, oracle.prim2con(w, g.cs2), nsteps, t_end=t_end)


def test_slab_bounds():
    assert slab_bounds(10, 3) == [(0, 4), (4, 7), (7, 10)]
    assert slab_bounds(8, 2, 4) == [(0, 4), (4, 8)]
    with pytest.raises(ValueError):
        slab_bounds(7, 2, 4)


@pytest.mark.parametrize("zbc", [0, 1])
@pytest.mark.parametrize("nslabs", [1, 3])
def test_local_exchange_matches_whole_grid(zbc, nslabs):
    g, w = _grid(zbc)
    ref, tr, kr = _whole(g, w, 3)
    slabs = [OracleSlab(g, z0, z1) for z0, z1 in slab_bounds(g.n[2], nslabs, 3)]
    for s, (z0, z1) in zip(slabs, slab_bounds(g.n[2], nslabs, 3)):
        s.set_primitive(w[:, z0:z1])
    dom = SlabDomain(LocalExchange(slabs, zbc))
    dom.loaded()
    dom.step(3)
    got = np.concatenate([s.interior() for s in slabs], axis=1)
    assert {(s.t, s.steps) for s in slabs} == {(tr, kr)}
    assert np.array_equal(got, ref)


def test_mutated_exchange_is_caught():
    """A slab that treats its upper neighbour as the end of the grid (ghost
    planes from the outflow rule instead of the neighbour's planes) no longer
    matches, so the comparison above has teeth."""
    g, w = _grid(0)
    ref, _, _ = _whole(g, w, 2)
    b = slab_bounds(g.n[2], 2, 3)
    slabs = [OracleSlab(g, z0, z1) for z0, z1 in b]
    for s, (z0, z1) in zip(slabs, b):
        s.set_primitive(w[:, z0:z1])
    ex = LocalExchange(slabs, 0)
    real = slabs[0].halo_unpack
    slabs[0].halo_unpack = (lambda level, side, buf:
                            slabs[0].halo_fill_outflow(level, 1) if side == 1 else real(level, side, buf))
    dom = SlabDomain(ex)
    dom.loaded()
    dom.step(2)
    got = np.concatenate([s.interior() for s in slabs], axis=1)
    assert not np.array_equal(got, ref)


def _worker(rank, world, port, zbc, nsteps, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g, w = _grid(zbc)
        z0, z1 = slab_bounds(g.n[2], world, 3)[rank]
        s = OracleSlab(g, z0, z1)
        s.set_primitive(w[:, z0:z1])
        dom = SlabDomain(DistExchange(s, rank, world, zbc, dist))
        dom.loaded()
        dom.step(nsteps)
        parts = [None] * world
        dist.all_gather_object(parts, (rank, s.t, s.steps, np.array(s.interior())))
        q.put(parts)
    finally:
        dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


@pytest.mark.parametrize("zbc,world", [(0, 2), (1, 2), (1, 3)])
def test_gloo_ranks_match_whole_grid(zbc, world):
    nsteps = 3
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, zbc, nsteps, q)) for r in range(world)]
    for p in procs:
        p.start()
    outs = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    g, w = _grid(zbc)
    ref, tr, kr = _whole(g, w, nsteps)
    for parts in outs:
        parts = sorted(parts, key=lambda x: x[0])
        assert {(t, k) for _, t, k, _ in parts} == {(tr, kr)}
        assert np.array_equal(np.concatenate([p[3] for p in parts], axis=1), ref)
