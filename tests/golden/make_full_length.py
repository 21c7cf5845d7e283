"""Write the oracle's state after the full step counts of the paper's test
configurations, in compact form, for the GPU parity tests.

Only ``oracle/`` (and the seeded input generators in ``workloads/``) are
called here: no value in these files comes from the CUDA path.  A full state
(84-131 MB per case) is too large to store, so each case keeps

* ``idx``/``val``: every field at a seeded random sample of 4096 cells, the
  three grid lines through the central cell and the eight corners;
* ``fmax``: max |u_f| over the grid, per field;
* ``psum_a``/``pmax_a`` (a = x, y, z): per field and per plane normal to axis
  a, the sum of u_f and the maximum of |u_f| over that plane;
* ``t``, ``steps``, the grid size and the step rule.

Cases (paper Sec. 3, with the grids and step counts of the benchmark
configurations):

hubble128_weno5 / hubble128_weno7
    Hubble-like expansion (Fig. 3 setup), 128^3 on [-5, 5]^3, exact
    initialisation at t0 = 10, CFL 0.3, 100 RK3 steps.
ellipsoidal128_weno7
    ellipsoidal flow (Fig. 2 setup), 128^3 on [-12, 12]^3, WENO7, 200 RK3
    steps at CFL 0.3 * 128/256, so that dt and the physical time reached match
    the 256^3 run.
batch_event160_weno5
    event 1 of the event-by-event size list used by the batch tests: lumpy
    data (seed 1605) on a 160^3 grid, WENO5, the fixed ensemble time step,
    100 RK3 steps.

Usage: python tests/golden/make_full_length.py [case ...]   (all by default)
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads as W  # noqa: E402

SAMPLE_SEED = 20161604
SAMPLE_CELLS = 4096
BATCH_SIZES = [(48, 48, 48), (160, 160, 160), (48, 160, 96), (130, 57, 75), (64, 64, 160), (100, 100, 100),
               (150, 49, 120), (77, 88, 99)]


def case(name):
    """(grid, primitives, nsteps) of a named case."""
    if name in ("hubble128_weno5", "hubble128_weno7"):
        g, w = W.hubble(N=128, scheme=int(name[-1]))
        return g, w, 100
    if name == "ellipsoidal128_weno7":
        g, w = W.ellipsoidal(N=128, scheme=7)
        g.cfl = 0.3 * 128 / 256
        return g, w, 200
    if name == "batch_event160_weno5":
        g, w = W.batch_event(1, BATCH_SIZES)
        return g, w, 100
    raise KeyError(name)


CASES = ["hubble128_weno5", "hubble128_weno7", "ellipsoidal128_weno7", "batch_event160_weno5"]


def sample_indices(n):
    """Flat indices (z, y, x order, x fastest) of the stored sample cells."""
    nx, ny, nz = n
    cells = nx * ny * nz
    rng = np.random.default_rng(SAMPLE_SEED)
    idx = set(rng.choice(cells, size=min(SAMPLE_CELLS, cells), replace=False).tolist())
    cx, cy, cz = nx // 2, ny // 2, nz // 2
    idx.update((cz * ny + cy) * nx + i for i in range(nx))
    idx.update((cz * ny + j) * nx + cx for j in range(ny))
    idx.update((k * ny + cy) * nx + cx for k in range(nz))
    for k in (0, nz - 1):
        for j in (0, ny - 1):
            for i in (0, nx - 1):
                idx.add((k * ny + j) * nx + i)
    return np.array(sorted(idx), dtype=np.int64)


def summarise(u, n):
    """The stored summary of a state u of shape (fields, nz, ny, nx)."""
    idx = sample_indices(n)
    flat = u.reshape(u.shape[0], -1)
    a = np.abs(u)
    return {
        "idx": idx,
        "val": flat[:, idx].copy(),
        "fmax": a.reshape(u.shape[0], -1).max(axis=1),
        "psum_x": u.sum(axis=(1, 2)), "pmax_x": a.max(axis=(1, 2)),
        "psum_y": u.sum(axis=(1, 3)), "pmax_y": a.max(axis=(1, 3)),
        "psum_z": u.sum(axis=(2, 3)), "pmax_z": a.max(axis=(2, 3)),
    }


def make(name):
    g, w, nsteps = case(name)
    c = oracle.make_cfg(g.n, g.dx, cs2=g.cs2, scheme=g.scheme, bc=g.bc, cfl=g.cfl, dt_fixed=g.dt_fixed,
                        eps=g.eps)
    u0 = oracle.prim2con(w, g.cs2)
    t0 = time.time()
    u, t, k = oracle.run(c, u0, nsteps, t=g.t0)
    wall = time.time() - t0
    out = summarise(u, g.n)
    out.update(n=np.array(g.n), steps=np.int64(k), t=np.float64(t), t_start=np.float64(g.t0),
               cfl=np.float64(g.cfl), dt_fixed=np.float64(g.dt_fixed), scheme=np.int64(g.scheme))
    path = os.path.join(HERE, "full_length_%s.npz" % name)
    np.savez_compressed(path, **out)
    print("%s: %d steps to t = %.15g in %.0f s (%d threads) -> %s" % (name, k, t, wall, oracle.max_threads(), path),
          flush=True)


if __name__ == "__main__":
    oracle.build()
    for name in sys.argv[1:] or CASES:
        make(name)
