"""Seeded synthetic initial data for the hydro workloads.

This module only produces inputs: primitive fields (e, v_x, v_y, v_z, n) on a
Cartesian grid plus the grid description.  It holds none of the numerical
scheme's arithmetic (no conserved-variable recovery, fluxes or reconstruction),
so the CUDA path and the CPU oracle can both consume the same arrays, each
converting them with its own code.

Arrays are numpy float64 of shape (5, nz, ny, nx), x fastest.  Cell centres are
origin + (i + 1/2) dx.  All random numbers come from numpy's PCG64 with the
stated seed.

Workloads (shapes follow the paper's tests, Sec. 3):
  sod         1+1D relativistic shock tube on [-1, 1] (Fig. 1)
  hubble      Hubble-like expansion on [-5, 5]^3 (Fig. 3)
  ellipsoidal Gaussian ellipsoid with linear, axis-scaled velocity (Fig. 2)
  lumpy       smooth sum of Gaussian hot spots, v = 0 (event-by-event data)
  smooth_periodic  small smooth periodic data for conservation / order tests
"""
from dataclasses import dataclass, field

import numpy as np

CS2 = 1.0 / 3.0


@dataclass
class Grid:
    n: tuple            # (nx, ny, nz)
    dx: tuple           # cell sizes
    origin: tuple       # lower corner of the box
    bc: tuple = (0, 0, 0)   # 0 outflow (copy edge cell), 1 periodic
    scheme: int = 5
    cfl: float = 0.3
    dt_fixed: float = 0.0       # > 0: constant time step instead of the CFL rule
    split: int = 0              # 0 global, 1 local Lax-Friedrichs splitting
    nq: int = 1                 # conserved charge densities (state fields 4 + nq)
    limiter: int = 0            # MUSTA-FORCE: 0 minmod, 1 MC, 2 van Leer, 3 superbee
    musta_stages: int = 2       # MUSTA-FORCE: stages of the FORCE flux
    charwise: int = 0           # WENO on 0 the components, 1 the characteristic fields
    mass: float = 0.0           # EOS p = cs2 (e - mass n_1); 0: p = cs2 e
    cs2: float = CS2
    eps: float = 1e-6
    t0: float = 0.0
    t_end: float = -1.0
    nsteps: int = 0
    name: str = ""
    extra: dict = field(default_factory=dict)

    def centres(self):
        """Cell-centre coordinates (x, y, z) as broadcastable arrays (nz, ny, nx)."""
        nx, ny, nz = self.n
        x = self.origin[0] + (np.arange(nx) + 0.5) * self.dx[0]
        y = self.origin[1] + (np.arange(ny) + 0.5) * self.dx[1]
        z = self.origin[2] + (np.arange(nz) + 0.5) * self.dx[2]
        return x[None, None, :], y[None, :, None], z[:, None, None]

    @property
    def cells(self):
        return int(self.n[0]) * int(self.n[1]) * int(self.n[2])


def _stack(g, e, vx, vy, vz, n):
    shape = (g.n[2], g.n[1], g.n[0])
    out = np.empty((5,) + shape)
    for i, a in enumerate((e, vx, vy, vz, n)):
        out[i] = np.broadcast_to(a, shape)
    return out


def sod(N=400, scheme=5):
    """Shock tube: left (e=1, n=1, v=0), right (e=0.1, n=0.125, v=0) split at
    x = 0 on [-1, 1], outflow boundaries, CFL 0.4, run to t = 0.4."""
    g = Grid(n=(N, 1, 1), dx=(2.0 / N, 2.0 / N, 2.0 / N), origin=(-1.0, -1.0 / N, -1.0 / N),
             bc=(0, 0, 0), scheme=scheme, cfl=0.4, t_end=0.4, nsteps=100000, name="sod")
    x, _, _ = g.centres()
    left = x < 0
    e = np.where(left, 1.0, 0.1)
    n = np.where(left, 1.0, 0.125)
    return g, _stack(g, e, 0.0, 0.0, 0.0, n)


def gas_sod(N=400, scheme=5, k=2.0 / 3.0, m=1.0):
    """Shock tube for the ideal gas p = k (e - m n) (adiabatic index 1 + k):
    left (n=1, p=1), right (n=0.125, p=0.1), both at rest, split at x = 0 on
    [-1, 1], outflow boundaries, CFL 0.4, run to t = 0.4; e = m n + p / k."""
    g = Grid(n=(N, 1, 1), dx=(2.0 / N, 2.0 / N, 2.0 / N), origin=(-1.0, -1.0 / N, -1.0 / N),
             bc=(0, 0, 0), scheme=scheme, cfl=0.4, cs2=k, mass=m, t_end=0.4, nsteps=100000, name="gas_sod")
    x, _, _ = g.centres()
    left = x < 0
    n = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    return g, _stack(g, m * n + p / k, 0.0, 0.0, 0.0, n)


def hubble(N=128, scheme=5, box=5.0, t0=10.0, e0=10.0, n0=1.0, nsteps=100, cfl=0.3):
    """Hubble-like flow u^mu = x^mu / tau, tau = sqrt(t^2 - r^2), started from
    its exact profile at t = t0: v = x / t0, e = e0 (t0/tau)^(3(1+cs2)),
    n = n0 (t0/tau)^3.  Box [-box, box]^3, outflow boundaries.  t0 must exceed
    the corner radius so that the flow is subluminal everywhere."""
    h = 2.0 * box / N
    g = Grid(n=(N, N, N), dx=(h, h, h), origin=(-box,) * 3, bc=(0, 0, 0), scheme=scheme,
             cfl=cfl, t0=t0, nsteps=nsteps, name="hubble", extra=dict(t0=t0, e0=e0, n0=n0))
    x, y, z = g.centres()
    r2 = x * x + y * y + z * z
    tau = np.sqrt(t0 * t0 - r2)
    e = e0 * (t0 / tau) ** (3.0 * (1.0 + CS2))
    n = n0 * (t0 / tau) ** 3
    return g, _stack(g, e, x / t0, y / t0, z / t0, n)


def ellipsoidal_charge(N=32, scheme=5, box=5.0, t0=10.0, e0=10.0, n0=1.0, axes=(2.0, 3.0, 4.0)):
    """Hubble background with an ellipsoidal charge profile
    n = n0 (t0/tau)^3 exp(-(t0^2/t^2)(x^2/2a^2 + y^2/2b^2 + z^2/2c^2)) at t = t0."""
    g, w = hubble(N=N, scheme=scheme, box=box, t0=t0, e0=e0, n0=n0)
    g.name = "ellipsoidal_charge"
    g.extra["axes"] = axes
    x, y, z = g.centres()
    a, b, c = axes
    w[4] *= np.exp(-(x * x / (2 * a * a) + y * y / (2 * b * b) + z * z / (2 * c * c)))
    return g, w


def ellipsoidal(N=256, scheme=7, box=12.0, e0=20.0, axes=(2.0, 3.0, 4.0), v_corner=0.9,
                nsteps=200, cfl=0.3):
    """Gaussian ellipsoid e = e0 exp(-x^2/2a^2 - y^2/2b^2 - z^2/2c^2) with
    linear velocity v_i = x_i / (t0 a_i^2); t0 is set so that the speed at the
    box corner is v_corner.  n = e / e0.  Box [-box, box]^3, outflow."""
    h = 2.0 * box / N
    a = np.asarray(axes, dtype=np.float64)
    t0 = box * np.sqrt(np.sum(1.0 / a ** 4)) / v_corner
    g = Grid(n=(N, N, N), dx=(h, h, h), origin=(-box,) * 3, bc=(0, 0, 0), scheme=scheme,
             cfl=cfl, nsteps=nsteps, name="ellipsoidal", extra=dict(t0=t0, e0=e0, axes=tuple(axes)))
    x, y, z = g.centres()
    e = e0 * np.exp(-x * x / (2 * a[0] ** 2) - y * y / (2 * a[1] ** 2) - z * z / (2 * a[2] ** 2))
    return g, _stack(g, e, x / (t0 * a[0] ** 2), y / (t0 * a[1] ** 2), z / (t0 * a[2] ** 2), e / e0)


def lumpy_params(seed=1604, blobs=20, radius=4.0, mu=1.0, sigma=0.5):
    """Seeded hot-spot parameters: centres uniform in a ball of radius
    `radius` (direction from 3 normals, radius r U^(1/3)), amplitudes
    lognormal(mu, sigma)."""
    rng = np.random.default_rng(seed)
    dirs = rng.standard_normal((blobs, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    rad = radius * rng.random(blobs) ** (1.0 / 3.0)
    centres = dirs * rad[:, None]
    amps = rng.lognormal(mean=mu, sigma=sigma, size=blobs)
    return centres, amps


def lumpy(n=(96, 96, 96), seed=1604, box=6.0, blobs=20, width=0.5, radius=4.0, mu=1.0,
          sigma=0.5, scheme=5, nsteps=50, cfl=0.3):
    """e = 0.1 + sum of `blobs` Gaussians of width `width` (parameters from
    lumpy_params); v = 0; n = e.  Box [-box, box] per axis with
    dx_d = 2 box / n_d (uneven boxes allowed)."""
    centres, amps = lumpy_params(seed, blobs, radius, mu, sigma)
    dx = tuple(2.0 * box / int(k) for k in n)
    g = Grid(n=tuple(int(k) for k in n), dx=dx, origin=(-box,) * 3, bc=(0, 0, 0), scheme=scheme,
             cfl=cfl, nsteps=nsteps, name="lumpy", extra=dict(seed=seed, width=width))
    x, y, z = g.centres()
    e = np.full((g.n[2], g.n[1], g.n[0]), 0.1)
    for c, A in zip(centres, amps):
        e += A * np.exp(-((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) / (2 * width * width))
    return g, _stack(g, e, 0.0, 0.0, 0.0, e)


def with_charges(g, w, nq=3):
    """Append nq - 1 further charge densities to primitive data w (shape
    (5, ...)): n_2 = n^2 / max n, n_3 = 1 + sin of the x coordinate, n_4 = 0.5.
    Returns data of shape (4 + nq, ...)."""
    x, _, _ = g.centres()
    n1 = w[4]
    extra = [n1 * n1 / n1.max(), np.broadcast_to(1.0 + 0.5 * np.sin(x), n1.shape), np.full(n1.shape, 0.5)]
    return np.concatenate([w, np.stack(extra[:nq - 1])]) if nq > 1 else w


def batch_sizes(events=256, seed=1604, lo=48, hi=160):
    """Per-event grid sizes (nx, ny, nz), each drawn uniformly from [lo, hi]."""
    out = []
    for i in range(events):
        rng = np.random.default_rng(seed + i)
        out.append(tuple(int(k) for k in rng.integers(lo, hi + 1, size=3)))
    return out


def batch_event(i, sizes, seed=1604, scheme=5, nsteps=100):
    """Event i of the event-by-event ensemble: lumpy data, seed seed + i, on
    batch_grid(i) (fixed ensemble time step)."""
    g, w = lumpy(n=sizes[i], seed=seed + i, scheme=scheme, nsteps=nsteps)
    g.dt_fixed = BATCH_DT
    g.name = "lumpy-event"
    return g, w


# Ensemble time step: CFL 0.3 on the finest grid of the ensemble (dx = 12/160)
# with the light-speed bound c = 1 on every characteristic speed, so every
# event is within CFL 0.3 and 100 steps reach t = 2.25 for all events (the
# lumpy events' near-vacuum outflow breaks the scheme at t ~ 3).
BATCH_DT = 0.3 * 12.0 / 160.0


def batch_grid(i, sizes, scheme=5, box=6.0, nsteps=100, dt=BATCH_DT):
    """Grid of event i (the data comes from batch_event or lumpy_params)."""
    n = sizes[i]
    return Grid(n=tuple(int(k) for k in n), dx=tuple(2.0 * box / int(k) for k in n), origin=(-box,) * 3,
                bc=(0, 0, 0), scheme=scheme, dt_fixed=dt, nsteps=nsteps, name="lumpy-event")


def smooth_periodic(n=(12, 12, 12), seed=7, amp=0.2, vamp=0.3, scheme=5, length=1.0):
    """Smooth random periodic data: a few low Fourier modes in e, v, n; the
    velocity field is scaled so that its largest speed is vamp."""
    rng = np.random.default_rng(seed)
    dx = tuple(length / k for k in n)
    g = Grid(n=tuple(n), dx=dx, origin=(0.0, 0.0, 0.0), bc=(1, 1, 1), scheme=scheme, name="periodic")
    x, y, z = g.centres()

    def field(base, a):
        f = np.full((n[2], n[1], n[0]), base, dtype=np.float64)
        for _ in range(3):
            k = rng.integers(-2, 3, size=3)
            ph = rng.random() * 2 * np.pi
            f = f + a * rng.random() * np.sin(2 * np.pi * (k[0] * x + k[1] * y + k[2] * z) / length + ph)
        return f
    e = field(1.0, amp)
    vx, vy, vz = field(0.0, 1.0), field(0.0, 1.0), field(0.0, 1.0)
    vmag = np.sqrt(vx * vx + vy * vy + vz * vz).max()
    s = vamp / vmag if vmag > 0 else 0.0   # largest speed is exactly vamp (< 1)
    nn = field(1.0, amp)
    return g, _stack(g, e, s * vx, s * vy, s * vz, nn)
