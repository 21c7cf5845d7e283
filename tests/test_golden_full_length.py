"""The oracle's stored full-length states (tests/golden/full_length_*.npz,
written by tests/golden/make_full_length.py from the oracle alone), checked on
the CPU against what they must satisfy independently of how they were made:

* the case metadata (grid, steps, CFL or fixed dt, time reached) matches the
  case definitions;
* the stored statistics agree with each other (maxima over planes of every
  axis give the same field maximum; plane sums of every axis give the same
  total; sampled values lie within the field maximum);
* Hubble-like expansion (paper Sec. 3, Fig. 3 setup): in the interior, far
  from the outflow boundaries, the sampled cells match the exact solution
  e = e0 (t0/tau)^(3(1+cs2)), v = x/t, n = n0 (t0/tau)^3 at the stored time;
* ellipsoidal flow (Fig. 2 setup): the data are mirror symmetric in x, y and
  z, so the plane sums of E and R are even, those of M_d odd along axis d and
  zero across the other axes, and the plane maxima are even."""
import numpy as np
import pytest

import oracle
import workloads as W
from exact import hubble as hubble_exact
from full_length import MFL, stored


@pytest.mark.parametrize("name", MFL.CASES)
def test_metadata_matches_case(name):
    g, w, nsteps = MFL.case(name)
    z = stored(name)
    assert tuple(int(k) for k in z["n"]) == tuple(g.n)
    assert int(z["steps"]) == nsteps and int(z["scheme"]) == g.scheme
    assert float(z["cfl"]) == g.cfl and float(z["dt_fixed"]) == g.dt_fixed and float(z["t_start"]) == g.t0
    if g.dt_fixed > 0:
        assert float(z["t"]) == pytest.approx(g.t0 + nsteps * g.dt_fixed, rel=1e-13)
    else:
        # the CFL rule: dt = cfl dx / max alpha with alpha < 1 gives dt > cfl dx
        assert float(z["t"]) > g.t0 + nsteps * g.cfl * min(g.dx)


@pytest.mark.parametrize("name", MFL.CASES)
def test_statistics_are_consistent(name):
    z = stored(name)
    fmax = z["fmax"]
    tot = [z["psum_" + a].sum(axis=1) for a in "xyz"]
    for a in "xyz":
        assert np.array_equal(z["pmax_" + a].max(axis=1), fmax), a
    scale = fmax * np.prod(z["n"])
    assert np.all(np.abs(tot[0] - tot[1]) <= 1e-13 * scale) and np.all(np.abs(tot[0] - tot[2]) <= 1e-13 * scale)
    assert np.all(np.abs(z["val"]) <= fmax[:, None])
    assert np.all(fmax > 0) and np.all(np.isfinite(z["val"]))
    assert np.all(np.diff(z["idx"]) > 0) and z["idx"][-1] < np.prod(z["n"])


@pytest.mark.parametrize("name", ["hubble128_weno5", "hubble128_weno7"])
def test_hubble_interior_matches_exact_solution(name):
    g, _, _ = MFL.case(name)
    z = stored(name)
    nx, ny, nz = g.n
    idx = z["idx"]
    cx = g.origin[0] + (idx % nx + 0.5) * g.dx[0]
    cy = g.origin[1] + ((idx // nx) % ny + 0.5) * g.dx[1]
    cz = g.origin[2] + (idx // (nx * ny) + 0.5) * g.dx[2]
    inside = (np.abs(cx) < 2.0) & (np.abs(cy) < 2.0) & (np.abs(cz) < 2.0)
    assert inside.sum() > 300
    p = oracle.con2prim(z["val"][:, inside].reshape(5, -1, 1, 1)).reshape(5, -1)
    e, vx, vy, vz, n = hubble_exact(cx[inside], cy[inside], cz[inside], float(z["t"]))
    assert np.abs(p[0] / e - 1).max() < 5e-7
    for got, want in ((p[1], vx), (p[2], vy), (p[3], vz)):
        assert np.abs(got - want).max() < 1e-7
    assert np.abs(p[4] / n - 1).max() < 1e-7


def test_ellipsoidal_mirror_symmetry():
    z = stored("ellipsoidal128_weno7")
    fmax = z["fmax"]
    N = int(z["n"][0])
    for d, a in enumerate("xyz"):
        ps, pm = z["psum_" + a], z["pmax_" + a]
        tol = 1e-14 * fmax * N * N
        for f in range(5):
            flipped = ps[f, ::-1]
            if f == 1 + d:
                assert np.all(np.abs(ps[f] + flipped) <= tol[f]), (a, f)        # odd along its own axis
            elif f in (1, 2, 3):
                assert np.all(np.abs(ps[f]) <= tol[f]), (a, f)                  # odd across the plane
            else:
                assert np.all(np.abs(ps[f] - flipped) <= tol[f]), (a, f)        # even
            assert np.all(np.abs(pm[f] - pm[f, ::-1]) <= 1e-14 * fmax[f]), (a, f)


def test_batch_event_reaches_the_ensemble_time():
    z = stored("batch_event160_weno5")
    assert float(z["t"]) == pytest.approx(100 * W.BATCH_DT, rel=1e-13)
