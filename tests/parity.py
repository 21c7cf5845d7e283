"""Helpers for GPU-vs-oracle parity tests."""
import numpy as np

import oracle

# parity tolerance: max relative error per field after the stated steps
TOL = 1e-11


def field_errors(a, b):
    """Normwise relative error per field: max|a-b| / max|b| (absolute if b == 0)."""
    out = []
    for f in range(a.shape[0]):
        den = np.abs(b[f]).max()
        num = np.abs(a[f] - b[f]).max()
        out.append(num / den if den > 0 else num)
    return np.array(out)


def oracle_cfg(g, dt_fixed=None):
    dt = getattr(g, "dt_fixed", 0.0) if dt_fixed is None else dt_fixed
    return oracle.make_cfg(g.n, g.dx, cs2=g.cs2, scheme=g.scheme, bc=g.bc, cfl=g.cfl, dt_fixed=dt, eps=g.eps,
                           split=getattr(g, "split", 0), nq=getattr(g, "nq", 1),
                           limiter=getattr(g, "limiter", 0), musta_k=getattr(g, "musta_stages", 2),
                           charw=getattr(g, "charwise", 0), mass=getattr(g, "mass", 0.0))


def run_oracle(g, w, nsteps, t0=0.0, t_end=-1.0):
    c = oracle_cfg(g)
    u0 = oracle.prim2con(w, g.cs2, getattr(g, "mass", 0.0))
    return oracle.run(c, u0, nsteps, t=t0, t_end=t_end)


def run_gpu(g, w, nsteps, t0=0.0, t_end=-1.0, use_primitive=True, u0=None):
    from paper_1604_03360_gb300 import Hydro
    with Hydro.from_grid(g) as h:
        if use_primitive:
            h.set_primitive(np.ascontiguousarray(w), t=t0)
        else:
            h.set_state(np.ascontiguousarray(u0), t=t0)
        h.step(nsteps, t_end)
        u = h.get_state()
        return u, h.t, h.steps


def assert_parity(g, w, nsteps, t0=0.0, t_end=-1.0, tol=TOL, use_primitive=True):
    ref, tr, kr = run_oracle(g, w, nsteps, t0, t_end)
    u0 = oracle.prim2con(w, g.cs2, getattr(g, "mass", 0.0))
    got, tg, kg = run_gpu(g, w, nsteps, t0, t_end, use_primitive=use_primitive, u0=u0)
    assert kg == kr, (kg, kr)
    assert abs(tg - tr) <= 1e-13 * max(1.0, abs(tr)), (tg, tr)
    err = field_errors(got, ref)
    assert np.all(err <= tol), err
    return err
