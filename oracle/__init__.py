"""Plain FP64 CPU oracle for the WENO5/WENO7 + RK3 relativistic hydro scheme.

TEST INFRASTRUCTURE ONLY.  This package is the independent checker of the CUDA
library: only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  The product path never imports, links or calls it,
and it shares no code, header or table with the CUDA sources.

The C source (``hydro_oracle.c``) follows the paper step by step: Eq. 1 (the
conservation law), Eq. 2 (the semi-discrete operator L), Sec. 1.2 (FD-WENO of
order 5 and 7) and the third-order Runge-Kutta integration of Sec. 1.  This
module only marshals numpy arrays into it.

State arrays are numpy float64 of shape (5, nz, ny, nx): fields
(E, M_x, M_y, M_z, R), x fastest.  Primitive arrays are (e, v_x, v_y, v_z, n).
"""
import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hydro_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

OK, ERR_ARG, ERR_OOM, ERR_UNPHYSICAL = 0, 1, 3, 4


def build(force=False, quiet=True):
    """Compile ``liboracle.so`` next to the source (gcc, no FMA contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-shared", "-fPIC", "-o", _LIB, _SRC, "-lm"]
    for extra in (["-fopenmp"], []):
        cmd = base[:1] + extra + base[1:]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode == 0:
            return _LIB
    raise RuntimeError("oracle build failed:\n" + res.stderr)


class Cfg(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32 * 3),
        ("r", ctypes.c_int32),
        ("bc", ctypes.c_int32 * 3),
        ("split", ctypes.c_int32),
        ("nq", ctypes.c_int32),
        ("limiter", ctypes.c_int32),
        ("musta_k", ctypes.c_int32),
        ("charw", ctypes.c_int32),
        ("dx", ctypes.c_double * 3),
        ("cs2", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("dt_fixed", ctypes.c_double),
        ("eps", ctypes.c_double),
        ("mass", ctypes.c_double),
    ]


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.POINTER
        d = ctypes.c_double
        vp = ctypes.c_void_p
        L.oc_con2prim.argtypes = [d, vp, vp]
        L.oc_prim2con.argtypes = [d, vp, vp]
        L.oc_flux.argtypes = [d, ctypes.c_int, vp, vp, vp]
        L.oc_flux_n.argtypes = [d, ctypes.c_int, ctypes.c_int, vp, vp, vp]
        L.oc_eigen.argtypes = [d, ctypes.c_int, vp, vp]
        L.oc_weno_left.argtypes = [ctypes.c_int, vp, d]
        L.oc_weno_left.restype = d
        L.oc_weno_tables.argtypes = [ctypes.c_int, vp, vp, vp]
        L.oc_alpha.argtypes = [P(Cfg), vp, vp]
        L.oc_L.argtypes = [P(Cfg), vp, vp, vp]
        L.oc_run.argtypes = [P(Cfg), vp, ctypes.c_int, d, P(d), P(ctypes.c_int64), vp, vp, vp, vp]
        L.oc_eps2.argtypes = [P(Cfg), vp, P(d)]
        L.oc_con2prim_n.argtypes = [d, d, ctypes.c_int, vp, ctypes.c_int64, vp]
        L.oc_prim2con_n.argtypes = [d, d, ctypes.c_int, vp, ctypes.c_int64, vp]
        L.oc_con2prim_gas.argtypes = [d, d, vp, vp]
        L.oc_con2prim_eos.argtypes = [d, d, vp, vp]
        L.oc_flux_eos.argtypes = [d, d, ctypes.c_int, ctypes.c_int, vp, vp, vp]
        L.oc_sound2.argtypes = [d, d, vp]
        L.oc_sound2.restype = d
        L.oc_eos_p.argtypes = [d, d, vp]
        L.oc_eos_p.restype = d
        L.oc_set_threads.argtypes = [ctypes.c_int]
        L.oc_limiter.argtypes = [ctypes.c_int, d, d]
        L.oc_limiter.restype = d
        L.oc_char_basis.argtypes = [d, ctypes.c_int, ctypes.c_int, vp, vp, vp]
        L.oc_invert.argtypes = [ctypes.c_int, vp, vp]
        L.oc_invert.restype = ctypes.c_int
        L.oc_get_max_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def _c(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a


def set_threads(n):
    """Number of OpenMP threads (0: library default)."""
    lib().oc_set_threads(int(n))


def max_threads():
    return lib().oc_get_max_threads()


def make_cfg(n, dx, cs2=1.0 / 3.0, scheme=5, bc=(0, 0, 0), cfl=0.3, dt_fixed=0.0, eps=1e-6, split=0, nq=1,
             limiter=0, musta_k=2, charw=0, mass=0.0):
    """n = (nx, ny, nz); scheme 5 (WENO5), 7 (WENO7) or 2 (MUSTA-FORCE + MUSCL);
    bc 0 outflow / 1 periodic; split 0 global / 1 local Lax-Friedrichs; nq
    conserved charges (state has 4 + nq fields); limiter 0 minmod, 1 MC,
    2 van Leer, 3 superbee; musta_k MUSTA stages; charw 0 component-wise,
    1 characteristic-wise WENO; mass m of the EOS p = cs2 (e - m n_1)
    (0: p = cs2 e)."""
    c = Cfg()
    for i in range(3):
        c.n[i] = int(n[i])
        c.dx[i] = float(dx[i])
        c.bc[i] = int(bc[i])
    c.r = {5: 3, 7: 4, 2: 1}[int(scheme)]
    c.cs2 = float(cs2)
    c.cfl = float(cfl)
    c.dt_fixed = float(dt_fixed)
    c.eps = float(eps)
    c.split = int(split)
    c.nq = int(nq)
    c.limiter = int(limiter)
    c.musta_k = int(musta_k)
    c.charw = int(charw)
    c.mass = float(mass)
    return c


def limiter(kind, a, b):
    """MUSCL slope limiter of the oracle (0 minmod, 1 MC, 2 van Leer, 3 superbee)."""
    return lib().oc_limiter(int(kind), float(a), float(b))


def _shape(c):
    return (4 + max(1, c.nq), c.n[2], c.n[1], c.n[0])


def con2prim(u, cs2=1.0 / 3.0, mass=0.0):
    """u: (4+q, ...) conserved (E, M, R_1..R_q) -> primitives (e, vx, vy, vz,
    n_1..n_q) for the EOS p = cs2 (e - mass n_1); NaN where unphysical."""
    u = _c(u)
    w = np.empty_like(u)
    n = u[0].size
    lib().oc_con2prim_n(cs2, mass, u.shape[0], _ptr(u), n, _ptr(w))
    return w


def prim2con(w, cs2=1.0 / 3.0, mass=0.0):
    w = _c(w)
    u = np.empty_like(w)
    lib().oc_prim2con_n(cs2, mass, w.shape[0], _ptr(w), w[0].size, _ptr(u))
    return u


def con2prim_gas(u, cs2, mass):
    """One cell (5 values) by the iterative recovery, whatever the mass
    (also m = 0); None if no physical state exists."""
    u = _c(u).reshape(-1)
    w = np.empty(5)
    return None if lib().oc_con2prim_gas(cs2, mass, _ptr(u), _ptr(w)) else w


def sound2(w, cs2=1.0 / 3.0, mass=0.0):
    """Squared sound speed of primitives w (e, vx, vy, vz, n_1)."""
    return lib().oc_sound2(cs2, mass, _ptr(_c(w).reshape(-1)))


def pressure(w, cs2=1.0 / 3.0, mass=0.0):
    return lib().oc_eos_p(cs2, mass, _ptr(_c(w).reshape(-1)))


def flux(d, u, cs2=1.0 / 3.0, mass=0.0):
    """Physical flux f_d(u) of one cell (u: 4 + q conserved values, q >= 1)."""
    u = _c(u).reshape(-1)
    w = np.empty(max(8, u.size))
    rc = lib().oc_con2prim_eos(cs2, mass, _ptr(u), _ptr(w))
    if rc:
        raise ValueError("unphysical state")
    f = np.empty(u.size)
    lib().oc_flux_eos(cs2, mass, int(d), u.size, _ptr(u), _ptr(w), _ptr(f))
    return f


def eigen(d, w, cs2=1.0 / 3.0):
    """(lambda_-, lambda_+) along d for primitives w = (e, vx, vy, vz, n)."""
    w = _c(w)
    lam = np.empty(2)
    lib().oc_eigen(cs2, int(d), _ptr(w), _ptr(lam))
    return lam


def char_basis(d, w, cs2=1.0 / 3.0):
    """(R, lam): right eigenvectors of df_d/du (columns; sound -, sound +,
    shear t1, shear t2, charges) at primitives w = (e, vx, vy, vz, n_1..n_q),
    and their eigenvalues."""
    w = _c(w)
    nf = w.size
    Rm = np.empty((nf, nf))
    lam = np.empty(nf)
    lib().oc_char_basis(cs2, int(d), nf, _ptr(w), _ptr(Rm), _ptr(lam))
    return Rm, lam


def invert(A):
    """Inverse by the oracle's Gauss-Jordan elimination (partial pivoting)."""
    A = _c(A)
    out = np.empty_like(A)
    if lib().oc_invert(A.shape[0], _ptr(A), _ptr(out)):
        raise ValueError("singular matrix")
    return out


def weno_left(r, v, eps=1e-6):
    v = _c(v)
    assert v.size == 2 * r - 1
    return lib().oc_weno_left(int(r), _ptr(v), float(eps))


def weno_tables(r):
    q = np.empty(r * r)
    t = np.empty(r * (r - 1) * r)
    d = np.empty(r)
    rc = lib().oc_weno_tables(int(r), _ptr(q), _ptr(t), _ptr(d))
    if rc:
        raise ValueError("r must be 3 or 4")
    return q.reshape(r, r), t.reshape(r, r - 1, r), d


def _check(rc, what):
    if rc == ERR_UNPHYSICAL:
        raise FloatingPointError(what + ": unphysical state (E <= 0 or |M| >= E)")
    if rc:
        raise RuntimeError("%s failed with code %d" % (what, rc))


def alpha(c, u):
    u = _c(u)
    assert u.shape == _shape(c), (u.shape, _shape(c))
    a = np.empty(3)
    _check(lib().oc_alpha(ctypes.byref(c), _ptr(u), _ptr(a)), "oc_alpha")
    return a


def L(c, u, alph):
    u = _c(u)
    assert u.shape == _shape(c)
    a = _c(alph)
    out = np.empty_like(u)
    _check(lib().oc_L(ctypes.byref(c), _ptr(u), _ptr(a), _ptr(out)), "oc_L")
    return out


def run(c, u, nsteps, t=0.0, t_end=-1.0, alpha_in=None, dt_in=None, record=False):
    """Advance a copy of u by up to nsteps RK3 steps.

    Returns (u_new, t_new, steps_done) or, with record=True,
    (u_new, t_new, steps_done, alphas[steps,3,3], dts[steps]).
    alpha_in/dt_in freeze the Lax-Friedrichs alphas and time steps.
    """
    u = _c(u).copy()
    assert u.shape == _shape(c)
    tt = ctypes.c_double(t)
    st = ctypes.c_int64(0)
    ain = _c(alpha_in).reshape(-1) if alpha_in is not None else None
    din = _c(dt_in).reshape(-1) if dt_in is not None else None
    if ain is not None:
        assert ain.size >= 9 * nsteps and din.size >= nsteps
    aout = np.zeros((max(nsteps, 1), 3, 3)) if record else None
    dout = np.zeros(max(nsteps, 1)) if record else None
    rc = lib().oc_run(
        ctypes.byref(c), _ptr(u), int(nsteps), float(t_end), ctypes.byref(tt), ctypes.byref(st),
        _ptr(ain) if ain is not None else None, _ptr(din) if din is not None else None,
        _ptr(aout) if record else None, _ptr(dout) if record else None)
    _check(rc, "oc_run")
    if record:
        k = st.value
        return u, tt.value, k, aout[:k].copy(), dout[:k].copy()
    return u, tt.value, st.value


def eps2(c, u):
    u = _c(u)
    out = ctypes.c_double(0.0)
    _check(lib().oc_eps2(ctypes.byref(c), _ptr(u), ctypes.byref(out)), "oc_eps2")
    return out.value
