"""Host-side test of the reverse-mode WENO5/WENO7 reconstructions used by the
adjoint pencil kernel (csrc/adj_weno.cuh).  The header also compiles as plain
C++; here it is built with g++ and checked against complex-step derivatives
of the forward reconstruction written out in numpy:

* one face: the window's cell adjoints (from the difference adjoints plus the
  centre term) against d(value)/d(v_i), for every integer-pipe choice, which
  must also agree bit for bit with each other;
* one pencil: the sweep's gbar+ and gbar- of every cell (outflow-style ghost
  cells, periodic wrap, and a pencil cut in two segments whose contributions
  add up) against the gradient of sum_j Fbar_j F_j, F_j the face flux of
  Sec. 1.2 from both biased reconstructions.

The numpy forward form of WENO5 is the textbook one (Jiang-Shu smoothness
indicators on the cell values, candidate values, linear weights 1/10, 6/10,
3/10); WENO7 uses the A, B, C smoothness forms of the device source on the
textbook candidates with linear weights (1, 12, 18, 4)/35.  Both are the
scaled forms the kernels use: b_k = 4 beta_k (WENO5), with eps scaled alike,
which leaves the weights unchanged."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1604_03360_gb300", "csrc")

SRC = r'''
#include "adj_weno.cuh"
using namespace hydro;

template <int R, int EMU>
static void face(const double* v, double eps, double rbar, double* vb)
{
    constexpr int S = 2 * R - 1;
    AdjWin<R> q;
    adj_win_init<R, (EMU & kEmuConst) != 0>(v, eps, q);
    double db[S - 1];
    adj_core<EMU>(q, eps, rbar, db);
    for (int i = 0; i < S; ++i) vb[i] = (i > 0 ? db[i - 1] : 0.0) - (i < S - 1 ? db[i] : 0.0);
    vb[R - 1] += rbar;
}
extern "C" void face_vjp(int r, int emu, const double* v, double eps, double rbar, double* vb)
{
    if (r == 3) {
        switch (emu) {
        case 0: face<3, 0>(v, eps, rbar, vb); break;
        case 1: face<3, 1>(v, eps, rbar, vb); break;
        case 3: face<3, 3>(v, eps, rbar, vb); break;
        default: face<3, 7>(v, eps, rbar, vb); break;
        }
    } else {
        switch (emu) {
        case 0: face<4, 0>(v, eps, rbar, vb); break;
        case 1: face<4, 1>(v, eps, rbar, vb); break;
        case 3: face<4, 3>(v, eps, rbar, vb); break;
        default: face<4, 7>(v, eps, rbar, vb); break;
        }
    }
}
// one pencil segment: cells m of g+-, lam and the outputs live at m + off of
// arrays of length n + 2 off; out-of-range cells are the caller's ghosts
template <int R>
static void sweep(int n, int off, const double* gp, const double* gm, const double* lam, double sc, double eps,
                  int j0, int j1, double* op, double* om, int* count)
{
    adj_sweep<R, kEmuConst | kEmuWeights>(
        j0, j1, eps, sc,
        [&](int m, double& a, double& b) { a = gp[m + off]; b = gm[m + off]; },
        [&](int m) { return (m >= 0 && m < n) ? lam[m] : 0.0; },
        [&](int m, double a, double b) {
            op[m + off] += a;
            om[m + off] += b;
            count[m + off] += 1;
        });
}
extern "C" void pencil_vjp(int r, int n, int off, const double* gp, const double* gm, const double* lam, double sc,
                           double eps, int j0, int j1, double* op, double* om, int* count)
{
    if (r == 3) sweep<3>(n, off, gp, gm, lam, sc, eps, j0, j1, op, om, count);
    else sweep<4>(n, off, gp, gm, lam, sc, eps, j0, j1, op, om, count);
}
'''


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    d = tmp_path_factory.mktemp("adjweno")
    src = d / "adj.cpp"
    src.write_text(SRC)
    so = d / "libadj.so"
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", "-I", CSRC, str(src), "-o",
                    str(so)], check=True)
    L = ctypes.CDLL(str(so))
    dp = ctypes.POINTER(ctypes.c_double)
    L.face_vjp.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_double, ctypes.c_double, dp]
    L.pencil_vjp.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp, ctypes.c_double, ctypes.c_double,
                             ctypes.c_int, ctypes.c_int, dp, dp, ctypes.POINTER(ctypes.c_int)]
    return L


def P(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ------------------------------------------------------------ numpy forward
def weno5_value(v, eps_s):
    """Left-biased WENO5-JS value at x_{j+1/2} from v_{j-2} .. v_{j+2}."""
    v0, v1, v2, v3, v4 = v
    beta = [13 / 12 * (v0 - 2 * v1 + v2) ** 2 + 0.25 * (v0 - 4 * v1 + 3 * v2) ** 2,
            13 / 12 * (v1 - 2 * v2 + v3) ** 2 + 0.25 * (v1 - v3) ** 2,
            13 / 12 * (v2 - 2 * v3 + v4) ** 2 + 0.25 * (3 * v2 - 4 * v3 + v4) ** 2]
    q = [(2 * v0 - 7 * v1 + 11 * v2) / 6, (-v1 + 5 * v2 + 2 * v3) / 6, (2 * v2 + 5 * v3 - v4) / 6]
    dc = [0.1, 0.6, 0.3]
    eps = eps_s / 4.0                       # b_k = 4 beta_k
    a = [dc[k] / (eps + beta[k]) ** 2 for k in range(3)]
    return sum(a[k] * q[k] for k in range(3)) / sum(a)


def weno7_value(v, eps_s):
    """Left-biased WENO7 value at x_{j+1/2} from v_{j-3} .. v_{j+3}."""
    d = [v[i + 1] - v[i] for i in range(6)]
    e = [d[i + 1] - d[i] for i in range(5)]
    A = [2 * d[0] - 7 * d[1] + 11 * d[2], -d[1] + 5 * d[2] + 2 * d[3], 2 * d[2] + 5 * d[3] - d[4],
         11 * d[3] - 7 * d[4] + 2 * d[5]]
    B = [2 * e[1] - e[0], e[2], e[2], 2 * e[3] - e[4]]
    C = [e[k + 1] - e[k] for k in range(4)]
    b = [A[k] ** 2 + 39 * B[k] ** 2 + 781 / 20 * C[k] ** 2 + eps_s for k in range(4)]
    q = [(-3 * v[0] + 13 * v[1] - 23 * v[2] + 25 * v[3]) / 12, (v[1] - 5 * v[2] + 13 * v[3] + 3 * v[4]) / 12,
         (-v[2] + 7 * v[3] + 7 * v[4] - v[5]) / 12, (3 * v[3] + 13 * v[4] - 5 * v[5] + v[6]) / 12]
    dc = [1 / 35, 12 / 35, 18 / 35, 4 / 35]
    a = [dc[k] / b[k] ** 2 for k in range(4)]
    return sum(a[k] * q[k] for k in range(4)) / sum(a)


VALUE = {3: weno5_value, 4: weno7_value}
H = 1e-30


def cs_grad(f, x):
    """Complex-step gradient of the real function f at x (exact to rounding)."""
    g = np.empty(len(x))
    for i in range(len(x)):
        z = np.array(x, dtype=complex)
        z[i] += 1j * H
        g[i] = f(z).imag / H
    return g


def windows(rng, r, n):
    """Windows with the spread of a smooth profile, of a jump and of noise."""
    S = 2 * r - 1
    out = []
    for c in range(n):
        kind = c % 3
        x = np.arange(S, dtype=float)
        if kind == 0:
            v = rng.uniform(0.5, 2.0) + 0.1 * np.sin(rng.uniform(0.2, 1.0) * x + rng.uniform(0, 6))
        elif kind == 1:
            v = np.where(x < rng.integers(1, S), rng.uniform(1, 3), rng.uniform(-1, 1))
        else:
            v = rng.normal(size=S)
        out.append(v * 10.0 ** rng.uniform(-3, 3))
    return out


@pytest.mark.parametrize("r", [3, 4])
def test_face_vjp_against_complex_step(lib, r):
    rng = np.random.default_rng(1604 + r)
    S = 2 * r - 1
    worst = 0.0
    for v in windows(rng, r, 300):
        scale = np.abs(v).max()
        for eps_s in (1e-6 * scale ** 2, 1e-12 * scale ** 2 + 1e-40):
            rbar = rng.normal()
            ref = rbar * cs_grad(lambda z: VALUE[r](z, eps_s), v)
            got = {}
            for emu in (0, 1, 3, 7):
                out = np.zeros(S)
                lib.face_vjp(r, emu, P(np.ascontiguousarray(v)), eps_s, rbar, P(out))
                got[emu] = out
            for emu in (1, 3, 7):
                assert np.array_equal(got[emu], got[0]), (emu, got[emu], got[0])
            err = np.abs(got[0] - ref).max() / (np.abs(ref).max() + abs(rbar) * 1e-300)
            worst = max(worst, err)
    assert worst < 1e-11, worst


def pencil_objective(gp, gm, lam, sc, eps_s, r, j0, j1, off):
    """sum_j Fbar_j (R+(g+ window) + R-(g- window)) over faces j0 .. j1."""
    G, n = r, len(lam)
    lam_at = lambda m: lam[m] if 0 <= m < n else 0.0  # noqa: E731
    tot = 0.0
    for j in range(j0, j1 + 1):
        fb = sc * (lam_at(j + 1) - lam_at(j))
        wp = [gp[m + off] for m in range(j - G + 1, j + G)]
        wm = [gm[m + off] for m in range(j + G, j - G + 1, -1)]   # mirrored: cells j+G .. j-G+2
        tot = tot + fb * (VALUE[r](wp, eps_s) + VALUE[r](wm, eps_s))
    return tot


@pytest.mark.parametrize("r", [3, 4])
@pytest.mark.parametrize("segs", ["whole", "split"])
def test_pencil_sweep_against_complex_step(lib, r, segs):
    rng = np.random.default_rng(7 + r)
    G, n = r, 23
    off = G + 1
    ne = n + 2 * off
    x = np.linspace(-1, 1, ne)
    gp = 2.0 + np.tanh(6 * x) + 0.05 * rng.normal(size=ne)
    gm = 1.5 - 0.5 * np.tanh(5 * (x - 0.2)) + 0.05 * rng.normal(size=ne)
    lam = rng.normal(size=n)
    sc, eps_s = 0.37, 1e-6
    # faces -1 .. n-1 (every face of a pencil of n cells), in one or two segments
    parts = [(-1, n - 1)] if segs == "whole" else [(-1, 10), (11, n - 1)]
    op, om = np.zeros(ne), np.zeros(ne)
    cnt = np.zeros(ne, dtype=np.int32)
    for j0, j1 in parts:
        c = np.zeros(ne, dtype=np.int32)
        lib.pencil_vjp(r, n, off, P(gp), P(gm), P(lam), sc, eps_s, j0, j1, P(op), P(om),
                       c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        # every cell of the segment's windows emitted exactly once
        lo, hi = j0 - G + 1, j1 + G
        assert np.all(c[lo + off:hi + off + 1] == 1) and c.sum() == hi - lo + 1, c
        cnt += c
    z = np.concatenate([gp, gm])

    def f(zz):
        return pencil_objective(zz[:ne], zz[ne:], lam, sc, eps_s, r, -1, n - 1, off)
    ref = cs_grad(f, z)
    got = np.concatenate([op, om])
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err < 1e-11, err
