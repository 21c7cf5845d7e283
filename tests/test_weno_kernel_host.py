"""The stage kernels' WENO5 / WENO7 reconstruction source (csrc/hydro_math.cuh:
the difference windows, their slides along a pencil and the cores that return
centre + M / D), compiled for the host with nvcc and run on the CPU:

* one face, left- and right-biased, against the definition of FD-WENO
  (tests/weno_definition.py, evaluated in floating point), for every
  integer-pipe choice, which must also agree with each other bit for bit;
* a pencil sweep that carries the window from face to face (the *_slide and
  *_slide_mirror functions the pencil kernels use) against fresh windows at
  every face, bit for bit.

Only the host build of the same source runs here; the device build is
checked against the oracle by the GPU parity tests."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest
import sympy as sp

from weno_definition import definition

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1604_03360_gb300", "csrc")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")

SRC = r'''
#include "hydro_math.cuh"
using namespace hydro;

template <int R, int EMU>
static void face(const double* v, double eps, int right, double* out)
{
    double M, D;
    if (right) weno_right<R, EMU>(v, eps, M, D);
    else weno_left<R, EMU>(v, eps, M, D);
    out[0] = M;
    out[1] = D;
}
extern "C" void face_md(int r, int emu, int right, const double* v, double eps, double* out)
{
    if (r == 3) {
        switch (emu) {
        case 0: face<3, 0>(v, eps, right, out); break;
        case 1: face<3, 1>(v, eps, right, out); break;
        case 3: face<3, 3>(v, eps, right, out); break;
        default: face<3, 7>(v, eps, right, out); break;
        }
    } else {
        switch (emu) {
        case 0: face<4, 0>(v, eps, right, out); break;
        case 1: face<4, 1>(v, eps, right, out); break;
        case 3: face<4, 3>(v, eps, right, out); break;
        default: face<4, 7>(v, eps, right, out); break;
        }
    }
}

// faces j = 0 .. n-2r+1 of the pencil g[0 .. n-1]: left-biased from
// g[j .. j+2r-2] and right-biased (mirrored) from g[j+1 .. j+2r-1], with the
// window carried from face to face; out: M, D left, M, D right per face
template <int R>
struct Win;
template <> struct Win<3> {
    using T = Diff5;
    static void fresh(const double* v, double e, T& q) { weno5_diffs<7>(v, e, q); }
    static void slide(const double* v, double e, T& q) { weno5_slide<7>(v, e, q); }
    static void slide_m(const double* m, double e, T& q) { weno5_slide_mirror<7>(m, e, q); }
    static void core(const T& q, double, double& M, double& D) { weno5_core<7>(q, M, D); }
};
template <> struct Win<4> {
    using T = Diff7;
    static void fresh(const double* v, double e, T& q) { weno7_diffs<7>(v, e, q); }
    static void slide(const double* v, double e, T& q) { weno7_slide<7>(v, e, q); }
    static void slide_m(const double* m, double e, T& q) { weno7_slide_mirror<7>(m, e, q); }
    static void core(const T& q, double, double& M, double& D) { weno7_core<7>(q, M, D); }
};
template <int R>
static void sweep(const double* g, int n, double eps, double* out)
{
    constexpr int S = 2 * R - 1;
    typename Win<R>::T qp, qm;
    for (int j = 0; j + S < n; ++j) {
        double m[S];
        for (int i = 0; i < S; ++i) m[i] = g[j + S - i];        // cells j+S .. j+1
        if (j == 0) {
            Win<R>::fresh(g, eps, qp);
            Win<R>::fresh(m, eps, qm);
        } else {
            Win<R>::slide(g + j, eps, qp);
            Win<R>::slide_m(m, eps, qm);
        }
        Win<R>::core(qp, eps, out[4 * j], out[4 * j + 1]);
        Win<R>::core(qm, eps, out[4 * j + 2], out[4 * j + 3]);
    }
}
extern "C" void pencil_md(int r, const double* g, int n, double eps, double* out)
{
    if (r == 3) sweep<3>(g, n, eps, out);
    else sweep<4>(g, n, eps, out);
}
'''


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    if not (os.path.exists(NVCC) or shutil.which("nvcc")):
        pytest.skip("nvcc is not available")
    d = tmp_path_factory.mktemp("wenohost")
    src = d / "weno_host.cu"
    src.write_text(SRC)
    so = d / "libweno_host.so"
    subprocess.run([NVCC, "-std=c++17", "-O2", "-shared", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
                    "-gencode", "arch=compute_103a,code=sm_103a", "-I", CSRC, str(src), "-o", str(so)], check=True)
    L = ctypes.CDLL(str(so))
    dp = ctypes.POINTER(ctypes.c_double)
    L.face_md.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, ctypes.c_double, dp]
    L.pencil_md.argtypes = [ctypes.c_int, dp, ctypes.c_int, ctypes.c_double, dp]
    return L


def P(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


_DEF = {}


def reference(r):
    """The definition's left-biased value as a float function of the window
    and of eps (in the definition's own scale)."""
    if r not in _DEF:
        v, qs, betas, lin = definition(r)
        eps = sp.symbols("eps")
        a = [lin[k] / (eps + betas[k]) ** 2 for k in range(r)]
        val = sum(a[k] * qs[k] for k in range(r)) / sum(a)
        _DEF[r] = sp.lambdify((v, eps), val, "math")
    return _DEF[r]


SCALE = {3: 4.0, 4: 36.0}      # b_k = SCALE beta_k on the kernels' inputs


def windows(rng, S, n):
    out = []
    for c in range(n):
        x = np.arange(S, dtype=float)
        kind = c % 3
        if kind == 0:
            w = rng.uniform(0.5, 2.0) + 0.1 * np.sin(rng.uniform(0.2, 1.0) * x + rng.uniform(0, 6))
        elif kind == 1:
            w = np.where(x < rng.integers(1, S), rng.uniform(1, 3), rng.uniform(-1, 1))
        else:
            w = rng.normal(size=S)
        out.append(w * 10.0 ** rng.uniform(-3, 3))
    return out


@pytest.mark.parametrize("r", [3, 4])
def test_face_against_definition(lib, r):
    S = 2 * r - 1
    ref = reference(r)
    rng = np.random.default_rng(11 + r)
    worst = 0.0
    for v in windows(rng, S, 300):
        scale = np.abs(v).max()
        for eps_s in (1e-6 * scale ** 2, 1e-3 * scale ** 2):
            for right in (0, 1):
                got = {}
                for emu in (0, 1, 3, 7):
                    out = np.zeros(2)
                    lib.face_md(r, emu, right, P(np.ascontiguousarray(v)), eps_s, P(out))
                    got[emu] = out
                for emu in (1, 3, 7):
                    assert np.array_equal(got[emu], got[0]), (emu, got[emu], got[0])
                w = v[::-1] if right else v
                value = w[r - 1] + got[0][0] / got[0][1]
                expect = ref(list(w), eps_s / SCALE[r])
                worst = max(worst, abs(value - expect) / scale)
    assert worst < 1e-13, worst


@pytest.mark.parametrize("r", [3, 4])
def test_pencil_sweep_equals_fresh_windows(lib, r):
    S = 2 * r - 1
    rng = np.random.default_rng(23 + r)
    n = 64
    x = np.linspace(-1, 1, n)
    g = np.ascontiguousarray(2.0 + np.tanh(8 * x) + 0.05 * rng.normal(size=n))
    eps_s = 1e-6
    nf = n - S
    out = np.zeros(4 * nf)
    lib.pencil_md(r, P(g), n, eps_s, P(out))
    for j in range(nf):
        left = np.zeros(2)
        right = np.zeros(2)
        lib.face_md(r, 7, 0, P(np.ascontiguousarray(g[j:j + S])), eps_s, P(left))
        lib.face_md(r, 7, 1, P(np.ascontiguousarray(g[j + 1:j + 1 + S])), eps_s, P(right))
        assert np.array_equal(out[4 * j:4 * j + 2], left), j
        assert np.array_equal(out[4 * j + 2:4 * j + 4], right), j
