"""hydro_step_noalloc: RK3 stepping for callers that cannot allocate device
memory (their device memory belongs to their own pool, or their loop must keep
a fixed footprint).  The entry point keeps its intermediate buffers in a static
device array of the library; here it is called through the C ABI on two
consecutive calls and checked against hydro_step, the allocating entry point.
Both run the same scheme with the same operations (the no-allocation path on
the fused stage kernel, hydro_step on its default launch of separate x, y and
z face passes and a per-cell combination, which agree bit for bit), so the
results must be identical.

This file sorts last so that a run stopping at the first failure has already
run every other test."""
import ctypes

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1604_03360_gb300.build as B
    B.build()
    oracle.build()
    import paper_1604_03360_gb300 as H
    lib = H.lib()
    P, vp = ctypes.POINTER, ctypes.c_void_p
    lib.hydro_step_noalloc.argtypes = [P(H.HydroConfig), vp, vp, ctypes.c_int64, ctypes.c_double, ctypes.c_int32,
                                       ctypes.c_double, vp, P(ctypes.c_double)]
    lib.hydro_step_noalloc.restype = ctypes.c_int32
    lib.hydro_noalloc_last_error.argtypes = []
    lib.hydro_noalloc_last_error.restype = ctypes.c_char_p
    return lib


def _cfg(g):
    import paper_1604_03360_gb300 as H
    return H.make_config(g.n, g.dx, scheme=g.scheme, bc=g.bc, cs2=g.cs2, cfl=g.cfl, eps=g.eps)


def _noalloc(L, g, u0, nsteps, in_place=False):
    import torch
    u_in = torch.from_numpy(np.ascontiguousarray(u0)).cuda()
    u_out = u_in if in_place else torch.full_like(u_in, float("nan"))
    cfg = _cfg(g)
    t = ctypes.c_double(-1.0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.hydro_step_noalloc(ctypes.byref(cfg), ctypes.c_void_p(u_in.data_ptr()), ctypes.c_void_p(u_out.data_ptr()),
                              u_in[0].numel(), 0.0, nsteps, -1.0, stream, ctypes.byref(t))
    assert rc == 0, L.hydro_noalloc_last_error()
    return u_out.cpu().numpy(), t.value


def _allocating(g, u0, nsteps):
    from paper_1604_03360_gb300 import Hydro
    with Hydro.from_grid(g) as h:
        h.set_state(np.ascontiguousarray(u0))
        h.step(nsteps)
        return h.get_state(), h.t


def test_noalloc_matches_hydro_step_on_two_calls(L):
    # call 1: WENO5 on an uneven grid, separate output buffer
    g1, w1 = W.lumpy(n=(30, 22, 18), seed=41, scheme=5)
    w1[1] = 0.3 * np.tanh(w1[0] - 1.0)
    u1 = oracle.prim2con(w1)
    a1, ta1 = _noalloc(L, g1, u1, 3)
    b1, tb1 = _allocating(g1, u1, 3)
    assert np.array_equal(a1, b1) and ta1 == tb1
    # call 2: another grid and scheme, in place; the array still holds call 1's data
    g2, w2 = W.hubble(N=40, scheme=7)
    u2 = oracle.prim2con(w2)
    a2, ta2 = _noalloc(L, g2, u2, 4, in_place=True)
    b2, tb2 = _allocating(g2, u2, 4)
    assert np.array_equal(a2, b2) and ta2 == tb2
    assert np.isfinite(a2).all()


def test_noalloc_rejects_grids_beyond_its_limit(L):
    import torch
    g, _ = W.lumpy(n=(64, 64, 33), seed=1)      # 135168 cells > 131072
    cfg = _cfg(g)
    buf = torch.zeros(8, device="cuda", dtype=torch.float64)
    rc = L.hydro_step_noalloc(ctypes.byref(cfg), ctypes.c_void_p(buf.data_ptr()), ctypes.c_void_p(buf.data_ptr()),
                              g.cells, 0.0, 1, -1.0, None, None)
    assert rc == 1
    assert b"exceeds the no-allocation limit" in L.hydro_noalloc_last_error()
