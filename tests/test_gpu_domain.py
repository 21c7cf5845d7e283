"""z-slab domain decomposition on one GPU: a grid cut into slabs (halo
handles driven one RK stage at a time, ghost planes exchanged and speeds
max-reduced between stages) must reproduce the whole-grid run bit for bit,
since every cell's arithmetic, every speed maximum and hence every dt are the
same.  The whole-grid run is itself parity-tested against the oracle."""
import numpy as np
import pytest

import workloads as W
from parity import run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1604_03360_gb300.build as B
    B.build()


def with_flow(g, w, scale=0.3):
    x, y, z = g.centres()
    sh = w[0].shape
    w[1] = np.broadcast_to(scale * np.tanh(x / 3.0) * np.ones_like(y), sh)
    w[2] = np.broadcast_to(-0.5 * scale * np.tanh((y - 0.5) / 2.0) * np.ones_like(z), sh)
    w[3] = np.broadcast_to(0.4 * scale * np.sin(z / 2.0) * np.ones_like(x), sh)
    return w


def run_slabs(g, w, nslabs, nsteps, device=None, t_end=-1.0, variant=None):
    from paper_1604_03360_gb300.domain import LocalExchange, SlabDomain, split_grid
    slabs, bounds = split_grid(g, nslabs)
    try:
        for s, (z0, z1) in zip(slabs, bounds):
            if variant is not None:
                s.set_launch(variant)
            s.set_primitive(np.ascontiguousarray(w[:, z0:z1]))
        dom = SlabDomain(LocalExchange(slabs, g.bc[2], device=device))
        dom.loaded()
        dom.step(nsteps, t_end)
        parts = [s.get_state() for s in slabs]
        ts = {(s.t, s.steps) for s in slabs}
        assert len(ts) == 1, ts
        t, k = ts.pop()
        return np.concatenate(parts, axis=1), t, k
    finally:
        for s in slabs:
            s.close()


def check(g, w, nslabs, nsteps, device=None, t_end=-1.0):
    ref, tr, kr = run_gpu(g, w, nsteps, t_end=t_end)
    got, tg, kg = run_slabs(g, w, nslabs, nsteps, device=device, t_end=t_end)
    assert (kg, tg) == (kr, tr)
    assert np.array_equal(got, ref), np.max(np.abs(got - ref))


@pytest.mark.parametrize("scheme", [5, 7, 2])
@pytest.mark.parametrize("nslabs", [2, 3])
def test_outflow_slabs_match_whole_grid(scheme, nslabs):
    g, w = W.lumpy(n=(21, 17, 26), seed=11, scheme=scheme)
    w = with_flow(g, w)
    check(g, w, nslabs, 5, device="cuda")


@pytest.mark.parametrize("scheme,variant", [(5, 7), (5, 8), (7, 6), (7, 7), (5, 10), (7, 11), (7, 12), (5, 12),
                                            (7, 13)])
def test_zpass_slabs_match_whole_grid(scheme, variant):
    """Slabs whose z faces come from the z pass (which reads the stored ghost
    planes) advance bit for bit like the whole grid on the fused kernel; so do
    slabs on the TMA-staged variants, whose tensor maps span the stored ghost
    planes (those need an even nx)."""
    g, w = W.lumpy(n=(22 if variant >= 10 else 21, 17, 26), seed=12, scheme=scheme)
    w = with_flow(g, w)
    ref, tr, kr = run_gpu(g, w, 4)
    got, tg, kg = run_slabs(g, w, 3, 4, device="cuda", variant=variant)
    assert (kg, tg) == (kr, tr)
    assert np.array_equal(got, ref), np.max(np.abs(got - ref))


@pytest.mark.parametrize("scheme", [5, 7, 2])
def test_periodic_slabs_match_whole_grid(scheme):
    g, w = W.smooth_periodic(n=(13, 11, 17), amp=0.3, vamp=0.5, seed=9, scheme=scheme)
    check(g, w, 3, 6, device="cuda")


def test_periodic_one_slab_wraps_onto_itself():
    g, w = W.smooth_periodic(n=(12, 10, 9), amp=0.3, vamp=0.5, seed=2, scheme=5)
    check(g, w, 1, 4, device="cuda")


def test_host_staging_thin_slabs_and_t_end():
    """Slabs exactly G = 4 planes thick (WENO7), staged through host memory,
    stopping at t_end mid-run."""
    g, w = W.lumpy(n=(18, 15, 16), seed=3, scheme=7)
    w = with_flow(g, w)
    ref, tr, kr = run_gpu(g, w, 10)
    check(g, w, 4, 10, device=None, t_end=0.5 * tr)


@pytest.mark.parametrize("scheme,variant", [(5, 2), (7, 1), (5, 4), (7, 3)])
def test_local_lf_zpass_slabs(scheme, variant):
    """Local-LF slabs on the z-pass launch: the z pass reads the exchanged
    ghost planes of u, the primitives and the speeds."""
    g, w = W.lumpy(n=(19, 15, 22), seed=31, scheme=scheme)
    w = with_flow(g, w)
    g.split = 1
    ref, tr, kr = run_gpu(g, w, 4)
    got, tg, kg = run_slabs(g, w, 3, 4, device="cuda", variant=variant)
    assert (kg, tg) == (kr, tr)
    assert np.array_equal(got, ref), np.max(np.abs(got - ref))


def test_local_lf_and_charges():
    g, w = W.lumpy(n=(16, 14, 20), seed=8, scheme=5)
    w = W.with_charges(g, with_flow(g, w), nq=3)
    g.nq, g.split = 3, 1
    check(g, w, 2, 4, device="cuda")


def test_halo_handle_rejects_whole_grid_calls():
    from paper_1604_03360_gb300 import HydroError
    from paper_1604_03360_gb300.domain import split_grid
    g, w = W.lumpy(n=(8, 8, 12), seed=1, scheme=5)
    slabs, bounds = split_grid(g, 2)
    try:
        s = slabs[0]
        s.set_primitive(np.ascontiguousarray(w[:, :6]))
        with pytest.raises(HydroError):
            s.step(1)
        with pytest.raises(HydroError):
            s.stage(5)
        assert s.halo_doubles() == (5 + 4) * 3 * 8 * 8
    finally:
        for s in slabs:
            s.close()


@pytest.mark.parametrize("scheme", [5, 7])
def test_charwise_slabs(scheme):
    g, w = W.lumpy(n=(17, 15, 22), seed=19, scheme=scheme)
    w = with_flow(g, w)
    g.charwise = 1
    check(g, w, 3, 4, device="cuda")


def test_gas_eos_slabs():
    g, w = W.lumpy(n=(17, 15, 22), seed=23, scheme=5)
    w = with_flow(g, w)
    w[0] = w[0] + w[4]
    g.cs2, g.mass = 2.0 / 3.0, 1.0
    check(g, w, 3, 4, device="cuda")


@pytest.mark.parametrize("scheme,variant,bc", [(7, None, (0, 0, 0)), (7, 7, (0, 1, 1)), (5, 8, (1, 0, 0)),
                                               (2, None, (0, 0, 0))])
def test_slabs_match_oracle(scheme, variant, bc):
    """The slab run against the CPU oracle directly (not only against the
    whole-grid GPU run): three slabs, six steps, outflow or periodic z."""
    import oracle
    from parity import TOL, field_errors, run_oracle
    g, w = W.lumpy(n=(23, 19, 27), seed=29, scheme=5 if scheme == 2 else scheme)
    w = with_flow(g, w)
    g.scheme, g.bc = scheme, bc
    oracle.build()
    ref, tr, kr = run_oracle(g, w, 6)
    got, tg, kg = run_slabs(g, w, 3, 6, device="cuda", variant=variant)
    assert kg == kr == 6 and abs(tg - tr) <= 1e-13 * tr
    err = field_errors(got, ref)
    assert np.all(err <= TOL), err
