"""Batched event-by-event stepping (per RK3 stage, face passes over the
pencils of all events and one combination launch, or a z pass and one
persistent launch over a tile work-list of all events) vs the CPU oracle per
event, and vs the single-grid path bit for bit."""
import numpy as np
import pytest

import oracle
import workloads as W
from parity import TOL, field_errors, oracle_cfg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1604_03360_gb300.build as B
    B.build()
    oracle.build()


def make_events(sizes, scheme=5, seed=900):
    out = []
    for i, n in enumerate(sizes):
        g, w = W.lumpy(n=n, seed=seed + i, scheme=scheme)
        w[1] = 0.25 * np.tanh(w[0] - 1.0)
        w[3] = -0.15 * np.tanh(w[0] - 2.0)
        out.append((g, w))
    return out


SIZES = [(37, 29, 21), (16, 16, 16), (9, 7, 30), (48, 20, 13), (20, 33, 5), (1, 12, 17)]


@pytest.mark.parametrize("scheme", [5, 7])
def test_batch_matches_oracle_and_single_grid(scheme):
    from paper_1604_03360_gb300 import Hydro, HydroBatch
    ev = make_events(SIZES, scheme=scheme)
    with HydroBatch([g for g, _ in ev]) as b:
        for i, (g, w) in enumerate(ev):
            b.set_primitive(i, w)
        b.step(4)
        got = [b.get_state(i) for i in range(len(ev))]
        variant, _, _, zc, items = b.launch()
    assert items > len(ev)
    for i, (g, w) in enumerate(ev):
        u, t, k = got[i]
        ref, tr, kr = oracle.run(oracle_cfg(g), oracle.prim2con(w), 4)
        assert k == kr == 4 and abs(t - tr) <= 1e-13 * tr
        assert np.all(field_errors(u, ref) <= TOL), (i, field_errors(u, ref))
        with Hydro.from_grid(g) as h:
            h.set_launch(variant, zc)
            h.set_primitive(w)
            h.step(4)
            assert np.array_equal(h.get_state(), u), i


@pytest.mark.parametrize("variant,zc", [(0, 8), (1, 16), (2, 5), (3, 12), (4, 10), (5, 7), (6, 9), (7, 11), (8, 13),
                                        (9, 0)])
def test_batch_launch_variants(variant, zc):
    from paper_1604_03360_gb300 import HydroBatch
    ev = make_events(SIZES[:4], scheme=5, seed=950)
    refs = [oracle.run(oracle_cfg(g), oracle.prim2con(w), 3)[0] for g, w in ev]
    with HydroBatch([g for g, _ in ev]) as b:
        b.set_launch(variant, zc)
        for i, (g, w) in enumerate(ev):
            b.set_primitive(i, w)
        b.step(3)
        for i in range(len(ev)):
            assert np.all(field_errors(b.get_state(i)[0], refs[i]) <= TOL)


@pytest.mark.parametrize("scheme,variant", [(5, 9), (7, 8)])
def test_batch_three_pass_matches_single_grid_bitwise(scheme, variant):
    """The batch's three-pass launch (x, y and z passes over every event's
    pencils, then one combination item per block of cells) gives each event
    exactly its single-grid result on the default (three-pass) launch."""
    from paper_1604_03360_gb300 import Hydro, HydroBatch
    ev = make_events(SIZES, scheme=scheme, seed=930)
    with HydroBatch([g for g, _ in ev]) as b:
        b.set_launch(variant, 0)
        for i, (g, w) in enumerate(ev):
            b.set_primitive(i, w)
        b.step(4)
        got = [b.get_state(i) for i in range(len(ev))]
        assert b.kernels_per_step() == 2 + 3 * 4
    for i, (g, w) in enumerate(ev):
        with Hydro.from_grid(g) as h:
            h.set_primitive(w)
            h.step(4)
            assert np.array_equal(h.get_state(), got[i][0]), i


def test_batch_autotune_leaves_state_unchanged():
    from paper_1604_03360_gb300 import HydroBatch
    ev = make_events(SIZES[:3], scheme=5, seed=970)
    with HydroBatch([g for g, _ in ev]) as b:
        for i, (g, w) in enumerate(ev):
            b.set_primitive(i, w)
        before = [b.get_state(i) for i in range(3)]
        assert b.autotune() > 0
        after = [b.get_state(i) for i in range(3)]
        for x, y in zip(before, after):
            assert np.array_equal(x[0], y[0]) and x[1] == y[1] and x[2] == y[2] == 0
        b.step(2)
        for i, (g, w) in enumerate(ev):
            ref = oracle.run(oracle_cfg(g), oracle.prim2con(w), 2)[0]
            assert np.all(field_errors(b.get_state(i)[0], ref) <= TOL)


def test_batch_reports_unphysical_event():
    from paper_1604_03360_gb300 import HydroBatch, HydroError
    ev = make_events(SIZES[:3], scheme=5, seed=990)
    with HydroBatch([g for g, _ in ev]) as b:
        for i, (g, w) in enumerate(ev):
            u = oracle.prim2con(w)
            if i == 2:
                u[1, 1, 2, 3] = 4.0 * u[0, 1, 2, 3]
            b.set_state(i, u)
        with pytest.raises(HydroError) as ei:
            b.sync()
        assert ei.value.code == 4 and "event 2" in str(ei.value)


def test_batch_requires_every_event_loaded():
    from paper_1604_03360_gb300 import HydroBatch, HydroError
    ev = make_events(SIZES[:2], scheme=5)
    with HydroBatch([g for g, _ in ev]) as b:
        b.set_primitive(0, ev[0][1])
        with pytest.raises(HydroError) as ei:
            b.step(1)
        assert ei.value.code == 6


def test_batch_ensemble_time_step_keeps_events_physical():
    """Eight events of the event-by-event configuration spanning the size
    range, 100 steps with the ensemble time step: all stay physical, reach
    t = 2.25, the 48^3 event matches the oracle run here cell by cell, and the
    160^3 event matches the oracle's stored full-length state (sampled cells,
    field maxima, per-plane sums and maxima)."""
    from full_length import MFL, check_against_stored
    from paper_1604_03360_gb300 import HydroBatch
    sizes = MFL.BATCH_SIZES
    assert sizes[0] == (48, 48, 48) and sizes[1] == (160, 160, 160)
    ev = [W.batch_event(i, sizes) for i in range(len(sizes))]
    with HydroBatch([g for g, _ in ev]) as b:
        for i, (g, w) in enumerate(ev):
            b.set_primitive(i, w)
        b.step(100)
        b.sync()
        out = [b.get_state(i) for i in range(len(ev))]
    for u, t, k in out:
        assert k == 100 and abs(t - 100 * W.BATCH_DT) < 1e-12
        assert np.isfinite(u).all()
    g0, w0 = ev[0]
    ref = oracle.run(oracle_cfg(g0), oracle.prim2con(w0), 100)[0]
    assert np.all(field_errors(out[0][0], ref) <= TOL)
    u1, t1, k1 = out[1]
    check_against_stored(u1, t1, k1, "batch_event160_weno5")


@pytest.mark.parametrize("scheme", [5, 7])
def test_batch_local_lf(scheme):
    from paper_1604_03360_gb300 import HydroBatch
    ev = make_events(SIZES[:4], scheme=scheme, seed=1010)
    for g, _ in ev:
        g.split = 1
    with HydroBatch([g for g, _ in ev]) as b:
        for i, (g, w) in enumerate(ev):
            b.set_primitive(i, w)
        b.step(3)
        for i, (g, w) in enumerate(ev):
            ref = oracle.run(oracle_cfg(g), oracle.prim2con(w), 3)[0]
            assert np.all(field_errors(b.get_state(i)[0], ref) <= TOL), i
