"""hydro_run_many: a stream of independent initial states on one grid (the
event-by-event use that motivates the paper's GPU code, Sec. 1), with the
copies in and out double-buffered against the steps.  Every item must give
bit for bit what set_state + step + get_state give, and match the oracle."""
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


def _items(n, scheme, dims=(29, 23, 19)):
    out = []
    for i in range(n):
        g, w = W.lumpy(n=dims, seed=300 + i, scheme=scheme)
        out.append(oracle.prim2con(w))
    return g, out


def _one_by_one(g, u0s, nsteps, t0):
    from paper_1604_03360_gb300 import Hydro
    res = []
    with Hydro.from_grid(g) as h:
        for u in u0s:
            h.set_state(np.ascontiguousarray(u), t=t0)
            h.step(nsteps)
            res.append((h.get_state(), h.t, h.steps))
    return res


@pytest.mark.parametrize("scheme", [5, 7])
def test_run_many_pinned_matches_one_by_one_and_oracle(scheme):
    import torch
    from paper_1604_03360_gb300 import Hydro
    g, u0s = _items(5, scheme)
    ins = [torch.from_numpy(u).pin_memory() for u in u0s]
    outs = [torch.full_like(x, float("nan")).pin_memory() for x in ins]
    with Hydro.from_grid(g) as h:
        h.run_many(ins, outs, nsteps=3, t0=0.5)
        last = h.get_state()
        t_last = h.t
    ref = _one_by_one(g, u0s, 3, 0.5)
    for o, (r, t, k) in zip(outs, ref):
        assert np.array_equal(o.numpy(), r)
    assert np.array_equal(last, ref[-1][0]) and t_last == ref[-1][1]
    want = oracle.run(oracle_cfg(g), u0s[2], 3, t=0.5)[0]
    assert np.all(field_errors(outs[2].numpy(), want) <= TOL)


def test_run_many_pageable_buffers_same_input_and_repeat_calls():
    """Pageable numpy buffers (copies do not overlap, results the same); one
    input buffer for every item; a second call reuses the staging buffers."""
    from paper_1604_03360_gb300 import Hydro
    g, u0s = _items(3, 5, dims=(24, 20, 1))
    outs = [np.empty_like(u0s[0]) for _ in range(4)]
    with Hydro.from_grid(g) as h:
        h.run_many([u0s[1]] * 4, outs, nsteps=2)
        for o in outs[1:]:
            assert np.array_equal(o, outs[0])
        outs2 = [np.empty_like(u) for u in u0s]
        h.run_many(u0s, outs2, nsteps=2)
    ref = _one_by_one(g, u0s, 2, 0.0)
    assert np.array_equal(outs[0], ref[1][0])
    for o, (r, _, _) in zip(outs2, ref):
        assert np.array_equal(o, r)


def test_run_many_reports_the_unphysical_item():
    from paper_1604_03360_gb300 import Hydro, HydroError
    g, u0s = _items(4, 5)
    bad = u0s[2].copy()
    bad[1, 3, 4, 5] = 2.0 * bad[0, 3, 4, 5]          # |M| > E
    outs = [np.empty_like(u) for u in u0s]
    with Hydro.from_grid(g) as h:
        with pytest.raises(HydroError) as ei:
            h.run_many([u0s[0], u0s[1], bad, u0s[3]], outs, nsteps=1)
        assert ei.value.code == 4 and "item 2" in str(ei.value)
        # the items before and after it are still computed
        h.run_many([u0s[3]], outs[:1], nsteps=1)
    ref = _one_by_one(g, [u0s[3]], 1, 0.0)
    assert np.array_equal(outs[0], ref[0][0]) and np.array_equal(outs[3], ref[0][0])


def test_run_many_argument_checks():
    from paper_1604_03360_gb300 import Hydro, HydroError
    g, u0s = _items(1, 5, dims=(12, 11, 10))
    with Hydro.from_grid(g) as h:
        h.run_many([], [], nsteps=1)                   # nothing to do
        with pytest.raises(ValueError):
            h.run_many(u0s, [], nsteps=1)
        with pytest.raises(HydroError):
            h.run_many(u0s, [np.empty_like(u0s[0])], nsteps=-1)
