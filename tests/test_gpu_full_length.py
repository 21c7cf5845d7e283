"""GPU vs oracle after the full step counts of the paper's test
configurations (Sec. 3): Hubble-like expansion at 128^3 for 100 steps
(WENO5 and WENO7) and ellipsoidal flow at 128^3 for 200 steps (WENO7, CFL
scaled by 128/256 so that dt and the physical time match the 256^3 run),
on the default launch.

The oracle needs minutes of host time per case, so its states come from
tests/golden/make_full_length.py (which calls only the oracle): sampled cells,
field maxima and per-plane sums and maxima (full_length.py).  One case, the
cheapest, is also recomputed here by the oracle and compared element by
element over the whole grid."""
import numpy as np
import pytest

import oracle
from full_length import MFL, check_against_stored
from parity import TOL, field_errors, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1604_03360_gb300.build as B
    B.build()
    oracle.build()


@pytest.mark.parametrize("name", ["hubble128_weno5", "hubble128_weno7", "ellipsoidal128_weno7"])
def test_full_length_against_stored_oracle(name):
    g, w, nsteps = MFL.case(name)
    u, t, k = run_gpu(g, w, nsteps, t0=g.t0)
    check_against_stored(u, t, k, name)


def test_hubble128_weno5_full_length_every_cell():
    """All 100 steps of the 128^3 Hubble configuration (WENO5), the oracle run
    in this process: every cell of every field within the tolerance."""
    g, w, nsteps = MFL.case("hubble128_weno5")
    ref, tr, kr = run_oracle(g, w, nsteps, t0=g.t0)
    got, tg, kg = run_gpu(g, w, nsteps, t0=g.t0)
    assert kg == kr == nsteps and abs(tg - tr) <= 1e-13 * tr
    err = field_errors(got, ref)
    assert np.all(err <= TOL), err
