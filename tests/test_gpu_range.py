"""Range of the device arithmetic that replaces IEEE division.

* The kernels' reciprocal (MUFU seed + one cubic Newton correction) against
  IEEE 1/x over the whole documented exponent range: at most one ulp off.
* The WENO face value uses one reciprocal of the product D+ D- of the two
  reconstructions' weight denominators; those products span a far wider range
  than the data.  Parity with the oracle (which normalises alpha_k / sum
  alpha) is checked on data scaled by 1e-8 .. 1e20 and with epsilon at both
  ends of its accepted range, where the plain product would underflow or
  overflow and the kernels must take their rescaled path."""
import numpy as np
import pytest

import oracle
import workloads as W
from parity import TOL, assert_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1604_03360_gb300.build as B
    B.build()
    oracle.build()


def _ulps(a, b):
    """|a - b| in units in the last place (a, b finite, of equal sign)."""
    ia, ib = a.view(np.int64), b.view(np.int64)
    return np.abs(ia - ib)


def test_rcp_within_one_ulp_of_ieee():
    import torch
    from paper_1604_03360_gb300 import eval_rcp
    rng = np.random.default_rng(31)
    n = 1 << 22
    # log-uniform magnitudes over the documented range 2^-1022 .. 2^1022, both signs
    x = np.ldexp(rng.uniform(1.0, 2.0, n), rng.integers(-1021, 1022, n)) * rng.choice([-1.0, 1.0], n)
    # exact powers of two, their neighbours and mantissas with long carry chains
    k = np.arange(-1021, 1022)
    special = np.concatenate([np.ldexp(1.0, k), np.nextafter(np.ldexp(1.0, k), np.inf),
                              np.nextafter(np.ldexp(2.0, k - 1), 0.0), np.ldexp(1.5, k), np.ldexp(1.0 + 2.0 ** -52, k),
                              -np.ldexp(1.0, k)])
    x = np.concatenate([x, special])
    y = eval_rcp(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = 1.0 / x
    assert np.all(np.sign(y) == np.sign(ref))
    u = _ulps(y, ref)
    assert u.max() <= 1, (u.max(), x[np.argmax(u)])
    exact = np.mean(u == 0)
    assert exact > 0.999, exact
    # powers of two are exact
    p2 = np.ldexp(1.0, k)
    assert np.array_equal(eval_rcp(torch.from_numpy(p2).cuda()).cpu().numpy(), 1.0 / p2)


@pytest.mark.parametrize("scheme", [5, 7])
@pytest.mark.parametrize("scale", [1e-8, 1e8, 1e12, 1e20])
def test_scaled_energy_density(scheme, scale):
    """Ellipsoidal flow with e multiplied by `scale` (p = e/3 is scale free,
    so the flow is the same up to the WENO epsilon).  At 1e12 and 1e20 the
    WENO7 denominators leave [2^-448, 2^448] and the rescaled face path runs;
    at 1e20 the plain product D+ D- would overflow."""
    g, w = W.ellipsoidal(N=36, scheme=scheme)
    w[0] *= scale
    g.cfl = 0.3 * 36 / 256
    assert_parity(g, w, 8)


def _uniform_block(scheme, eps):
    """Lumpy data clipped from below, so most of the box is exactly uniform
    (every difference there is exactly zero), with a smooth flow elsewhere."""
    g, w = W.lumpy(n=(26, 21, 19), seed=44, scheme=scheme)
    w[0] = np.maximum(w[0], 0.6)
    w[4] = w[0].copy()
    w[1] = np.where(w[0] > 0.6, 0.2 * np.tanh(w[0] - 1.0), 0.0)
    g.eps = eps
    return g, w


@pytest.mark.parametrize("scheme", [5, 7])
def test_smallest_epsilon_on_uniform_block(scheme):
    """eps = 1e-40: in the uniform region beta = 0, so each denominator is a
    power of eps (about 1e-227 for WENO7) and D+ D- would underflow."""
    g, w = _uniform_block(scheme, 1e-40)
    assert_parity(g, w, 6)


@pytest.mark.parametrize("scheme", [5, 7])
def test_largest_epsilon_linear_weights(scheme):
    """eps = 1e30: the weights are the linear ones and D ~ eps^(2(r-1))."""
    g, w = W.smooth_periodic(n=(19, 13, 11), amp=0.3, vamp=0.5, seed=9, scheme=scheme)
    g.eps = 1e30
    g.cfl = 0.4
    assert_parity(g, w, 6)
    g, w = _uniform_block(scheme, 1e30)
    assert_parity(g, w, 6)


def test_epsilon_outside_range_rejected():
    from paper_1604_03360_gb300 import Hydro, HydroError
    for eps in (1e-41, 1e31):
        with pytest.raises(HydroError) as ei:
            Hydro((8, 8, 8), (0.1, 0.1, 0.1), eps=eps)
        assert ei.value.code == 1 and "weno_eps" in str(ei.value)
