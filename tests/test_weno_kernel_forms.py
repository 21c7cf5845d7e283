"""The difference-basis forms of the stage kernels' WENO5 / WENO7
reconstructions (csrc/hydro_math.cuh: weno5_core, weno7_core and the carried
window terms) against the definition of FD-WENO (Sec. 1.2), in exact
arithmetic with sympy.  The definition is derived from scratch in
tests/weno_definition.py: each candidate is the polynomial of degree r-1
whose cell averages over its stencil are the point values, q_k its value at
x_{j+1/2}, the linear weights make sum_k d_k q_k the value of the polynomial
of degree 2r-2 over the whole window, and beta_k = sum_l int
(d^l p_k / dxi^l)^2 over the centre cell.

What is checked is the algebra the kernels rely on (their FP64 arithmetic
is checked against the oracle on the GPU):
* the smoothness sums b_k are fixed multiples of beta_k (4 for WENO5, 36 for
  WENO7 with the kernel's integer-coefficient forms), so the kernels' eps_s
  = 16 eps (WENO5) and 144 eps (WENO7), applied to the split flux g = 2 f,
  give the definition's weights;
* the centre-relative numerators m_k, with the weights of D, equal the
  candidate values less the centre value times the linear weights (WENO7:
  m_k = (1, 12, 18, 4)_k (A_k + B_k), 12 x 35 d_k (q_k - v_3));
* the terms the pencil sweeps carry from face to face (WENO5 13/3 s_k^2,
  WENO7 781/20 C_k^2) depend only on the cells of stencil k, and the shifted
  forms (A0 and A3 through B0 and B3, m1 = A1 + e2) are the same values."""
import pytest
import sympy as sp

from weno_definition import definition  # noqa: E402


def diffs(v, n):
    return [v[i + 1] - v[i] for i in range(n)]


def test_weno5_forms():
    v, qs, betas, lin = definition(3)
    d = diffs(v, 4)
    s = [d[k + 1] - d[k] for k in range(3)]
    t = [3 * d[1] - d[0], d[1] + d[2], 3 * d[2] - d[3]]
    for k in range(3):
        # the carried term 13/3 s_k^2: s_k is the second difference of stencil k's cells
        assert sp.expand(s[k] - (v[k] - 2 * v[k + 1] + v[k + 2])) == 0
        assert sp.expand(sp.Rational(13, 3) * s[k] ** 2 + t[k] ** 2 - 4 * betas[k]) == 0
    assert [10 * w for w in lin] == [1, 6, 3]
    m = [sp.Rational(5, 6) * d[1] - d[0] / 3, 2 * d[2] + d[1], 2 * d[2] - d[3] / 2]
    for k in range(3):
        assert sp.expand(m[k] - 10 * lin[k] * (qs[k] - v[2])) == 0


def test_weno7_forms():
    v, qs, betas, lin = definition(4)
    d = diffs(v, 6)
    e = [d[i + 1] - d[i] for i in range(5)]
    Cf = [e[k + 1] - e[k] for k in range(4)]
    B = [2 * e[1] - e[0], e[2], e[2], 2 * e[3] - e[4]]
    A = [6 * d[2] + 2 * B[0] + e[1], 2 * d[3] + 5 * d[2] - d[1], 5 * d[3] + 2 * d[2] - d[4],
         6 * d[3] - 2 * B[3] - e[3]]
    # the shifted forms of A0 and A3 are the integer-coefficient ones
    assert sp.expand(A[0] - (2 * d[0] - 7 * d[1] + 11 * d[2])) == 0
    assert sp.expand(A[3] - (11 * d[3] - 7 * d[4] + 2 * d[5])) == 0
    for k in range(4):
        # the carried term 781/20 C_k^2: C_k is the third difference of stencil k's cells
        assert sp.expand(Cf[k] - (v[k + 3] - 3 * v[k + 2] + 3 * v[k + 1] - v[k])) == 0
        b = A[k] ** 2 + 39 * B[k] ** 2 + sp.Rational(781, 20) * Cf[k] ** 2
        assert sp.expand(b - 36 * betas[k]) == 0
    assert [35 * w for w in lin] == [1, 12, 18, 4]
    # the numerators, with M and D both taken 12 times larger
    dc = [1, 12, 18, 4]
    m = [A[0] + B[0], 12 * (A[1] + B[1]), 18 * (A[2] + B[2]), 4 * (A[3] + B[3])]
    for k in range(4):
        assert sp.expand(m[k] - 12 * 35 * lin[k] * (qs[k] - v[3])) == 0
        assert sp.expand(m[k] - dc[k] * (A[k] + B[k])) == 0
    assert sp.expand((A[1] + e[2]) - (-d[1] + 4 * d[2] + 3 * d[3])) == 0
    # the weights of D' = 12 sum_k 35 d_k P_k
    assert [12 * c for c in dc] == [12, 144, 216, 48]


@pytest.mark.parametrize("r", [3, 4])
def test_scaled_weights_equal_the_definition(r):
    """With b_k = s beta_k (s = 4 or 36) and eps_s = s eps the normalised
    weights are the definition's, for any eps and beta."""
    scale = {3: 4, 4: 36}[r]
    eps = sp.symbols("eps", positive=True)
    beta = sp.symbols("beta0:%d" % r, positive=True)
    _, _, _, lin = definition(r)
    a = [lin[k] / (eps + beta[k]) ** 2 for k in range(r)]
    ab = [lin[k] / (scale * eps + scale * beta[k]) ** 2 for k in range(r)]
    for k in range(r):
        assert sp.simplify(a[k] / sum(a) - ab[k] / sum(ab)) == 0
