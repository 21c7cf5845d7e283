"""Exact solutions of ideal relativistic hydrodynamics with p = k e, used to pin
the CPU oracle.  Written from the physics, independently of the oracle's code.

* Relativistic Sod shock tube (the 1+1D test of the paper's Sec. 3, Fig. 1):
  left rarefaction + contact + right shock.  For p = k e the rarefaction keeps
  the Riemann invariant artanh(v) + sqrt(k)/(1+k) ln e fixed; across the
  shock the relative velocity obeys
  v_rel^2 = (p_b - p_a)(e_b - e_a) / ((e_a + p_b)(e_b + p_a)); the passive
  charge follows n ~ s ~ e^(1/(1+k)) in the fan and the current jump
  condition across the shock.
* Hubble-like flow (Sec. 3, Fig. 3): u^mu = x^mu / tau, tau = sqrt(t^2 - r^2),
  e = e0 (t0/tau)^(3(1+k)), n = n0 (t0/tau)^3.  Any charge profile that is a
  function of x^mu / t only is carried along (u.d s = 0), e.g. an ellipsoidal
  Gaussian in x/t.
"""
import numpy as np
from scipy.optimize import brentq


def t_mu_nu(e, v, n, k):
    """Conserved densities from primitives by the definition of T^{mu nu} and
    N^mu (v: (..., 3)): returns (T00, T0i[3], N0)."""
    v = np.asarray(v, dtype=np.float64)
    g2 = 1.0 / (1.0 - np.sum(v * v, axis=-1))
    p = k * e
    T00 = (e + p) * g2 - p
    T0i = ((e + p) * g2)[..., None] * v
    N0 = n * np.sqrt(g2)
    return T00, T0i, N0


class SodExact:
    def __init__(self, eL=1.0, nL=1.0, eR=0.1, nR=0.125, k=1.0 / 3.0, x0=0.0):
        self.eL, self.nL, self.eR, self.nR, self.k, self.x0 = eL, nL, eR, nR, k, x0
        c = np.sqrt(k)
        self.c = c

        def v_rare(es):
            return np.tanh(c / (1.0 + k) * np.log(eL / es))

        def v_shock(es):
            pa, pb = k * eR, k * es
            return np.sqrt((pb - pa) * (es - eR) / ((eR + pb) * (es + pa)))

        es = brentq(lambda e: v_rare(e) - v_shock(e), eR * (1 + 1e-12), eL * (1 - 1e-12), xtol=1e-15, rtol=1e-15)
        vs = v_shock(es)
        self.e_star, self.v_star = es, vs
        ps = k * es
        W = (es + ps) / (1.0 - vs * vs)
        self.V_shock = (W * vs * vs + ps - k * eR) / (W * vs)
        gs = 1.0 / np.sqrt(1.0 - vs * vs)
        self.n_star_L = nL * (es / eL) ** (1.0 / (1.0 + k))
        self.n_star_R = nR * self.V_shock / (gs * (self.V_shock - vs))
        self.xi_head = -c
        self.xi_tail = (vs - c) / (1.0 - vs * c)

    def jump_residuals(self):
        """Rankine-Hugoniot residuals of energy, momentum and charge across the shock."""
        k, es, vs, V = self.k, self.e_star, self.v_star, self.V_shock
        Tb, Mb, Nb = t_mu_nu(es, np.array([vs, 0, 0]), self.n_star_R, k)
        Ta, Ma, Na = t_mu_nu(self.eR, np.array([0.0, 0, 0]), self.nR, k)
        ps, pa = k * es, k * self.eR
        Wb = (es + ps) / (1 - vs * vs)
        fb_E, fa_E = Mb[0], 0.0
        fb_M, fa_M = Wb * vs * vs + ps, pa
        fb_N, fa_N = Nb * vs, 0.0
        return ((Tb - Ta) * V - (fb_E - fa_E), (Mb[0] - Ma[0]) * V - (fb_M - fa_M), (Nb - Na) * V - (fb_N - fa_N))

    def __call__(self, x, t):
        """(e, v, n) at positions x and time t > 0."""
        k, c = self.k, self.c
        xi = (np.asarray(x, dtype=np.float64) - self.x0) / t
        e = np.empty_like(xi)
        v = np.empty_like(xi)
        n = np.empty_like(xi)
        L = xi < self.xi_head
        F = (xi >= self.xi_head) & (xi < self.xi_tail)
        CL = (xi >= self.xi_tail) & (xi < self.v_star)
        CR = (xi >= self.v_star) & (xi < self.V_shock)
        R = xi >= self.V_shock
        e[L], v[L], n[L] = self.eL, 0.0, self.nL
        vf = (xi[F] + c) / (1.0 + xi[F] * c)
        ef = self.eL * ((1.0 - vf) / (1.0 + vf)) ** ((1.0 + k) / (2.0 * c))
        e[F], v[F], n[F] = ef, vf, self.nL * (ef / self.eL) ** (1.0 / (1.0 + k))
        e[CL], v[CL], n[CL] = self.e_star, self.v_star, self.n_star_L
        e[CR], v[CR], n[CR] = self.e_star, self.v_star, self.n_star_R
        e[R], v[R], n[R] = self.eR, 0.0, self.nR
        return e, v, n


def hubble(x, y, z, t, t0=10.0, e0=10.0, n0=1.0, k=1.0 / 3.0, axes=None):
    """Exact Hubble-like flow at time t (optionally with the ellipsoidal charge
    profile exp(-(x^2/2a^2 + y^2/2b^2 + z^2/2c^2) t0^2 / t^2))."""
    tau = np.sqrt(t * t - (x * x + y * y + z * z))
    e = e0 * (t0 / tau) ** (3.0 * (1.0 + k))
    n = n0 * (t0 / tau) ** 3
    if axes is not None:
        a, b, c = axes
        n = n * np.exp(-(t0 * t0 / (t * t)) * (x * x / (2 * a * a) + y * y / (2 * b * b) + z * z / (2 * c * c)))
    return e, x / t, y / t, z / t, n
