"""Exact solutions of ideal relativistic hydrodynamics with p = k e, used to pin
the CPU oracle.  Written from the physics, independently of the oracle's code.

* Relativistic Sod shock tube (the 1+1D test of the paper's Sec. 3, Fig. 1):
  left rarefaction + contact + right shock.  For p = k e the rarefaction keeps
  the Riemann invariant artanh(v) + sqrt(k)/(1+k) ln e fixed; across the
  shock the relative velocity obeys
  v_rel^2 = (p_b - p_a)(e_b - e_a) / ((e_a + p_b)(e_b + p_a)); the passive
  charge follows n ~ s ~ e^(1/(1+k)) in the fan and the current jump
  condition across the shock.
* Relativistic shock tube for an ideal gas with rest mass (the general EOS
  p = k (e - m n)): rarefaction by its Riemann invariant, shock by solving
  the jump conditions of Eq. 1.
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


def t_mu_nu_p(e, p, v, n):
    """As t_mu_nu for any pressure p (a general EOS)."""
    v = np.asarray(v, dtype=np.float64)
    g2 = 1.0 / (1.0 - np.sum(v * v, axis=-1))
    return (e + p) * g2 - p, ((e + p) * g2)[..., None] * v, n * np.sqrt(g2)


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


class GasRiemannExact:
    """Relativistic shock tube for the ideal gas p = k (e - m n) (adiabatic
    index 1 + k, rest mass m per unit charge), both sides at rest, p_L > p_R:
    left rarefaction + contact + right shock.  Built from first principles:

    * rarefaction: isentropic, p ~ (m n)^(1+k), and along the fan the
      Riemann invariant artanh(v) + int dp / ((e + p) c_s) is constant
      (c_s^2 = (1+k) p / (e+p)); inside the fan (v - c_s)/(1 - v c_s) = x/t;
    * shock: the jump conditions [F - V U] = 0 of Eq. 1 for N^0, T^00, T^0x
      across a discontinuity moving at speed V into the state at rest,
      solved numerically for the state behind it.
    """

    def __init__(self, nL=1.0, pL=1.0, nR=0.125, pR=0.1, k=2.0 / 3.0, m=1.0, x0=0.0):
        from scipy.integrate import quad
        self.nL, self.pL, self.nR, self.pR, self.k, self.m, self.x0 = nL, pL, nR, pR, k, m, x0
        self.G = 1.0 + k
        self.eL, self.eR = m * nL + pL / k, m * nR + pR / k
        self._quad = quad
        ps = brentq(lambda p: self.v_rare(p) - self.v_shock(p)[0], pR * (1 + 1e-9), pL * (1 - 1e-9),
                    xtol=1e-14, rtol=1e-14)
        self.p_star = ps
        self.v_star, self.n_star_R, self.V_shock = self.v_shock(ps)
        self.n_star_L = self.n_isen(ps)
        self.cL = self.cs(self.eL, pL)
        cS = self.cs(self.e_of(self.n_star_L, ps), ps)
        self.xi_head = -self.cL
        self.xi_tail = (self.v_star - cS) / (1.0 - self.v_star * cS)

    def e_of(self, n, p):
        return self.m * n + p / self.k

    def cs(self, e, p):
        return np.sqrt(self.G * p / (e + p))

    def n_isen(self, p):
        """charge density on the left isentrope through (n_L, p_L)"""
        return self.nL * (p / self.pL) ** (1.0 / self.G)

    def _dinv(self, p):
        e = self.e_of(self.n_isen(p), p)
        return 1.0 / ((e + p) * self.cs(e, p))

    def v_rare(self, p):
        """flow speed behind the left rarefaction at pressure p (< p_L)"""
        return np.tanh(self._quad(self._dinv, p, self.pL, epsabs=0, epsrel=1e-13, limit=200)[0])

    def v_shock(self, pb):
        """(v_b, n_b, V) behind a right-moving shock of pressure pb into the
        state at rest (n_R, p_R)."""
        from scipy.optimize import fsolve
        nR, pR, eR, k, m = self.nR, self.pR, self.eR, self.k, self.m

        def res(x):
            nb, vb, V = x
            if not (nb > 0 and abs(vb) < 1):
                return [1e3, 1e3, 1e3]
            Wb = 1.0 / np.sqrt(1.0 - vb * vb)
            eb = self.e_of(nb, pb)
            A = (eb + pb) * Wb * Wb
            return [nb * Wb * (vb - V) + nR * V,                  # N^0
                    A * vb - V * (A - pb) + V * eR,                # T^00
                    A * vb * (vb - V) + pb - pR]                   # T^0x
        best = None
        for vb0 in (0.1, 0.3, 0.5, 0.7):
            for V0 in (0.5, 0.8, 0.95):
                x, info, ier, _ = fsolve(res, [2 * nR, vb0, V0], full_output=True, xtol=1e-14)
                if ier == 1 and x[0] > 0 and 0 < x[1] < x[2] < 1 and max(abs(np.array(res(x)))) < 1e-12:
                    best = x
                    break
            if best is not None:
                break
        if best is None:
            raise RuntimeError("no shock solution at p = %g" % pb)
        nb, vb, V = best
        return vb, nb, V

    def jump_residuals(self):
        Wb = 1.0 / np.sqrt(1.0 - self.v_star ** 2)
        eb, pb, V = self.e_of(self.n_star_R, self.p_star), self.p_star, self.V_shock
        A = (eb + pb) * Wb * Wb
        return (self.n_star_R * Wb * (self.v_star - V) + self.nR * V,
                A * self.v_star - V * (A - pb) + V * self.eR,
                A * self.v_star * (self.v_star - V) + pb - self.pR)

    def __call__(self, x, t):
        """(e, v, n, p) at positions x and time t > 0."""
        xi = (np.asarray(x, dtype=np.float64) - self.x0) / t
        p = np.empty_like(xi)
        v = np.empty_like(xi)
        n = np.empty_like(xi)
        for i, s in enumerate(xi):
            if s < self.xi_head:
                p[i], v[i], n[i] = self.pL, 0.0, self.nL
            elif s < self.xi_tail:
                def g(pp):
                    vv = self.v_rare(pp)
                    c = self.cs(self.e_of(self.n_isen(pp), pp), pp)
                    return (vv - c) / (1.0 - vv * c) - s
                pp = brentq(g, self.p_star * (1 - 1e-12), self.pL, xtol=1e-15, rtol=1e-14)
                p[i], v[i], n[i] = pp, self.v_rare(pp), self.n_isen(pp)
            elif s < self.v_star:
                p[i], v[i], n[i] = self.p_star, self.v_star, self.n_star_L
            elif s < self.V_shock:
                p[i], v[i], n[i] = self.p_star, self.v_star, self.n_star_R
            else:
                p[i], v[i], n[i] = self.pR, 0.0, self.nR
        return self.e_of(n, p), v, n, p


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
