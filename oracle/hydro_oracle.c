/*
 * hydro_oracle.c -- plain, slow FP64 CPU oracle for the finite-difference
 * WENO5/WENO7 scheme with third-order Runge-Kutta time stepping for 3+1D
 * ideal relativistic hydrodynamics (Sikorski et al., "Relativistic
 * hydrodynamics on graphics processing units", arXiv:1604.03360).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent checker of the
 * CUDA path.  Only the test suite, the smoke check and the benchmark's CPU
 * baseline leg may load it; the product library never calls it and shares
 * no code, header or table with it.
 *
 * What it computes, step by step, in the paper's order:
 *   Eq. 1 (Sec. 1)   du/dt + sum_i d f_i(u)/dx_i = 0, u = (E, M_x, M_y, M_z, R):
 *                    energy density T^00, momentum densities T^0i and one
 *                    conserved charge density n*gamma.  Ideal fluid,
 *                    T^{mu nu} = (e+p) u^mu u^nu - p g^{mu nu}, EOS p = cs2*e.
 *   Eq. 2 (Sec. 1)   L(u) = sum_i (F_i(x - e_i/2) - F_i(x + e_i/2)) / |e_i|.
 *   Sec. 1.2         F at the half-cell faces by finite-difference WENO of
 *                    order 5 (r = 3) or 7 (r = 4), applied component-wise to
 *                    the Lax-Friedrichs split fluxes f^+- = (f +- alpha u)/2,
 *                    alpha per direction = max |characteristic speed| over the
 *                    grid (global Lax-Friedrichs).
 *   Sec. 1           third-order Runge-Kutta in time (variant not named):
 *                    the SSP (Shu-Osher) form
 *                    u1 = u + dt L(u); u2 = 3/4 u + 1/4 (u1 + dt L(u1));
 *                    u' = 1/3 u + 2/3 (u2 + dt L(u2)).
 *
 * Readings where the paper is silent (kept identical on both sides): the EOS
 * p = cs2 e; component-wise reconstruction; global LF splitting recomputed
 * from every stage's input; dt = cfl * min_d dx_d / max_d alpha_d over the
 * directions with more than one cell, clipped to t_end; outflow boundaries
 * copy the edge cell into the ghost cells (zeroth-order extrapolation of the
 * conserved variables); periodic boundaries wrap; directions with a single
 * cell contribute no flux difference.
 * General EOS (mass m > 0): p = cs2 (e - m n_1), the ideal gas of adiabatic
 * index 1 + cs2 whose rest mass is m per unit of the first charge (m = 0 is
 * p = cs2 e).  The first charge then enters the pressure; the primitive
 * recovery solves for p by bracketed Newton iteration, and the Lax-Friedrichs
 * speeds use c_s^2 = (1 + cs2) p / (e + p).  WENO (component-wise, global or
 * local LF) only.
 * Several conserved charges (nq > 1): the state is (E, M, R_1..R_nq); every
 * charge is a passive density advected like R (flux R_k v_d, n_k = R_k / gamma),
 * since p = cs2 e does not depend on them.
 * MUSTA-FORCE + MUSCL (r = 1, Sec. 1.1, second order): the state is
 * reconstructed linearly in each cell, component-wise on the conserved
 * variables, with the slope limited by `limiter` (u_L = u_j + s_j/2,
 * u_R = u_{j+1} - s_{j+1}/2; an unphysical reconstructed state falls back to
 * the cell average).  The face flux is MUSTA: musta_k stages of the centred
 * FORCE flux F = (F_LF + F_LW)/2 on the local states, with the local ratio
 * dt/dx = 0.9 / S, S = max |lambda| over the two local states; between
 * stages the local states are advanced as a predictor (u_L -= r (F - f_L),
 * u_R -= r (f_R - F)).  If the Lax-Wendroff state is unphysical the stage
 * flux is F_LF; if a predicted state is unphysical the iteration stops.
 * Characteristic-wise variant (charw = 1, with global LF): at the face
 * j+1/2 along d the split fluxes of both stencils are projected on the
 * characteristic fields of the face state -- the primitives of the mean of
 * the conserved states of cells j and j+1 -- with the left eigenvectors
 * L = R^-1 of df_d/du there; every field is reconstructed as above and the
 * face flux is R times the reconstructed fields.  R (oc_char_basis) is
 * derived in closed form, each column the change of u for a unit change of
 * e (sound waves), of one transverse velocity (shear waves) or of one
 * charge density; L comes from Gauss-Jordan elimination (oc_invert).
 * Local Lax-Friedrichs variant (split = 1): the face j+1/2 along d uses
 * alpha = max over the 2r cells j-r+1 .. j+r (the union of both biased
 * stencils) of max(|lambda_-|, |lambda_+|) along d; the time step still uses
 * the global speeds.
 *
 * Built with -O2 -ffp-contract=off (no FMA contraction) so that x86-64 and
 * aarch64 hosts give identical bits.  OpenMP (if present) only splits the
 * independent per-cell and per-pencil loops; the maxima are order
 * independent, so results do not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Oracle configuration (its own type: nothing is shared with the library). */
typedef struct {
    int32_t n[3];      /* interior cells along x, y, z (x fastest in memory) */
    int32_t r;         /* WENO parameter: 3 -> WENO5, 4 -> WENO7 */
    int32_t bc[3];     /* 0: outflow (copy edge cell), 1: periodic */
    int32_t split;     /* 0: global Lax-Friedrichs, 1: local Lax-Friedrichs */
    int32_t nq;        /* conserved charge densities R_1..R_nq (0 or 1: one) */
    int32_t limiter;   /* MUSCL slope limiter: 0 minmod, 1 MC, 2 van Leer, 3 superbee */
    int32_t musta_k;   /* MUSTA stages (>= 1; 1 is plain FORCE) */
    int32_t charw;     /* WENO on: 0 the components of u, 1 the characteristic fields */
    double dx[3];      /* cell sizes |e_i| */
    double cs2;        /* EOS p = cs2 * e */
    double cfl;
    double dt_fixed;   /* > 0: use this dt instead of the CFL rule */
    double eps;        /* WENO epsilon in alpha_k = d_k / (eps + beta_k)^2 */
    double mass;       /* EOS p = cs2 (e - mass n_1); 0: p = cs2 e */
} oc_cfg;

enum { OC_OK = 0, OC_ERR_ARG = 1, OC_ERR_UNPHYSICAL = 4, OC_ERR_OOM = 3 };
#define MAXF 8   /* E, M_x, M_y, M_z and up to four charges */
#define NFMAX_M 8
static int nfields(const void *cfg);

/* ------------------------------------------------------------------------ */
/* Thermodynamics and fluxes (Eq. 1)                                        */
/* ------------------------------------------------------------------------ */

/* Conserved (E, M, R) -> primitive (e, v, n) for p = k e.  With
 * W = (e+p) gamma^2: E = W - p, M = W v, so (E + k e)^2 - M^2 =
 * (1+k) e (E + k e), i.e. k e^2 + (1-k) E e - (E^2 - M^2) = 0; the positive
 * root is written in the cancellation-free form.  v = M / (E + p),
 * n = R / gamma.  Returns nonzero for E <= 0 or |M| >= E (no physical
 * state) or NaN input. */
int oc_con2prim(double k, const double *u, double *w)
{
    const double E = u[0], mx = u[1], my = u[2], mz = u[3], R = u[4];
    const double m2 = mx * mx + my * my + mz * mz;
    const double d = E * E - m2;
    if (!(E > 0.0) || !(d > 0.0)) return 1;
    const double b = (1.0 - k) * E;
    const double e = 2.0 * d / (b + sqrt(b * b + 4.0 * k * d));
    const double p = k * e;
    const double vx = mx / (E + p), vy = my / (E + p), vz = mz / (E + p);
    const double v2 = vx * vx + vy * vy + vz * vz;
    w[0] = e;
    w[1] = vx;
    w[2] = vy;
    w[3] = vz;
    w[4] = R * sqrt(1.0 - v2);
    return 0;
}

/* Primitive (e, v, n) -> conserved: E = (e+p) gamma^2 - p, M = (e+p) gamma^2 v,
 * R = n gamma. */
void oc_prim2con(double k, const double *w, double *u)
{
    const double e = w[0], vx = w[1], vy = w[2], vz = w[3], n = w[4];
    const double p = k * e;
    const double g2 = 1.0 / (1.0 - (vx * vx + vy * vy + vz * vz));
    const double W = (e + p) * g2;
    u[0] = W - p;
    u[1] = W * vx;
    u[2] = W * vy;
    u[3] = W * vz;
    u[4] = n * sqrt(g2);
}

/* Physical flux along direction d (Eq. 1): f_d(E) = M_d = T^{0d},
 * f_d(M_j) = M_j v_d + p delta_jd = T^{jd}, f_d(R) = R v_d = n u^d. */
void oc_flux_n(double k, int d, int nf, const double *u, const double *w, double *f)
{
    const double p = k * w[0];
    const double vd = w[1 + d];
    f[0] = u[1 + d];
    f[1] = u[1] * vd + (d == 0 ? p : 0.0);
    f[2] = u[2] * vd + (d == 1 ? p : 0.0);
    f[3] = u[3] * vd + (d == 2 ? p : 0.0);
    for (int q = 4; q < nf; ++q) f[q] = u[q] * vd;   /* charges: R_q v_d */
}

void oc_flux(double k, int d, const double *u, const double *w, double *f) { oc_flux_n(k, d, 5, u, w, f); }

/* Characteristic (sound-wave) speeds along d for p = k e:
 * lambda_+- = [v_d (1-k) +- sqrt(k) sqrt((1-v^2)(1 - v_d^2 - k (v^2 - v_d^2)))]
 *             / (1 - k v^2).  The other three eigenvalues equal v_d and lie
 * between these two. */
void oc_eigen(double k, int d, const double *w, double *lam)
{
    const double vx = w[1], vy = w[2], vz = w[3];
    const double v2 = vx * vx + vy * vy + vz * vz;
    const double vd = w[1 + d];
    const double root = sqrt(k) * sqrt((1.0 - v2) * (1.0 - vd * vd - k * (v2 - vd * vd)));
    const double den = 1.0 - k * v2;
    lam[0] = (vd * (1.0 - k) - root) / den;
    lam[1] = (vd * (1.0 - k) + root) / den;
}

/* ------------------------------------------------------------------------ */
/* General equation of state p(e, n) = k (e - m n_1)                         */
/* ------------------------------------------------------------------------ */
/* The ideal gas with adiabatic index 1 + k whose rest mass is m per unit of
 * the first charge: n_1 m is the rest-mass density, e - m n_1 the internal
 * energy density.  m = 0 is the EOS p = k e above.  Sound speed squared
 * c_s^2 = dp/de + n/(e+p) dp/dn = k (e + p - m n) / (e + p) = (1 + k) p / (e + p). */
double oc_eos_p(double k, double m, const double *w) { return m == 0.0 ? k * w[0] : k * (w[0] - m * w[4]); }

double oc_sound2(double k, double m, const double *w)
{
    if (m == 0.0) return k;
    const double p = oc_eos_p(k, m, w);
    return (1.0 + k) * p / (w[0] + p);
}

/* Conserved -> primitive for m >= 0 by bracketed Newton iteration on the
 * pressure: with v = M / (E + p), e = E - M.v, n = R sqrt(1 - v^2),
 * f(p) = k (e - m n) - p is decreasing (f' = v^2 c_s^2 - 1 < 0); f(0) > 0
 * is required (positive internal energy) and f <= 0 at the pressure of the
 * m = 0 state (an upper bracket).  A Newton step that leaves the bracket is
 * replaced by bisection.  Stops at f = 0, when the update no longer changes
 * p, or when it is below 1e-15 p (at most 200 steps).  Returns nonzero if no
 * physical state exists. */
int oc_con2prim_gas(double k, double m, const double *u, double *w)
{
    const double E = u[0], R = u[4];
    const double M2 = u[1] * u[1] + u[2] * u[2] + u[3] * u[3];
    const double dd = E * E - M2;
    if (!(E > 0.0) || !(dd > 0.0) || !(R >= 0.0)) return 1;
    const double b = (1.0 - k) * E;
    const double hi0 = k * (2.0 * dd / (b + sqrt(b * b + 4.0 * k * dd)));   /* pressure if m = 0 */
    double lo = 0.0, hi = hi0;
    /* f and f' at p */
    double p = hi, f = 0.0, fp = -1.0;
    {
        const double v2 = M2 / (E * E);
        const double f0 = k * ((E - M2 / E) - m * R * sqrt(1.0 - v2));
        if (!(f0 > 0.0)) return 1;
    }
    for (int it = 0; it < 200; ++it) {
        const double h = E + p, v2 = M2 / (h * h);
        const double e = E - M2 / h, n = R * sqrt(1.0 - v2);
        f = k * (e - m * n) - p;
        if (f == 0.0) break;                      /* p is the root */
        const double cs2 = (1.0 + k) * p / (e + p);
        fp = v2 * cs2 - 1.0;
        if (f > 0.0) lo = p;
        else hi = p;
        double pn = p - f / fp;
        if (pn == p) break;                       /* the update is below the rounding of p */
        if (!(pn > lo && pn < hi)) pn = 0.5 * (lo + hi);
        const double dp = fabs(pn - p);
        p = pn;
        if (dp <= 1e-15 * p) break;
    }
    if (!(p > 0.0)) return 1;
    const double h = E + p;
    w[0] = E - M2 / h;
    w[1] = u[1] / h;
    w[2] = u[2] / h;
    w[3] = u[3] / h;
    w[4] = R * sqrt(1.0 - (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]));
    return 0;
}

int oc_con2prim_eos(double k, double m, const double *u, double *w)
{
    return m == 0.0 ? oc_con2prim(k, u, w) : oc_con2prim_gas(k, m, u, w);
}

/* Primitive -> conserved for the general EOS (same definitions as oc_prim2con). */
void oc_prim2con_eos(double k, double m, const double *w, double *u)
{
    if (m == 0.0) {
        oc_prim2con(k, w, u);
        return;
    }
    const double e = w[0], vx = w[1], vy = w[2], vz = w[3], n = w[4];
    const double p = oc_eos_p(k, m, w);
    const double g2 = 1.0 / (1.0 - (vx * vx + vy * vy + vz * vz));
    const double W = (e + p) * g2;
    u[0] = W - p;
    u[1] = W * vx;
    u[2] = W * vy;
    u[3] = W * vz;
    u[4] = n * sqrt(g2);
}

/* Flux of Eq. 1 with p from the general EOS (oc_flux_n for m = 0). */
void oc_flux_eos(double k, double m, int d, int nf, const double *u, const double *w, double *f)
{
    const double p = oc_eos_p(k, m, w);
    const double vd = w[1 + d];
    f[0] = u[1 + d];
    for (int j = 0; j < 3; ++j) f[1 + j] = u[1 + j] * vd + (d == j ? p : 0.0);
    for (int q = 4; q < nf; ++q) f[q] = u[q] * vd;
}

/* Right eigenvectors of the flux Jacobian A_d = df_d/du at the primitive
 * state w = (e, v, n_1..n_q), as the columns of Rm (nf x nf, row-major,
 * rows E, M_x, M_y, M_z, R_1..R_q).  Each column is the change of u that
 * belongs to a unit change of one primitive quantity along one wave family,
 * derived from dF = lambda dU for T^{mu nu} of an ideal fluid with p = k e
 * (h = (1+k) e, K = h gamma^2, Q = d(K) = gamma^2 dh + 2 h gamma^4 v.dv):
 *   col 0, 1  sound waves lambda_-, lambda_+ (oc_eigen), de = 1:
 *             dv_d = k (1 - lambda v_d) / (K (lambda - v_d)),
 *             dv_t = -lambda k v_t / (K (lambda - v_d)) (t != d),
 *             dE = Q - k, dM_i = Q v_i + K dv_i, dR_q = R_q dv_d / (lambda - v_d);
 *   col 2, 3  shear waves along t1 = (d+1)%3, t2 = (d+2)%3, lambda = v_d,
 *             dv_t = 1 (de = dv_d = 0, dn = 0): Q = 2 h gamma^4 v_t,
 *             dE = Q, dM_i = Q v_i + K delta_it, dR_q = n_q gamma^3 v_t;
 *   col 4+q   charge q, lambda = v_d, dn_q = 1: dR_q = gamma, all else 0.
 * lam (optional) receives the eigenvalue of every column.  The normalisation
 * (unit primitive change) fixes the scale of the characteristic fields. */
void oc_char_basis(double k, int d, int nf, const double *w, double *Rm, double *lam)
{
    const double e = w[0], v[3] = {w[1], w[2], w[3]};
    const double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    const double g2 = 1.0 / (1.0 - v2), gam = sqrt(g2);
    const double h = (1.0 + k) * e, K = h * g2;
    const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    double ls[2];
    oc_eigen(k, d, w, ls);
    for (int i = 0; i < nf * nf; ++i) Rm[i] = 0.0;
    for (int s = 0; s < 2; ++s) {                 /* sound waves */
        const double l = ls[s];
        double dv[3];
        dv[d] = k * (1.0 - l * v[d]) / (K * (l - v[d]));
        dv[t1] = -l * k * v[t1] / (K * (l - v[d]));
        dv[t2] = -l * k * v[t2] / (K * (l - v[d]));
        const double vdv = v[0] * dv[0] + v[1] * dv[1] + v[2] * dv[2];
        const double Q = g2 * (1.0 + k) + 2.0 * h * g2 * g2 * vdv;
        Rm[0 * nf + s] = Q - k;
        for (int i = 0; i < 3; ++i) Rm[(1 + i) * nf + s] = Q * v[i] + K * dv[i];
        for (int q = 4; q < nf; ++q) Rm[q * nf + s] = w[q] * gam * dv[d] / (l - v[d]);
    }
    const int ts[2] = {t1, t2};
    for (int s = 0; s < 2; ++s) {                 /* shear waves */
        const int t = ts[s];
        const double Q = 2.0 * h * g2 * g2 * v[t];
        Rm[0 * nf + 2 + s] = Q;
        for (int i = 0; i < 3; ++i) Rm[(1 + i) * nf + 2 + s] = Q * v[i] + (i == t ? K : 0.0);
        for (int q = 4; q < nf; ++q) Rm[q * nf + 2 + s] = w[q] * gam * g2 * v[t];
    }
    for (int q = 4; q < nf; ++q) Rm[q * nf + q] = gam;   /* charges */
    if (lam) {
        lam[0] = ls[0];
        lam[1] = ls[1];
        for (int c = 2; c < nf; ++c) lam[c] = v[d];
    }
}

/* Inverse of the nf x nf matrix A (row-major) by Gauss-Jordan elimination
 * with partial pivoting.  Returns nonzero if a pivot vanishes. */
int oc_invert(int nf, const double *A, double *Ainv)
{
    double M[MAXF][2 * MAXF];
    for (int i = 0; i < nf; ++i)
        for (int j = 0; j < 2 * nf; ++j) M[i][j] = j < nf ? A[i * nf + j] : (j - nf == i ? 1.0 : 0.0);
    for (int c = 0; c < nf; ++c) {
        int piv = c;
        for (int i = c + 1; i < nf; ++i)
            if (fabs(M[i][c]) > fabs(M[piv][c])) piv = i;
        if (!(fabs(M[piv][c]) > 0.0)) return 1;
        if (piv != c)
            for (int j = 0; j < 2 * nf; ++j) {
                const double t = M[c][j];
                M[c][j] = M[piv][j];
                M[piv][j] = t;
            }
        const double pv = M[c][c];
        for (int j = 0; j < 2 * nf; ++j) M[c][j] /= pv;
        for (int i = 0; i < nf; ++i) {
            if (i == c) continue;
            const double f = M[i][c];
            for (int j = 0; j < 2 * nf; ++j) M[i][j] -= f * M[c][j];
        }
    }
    for (int i = 0; i < nf; ++i)
        for (int j = 0; j < nf; ++j) Ainv[i * nf + j] = M[i][nf + j];
    return 0;
}

/* ------------------------------------------------------------------------ */
/* WENO reconstruction (Sec. 1.2; Jiang-Shu / Shu finite-difference WENO)    */
/* ------------------------------------------------------------------------ */
/* Left-biased value at x_{j+1/2} from v[0..2r-2] = v_{j-r+1} .. v_{j+r-1}.
 * Candidate k (k = 0..r-1) uses cells j-r+1+k .. j+k, i.e. v[k .. k+r-1].
 * p_k is the degree r-1 polynomial whose averages over those cells equal the
 * values; q_k = p_k(x_{j+1/2}); p_k(xi) = sum_i c_i xi^i about x_j in units of
 * dx.  Tables: numerators over a common denominator per row. */

/* q_k = sum_m QN[k][m] v[k+m] / QD */
static const double Q5N[3][3] = {{2, -7, 11}, {-1, 5, 2}, {2, 5, -1}};
static const double Q5D = 6;
static const double Q7N[4][4] = {{-3, 13, -23, 25}, {1, -5, 13, 3}, {-1, 7, 7, -1}, {3, 13, -5, 1}};
static const double Q7D = 12;
/* Taylor coefficients c_1 .. c_{r-1} of p_k: c_i = sum_m TN[k][i-1][m] v[k+m] / TD[i-1] */
static const double T5N[3][2][3] = {
    {{1, -4, 3}, {1, -2, 1}},
    {{-1, 0, 1}, {1, -2, 1}},
    {{-3, 4, -1}, {1, -2, 1}}};
static const double T5D[2] = {2, 2};
static const double T7N[4][3][4] = {
    {{-7, 33, -69, 43}, {-1, 4, -5, 2}, {-1, 3, -3, 1}},
    {{5, -27, 15, 7}, {0, 1, -2, 1}, {-1, 3, -3, 1}},
    {{-7, -15, 27, -5}, {1, -2, 1, 0}, {-1, 3, -3, 1}},
    {{-43, 69, -33, 7}, {2, -5, 4, -1}, {-1, 3, -3, 1}}};
static const double T7D[3] = {24, 2, 6};
/* optimal (linear) weights */
static const double D5[3] = {1.0 / 10, 6.0 / 10, 3.0 / 10};
static const double D7[4] = {1.0 / 35, 12.0 / 35, 18.0 / 35, 4.0 / 35};

static double falling(int a, int l)
{
    double f = 1.0;
    for (int i = 0; i < l; ++i) f *= (double)(a - i);
    return f;
}

/* Smoothness indicator, the Jiang-Shu definition written out:
 * beta = sum_{l=1}^{r-1} int_{-1/2}^{1/2} (d^l p / d xi^l)^2 d xi. */
static double smoothness(int r, const double *c /* c[1..r-1] used */)
{
    double beta = 0.0;
    for (int l = 1; l < r; ++l)
        for (int a = l; a < r; ++a)
            for (int b = l; b < r; ++b) {
                const int pw = (a - l) + (b - l);
                if (pw & 1) continue; /* odd moments of [-1/2, 1/2] vanish */
                const double mom = 1.0 / ((double)(pw + 1) * ldexp(1.0, pw));
                beta += falling(a, l) * falling(b, l) * c[a] * c[b] * mom;
            }
    return beta;
}

double oc_weno_left(int r, const double *v, double eps)
{
    double q[4], beta[4], alpha[4], sum = 0.0;
    for (int k = 0; k < r; ++k) {
        double c[4] = {0, 0, 0, 0};
        q[k] = 0.0;
        for (int m = 0; m < r; ++m)
            q[k] += (r == 3 ? Q5N[k][m] : Q7N[k][m]) * v[k + m];
        q[k] /= (r == 3 ? Q5D : Q7D);
        for (int i = 1; i < r; ++i) {
            for (int m = 0; m < r; ++m)
                c[i] += (r == 3 ? T5N[k][i - 1][m] : T7N[k][i - 1][m]) * v[k + m];
            c[i] /= (r == 3 ? T5D[i - 1] : T7D[i - 1]);
        }
        beta[k] = smoothness(r, c);
        const double dk = (r == 3 ? D5[k] : D7[k]);
        alpha[k] = dk / ((eps + beta[k]) * (eps + beta[k]));
        sum += alpha[k];
    }
    double out = 0.0;
    for (int k = 0; k < r; ++k) out += (alpha[k] / sum) * q[k];
    return out;
}

/* Right-biased value at x_{j+1/2} from v_{j-r+2} .. v_{j+r}: the mirror image. */
static double weno_right(int r, const double *v, double eps)
{
    double m[7];
    for (int i = 0; i < 2 * r - 1; ++i) m[i] = v[2 * r - 2 - i];
    return oc_weno_left(r, m, eps);
}

/* Coefficient tables, exported so tests can compare them with a symbolic
 * derivation from the definition.  q: r*r, taylor: r*(r-1)*r, d: r. */
int oc_weno_tables(int r, double *q, double *taylor, double *d)
{
    if (r != 3 && r != 4) return OC_ERR_ARG;
    for (int k = 0; k < r; ++k) {
        d[k] = (r == 3 ? D5[k] : D7[k]);
        for (int m = 0; m < r; ++m) {
            q[k * r + m] = (r == 3 ? Q5N[k][m] / Q5D : Q7N[k][m] / Q7D);
            for (int i = 1; i < r; ++i)
                taylor[(k * (r - 1) + (i - 1)) * r + m] =
                    (r == 3 ? T5N[k][i - 1][m] / T5D[i - 1] : T7N[k][i - 1][m] / T7D[i - 1]);
        }
    }
    return OC_OK;
}

/* ------------------------------------------------------------------------ */
/* Grid helpers and boundary conditions                                     */
/* ------------------------------------------------------------------------ */
static int g_threads = 0;
void oc_set_threads(int n) { g_threads = n; }
int oc_get_max_threads(void)
{
#ifdef _OPENMP
    return g_threads > 0 ? g_threads : omp_get_max_threads();
#else
    return 1;
#endif
}

static int active(const oc_cfg *c, int d) { return c->n[d] > 1; }
static int nfields(const void *cfg)
{
    const oc_cfg *c = (const oc_cfg *)cfg;
    return 4 + (c->nq > 1 ? c->nq : 1);
}

/* index of the interior cell that supplies (possibly ghost) coordinate i */
static int bc_src(const oc_cfg *c, int d, int i)
{
    const int n = c->n[d];
    if (i >= 0 && i < n) return i;
    if (c->bc[d] == 1) return ((i % n) + n) % n;
    return i < 0 ? 0 : n - 1;
}

static int64_t cell(const oc_cfg *c, int i, int j, int k)
{
    return ((int64_t)k * c->n[1] + j) * c->n[0] + i;
}

static int cfg_ok(const oc_cfg *c)
{
    if (!c) return 0;
    for (int d = 0; d < 3; ++d)
        if (c->n[d] < 1 || !(c->dx[d] > 0) || (c->bc[d] != 0 && c->bc[d] != 1)) return 0;
    if (c->r != 1 && c->r != 3 && c->r != 4) return 0;
    if (c->r == 1 && (c->limiter < 0 || c->limiter > 3 || c->musta_k < 1 || c->split != 0 || c->nq > 1)) return 0;
    if (c->split != 0 && c->split != 1) return 0;
    if (c->charw != 0 && (c->charw != 1 || c->r == 1)) return 0;
    if (!(c->mass >= 0.0) || (c->mass > 0.0 && (c->r == 1 || c->charw))) return 0;
    if (c->nq < 0 || c->nq > MAXF - 4) return 0;
    if (!(c->cs2 > 0 && c->cs2 < 1) || !(c->eps > 0)) return 0;
    for (int d = 0; d < 3; ++d)
        if (active(c, d) && c->bc[d] == 1 && c->n[d] < (c->r == 1 ? 2 : c->r)) return 0;
    return 1;
}

/* alpha_d = max over interior cells of max(|lambda_-|, |lambda_+|). */
int oc_alpha(const oc_cfg *c, const double *u, double *alpha)
{
    if (!cfg_ok(c)) return OC_ERR_ARG;
    const int64_t N = (int64_t)c->n[0] * c->n[1] * c->n[2];
    double a0 = 0, a1 = 0, a2 = 0;
    int bad = 0;
#pragma omp parallel for reduction(max : a0, a1, a2) reduction(| : bad) num_threads(oc_get_max_threads())
    for (int64_t q = 0; q < N; ++q) {
        double uu[MAXF], w[MAXF], lam[2];
        for (int f = 0; f < 5; ++f) uu[f] = u[f * N + q];
        if (oc_con2prim_eos(c->cs2, c->mass, uu, w)) {
            bad |= 1;
            continue;
        }
        const double cs2 = oc_sound2(c->cs2, c->mass, w);
        oc_eigen(cs2, 0, w, lam);
        a0 = fmax(a0, fmax(fabs(lam[0]), fabs(lam[1])));
        oc_eigen(cs2, 1, w, lam);
        a1 = fmax(a1, fmax(fabs(lam[0]), fabs(lam[1])));
        oc_eigen(cs2, 2, w, lam);
        a2 = fmax(a2, fmax(fabs(lam[0]), fabs(lam[1])));
    }
    alpha[0] = a0;
    alpha[1] = a1;
    alpha[2] = a2;
    return bad ? OC_ERR_UNPHYSICAL : OC_OK;
}

/* ------------------------------------------------------------------------ */
/* MUSCL + MUSTA-FORCE (Sec. 1.1)                                            */
/* ------------------------------------------------------------------------ */
static double minmod2(double a, double b)
{
    if (a * b <= 0.0) return 0.0;
    return fabs(a) < fabs(b) ? a : b;
}

/* limited slope from the backward and forward differences a, b */
double oc_limiter(int kind, double a, double b)
{
    if (a * b <= 0.0) return 0.0;
    switch (kind) {
    case 0: /* minmod */
        return minmod2(a, b);
    case 1: /* monotonized central: minmod(2a, (a+b)/2, 2b) */
        return minmod2(minmod2(2.0 * a, 0.5 * (a + b)), 2.0 * b);
    case 2: /* van Leer: harmonic mean */
        return 2.0 * a * b / (a + b);
    default: { /* superbee: maxmod(minmod(2a, b), minmod(a, 2b)) */
        const double s1 = minmod2(2.0 * a, b), s2 = minmod2(a, 2.0 * b);
        return fabs(s1) > fabs(s2) ? s1 : s2;
    }
    }
}

static double max_speed(const oc_cfg *c, int d, const double *w)
{
    double lam[2];
    oc_eigen(c->cs2, d, w, lam);
    return fmax(fabs(lam[0]), fabs(lam[1]));
}

/* MUSTA-FORCE flux along d between local states uL, uR (5 values each).
 * Returns nonzero if the initial local states are unphysical. */
static int musta_force(const oc_cfg *c, int d, const double *uL0, const double *uR0, double *F)
{
    double uL[NFMAX_M], uR[NFMAX_M], wL[NFMAX_M], wR[NFMAX_M], fL[NFMAX_M], fR[NFMAX_M];
    memcpy(uL, uL0, sizeof(double) * 5);
    memcpy(uR, uR0, sizeof(double) * 5);
    if (oc_con2prim(c->cs2, uL, wL) || oc_con2prim(c->cs2, uR, wR)) return 1;
    for (int l = 1; l <= c->musta_k; ++l) {
        oc_flux_n(c->cs2, d, 5, uL, wL, fL);
        oc_flux_n(c->cs2, d, 5, uR, wR, fR);
        const double S = fmax(max_speed(c, d, wL), max_speed(c, d, wR));
        const double r = 0.9 / S;               /* local dt / dx */
        double uLW[NFMAX_M], wLW[NFMAX_M], fLW[NFMAX_M], Flf[NFMAX_M];
        for (int k = 0; k < 5; ++k) {
            Flf[k] = 0.5 * (fL[k] + fR[k]) - 0.5 / r * (uR[k] - uL[k]);
            uLW[k] = 0.5 * (uL[k] + uR[k]) - 0.5 * r * (fR[k] - fL[k]);
        }
        if (oc_con2prim(c->cs2, uLW, wLW)) {
            for (int k = 0; k < 5; ++k) F[k] = Flf[k];
        } else {
            oc_flux_n(c->cs2, d, 5, uLW, wLW, fLW);
            for (int k = 0; k < 5; ++k) F[k] = 0.5 * (Flf[k] + fLW[k]);
        }
        if (l == c->musta_k) break;
        double nL[NFMAX_M], nR[NFMAX_M], vL[NFMAX_M], vR[NFMAX_M];
        for (int k = 0; k < 5; ++k) {
            nL[k] = uL[k] - r * (F[k] - fL[k]);
            nR[k] = uR[k] - r * (fR[k] - F[k]);
        }
        if (oc_con2prim(c->cs2, nL, vL) || oc_con2prim(c->cs2, nR, vR)) break;
        memcpy(uL, nL, sizeof uL);
        memcpy(uR, nR, sizeof uR);
        memcpy(wL, vL, sizeof wL);
        memcpy(wR, vR, sizeof wR);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* The semi-discrete operator L(u) of Eq. 2                                 */
/* ------------------------------------------------------------------------ */
/* L = sum_d (F_d(j - 1/2) - F_d(j + 1/2)) / dx_d with
 * F(j+1/2) = WENO_left(f^+_{j-r+1..j+r-1}) + WENO_right(f^-_{j-r+2..j+r}),
 * f^+- = (f_d(u) +- alpha_d u) / 2, ghost cells from the boundary rule. */
int oc_L(const oc_cfg *c, const double *u, const double *alpha, double *L)
{
    if (!cfg_ok(c)) return OC_ERR_ARG;
    const int r = c->r, G = (r == 1 ? 2 : r);
    const int NF = nfields(c);
    const int64_t N = (int64_t)c->n[0] * c->n[1] * c->n[2];
    int bad = 0;
#pragma omp parallel for num_threads(oc_get_max_threads())
    for (int64_t q = 0; q < NF * N; ++q) L[q] = 0.0;

    for (int d = 0; d < 3; ++d) {
        if (!active(c, d)) continue;
        const int nd = c->n[d];
        const int da = (d + 1) % 3, db = (d + 2) % 3; /* the two other axes */
        const int64_t npen = (int64_t)c->n[da] * c->n[db];
        const int len = nd + 2 * G;
#pragma omp parallel for reduction(| : bad) num_threads(oc_get_max_threads())
        for (int64_t pen = 0; pen < npen; ++pen) {
            const int ia = (int)(pen % c->n[da]), ib = (int)(pen / c->n[da]);
            double *fp = malloc(sizeof(double) * NF * len);
            double *fm = malloc(sizeof(double) * NF * len);
            double *F = malloc(sizeof(double) * NF * (nd + 1));
            double *fr = malloc(sizeof(double) * NF * len);    /* physical flux (local LF) */
            double *ur = malloc(sizeof(double) * NF * len);    /* state (local LF) */
            double *sp = malloc(sizeof(double) * len);         /* max |lambda| along d (local LF) */
            if (!fp || !fm || !F || !fr || !ur || !sp) {
                bad |= 2;
                free(fp); free(fm); free(F); free(fr); free(ur); free(sp);
                continue;
            }
            /* split fluxes at every cell of the pencil, ghosts included */
            for (int m = 0; m < len; ++m) {
                int ijk[3];
                ijk[d] = bc_src(c, d, m - G);
                ijk[da] = ia;
                ijk[db] = ib;
                const int64_t q = cell(c, ijk[0], ijk[1], ijk[2]);
                double uu[MAXF], w[MAXF], f[MAXF];
                for (int k = 0; k < NF; ++k) uu[k] = u[k * N + q];
                if (oc_con2prim_eos(c->cs2, c->mass, uu, w)) {
                    bad |= 1;
                    for (int k = 0; k < 5; ++k) w[k] = 0.0;
                }
                oc_flux_eos(c->cs2, c->mass, d, NF, uu, w, f);
                for (int k = 0; k < NF; ++k) {
                    fp[k * len + m] = 0.5 * (f[k] + alpha[d] * uu[k]);
                    fm[k * len + m] = 0.5 * (f[k] - alpha[d] * uu[k]);
                    fr[k * len + m] = f[k];
                    ur[k * len + m] = uu[k];
                }
                double lam[2];
                oc_eigen(oc_sound2(c->cs2, c->mass, w), d, w, lam);
                sp[m] = fmax(fabs(lam[0]), fabs(lam[1]));
            }
            /* face fluxes: F[s] sits at face s - 1/2, s = 0..nd */
            for (int s = 0; s <= nd; ++s) {
                const int j = s - 1 + G; /* padded index of the cell left of the face */
                if (r == 1) {
                    /* MUSCL states at the face from cells j-1 .. j+2, then MUSTA-FORCE */
                    double uL[NFMAX_M], uR[NFMAX_M], u0[NFMAX_M], u1[NFMAX_M], wtmp[NFMAX_M], Ff[NFMAX_M];
                    for (int k = 0; k < 5; ++k) {
                        const double *v = ur + k * len;
                        const double sl = oc_limiter(c->limiter, v[j] - v[j - 1], v[j + 1] - v[j]);
                        const double sr = oc_limiter(c->limiter, v[j + 1] - v[j], v[j + 2] - v[j + 1]);
                        u0[k] = v[j];
                        u1[k] = v[j + 1];
                        uL[k] = v[j] + 0.5 * sl;
                        uR[k] = v[j + 1] - 0.5 * sr;
                    }
                    if (oc_con2prim(c->cs2, uL, wtmp)) memcpy(uL, u0, sizeof uL);
                    if (oc_con2prim(c->cs2, uR, wtmp)) memcpy(uR, u1, sizeof uR);
                    if (musta_force(c, d, uL, uR, Ff)) {
                        bad |= 1;
                        for (int k = 0; k < 5; ++k) Ff[k] = 0.0;
                    }
                    for (int k = 0; k < NF; ++k) F[k * (nd + 1) + s] = Ff[k];
                    continue;
                }
                if (c->split == 1) {
                    /* local LF: split again with this face's own alpha */
                    double af = 0.0;
                    for (int m = j - r + 1; m <= j + r; ++m) af = fmax(af, sp[m]);
                    for (int k = 0; k < NF; ++k) {
                        double vp[7], vm[7];
                        for (int i = 0; i < 2 * r - 1; ++i) {
                            const int a = j - r + 1 + i, b = j - r + 2 + i;
                            vp[i] = 0.5 * (fr[k * len + a] + af * ur[k * len + a]);
                            vm[i] = 0.5 * (fr[k * len + b] - af * ur[k * len + b]);
                        }
                        F[k * (nd + 1) + s] = oc_weno_left(r, vp, c->eps) + weno_right(r, vm, c->eps);
                    }
                    continue;
                }
                if (c->charw == 1) {
                    /* characteristic fields at the face state: the mean of the
                     * conserved states of the two cells beside the face */
                    double ub[MAXF], wb[MAXF], Rm[MAXF * MAXF], Lm[MAXF * MAXF], Fc[MAXF];
                    for (int k = 0; k < NF; ++k) ub[k] = 0.5 * (ur[k * len + j] + ur[k * len + j + 1]);
                    if (oc_con2prim(c->cs2, ub, wb)) {
                        bad |= 1;
                        continue;
                    }
                    for (int q = 5; q < NF; ++q) wb[q] = ub[q] * sqrt(1.0 - (wb[1] * wb[1] + wb[2] * wb[2] + wb[3] * wb[3]));
                    oc_char_basis(c->cs2, d, NF, wb, Rm, NULL);
                    if (oc_invert(NF, Rm, Lm)) {
                        bad |= 1;
                        continue;
                    }
                    for (int ch = 0; ch < NF; ++ch) {
                        double vp[7], vm[7];
                        for (int i = 0; i < 2 * r - 1; ++i) {
                            vp[i] = 0.0;
                            vm[i] = 0.0;
                            for (int k = 0; k < NF; ++k) {
                                vp[i] += Lm[ch * NF + k] * fp[k * len + j - r + 1 + i];
                                vm[i] += Lm[ch * NF + k] * fm[k * len + j - r + 2 + i];
                            }
                        }
                        Fc[ch] = oc_weno_left(r, vp, c->eps) + weno_right(r, vm, c->eps);
                    }
                    for (int k = 0; k < NF; ++k) {
                        double acc = 0.0;
                        for (int ch = 0; ch < NF; ++ch) acc += Rm[k * NF + ch] * Fc[ch];
                        F[k * (nd + 1) + s] = acc;
                    }
                    continue;
                }
                for (int k = 0; k < NF; ++k) {
                    const double *vp = fp + k * len + (j - r + 1);
                    const double *vm = fm + k * len + (j - r + 2);
                    F[k * (nd + 1) + s] = oc_weno_left(r, vp, c->eps) + weno_right(r, vm, c->eps);
                }
            }
            for (int s = 0; s < nd; ++s) {
                int ijk[3];
                ijk[d] = s;
                ijk[da] = ia;
                ijk[db] = ib;
                const int64_t q = cell(c, ijk[0], ijk[1], ijk[2]);
                for (int k = 0; k < NF; ++k)
                    L[k * N + q] += (F[k * (nd + 1) + s] - F[k * (nd + 1) + s + 1]) / c->dx[d];
            }
            free(fp);
            free(fm);
            free(F);
            free(fr);
            free(ur);
            free(sp);
        }
    }
    if (bad & 2) return OC_ERR_OOM;
    return bad ? OC_ERR_UNPHYSICAL : OC_OK;
}

/* ------------------------------------------------------------------------ */
/* Time stepping (Sec. 1: third-order Runge-Kutta, SSP form)                 */
/* ------------------------------------------------------------------------ */
static double cfl_dt(const oc_cfg *c, const double *alpha)
{
    if (c->dt_fixed > 0) return c->dt_fixed;
    int any = 0;
    for (int d = 0; d < 3; ++d) any |= active(c, d);
    double mindx = INFINITY, amax = 0.0;
    for (int d = 0; d < 3; ++d) {
        if (any && !active(c, d)) continue;
        mindx = fmin(mindx, c->dx[d]);
        amax = fmax(amax, alpha[d]);
    }
    return c->cfl * mindx / amax;
}

/* One RK3 stage: out = a*un + b*(us + dt*L(us; alpha)) (a = 0 for stage 1). */
static int rk_stage(const oc_cfg *c, const double *un, const double *us, const double *alpha,
                    double dt, double a, double b, double *out, double *Lbuf)
{
    const int rc = oc_L(c, us, alpha, Lbuf);
    if (rc) return rc;
    const int64_t M = (int64_t)nfields(c) * c->n[0] * c->n[1] * c->n[2];
#pragma omp parallel for num_threads(oc_get_max_threads())
    for (int64_t q = 0; q < M; ++q) {
        const double s = us[q] + dt * Lbuf[q];
        out[q] = (a == 0.0) ? s : a * un[q] + b * s;
    }
    return OC_OK;
}

/* Advance u in place by up to nsteps RK3 steps, stopping when t reaches
 * t_end (t_end < 0: no limit).  If alpha_in/dt_in are given, those frozen
 * values replace the computed ones (alpha_in[step*9 + stage*3 + d],
 * dt_in[step]).  alpha_out/dt_out (optional) record the values used.
 * *t and *steps are updated.  Returns 0 or an error code. */
int oc_run(const oc_cfg *c, double *u, int nsteps, double t_end, double *t, int64_t *steps,
           const double *alpha_in, const double *dt_in, double *alpha_out, double *dt_out)
{
    if (!cfg_ok(c) || nsteps < 0 || !t) return OC_ERR_ARG;
    const int64_t M = (int64_t)nfields(c) * c->n[0] * c->n[1] * c->n[2];
    double *u1 = malloc(sizeof(double) * M), *u2 = malloc(sizeof(double) * M);
    double *Lb = malloc(sizeof(double) * M);
    int rc = OC_OK;
    if (!u1 || !u2 || !Lb) rc = OC_ERR_OOM;
    for (int s = 0; s < nsteps && rc == OC_OK; ++s) {
        double a0[3], a1[3], a2[3], dt;
        if (alpha_in) {
            memcpy(a0, alpha_in + 9 * s, sizeof a0);
            dt = dt_in[s];
        } else {
            if ((rc = oc_alpha(c, u, a0))) break;
            dt = cfl_dt(c, a0);
            if (t_end >= 0 && *t + dt > t_end) dt = t_end - *t;
            if (!(dt > 0)) break;
        }
        if ((rc = rk_stage(c, u, u, a0, dt, 0.0, 1.0, u1, Lb))) break;
        if (alpha_in) memcpy(a1, alpha_in + 9 * s + 3, sizeof a1);
        else if ((rc = oc_alpha(c, u1, a1))) break;
        if ((rc = rk_stage(c, u, u1, a1, dt, 0.75, 0.25, u2, Lb))) break;
        if (alpha_in) memcpy(a2, alpha_in + 9 * s + 6, sizeof a2);
        else if ((rc = oc_alpha(c, u2, a2))) break;
        if ((rc = rk_stage(c, u, u2, a2, dt, 1.0 / 3.0, 2.0 / 3.0, u, Lb))) break;
        if (alpha_out) {
            memcpy(alpha_out + 9 * s, a0, sizeof a0);
            memcpy(alpha_out + 9 * s + 3, a1, sizeof a1);
            memcpy(alpha_out + 9 * s + 6, a2, sizeof a2);
        }
        if (dt_out) dt_out[s] = dt;
        *t += dt;
        if (steps) *steps += 1;
    }
    free(u1);
    free(u2);
    free(Lb);
    return rc;
}

/* Momentum anisotropy eps_2 = sum(T^xx - T^yy) / sum(T^xx + T^yy) over the
 * interior cells, T^ij = (e+p) gamma^2 v_i v_j + p delta_ij = M_i v_j + p delta_ij.
 * Serial sum in memory order. */
int oc_eps2(const oc_cfg *c, const double *u, double *out)
{
    if (!cfg_ok(c)) return OC_ERR_ARG;
    const int64_t N = (int64_t)c->n[0] * c->n[1] * c->n[2];
    double num = 0.0, den = 0.0;
    for (int64_t q = 0; q < N; ++q) {
        double uu[MAXF], w[MAXF];
        for (int f = 0; f < 5; ++f) uu[f] = u[f * N + q];
        if (oc_con2prim_eos(c->cs2, c->mass, uu, w)) return OC_ERR_UNPHYSICAL;
        const double p = oc_eos_p(c->cs2, c->mass, w);
        const double txx = uu[1] * w[1] + p, tyy = uu[2] * w[2] + p;
        num += txx - tyy;
        den += txx + tyy;
    }
    *out = num / den;
    return OC_OK;
}

/* Array versions of the point functions, for tests. */
/* (E, M, R_1..R_q) <-> (e, v, n_1..n_q) for nf = 4 + q fields of n cells. */
int oc_con2prim_n(double k, double m, int nf, const double *u, int64_t n, double *w)
{
    int bad = 0;
    if (nf < 5 || nf > MAXF) return OC_ERR_ARG;
    for (int64_t q = 0; q < n; ++q) {
        double uu[MAXF], ww[MAXF];
        for (int f = 0; f < nf; ++f) uu[f] = u[f * n + q];
        if (oc_con2prim_eos(k, m, uu, ww)) {
            bad = 1;
            for (int f = 0; f < nf; ++f) ww[f] = NAN;
        } else {
            const double v2 = ww[1] * ww[1] + ww[2] * ww[2] + ww[3] * ww[3];
            for (int f = 5; f < nf; ++f) ww[f] = uu[f] * sqrt(1.0 - v2);
        }
        for (int f = 0; f < nf; ++f) w[f * n + q] = ww[f];
    }
    return bad ? OC_ERR_UNPHYSICAL : OC_OK;
}

void oc_prim2con_n(double k, double m, int nf, const double *w, int64_t n, double *u)
{
    for (int64_t q = 0; q < n; ++q) {
        double uu[MAXF], ww[MAXF];
        for (int f = 0; f < nf; ++f) ww[f] = w[f * n + q];
        oc_prim2con_eos(k, m, ww, uu);
        const double g = 1.0 / sqrt(1.0 - (ww[1] * ww[1] + ww[2] * ww[2] + ww[3] * ww[3]));
        for (int f = 5; f < nf; ++f) uu[f] = ww[f] * g;
        for (int f = 0; f < nf; ++f) u[f * n + q] = uu[f];
    }
}
