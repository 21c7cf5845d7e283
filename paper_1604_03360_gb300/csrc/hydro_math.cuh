// hydro_math.cuh -- FP64 device arithmetic of the relativistic hydro scheme
// (Sikorski et al., arXiv:1604.03360): conserved->primitive recovery for
// p = cs2 e, the fluxes of Eq. 1, the characteristic speeds used by the
// Lax-Friedrichs splitting, and finite-difference WENO5 / WENO7 (Sec. 1.2).
//
// GB300 design notes.  On this part the FP64 pipe issues ~2 FMA per clock per
// SM while FP32/INT issue ~60x more, so every FP64 instruction counts:
//  * reconstructions return a fraction N/D (one reciprocal per face instead of
//    one division per weight);
//  * the Lax-Friedrichs split works on g = f +- alpha u = 2 f^{+-} and the
//    smoothness indicators are rescaled by powers of two (or 9 for WENO7)
//    with epsilon rescaled to match -- exact rescalings that leave the
//    nonlinear weights unchanged;
//  * reciprocals take the MUFU seed (rcp.approx.ftz.f64, on the SFU pipe) and
//    one cubically convergent Newton correction on the FP64 pipe.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "fp64_int.cuh"

namespace hydro {

// 1/x for finite, normal, positive or negative x.  Seed r0 from the MUFU
// approximation, then the series (Newton-Raphson of order three) correction
// r = r0 (1 + e + e^2), e = 1 - x r0, whose relative error is e^3 (Muller et
// al., Handbook of Floating-Point Arithmetic, Newton-Raphson division).  The
// result is within about one ulp of 1/x; it is not correctly rounded.
__device__ __forceinline__ double rcp(double x)
{
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    const double e = fma(-x, r, 1.0);
    const double t = fma(e, e, e);
    return fma(r, t, r);
}

// Conserved -> primitive for p = k e (positive root of
// k e^2 + (1-k) E e - (E^2 - M^2) = 0 in cancellation-free form).
// Returns false for E <= 0, |M| >= E or NaN.  Outputs p, v and e.
__device__ __forceinline__ bool con2prim(double k, double E, double mx, double my, double mz,
                                         double& p, double& vx, double& vy, double& vz, double& e)
{
    const double m2 = fma(mx, mx, fma(my, my, mz * mz));
    const double d = fma(E, E, -m2);
    if (!(E > 0.0) || !(d > 0.0)) return false;
    const double b = (1.0 - k) * E;
    const double s = sqrt(fma(b, b, 4.0 * k * d));
    e = (2.0 * d) * rcp(b + s);
    p = k * e;
    const double ih = rcp(E + p);
    vx = mx * ih;
    vy = my * ih;
    vz = mz * ih;
    return true;
}

// Conserved -> primitive for the general EOS p = k (e - m n), m > 0 (n = R /
// gamma, the first charge).  The pressure solves f(p) = k (e(p) - m n(p)) - p
// = 0 with v = M / (E + p), e = E - M.v, n = R sqrt(1 - v^2); f is decreasing
// (f' = v^2 c_s^2 - 1), f(0) > 0 is required (positive internal energy) and the
// p = k e pressure brackets the root from above.  Newton steps that leave the
// bracket are replaced by bisection; stops at f = 0, when the update no longer
// changes p, or when it is below 1e-15 p (at most 100 steps).  Returns false
// when no physical state exists.
static __device__ __noinline__ bool con2prim_gas(double k, double m, double E, double mx, double my, double mz, double R,
                                          double& p, double& vx, double& vy, double& vz, double& e)
{
    const double M2 = fma(mx, mx, fma(my, my, mz * mz));
    const double d = fma(E, E, -M2);
    if (!(E > 0.0) || !(d > 0.0) || !(R >= 0.0)) return false;
    const double iE = rcp(E);
    const double v20 = M2 * iE * iE;
    if (!(k * fma(-m * R, sqrt(1.0 - v20), fma(-M2, iE, E)) > 0.0)) return false;   // f(0) > 0
    const double b = (1.0 - k) * E;
    double hi = k * ((2.0 * d) * rcp(b + sqrt(fma(b, b, 4.0 * k * d))));
    double lo = 0.0, x = hi;
    for (int it = 0; it < 100; ++it) {
        const double ih = rcp(E + x);
        const double v2 = M2 * ih * ih;
        const double ee = fma(-M2, ih, E);
        const double n = R * sqrt(1.0 - v2);
        const double f = fma(k, fma(-m, n, ee), -x);
        if (f == 0.0) break;                      // x is the root
        const double fp = fma(v2 * (1.0 + k) * x, rcp(ee + x), -1.0);
        if (f > 0.0) lo = x;
        else hi = x;
        double xn = fma(-f, rcp(fp), x);
        if (xn == x) break;                       // the update is below the rounding of x
        if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
        const double dx = fabs(xn - x);
        x = xn;
        if (dx <= 1e-15 * x) break;
    }
    if (!(x > 0.0)) return false;
    const double ih = rcp(E + x);
    p = x;
    e = fma(-M2, ih, E);
    vx = mx * ih;
    vy = my * ih;
    vz = mz * ih;
    return true;
}

// squared sound speed of the general EOS: (1 + k) p / (e + p)
__device__ __forceinline__ double sound2_gas(double k, double p, double e) { return (1.0 + k) * p * rcp(e + p); }

// max(|lambda_+|, |lambda_-|) along each axis for p = k e, where
// lambda_+- = (v_d (1-k) +- sqrt(k (1-v^2)(1 - k v^2 - (1-k) v_d^2))) / (1 - k v^2);
// with a positive denominator and a non-negative root the larger magnitude is
// (|v_d| (1-k) + root) / (1 - k v^2).
__device__ __forceinline__ void max_speeds(double k, double vx, double vy, double vz, double out[3])
{
    const double v2 = fma(vx, vx, fma(vy, vy, vz * vz));
    const double one_kv2 = fma(-k, v2, 1.0);
    const double kq = k * (1.0 - v2);
    const double iden = rcp(one_kv2);
    const double omk = 1.0 - k;
    const double v[3] = {vx, vy, vz};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double rad = kq * fma(-omk * v[d], v[d], one_kv2);
        out[d] = fma(fabs(v[d]), omk, sqrt(rad)) * iden;
    }
}

// ---------------------------------------------------------------------------
// FD-WENO reconstruction (Jiang-Shu smoothness indicators, Sec. 1.2).
// weno_left: value at x_{j+1/2} from v[0..S-1] = v_{j-r+1} .. v_{j+r-1}.
// Result = N / D.  Candidate k uses v[k..k+r-1].
// ---------------------------------------------------------------------------

// r = 3.  With inputs g = 2 f the indicator b_k = 13/3 (2nd diff)^2 +
// (1st-derivative form)^2 equals 16 beta_k(f); eps_s must be 16 eps.
// N and D are the weight-normalised sums multiplied by 10 prod_k (eps+beta_k)^2.
// All linear forms are built from the differences d_i = v_{i+1} - v_i:
// 2nd differences s_k = d_{k+1} - d_k, first-derivative forms
// t0 = 3 d1 - d0, t1 = d1 + d2, t2 = 3 d2 - d3 (same values as the
// Jiang-Shu forms a - 4b + 3c, d - b, -3c + 4d - e).
//
// The differences of a window do not depend on the face it serves, so a sweep
// along a pencil carries them from one face to the next (Diff5 / Diff7): the
// window v_{j-r+1} .. v_{j+r-1} of face j+1/2 shares all but one difference
// of each order with the window of face j+3/2.  weno5 / weno7 compute them
// afresh; the *_slide functions update them for a window moved by one cell,
// with the same operations on the same operands, so a sweep gives the same
// bits as fresh windows.  The reconstruction functions are host functions
// too, so the same source also runs on the CPU (a host test checks it against
// the WENO definition and the sweeps against fresh windows).
struct Diff5 {
    double d[4];     // d_i = v_{i+1} - v_i
    double cs[3];    // 13/3 s_k^2 + eps_s, s_k = d_{k+1} - d_k
};

// EMU selects operations that run on the integer pipe (fp64_int.cuh) instead
// of the FP64 unit: kEmuConst the products with constants, kEmuWeights the
// squares and products of the nonlinear weights, kEmuFace the last products
// of the weighted sums and of the face combination.  Every choice gives the
// same bits.  (The flags kEmuConst, kEmuWeights and kEmuFace are defined in
// fp64_int.cuh.)
// the squares / the products of the nonlinear weights on the integer pipe
__host__ __device__ constexpr bool emu_wsq(int emu) { return (emu & kEmuWeights) != 0; }
__host__ __device__ constexpr bool emu_wprod(int emu) { return (emu & kEmuWeights) != 0; }

// The second-difference term 13/3 s_k^2 + eps of b_k depends on the three
// cells of stencil k only, so it is carried with the differences (as
// WENO7's third-difference term is).
template <bool EC>
__host__ __device__ __forceinline__ double w5_sterm(double s, double eps_s)
{
    return fma(xmul<EC>(13.0 / 3.0, s), s, eps_s);
}

template <int EMU = 0>
__host__ __device__ __forceinline__ void weno5_diffs(const double* v, double eps_s, Diff5& q)
{
    constexpr bool EC = (EMU & kEmuConst) != 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) q.d[i] = v[i + 1] - v[i];
#pragma unroll
    for (int k = 0; k < 3; ++k) q.cs[k] = w5_sterm<EC>(q.d[k + 1] - q.d[k], eps_s);
}

// window moved one cell up the array (v is the new window): the new cell
// enters at v[4]
template <int EMU = 0>
__host__ __device__ __forceinline__ void weno5_slide(const double* v, double eps_s, Diff5& q)
{
    constexpr bool EC = (EMU & kEmuConst) != 0;
#pragma unroll
    for (int i = 0; i < 3; ++i) q.d[i] = q.d[i + 1];
#pragma unroll
    for (int k = 0; k < 2; ++k) q.cs[k] = q.cs[k + 1];
    q.d[3] = v[4] - v[3];
    q.cs[2] = w5_sterm<EC>(q.d[3] - q.d[2], eps_s);
}

// mirrored window moved one cell (m is the new mirrored window): the new
// cell enters at m[0]
template <int EMU = 0>
__host__ __device__ __forceinline__ void weno5_slide_mirror(const double* m, double eps_s, Diff5& q)
{
    constexpr bool EC = (EMU & kEmuConst) != 0;
#pragma unroll
    for (int i = 3; i > 0; --i) q.d[i] = q.d[i - 1];
#pragma unroll
    for (int k = 2; k > 0; --k) q.cs[k] = q.cs[k - 1];
    q.d[0] = m[1] - m[0];
    q.cs[0] = w5_sterm<EC>(q.d[1] - q.d[0], eps_s);
}

// Result: the reconstruction is v[2] + M / D (the centre value plus a
// correction), see weno_left.
template <int EMU = 0>
__host__ __device__ __forceinline__ void weno5_core(const Diff5& q, double& M, double& D)
{
    constexpr bool EC = (EMU & kEmuConst) != 0;
    const double d0 = q.d[0], d1 = q.d[1], d2 = q.d[2], d3 = q.d[3];
    const double t0 = fma(3.0, d1, -d0), t1 = d1 + d2, t2 = fma(3.0, d2, -d3);
    const double b0 = fma(t0, t0, q.cs[0]);
    const double b1 = fma(t1, t1, q.cs[1]);
    const double b2 = fma(t2, t2, q.cs[2]);
    constexpr bool ES = emu_wsq(EMU), EP = emu_wprod(EMU);
    const double w0 = xmul<ES>(b0, b0), w1 = xmul<ES>(b1, b1), w2 = xmul<ES>(b2, b2);
    const double P0 = xmul<EP>(w1, w2), P1 = xmul<EP>(w0, w2), P2 = xmul<EP>(w0, w1);
    // 10 d_k (q_k - c), c = v[2]: d = (1, 6, 3)/10, q0 = (2a-7b+11c)/6 =
    // c - d0/3 + 5 d1/6, q1 = (-b+5c+2d)/6 = c + (d1 + 2 d2)/6,
    // q2 = (2c+5d-e)/6 = c + (4 d2 - d3)/6
    const double m0 = fma(5.0 / 6.0, d1, xmul<EC>(-1.0 / 3.0, d0));
    const double m1 = fma(2.0, d2, d1);
    const double m2 = fma(-0.5, d3, xmul_pow2<EC, 1>(d2));
    M = fma(m0, P0, fma(m1, P1, xmul<(EMU & kEmuFace) != 0>(m2, P2)));
    D = fma(3.0, P2, fma(6.0, P1, P0));
}

template <int EMU = 0>
__host__ __device__ __forceinline__ void weno5(double a, double b, double c, double d, double e, double eps_s,
                                      double& M, double& D)
{
    const double v[5] = {a, b, c, d, e};
    Diff5 q;
    weno5_diffs<EMU>(v, eps_s, q);
    weno5_core<EMU>(q, M, D);
}

// r = 4 (Balsara-Shu weights from the same definition).  For the cubic
// candidate p_k(xi) = sum c_i xi^i about x_j, beta = (c1 + c3/4)^2 +
// 13/3 c2^2 + 781/20 c3^2.  With A = 6 (c1 + c3/4), B = 2 c2, C = 6 c3
// (integer-coefficient forms) and inputs g = 2 f:
// b_k = A^2 + 39 B^2 + 781/20 C^2 = 144 beta_k(f); eps_s must be 144 eps.
// N and D are multiplied by 420 prod_k (eps+beta_k)^2 (35 from the linear
// weights, 12 from the candidate forms).
// In the difference basis d_i = v_{i+1} - v_i, e_i = d_{i+1} - d_i:
// C_k = e_{k+1} - e_k (third differences); B0 = 2 e1 - e0, B1 = B2 = e2,
// B3 = 2 e3 - e4; A0 = 2 d0 - 7 d1 + 11 d2, A1 = -d1 + 5 d2 + 2 d3,
// A2 = 2 d2 + 5 d3 - d4, A3 = 11 d3 - 7 d4 + 2 d5 (identical values to the
// forms written on the cell values).  The term 781/20 C_k^2 + eps depends on
// the cells of stencil k only, so it is carried with the differences.
struct Diff7 {
    double d[6];     // d_i = v_{i+1} - v_i
    double e[5];     // e_i = d_{i+1} - d_i
    double ct[4];    // 781/20 C_k^2 + eps_s, C_k = e_{k+1} - e_k
};

template <bool EC>
__host__ __device__ __forceinline__ double w7_cterm(double C, double eps_s)
{
    return fma(xmul<EC>(781.0 / 20.0, C), C, eps_s);
}

template <int EMU = 0>
__host__ __device__ __forceinline__ void weno7_diffs(const double* v, double eps_s, Diff7& q)
{
    constexpr bool EC = (EMU & kEmuConst) != 0;
#pragma unroll
    for (int i = 0; i < 6; ++i) q.d[i] = v[i + 1] - v[i];
#pragma unroll
    for (int i = 0; i < 5; ++i) q.e[i] = q.d[i + 1] - q.d[i];
#pragma unroll
    for (int k = 0; k < 4; ++k) q.ct[k] = w7_cterm<EC>(q.e[k + 1] - q.e[k], eps_s);
}

// window moved one cell up the array: the new cell enters at v[6]
template <int EMU = 0>
__host__ __device__ __forceinline__ void weno7_slide(const double* v, double eps_s, Diff7& q)
{
    constexpr bool EC = (EMU & kEmuConst) != 0;
#pragma unroll
    for (int i = 0; i < 5; ++i) q.d[i] = q.d[i + 1];
#pragma unroll
    for (int i = 0; i < 4; ++i) q.e[i] = q.e[i + 1];
#pragma unroll
    for (int k = 0; k < 3; ++k) q.ct[k] = q.ct[k + 1];
    q.d[5] = v[6] - v[5];
    q.e[4] = q.d[5] - q.d[4];
    q.ct[3] = w7_cterm<EC>(q.e[4] - q.e[3], eps_s);
}

// mirrored window moved one cell: the new cell enters at m[0]
template <int EMU = 0>
__host__ __device__ __forceinline__ void weno7_slide_mirror(const double* m, double eps_s, Diff7& q)
{
    constexpr bool EC = (EMU & kEmuConst) != 0;
#pragma unroll
    for (int i = 5; i > 0; --i) q.d[i] = q.d[i - 1];
#pragma unroll
    for (int i = 4; i > 0; --i) q.e[i] = q.e[i - 1];
#pragma unroll
    for (int k = 3; k > 0; --k) q.ct[k] = q.ct[k - 1];
    q.d[0] = m[1] - m[0];
    q.e[0] = q.d[1] - q.d[0];
    q.ct[0] = w7_cterm<EC>(q.e[1] - q.e[0], eps_s);
}

// Result: the reconstruction is v[3] + M / D, see weno_left.
template <int EMU = 0>
__host__ __device__ __forceinline__ void weno7_core(const Diff7& q, double& M, double& D)
{
    constexpr bool EC = (EMU & kEmuConst) != 0;
    const double d0 = q.d[0], d1 = q.d[1], d2 = q.d[2], d3 = q.d[3], d4 = q.d[4], d5 = q.d[5];
    const double e0 = q.e[0], e1 = q.e[1], e2 = q.e[2], e3 = q.e[3], e4 = q.e[4];
    const double B0 = fma(2.0, e1, -e0), B12 = e2, B3 = fma(2.0, e3, -e4);
    // A0 = 2 d0 - 7 d1 + 11 d2 = 6 d2 + 2 B0 + e1, A3 = 11 d3 - 7 d4 + 2 d5 =
    // 6 d3 - 2 B3 - e3
    const double A0 = fma(6.0, d2, fma(2.0, B0, e1));
    const double A1 = fma(2.0, d3, fma(5.0, d2, -d1));
    const double A2 = fma(5.0, d3, fma(2.0, d2, -d4));
    const double A3 = fma(6.0, d3, fma(-2.0, B3, -e3));
    const double b39 = xmul_small<EC, 39, 6, 0>(B12);
    const double b0 = fma(A0, A0, fma(xmul_small<EC, 39, 6, 0>(B0), B0, q.ct[0]));
    const double b1 = fma(A1, A1, fma(b39, B12, q.ct[1]));
    const double b2 = fma(A2, A2, fma(b39, B12, q.ct[2]));
    const double b3 = fma(A3, A3, fma(xmul_small<EC, 39, 6, 0>(B3), B3, q.ct[3]));
    constexpr bool ES = emu_wsq(EMU), EP = emu_wprod(EMU);
    const double w0 = xmul<ES>(b0, b0), w1 = xmul<ES>(b1, b1), w2 = xmul<ES>(b2, b2), w3 = xmul<ES>(b3, b3);
    const double p01 = xmul<EP>(w0, w1), p23 = xmul<EP>(w2, w3);
    const double P0 = xmul<EP>(w1, p23), P1 = xmul<EP>(w0, p23), P2 = xmul<EP>(p01, w3), P3 = xmul<EP>(p01, w2);
    // 35 d_k (q_k - v3), d = (1, 12, 18, 4)/35, in the difference basis:
    // q0 - v3 = (3 d0 - 10 d1 + 13 d2)/12, q1 - v3 = (-d1 + 4 d2 + 3 d3)/12,
    // q2 - v3 = (d2 + 6 d3 - d4)/12, q3 - v3 = (9 d3 - 4 d4 + d5)/12.  Each
    // numerator is A_k + B_k of the smoothness forms (3 d0 - 10 d1 + 13 d2 =
    // A0 + B0, and so on), so with M and D both taken 12 times larger
    // m_k = 12 x 35 d_k (q_k - v3) = (1, 12, 18, 4)_k (A_k + B_k): one
    // addition each, the factors on the integer pipe
    const double m0 = A0 + B0;
    const double m1 = xmul_small<EC, 3, 2, 2>(A1 + B12);
    const double m2 = xmul_small<EC, 9, 4, 1>(A2 + B12);
    const double m3 = xmul_pow2<EC, 2>(A3 + B3);
    M = fma(m0, P0, fma(m1, P1, fma(m2, P2, xmul<(EMU & kEmuFace) != 0>(m3, P3))));
    D = fma(48.0, P3, fma(216.0, P2, fma(144.0, P1, xmul_small<EC, 3, 2, 2>(P0))));
}

template <int EMU = 0>
__host__ __device__ __forceinline__ void weno7(const double* v, double eps_s, double& M, double& D)
{
    Diff7 q;
    weno7_diffs<EMU>(v, eps_s, q);
    weno7_core<EMU>(q, M, D);
}

// Left-biased value at x_{j+1/2} from v[0..S-1] = v_{j-r+1} .. v_{j+r-1}: the
// centre value v[r-1] = v_j plus M / D, where D = sum_k d_k alpha_k and
// M = sum_k d_k alpha_k (q_k - v_j) up to one common positive factor (q_k the
// candidate values, alpha_k = 1/(eps+beta_k)^2); candidate k uses v[k..k+r-1].
template <int R, int EMU = 0>
__host__ __device__ __forceinline__ void weno_left(const double* v, double eps_s, double& M, double& D)
{
    if constexpr (R == 3) weno5<EMU>(v[0], v[1], v[2], v[3], v[4], eps_s, M, D);
    else weno7<EMU>(v, eps_s, M, D);
}

// Right-biased value at x_{j-1/2} of the stencil centred on j: the mirror
// image, again v[r-1] + M / D.
template <int R, int EMU = 0>
__host__ __device__ __forceinline__ void weno_right(const double* v, double eps_s, double& M, double& D)
{
    if constexpr (R == 3) {
        weno5<EMU>(v[4], v[3], v[2], v[1], v[0], eps_s, M, D);
    } else {
        const double m[7] = {v[6], v[5], v[4], v[3], v[2], v[1], v[0]};
        weno7<EMU>(m, eps_s, M, D);
    }
}

// 2^(1023 - e) for the biased exponent e of x (e clamped to 1 .. 2045, so
// the factor is a normal number): x times it lies in [1, 2) for normal x.
__device__ __forceinline__ double pow2_unscale(double x)
{
    int e = (int)(((unsigned)__double2hiint(x) >> 20) & 0x7ffu);
    e = min(max(e, 1), 2045);
    return __hiloint2double((2046 - e) << 20, 0);
}

// Face value (cp + Mp/Dp) + (cm + Mm/Dm) with one reciprocal; cp, cm are the
// centre values of the two stencils.
//
// Dynamic range.  Dp and Dm are products of r - 1 squared smoothness terms
// (eps + beta)^2, so they span a far wider range than the data: Dp Dm can
// overflow (then the correction would silently vanish) or underflow (then
// rcp.approx.ftz gives inf).  When either D leaves [2^-448, 2^448] -- checked
// with integer operations on the exponent fields, off the FP64 pipe -- both
// sides are first scaled by exact powers of two into [1, 2).  That leaves
// M/D unchanged, and inside the range the result is the same as before bit
// for bit.  The scaled path holds while each D and M is a finite normal
// number: eps >= 1e-40 (checked at set-up) and split-flux differences below
// about 1e24 (WENO7) or 1e37 (WENO5).
__device__ __forceinline__ double face_sum_rescaled(double Mp, double Dp, double cp, double Mm, double Dm, double cm)
{
    const double sp = pow2_unscale(Dp), sm = pow2_unscale(Dm);
    Mp *= sp;
    Dp *= sp;
    Mm *= sm;
    Dm *= sm;
    return fma(fma(Mp, Dm, Mm * Dp), rcp(Dp * Dm), cp + cm);
}

constexpr unsigned kFaceExpLo = 1023u - 448u, kFaceExpSpan = 896u;

template <int EMU = 0>
__device__ __forceinline__ double face_sum(double Mp, double Dp, double cp, double Mm, double Dm, double cm)
{
    constexpr bool EF = (EMU & kEmuFace) != 0;
    const unsigned ep = ((unsigned)__double2hiint(Dp) >> 20) - kFaceExpLo;
    const unsigned em = ((unsigned)__double2hiint(Dm) >> 20) - kFaceExpLo;
    if (max(ep, em) > kFaceExpSpan) return face_sum_rescaled(Mp, Dp, cp, Mm, Dm, cm);
    return fma(fma(Mp, Dm, xmul<EF>(Mm, Dp)), rcp(xmul<EF>(Dp, Dm)), cp + cm);
}

template <int R> struct SchemeConst;
template <> struct SchemeConst<3> { static constexpr double eps_scale = 16.0; };
template <> struct SchemeConst<4> { static constexpr double eps_scale = 144.0; };

}  // namespace hydro
