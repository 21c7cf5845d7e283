// adj_weno.cuh -- reverse mode (vector-Jacobian product) of the scaled WENO5
// and WENO7 face reconstructions of hydro_math.cuh (Sec. 1.2), written for a
// sweep along one pencil, with the smoothness indicators differentiated as
// they are (smooth weights, epsilon > 0).
//
// Forward form of one reconstruction from the window v[0 .. 2r-2]: in the
// difference basis d_i = v_{i+1} - v_i (and their differences), b_k = eps_s +
// (smoothness forms of stencil k)^2, w_k = b_k^2, P_k = prod_{m!=k} w_m,
// D = sum_k dc_k P_k, M = sum_k m_k P_k with m_k the centre-relative candidate
// forms (linear in d), value = v[r-1] + M / D.
//
// Reverse form: Rbar (the adjoint of the value) goes to the centre cell
// directly, and M / D sends its adjoint through P -> w -> b -> the smoothness
// forms and m_k onto the differences: db_i, the adjoint of d_i.  Along a
// pencil the differences are shared by consecutive faces, so both the
// forward differences and their adjoints are carried from face to face: the
// sweep takes one new difference per face and side, accumulates db into the
// adjoints of the differences still in some window, and a difference leaving
// every window sends +-its adjoint to its two cells (d_i = v_{i+1} - v_i).
//
// EMU selects products computed on the integer pipe (fp64_int.cuh; the same
// bits): kEmuConst the products with constants, kEmuWeights those of w and P
// and their reverse (wbar), kEmuFace the other products of the reverse sweep.
// A product kept on the FP64 unit is an explicitly rounded multiply, so the
// compiler never contracts it into an FMA with a later add and every choice
// gives the same bits.
//
// The header also compiles as plain C++ (host, with 1/x for the reciprocal),
// so the same source is checked on the host against complex-step derivatives
// of the forward formulas.
#pragma once
#include <cmath>

#include "fp64_int.cuh"
#ifdef __CUDACC__
#include "hydro_math.cuh"
#endif

namespace hydro {

// x * y on the integer pipe (E) or the FP64 unit, never contracted
template <bool E>
HYDRO_HD double pmul(double x, double y)
{
    if constexpr (E) {
        return dmul_int(x, y);
    } else {
#ifdef __CUDA_ARCH__
        return __dmul_rn(x, y);
#else
        return x * y;
#endif
    }
}

HYDRO_HD double adj_rcp(double x)
{
#ifdef __CUDA_ARCH__
    return rcp(x);
#else
    return 1.0 / x;
#endif
}

// Forward differences of one window that the reverse form needs, carried
// along the sweep.  WENO5: d (4) and s_k = d_{k+1} - d_k (13/3 s_k is formed
// per face, on the integer pipe: carrying it too costs a CTA per SM).
// WENO7: d (6), e_i = d_{i+1} - d_i (5), C_k = e_{k+1} - e_k, kC_k = 781/20
// C_k and ct_k = kC_k C_k + eps_s (the third-difference term of b_k).
template <int R> struct AdjWin;
template <> struct AdjWin<3> { double d[4], s[3]; };
template <> struct AdjWin<4> { double d[6], e[5], C[4], kC[4], ct[4]; };

template <bool EC>
HYDRO_HD void adj_win_fill(AdjWin<3>& q, double)
{
    for (int k = 0; k < 3; ++k) q.s[k] = q.d[k + 1] - q.d[k];
}
template <bool EC>
HYDRO_HD void adj_win_fill(AdjWin<4>& q, double eps_s)
{
    for (int i = 0; i < 5; ++i) q.e[i] = q.d[i + 1] - q.d[i];
    for (int k = 0; k < 4; ++k) {
        q.C[k] = q.e[k + 1] - q.e[k];
        q.kC[k] = xmul<EC>(781.0 / 20.0, q.C[k]);
        q.ct[k] = fma(q.kC[k], q.C[k], eps_s);
    }
}

// the window v[0 .. 2R-2], differences formed afresh
template <int R, bool EC>
HYDRO_HD void adj_win_init(const double* v, double eps_s, AdjWin<R>& q)
{
    for (int i = 0; i < 2 * R - 2; ++i) q.d[i] = v[i + 1] - v[i];
    adj_win_fill<EC>(q, eps_s);
}

// the window moved one cell up its array: dn = v[2R-2] - v[2R-3] of the new
// window enters at the top; the others are the previous window's
template <bool EC>
HYDRO_HD void adj_win_top(AdjWin<3>& q, double dn, double)
{
    for (int i = 0; i < 3; ++i) q.d[i] = q.d[i + 1];
    for (int k = 0; k < 2; ++k) q.s[k] = q.s[k + 1];
    q.d[3] = dn;
    q.s[2] = q.d[3] - q.d[2];
}
template <bool EC>
HYDRO_HD void adj_win_top(AdjWin<4>& q, double dn, double eps_s)
{
    for (int i = 0; i < 5; ++i) q.d[i] = q.d[i + 1];
    for (int i = 0; i < 4; ++i) q.e[i] = q.e[i + 1];
    for (int k = 0; k < 3; ++k) {
        q.C[k] = q.C[k + 1];
        q.kC[k] = q.kC[k + 1];
        q.ct[k] = q.ct[k + 1];
    }
    q.d[5] = dn;
    q.e[4] = q.d[5] - q.d[4];
    q.C[3] = q.e[4] - q.e[3];
    q.kC[3] = xmul<EC>(781.0 / 20.0, q.C[3]);
    q.ct[3] = fma(q.kC[3], q.C[3], eps_s);
}

// a mirrored window moved one cell: dn = m[1] - m[0] of the new window
// enters at the bottom
template <bool EC>
HYDRO_HD void adj_win_bottom(AdjWin<3>& q, double dn, double)
{
    for (int i = 3; i > 0; --i) q.d[i] = q.d[i - 1];
    for (int k = 2; k > 0; --k) q.s[k] = q.s[k - 1];
    q.d[0] = dn;
    q.s[0] = q.d[1] - q.d[0];
}
template <bool EC>
HYDRO_HD void adj_win_bottom(AdjWin<4>& q, double dn, double eps_s)
{
    for (int i = 5; i > 0; --i) q.d[i] = q.d[i - 1];
    for (int i = 4; i > 0; --i) q.e[i] = q.e[i - 1];
    for (int k = 3; k > 0; --k) {
        q.C[k] = q.C[k - 1];
        q.kC[k] = q.kC[k - 1];
        q.ct[k] = q.ct[k - 1];
    }
    q.d[0] = dn;
    q.e[0] = q.d[1] - q.d[0];
    q.C[0] = q.e[1] - q.e[0];
    q.kC[0] = xmul<EC>(781.0 / 20.0, q.C[0]);
    q.ct[0] = fma(q.kC[0], q.C[0], eps_s);
}

// WENO5: db[0 .. 3] = Rbar * d(M / D)/d(d_i).  Smoothness forms t_k (first
// derivative: 3 d1 - d0, d1 + d2, 3 d2 - d3) and s_k; linear weights
// dc = (1, 6, 3); m_k = 10 dc_k (q_k - v_2) = (5 d1 / 6 - d0 / 3,
// 2 d2 + d1, 2 d2 - d3 / 2).
template <int EMU>
HYDRO_HD void adj_core(const AdjWin<3>& q, double eps_s, double Rbar, double* db)
{
    constexpr bool EC = (EMU & kEmuConst) != 0, EW = (EMU & kEmuWeights) != 0, EF = (EMU & kEmuFace) != 0;
    const double d0 = q.d[0], d1 = q.d[1], d2 = q.d[2], d3 = q.d[3];
    const double ks0 = xmul<EC>(13.0 / 3.0, q.s[0]), ks1 = xmul<EC>(13.0 / 3.0, q.s[1]);
    const double ks2 = xmul<EC>(13.0 / 3.0, q.s[2]);
    const double t0 = fma(3.0, d1, -d0), t1 = d1 + d2, t2 = fma(3.0, d2, -d3);
    const double b0 = fma(ks0, q.s[0], fma(t0, t0, eps_s));
    const double b1 = fma(ks1, q.s[1], fma(t1, t1, eps_s));
    const double b2 = fma(ks2, q.s[2], fma(t2, t2, eps_s));
    const double w0 = pmul<EW>(b0, b0), w1 = pmul<EW>(b1, b1), w2 = pmul<EW>(b2, b2);
    const double P0 = pmul<EW>(w1, w2), P1 = pmul<EW>(w0, w2), P2 = pmul<EW>(w0, w1);
    const double m0 = fma(5.0 / 6.0, d1, xmul<EC>(-1.0 / 3.0, d0));
    const double m1 = fma(2.0, d2, d1);
    const double m2 = fma(-0.5, d3, xmul_pow2<EC, 1>(d2));
    const double M = fma(m0, P0, fma(m1, P1, pmul<EF>(m2, P2)));
    const double D = fma(3.0, P2, fma(6.0, P1, P0));
    // reverse: value = c + M / D
    const double iD = adj_rcp(D);
    const double Mb = pmul<EF>(Rbar, iD);
    const double Db = -pmul<EF>(Mb, pmul<EF>(M, iD));
    const double Pb0 = fma(Mb, m0, Db), Pb1 = fma(Mb, m1, xmul_small<EC, 3, 2, 1>(Db));
    const double Pb2 = fma(Mb, m2, xmul_small<EC, 3, 2, 0>(Db));
    const double mb0 = pmul<EF>(Mb, P0), mb1 = pmul<EF>(Mb, P1), mb2 = pmul<EF>(Mb, P2);
    // w_k = b_k^2 enters every P_m with m != k
    const double wb0 = fma(Pb1, w2, pmul<EW>(Pb2, w1)), wb1 = fma(Pb0, w2, pmul<EW>(Pb2, w0));
    const double wb2 = fma(Pb0, w1, pmul<EW>(Pb1, w0));
    // b_k = eps + t_k^2 + 13/3 s_k^2: tbar = 4 t b wbar, sbar = 4 (13/3) s b wbar
    const double g0 = pmul<EF>(xmul_pow2<EC, 2>(b0), wb0), g1 = pmul<EF>(xmul_pow2<EC, 2>(b1), wb1);
    const double g2 = pmul<EF>(xmul_pow2<EC, 2>(b2), wb2);
    const double tb0 = pmul<EF>(t0, g0), tb1 = pmul<EF>(t1, g1), tb2 = pmul<EF>(t2, g2);
    const double sb0 = pmul<EF>(ks0, g0), sb1 = pmul<EF>(ks1, g1), sb2 = pmul<EF>(ks2, g2);
    // transposes of t_k, s_k (s_k = d_{k+1} - d_k) and m_k onto the d_i
    db[0] = fma(-1.0 / 3.0, mb0, -(tb0 + sb0));
    db[1] = fma(3.0, tb0, fma(5.0 / 6.0, mb0, (tb1 + mb1) + (sb0 - sb1)));
    db[2] = fma(3.0, tb2, fma(2.0, mb1 + mb2, tb1 + (sb1 - sb2)));
    db[3] = fma(-0.5, mb2, sb2 - tb2);
}

// WENO7: db[0 .. 5].  b_k = A_k^2 + 39 B_k^2 + ct_k with (in d)
// A = (2 d0 - 7 d1 + 11 d2, -d1 + 5 d2 + 2 d3, 2 d2 + 5 d3 - d4,
// 11 d3 - 7 d4 + 2 d5), B = (2 e1 - e0, e2, e2, 2 e3 - e4), C_k = e_{k+1} - e_k;
// dc = (1, 12, 18, 4); m_k = 35 dc_k (q_k - v_3) = (d0/4 - 5 d1/6 + 13 d2/12,
// -d1 + 4 d2 + 3 d3, 3 (d2 - d4)/2 + 9 d3, 3 d3 - 4 d4/3 + d5/3).  The
// forward forms are those of weno7_core (A0 and A3 through B0 and B3, m1 as
// A1 + e2), the same values.
template <int EMU>
HYDRO_HD void adj_core(const AdjWin<4>& q, double eps_s, double Rbar, double* db)
{
    constexpr bool EC = (EMU & kEmuConst) != 0, EW = (EMU & kEmuWeights) != 0, EF = (EMU & kEmuFace) != 0;
    (void)eps_s;
    const double d0 = q.d[0], d1 = q.d[1], d2 = q.d[2], d3 = q.d[3], d4 = q.d[4], d5 = q.d[5];
    const double e0 = q.e[0], e1 = q.e[1], e2 = q.e[2], e3 = q.e[3], e4 = q.e[4];
    const double B0 = fma(2.0, e1, -e0), B12 = e2, B3 = fma(2.0, e3, -e4);
    const double A0 = fma(6.0, d2, fma(2.0, B0, e1));
    const double A1 = fma(2.0, d3, fma(5.0, d2, -d1));
    const double A2 = fma(5.0, d3, fma(2.0, d2, -d4));
    const double A3 = fma(6.0, d3, fma(-2.0, B3, -e3));
    const double kB0 = xmul_small<EC, 39, 6, 0>(B0), kB12 = xmul_small<EC, 39, 6, 0>(B12);
    const double kB3 = xmul_small<EC, 39, 6, 0>(B3);
    const double b0 = fma(A0, A0, fma(kB0, B0, q.ct[0]));
    const double b1 = fma(A1, A1, fma(kB12, B12, q.ct[1]));
    const double b2 = fma(A2, A2, fma(kB12, B12, q.ct[2]));
    const double b3 = fma(A3, A3, fma(kB3, B3, q.ct[3]));
    const double w0 = pmul<EW>(b0, b0), w1 = pmul<EW>(b1, b1), w2 = pmul<EW>(b2, b2), w3 = pmul<EW>(b3, b3);
    const double w01 = pmul<EW>(w0, w1), w23 = pmul<EW>(w2, w3), w02 = pmul<EW>(w0, w2);
    const double w03 = pmul<EW>(w0, w3), w12 = pmul<EW>(w1, w2), w13 = pmul<EW>(w1, w3);
    const double P0 = pmul<EW>(w1, w23), P1 = pmul<EW>(w0, w23), P2 = pmul<EW>(w01, w3), P3 = pmul<EW>(w01, w2);
    const double m0 = fma(13.0 / 12.0, d2, fma(-5.0 / 6.0, d1, xmul_pow2<EC, -2>(d0)));
    const double m1 = A1 + B12;
    const double m2 = fma(9.0, d3, xmul_small<EC, 3, 2, -1>(d2 - d4));
    const double m3 = fma(3.0, d3, fma(-4.0 / 3.0, d4, xmul<EC>(1.0 / 3.0, d5)));
    const double M = fma(m0, P0, fma(m1, P1, fma(m2, P2, pmul<EF>(m3, P3))));
    const double D = fma(4.0, P3, fma(18.0, P2, fma(12.0, P1, P0)));
    // reverse: value = c + M / D
    const double iD = adj_rcp(D);
    const double Mb = pmul<EF>(Rbar, iD);
    const double Db = -pmul<EF>(Mb, pmul<EF>(M, iD));
    const double Pb0 = fma(Mb, m0, Db), Pb1 = fma(Mb, m1, xmul_small<EC, 3, 2, 2>(Db));
    const double Pb2 = fma(Mb, m2, xmul_small<EC, 9, 4, 1>(Db)), Pb3 = fma(Mb, m3, xmul_pow2<EC, 2>(Db));
    const double mb0 = pmul<EF>(Mb, P0), mb1 = pmul<EF>(Mb, P1), mb2 = pmul<EF>(Mb, P2), mb3 = pmul<EF>(Mb, P3);
    // leave-two-out products for wbar
    const double wb0 = fma(Pb1, w23, fma(Pb2, w13, pmul<EW>(Pb3, w12)));
    const double wb1 = fma(Pb0, w23, fma(Pb2, w03, pmul<EW>(Pb3, w02)));
    const double wb2 = fma(Pb0, w13, fma(Pb1, w03, pmul<EW>(Pb3, w01)));
    const double wb3 = fma(Pb0, w12, fma(Pb1, w02, pmul<EW>(Pb2, w01)));
    // Abar = 4 A b wbar, Bbar = 4 (39 B) b wbar, Cbar = 4 (781/20 C) b wbar
    const double g0 = pmul<EF>(xmul_pow2<EC, 2>(b0), wb0), g1 = pmul<EF>(xmul_pow2<EC, 2>(b1), wb1);
    const double g2 = pmul<EF>(xmul_pow2<EC, 2>(b2), wb2), g3 = pmul<EF>(xmul_pow2<EC, 2>(b3), wb3);
    const double Ab0 = pmul<EF>(A0, g0), Ab1 = pmul<EF>(A1, g1), Ab2 = pmul<EF>(A2, g2), Ab3 = pmul<EF>(A3, g3);
    const double Bb0 = pmul<EF>(kB0, g0), Bb1 = pmul<EF>(kB12, g1), Bb2 = pmul<EF>(kB12, g2);
    const double Bb3 = pmul<EF>(kB3, g3);
    const double Cb0 = pmul<EF>(q.kC[0], g0), Cb1 = pmul<EF>(q.kC[1], g1), Cb2 = pmul<EF>(q.kC[2], g2);
    const double Cb3 = pmul<EF>(q.kC[3], g3);
    // (B, C) -> e
    const double eb0 = -Bb0 - Cb0;
    const double eb1 = fma(2.0, Bb0, Cb0 - Cb1);
    const double eb2 = Bb1 + Bb2 + (Cb1 - Cb2);
    const double eb3 = fma(2.0, Bb3, Cb2 - Cb3);
    const double eb4 = Cb3 - Bb3;
    // (A, e, m) -> d
    db[0] = fma(2.0, Ab0, fma(0.25, mb0, -eb0));
    db[1] = fma(-7.0, Ab0, fma(-5.0 / 6.0, mb0, (eb0 - eb1) - (Ab1 + mb1)));
    db[2] = fma(11.0, Ab0, fma(5.0, Ab1, fma(2.0, Ab2, fma(13.0 / 12.0, mb0, fma(4.0, mb1, fma(1.5, mb2, eb1 - eb2))))));
    db[3] = fma(2.0, Ab1, fma(5.0, Ab2, fma(11.0, Ab3, fma(3.0, mb1 + mb3, fma(9.0, mb2, eb2 - eb3)))));
    db[4] = fma(-7.0, Ab3, fma(-1.5, mb2, fma(-4.0 / 3.0, mb3, (eb3 - eb4) - Ab2)));
    db[5] = fma(2.0, Ab3, fma(1.0 / 3.0, mb3, eb4));
}

// Reverse sweep over faces j0 .. j1 of one pencil (face j between cells j and
// j+1) of the face flux F_j = R+(g+ of cells j-r+1 .. j+r-1) + R-(g- of cells
// j-r+2 .. j+r), R- the mirror image of R+, with face adjoints
// Fbar_j = sc (lam(j+1) - lam(j)).
//   load(m, gp, gm): the split fluxes g+, g- of cell m (any m: the caller
//     applies the boundary rule);
//   lam(m): the stage-output adjoint of cell m (0 outside the grid);
//   emit(m, vp, vm): this segment's whole contribution to gbar+ and gbar- of
//     cell m, called once for every m = j0-r+1 .. j1+r, in increasing order.
// Per face and side: one new difference, the reverse form onto the window's
// differences, and one cell completed.  After the last face the windows
// drain through 2r-1 more steps without faces.
template <int R, int EMU, class Load, class Lam, class Emit>
HYDRO_HD void adj_sweep(int j0, int j1, double eps_s, double sc, Load load, Lam lam, Emit emit)
{
    constexpr int G = R, S = 2 * R - 1, ND = 2 * R - 2;
    constexpr bool EC = (EMU & kEmuConst) != 0;
    AdjWin<R> qp, qm;        // + side: cells j-G+1 .. j+G-1; - side mirrored: cells j+G .. j-G+2
    double gp_top, gp_next, gm_top;
    {
        double gp[S + 1], gm[S + 1];
        for (int i = 0; i <= S; ++i) load(j0 - G + 1 + i, gp[i], gm[i]);
        adj_win_init<R, EC>(gp, eps_s, qp);
        double m[S];
        for (int i = 0; i < S; ++i) m[i] = gm[S - i];
        adj_win_init<R, EC>(m, eps_s, qm);
        gp_top = gp[S - 1];
        gp_next = gp[S];
        gm_top = gm[S];
    }
    // adjoints of the differences in a window: dp[i] of d_{j-G+1+i} (+ side),
    // dm[i] of d_{j-G+2+i} (- side; d_c = g_{c+1} - g_c)
    double dp[ND], dm[ND];
    for (int i = 0; i < ND; ++i) dp[i] = dm[i] = 0.0;
    double fb[G + 1];        // fb[G - i] = Fbar of face j - i
    for (int i = 0; i <= G; ++i) fb[i] = 0.0;
    double prevp = 0.0;      // + side: the adjoint of d_{j-G} (completed at face j-1)
    double pm1 = 0.0, pm2 = 0.0;  // - side: those of d_{j-G+1}, d_{j-G}
    double lamL = lam(j0);
    for (int j = j0; j <= j1 + 2 * G - 1; ++j) {
        for (int i = 0; i < G; ++i) fb[i] = fb[i + 1];
        if (j <= j1) {
            const double lamR = lam(j + 1);
            const double Fb = sc * (lamR - lamL);
            lamL = lamR;
            fb[G] = Fb;
            double bp[ND], bm[ND];
            adj_core<EMU>(qp, eps_s, Fb, bp);
            adj_core<EMU>(qm, eps_s, Fb, bm);
            for (int i = 0; i < ND - 1; ++i) dp[i] += bp[i];
            dp[ND - 1] = bp[ND - 1];
            // mirrored difference i is -d_{j+G-1-i}
            for (int i = 1; i < ND; ++i) dm[ND - 1 - i] -= bm[i];
            dm[ND - 1] = -bm[0];
        } else {
            fb[G] = 0.0;
            dp[ND - 1] = 0.0;
            dm[ND - 1] = 0.0;
        }
        // cell j-G+1 is complete: its centre term (+ side: face j-G+1, - side:
        // face j-G) and the adjoints of its two differences
        const double vp = fb[1] + prevp - dp[0];
        const double vm = fb[0] + pm2 - pm1;
        prevp = dp[0];
        pm2 = pm1;
        pm1 = dm[0];
        emit(j - G + 1, vp, vm);
        for (int i = 0; i < ND - 1; ++i) {
            dp[i] = dp[i + 1];
            dm[i] = dm[i + 1];
        }
        // the windows of face j+1: + side gains cell j+G, - side cell j+G+1
        if (j + 1 <= j1) {
            double gpn, gmn;
            load(j + G + 1, gpn, gmn);
            adj_win_top<EC>(qp, gp_next - gp_top, eps_s);
            gp_top = gp_next;
            gp_next = gpn;
            adj_win_bottom<EC>(qm, gm_top - gmn, eps_s);
            gm_top = gmn;
        }
    }
}

}  // namespace hydro
