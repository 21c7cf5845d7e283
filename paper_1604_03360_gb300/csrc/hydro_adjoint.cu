// hydro_adjoint.cu -- reverse mode (vector-Jacobian product) of N steps of the
// WENO + SSP-RK3 scheme, with the Lax-Friedrichs speeds and the time steps
// frozen at their forward values (their maxima are not differentiable), and
// the momentum-anisotropy observable eps_2 with its gradient.
//
// Forward with recording: every step stores its speeds (stage inputs) and dt;
// the state is checkpointed every `ckpt_every` steps.  Backward, segment by
// segment from the last: recompute the segment from its checkpoint with
// frozen stages, keeping every stage input (u and its primitives) of every
// step of the segment, then for each step (last first) run the three stage
// adjoints in reverse:
//   u_out = ca u_n + cb (u_s + dt L(u_s))  =>
//   lam_s = cb lam_out + J_L(u_s)^T (cb dt lam_out),  lam_n += ca lam_out.
// J_L^T mu is a sum over axes.  One thread per (axis, field, pencil) sweeps
// the pencil's faces with a register window: face adjoint
// F~bar_{j+1/2} = hdx (mu_{j+1} - mu_j), reverse-mode WENO of both biased
// reconstructions into the split-flux adjoints gbar+-, ghost-cell
// contributions folded back onto their source cells by the boundary rule (no
// atomics anywhere); then one cell kernel applies, summed over the axes,
//   ubar = sum_d J_f_d(u)^T (gbar+_d + gbar-_d) + alpha_d (gbar+_d - gbar-_d).
// A warp's pencils are consecutive in the fastest index of the array it
// sweeps, so y and z pencils read and write coalesced rows.  x pencils would
// not (consecutive threads a row apart), so their inputs are first
// transposed into an x-slowest layout (y fastest, then z, then x), swept
// there as the slowest axis by the same kernel, and their outputs transposed
// back: the same operations on the same operands, so the same bits.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "hydro_common.cuh"

namespace hydro {

// ---------------------------------------------------------------- WENO VJPs
// The scaled reconstructions of weno5 / weno7 (hydro_math.cuh), written in
// their difference bases: b_k = eps_s + (smoothness forms)^2, w_k = b_k^2,
// P_k = prod_{m!=k} w_m, N = sum n_k P_k, D = sum dc_k P_k, value = N / D.
// vb (+)= Rbar * d(N/D)/dv: the forward values once, then the reverse sweep
// N, D -> P -> w -> b -> (smoothness forms, n) -> v.  EMU selects products
// computed on the integer pipe (fp64_int.cuh; the same bits): kEmuConst the
// products with constants, kEmuWeights those of w and P and their reverse
// (wbar), kEmuFace the other products of the reverse sweep.  ACC: accumulate
// into vb[0 .. 2R-3] (else overwrite them); vb[2R-2], the newest cell of a
// sliding window, is always overwritten.  Checked against complex-step derivatives of
// the forward formulas (1e-14 WENO5, 2e-14 WENO7).
// x * y on the integer pipe (E) or the FP64 unit; the FP64 product is never
// contracted into an FMA with a later add, so both give the same bits
template <bool E>
__device__ __forceinline__ double pmul(double x, double y)
{
    if constexpr (E) return dmul_int(x, y);
    else return __dmul_rn(x, y);
}

template <bool ACC>
__device__ __forceinline__ void vjp_out(double& dst, double x)
{
    if constexpr (ACC) dst += x;
    else dst = x;
}

template <int EMU, bool ACC>
__device__ __forceinline__ void weno5_vjp(const double* v, double eps_s, double Rbar, double* vb)
{
    constexpr bool EC = (EMU & kEmuConst) != 0, EW = (EMU & kEmuWeights) != 0, EF = (EMU & kEmuFace) != 0;
    const double d0 = v[1] - v[0], d1 = v[2] - v[1], d2 = v[3] - v[2], d3 = v[4] - v[3];
    const double s0 = d1 - d0, s1 = d2 - d1, s2 = d3 - d2;
    const double t0 = fma(3.0, d1, -d0), t1 = d1 + d2, t2 = fma(3.0, d2, -d3);
    const double ks0 = xmul<EC>(13.0 / 3.0, s0), ks1 = xmul<EC>(13.0 / 3.0, s1), ks2 = xmul<EC>(13.0 / 3.0, s2);
    const double b0 = fma(ks0, s0, fma(t0, t0, eps_s));
    const double b1 = fma(ks1, s1, fma(t1, t1, eps_s));
    const double b2 = fma(ks2, s2, fma(t2, t2, eps_s));
    const double w0 = pmul<EW>(b0, b0), w1 = pmul<EW>(b1, b1), w2 = pmul<EW>(b2, b2);
    const double P0 = pmul<EW>(w1, w2), P1 = pmul<EW>(w0, w2), P2 = pmul<EW>(w0, w1);
    // candidates scaled by the linear weights (1, 6, 3)/10 x 10
    const double n0 = fma(11.0 / 6.0, v[2], fma(-7.0 / 6.0, v[1], xmul<EC>(1.0 / 3.0, v[0])));
    const double n1 = fma(2.0, v[3], fma(5.0, v[2], -v[1]));
    const double n2 = fma(-0.5, v[4], fma(2.5, v[3], v[2]));
    const double N = fma(n0, P0, fma(n1, P1, pmul<EF>(n2, P2)));
    const double D = fma(3.0, P2, fma(6.0, P1, P0));
    // reverse: value = N / D
    const double iD = rcp(D);
    const double Nb = pmul<EF>(Rbar, iD);
    const double Db = -pmul<EF>(Nb, pmul<EF>(N, iD));
    const double Pb0 = fma(Nb, n0, Db), Pb1 = fma(Nb, n1, xmul_small<EC, 3, 2, 1>(Db));
    const double Pb2 = fma(Nb, n2, xmul_small<EC, 3, 2, 0>(Db));
    const double nb0 = pmul<EF>(Nb, P0), nb1 = pmul<EF>(Nb, P1), nb2 = pmul<EF>(Nb, P2);
    // w_k = b_k^2 enters every P_m with m != k
    const double wb0 = fma(Pb1, w2, pmul<EW>(Pb2, w1)), wb1 = fma(Pb0, w2, pmul<EW>(Pb2, w0));
    const double wb2 = fma(Pb0, w1, pmul<EW>(Pb1, w0));
    // b_k = eps + t_k^2 + 13/3 s_k^2: tbar = 4 t b wbar, sbar = 4 (13/3) s b wbar
    const double q0 = pmul<EF>(xmul_pow2<EC, 2>(b0), wb0), q1 = pmul<EF>(xmul_pow2<EC, 2>(b1), wb1);
    const double q2 = pmul<EF>(xmul_pow2<EC, 2>(b2), wb2);
    const double tb0 = pmul<EF>(t0, q0), tb1 = pmul<EF>(t1, q1), tb2 = pmul<EF>(t2, q2);
    const double sb0 = pmul<EF>(ks0, q0), sb1 = pmul<EF>(ks1, q1), sb2 = pmul<EF>(ks2, q2);
    // transposes of t_k, s_k and n_k written on the cell values
    vjp_out<ACC>(vb[0], fma(1.0 / 3.0, nb0, tb0 + sb0));
    vjp_out<ACC>(vb[1], fma(-7.0 / 6.0, nb0, fma(-4.0, tb0, fma(-2.0, sb0, sb1 - nb1 - tb1))));
    vjp_out<ACC>(vb[2], fma(11.0 / 6.0, nb0, fma(5.0, nb1, fma(3.0, tb0 - tb2, fma(-2.0, sb1, nb2 + sb0 + sb2)))));
    vjp_out<ACC>(vb[3], fma(2.0, nb1, fma(2.5, nb2, fma(4.0, tb2, fma(-2.0, sb2, tb1 + sb1)))));
    vb[4] = fma(-0.5, nb2, sb2 - tb2);
}

// WENO7 in the difference basis of weno7 (A, B, C forms, b_k = eps + A^2 +
// 39 B^2 + 781/20 C^2); the reverse sweep takes the leave-two-out products
// for wbar and (A, B, C, n) -> (e, d) -> v for the transposes.
template <int EMU, bool ACC>
__device__ __forceinline__ void weno7_vjp(const double* v, double eps_s, double Rbar, double* vb)
{
    constexpr bool EC = (EMU & kEmuConst) != 0, EW = (EMU & kEmuWeights) != 0, EF = (EMU & kEmuFace) != 0;
    constexpr double kc = 781.0 / 20.0;
    double d[6], e[5];
#pragma unroll
    for (int i = 0; i < 6; ++i) d[i] = v[i + 1] - v[i];
#pragma unroll
    for (int i = 0; i < 5; ++i) e[i] = d[i + 1] - d[i];
    const double C0 = e[1] - e[0], C1 = e[2] - e[1], C2 = e[3] - e[2], C3 = e[4] - e[3];
    const double B0 = fma(2.0, e[1], -e[0]), B12 = e[2], B3 = fma(2.0, e[3], -e[4]);
    const double A0 = fma(6.0, d[2], fma(2.0, B0, e[1]));
    const double A1 = fma(2.0, d[3], fma(5.0, d[2], -d[1]));
    const double A2 = fma(5.0, d[3], fma(2.0, d[2], -d[4]));
    const double A3 = fma(6.0, d[3], fma(-2.0, B3, -e[3]));
    const double kB0 = xmul_small<EC, 39, 6, 0>(B0), kB12 = xmul_small<EC, 39, 6, 0>(B12);
    const double kB3 = xmul_small<EC, 39, 6, 0>(B3);
    const double kC0 = xmul<EC>(kc, C0), kC1 = xmul<EC>(kc, C1), kC2 = xmul<EC>(kc, C2), kC3 = xmul<EC>(kc, C3);
    const double b0 = fma(A0, A0, fma(kB0, B0, fma(kC0, C0, eps_s)));
    const double b1 = fma(A1, A1, fma(kB12, B12, fma(kC1, C1, eps_s)));
    const double b2 = fma(A2, A2, fma(kB12, B12, fma(kC2, C2, eps_s)));
    const double b3 = fma(A3, A3, fma(kB3, B3, fma(kC3, C3, eps_s)));
    const double w0 = pmul<EW>(b0, b0), w1 = pmul<EW>(b1, b1), w2 = pmul<EW>(b2, b2), w3 = pmul<EW>(b3, b3);
    const double w01 = pmul<EW>(w0, w1), w23 = pmul<EW>(w2, w3), w02 = pmul<EW>(w0, w2);
    const double w03 = pmul<EW>(w0, w3), w12 = pmul<EW>(w1, w2), w13 = pmul<EW>(w1, w3);
    const double P0 = pmul<EW>(w1, w23), P1 = pmul<EW>(w0, w23), P2 = pmul<EW>(w01, w3), P3 = pmul<EW>(w01, w2);
    // candidates scaled by the linear weights (1, 12, 18, 4)/35 x 35
    const double n0 = fma(25.0 / 12.0, v[3], fma(-23.0 / 12.0, v[2], fma(13.0 / 12.0, v[1], xmul_pow2<EC, -2>(-v[0]))));
    const double n1 = fma(3.0, v[4], fma(13.0, v[3], fma(-5.0, v[2], v[1])));
    const double n2 = fma(10.5, v[3] + v[4], xmul_small<EC, 3, 2, -1>(-(v[2] + v[5])));
    const double n3 = fma(13.0 / 3.0, v[4], fma(-5.0 / 3.0, v[5], fma(1.0 / 3.0, v[6], v[3])));
    const double N = fma(n0, P0, fma(n1, P1, fma(n2, P2, pmul<EF>(n3, P3))));
    const double D = fma(4.0, P3, fma(18.0, P2, fma(12.0, P1, P0)));
    // reverse: value = N / D
    const double iD = rcp(D);
    const double Nb = pmul<EF>(Rbar, iD);
    const double Db = -pmul<EF>(Nb, pmul<EF>(N, iD));
    const double Pb0 = fma(Nb, n0, Db), Pb1 = fma(Nb, n1, xmul_small<EC, 3, 2, 2>(Db));
    const double Pb2 = fma(Nb, n2, xmul_small<EC, 9, 4, 1>(Db)), Pb3 = fma(Nb, n3, xmul_pow2<EC, 2>(Db));
    const double nb0 = pmul<EF>(Nb, P0), nb1 = pmul<EF>(Nb, P1), nb2 = pmul<EF>(Nb, P2), nb3 = pmul<EF>(Nb, P3);
    const double wb0 = fma(Pb1, w23, fma(Pb2, w13, pmul<EW>(Pb3, w12)));
    const double wb1 = fma(Pb0, w23, fma(Pb2, w03, pmul<EW>(Pb3, w02)));
    const double wb2 = fma(Pb0, w13, fma(Pb1, w03, pmul<EW>(Pb3, w01)));
    const double wb3 = fma(Pb0, w12, fma(Pb1, w02, pmul<EW>(Pb2, w01)));
    // b_k = eps + A^2 + 39 B^2 + kc C^2: Abar = 4 A b wbar, Bbar = 4 (39 B) b wbar, ...
    const double q0 = pmul<EF>(xmul_pow2<EC, 2>(b0), wb0), q1 = pmul<EF>(xmul_pow2<EC, 2>(b1), wb1);
    const double q2 = pmul<EF>(xmul_pow2<EC, 2>(b2), wb2), q3 = pmul<EF>(xmul_pow2<EC, 2>(b3), wb3);
    const double Ab0 = pmul<EF>(A0, q0), Ab1 = pmul<EF>(A1, q1), Ab2 = pmul<EF>(A2, q2), Ab3 = pmul<EF>(A3, q3);
    const double Bb0 = pmul<EF>(kB0, q0), Bb1 = pmul<EF>(kB12, q1), Bb2 = pmul<EF>(kB12, q2);
    const double Bb3 = pmul<EF>(kB3, q3);
    const double Cb0 = pmul<EF>(kC0, q0), Cb1 = pmul<EF>(kC1, q1), Cb2 = pmul<EF>(kC2, q2);
    const double Cb3 = pmul<EF>(kC3, q3);
    // transposes: (B, C) -> e, (A, e) -> d, d -> v, n -> v
    const double eb0 = -Bb0 - Cb0;
    const double eb1 = fma(2.0, Bb0, Cb0 - Cb1);
    const double eb2 = Bb1 + Bb2 + (Cb1 - Cb2);
    const double eb3 = fma(2.0, Bb3, Cb2 - Cb3);
    const double eb4 = Cb3 - Bb3;
    const double db0 = fma(2.0, Ab0, -eb0);
    const double db1 = fma(-7.0, Ab0, (eb0 - eb1) - Ab1);
    const double db2 = fma(11.0, Ab0, fma(5.0, Ab1, fma(2.0, Ab2, eb1 - eb2)));
    const double db3 = fma(2.0, Ab1, fma(5.0, Ab2, fma(11.0, Ab3, eb2 - eb3)));
    const double db4 = fma(-7.0, Ab3, (eb3 - eb4) - Ab2);
    const double db5 = fma(2.0, Ab3, eb4);
    vjp_out<ACC>(vb[0], fma(-0.25, nb0, -db0));
    vjp_out<ACC>(vb[1], fma(13.0 / 12.0, nb0, nb1 + (db0 - db1)));
    vjp_out<ACC>(vb[2], fma(-23.0 / 12.0, nb0, fma(-5.0, nb1, fma(-1.5, nb2, db1 - db2))));
    vjp_out<ACC>(vb[3], fma(25.0 / 12.0, nb0, fma(13.0, nb1, fma(10.5, nb2, nb3 + (db2 - db3)))));
    vjp_out<ACC>(vb[4], fma(3.0, nb1, fma(10.5, nb2, fma(13.0 / 3.0, nb3, db3 - db4))));
    vjp_out<ACC>(vb[5], fma(-1.5, nb2, fma(-5.0 / 3.0, nb3, db4 - db5)));
    vb[6] = fma(1.0 / 3.0, nb3, db5);
}

// the left-biased reconstruction of the face from the 2R-1 cells v
template <int R, int EMU, bool ACC = true>
__device__ __forceinline__ void weno_left_vjp(const double* v, double eps_s, double Rbar, double* vb)
{
    static_assert(R == 3 || R == 4, "WENO5 or WENO7");
    if constexpr (R == 3) weno5_vjp<EMU, ACC>(v, eps_s, Rbar, vb);
    else weno7_vjp<EMU, ACC>(v, eps_s, Rbar, vb);
}

// the right-biased one: the left form on the mirrored cells; vb[2R-2] is
// overwritten, the others accumulate
template <int R, int EMU>
__device__ __forceinline__ void weno_right_vjp(const double* v, double eps_s, double Rbar, double* vb)
{
    constexpr int S = 2 * R - 1;
    double m[S], mb[S];
#pragma unroll
    for (int i = 0; i < S; ++i) m[i] = v[S - 1 - i];
    weno_left_vjp<R, EMU, false>(m, eps_s, Rbar, mb);
    vb[S - 1] = mb[0];
#pragma unroll
    for (int i = 1; i < S; ++i) vb[S - 1 - i] += mb[i];
}

// ------------------------------------------------------------ adjoint kernels
// The pencils of one physical axis ("job"), in the layout of its arrays
// (dimensions n, fastest first): the job sweeps layout axis d; phys is the
// physical axis (its speed, momentum and pressure term), wv the field of w
// holding the velocity along it.
struct AdjPencilJob {
    const double* u;                    // stage input state (5 fields)
    const double* w;                    // its p (field 0) and the velocity (field wv)
    const double* lam;                  // adjoint of the stage output (5 fields)
    double* gpo;                        // out: adjoint of g+ along the axis, 5 fields
    double* gmo;                        // out: adjoint of g-, same layout
    int n[3], d, phys, wv, bc;
    double hdx;
    int nseg;                           // 1, or 2: each pencil's faces split in two halves
    long long count;                    // threads: segments x 5 fields x pencils
};
struct AdjPencilArgs {
    AdjPencilJob job[3];
    int njob;
    const unsigned long long* rec;      // step record: speeds [3 stages][3 axes], dt
    long long fs;
    int stage;
    double cb, eps_s;
};

template <int R, int EMU, int MINB>
__global__ void __launch_bounds__(128, MINB) adj_pencil_kernel(const AdjPencilArgs a)
{
    constexpr int G = R, Wn = 2 * R;
    // thread -> (job, field, pencil): the jobs' ranges follow one another
    long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    int jb = 0;
    while (jb < a.njob && tid >= a.job[jb].count) tid -= a.job[jb++].count;
    if (jb >= a.njob) return;
    const AdjPencilJob& J = a.job[jb];
    const int d = J.d;
    const int nd = J.n[d];
    const int da = d == 0 ? 1 : 0, db = d == 2 ? 1 : 2;
    const long long npen = (long long)J.n[da] * J.n[db];
    const int seg = (int)(tid / (5 * npen));
    const long long rem = tid % (5 * npen);
    const int k = (int)(rem / npen);
    const long long pen = rem % npen;
    // faces j0 .. j1 of this segment (face j lies between cells j and j+1);
    // with two segments the cells jm-G+1 .. jm+G-1 receive contributions from
    // both, and (periodic) the G cells at each end from the other segment's
    // ghost folds: those are accumulated by exactly two commutative adds into
    // zeroed outputs, so the sums do not depend on the order
    const bool split = J.nseg == 2;
    const int jm = (nd - 1) / 2;
    const int j0 = (split && seg == 1) ? jm : -1;
    const int j1 = (split && seg == 0) ? jm - 1 : nd - 1;
    const int ph = J.phys;
    double* const gpo = J.gpo;
    double* const gmo = J.gmo;
    auto stride = [&](int e) { return e == 0 ? 1LL : (e == 1 ? (long long)J.n[0] : (long long)J.n[0] * J.n[1]); };
    const long long base = (pen % J.n[da]) * stride(da) + (pen / J.n[da]) * stride(db);
    const long long stp = stride(d);
    const long long fs = a.fs;
    const double alpha = __longlong_as_double((long long)a.rec[3 * (a.stage - 1) + ph]);
    const double dt = __longlong_as_double((long long)a.rec[9]);
    const double sc = a.cb * dt * J.hdx;
    const int bcd = J.bc;
    const double* const U = J.u;
    const double* const Wv = J.w + (long long)J.wv * fs;
    const double* const P = J.w;
    const double* const lam = J.lam;

    auto gval = [&](int m, double& gpv, double& gmv) {
        const long long q = base + (long long)bc_map(m, nd, bcd) * stp;
        const double uk = U[k * fs + q];
        const double vd = Wv[q];
        double f;
        if (k == 0) f = U[(1 + ph) * fs + q];
        else f = uk * vd + (k == 1 + ph ? P[q] : 0.0);
        gpv = fma(alpha, uk, f);
        gmv = fma(-alpha, uk, f);
    };
    double gpw[Wn], gmw[Wn], ap[Wn], am[Wn];
#pragma unroll
    for (int i = 0; i < Wn; ++i) {
        gval(j0 - G + 1 + i, gpw[i], gmw[i]);
        ap[i] = am[i] = 0.0;
    }
    // Ghost contributions fold onto the cells they copy.  Cells are emitted
    // in increasing order, ghosts below 0 first and above nd - 1 last, so:
    // outflow sums the low ghosts in (lo_p, lo_m) and adds them to cell 0, and
    // adds the high ghosts to cell nd - 1 after it is stored; periodic (one
    // segment) stores the low ghosts into cells nd - G .. nd - 1, which then
    // add their own values, and adds the high ghosts to cells 0 .. G - 1; with
    // two segments every such cell is accumulated by atomic adds.
    const bool periodic = bcd == 1;
    const bool periodic_split = split && periodic;
    double lo_p = 0.0, lo_m = 0.0;
    auto shared_cell = [&](int m) {
        return split && ((m >= jm - G + 1 && m <= jm + G - 1) || (periodic_split && (m < G || m >= nd - G)));
    };
    auto put = [&](long long q, double vp, double vm, int how) {   // how: 0 store, 1 add, 2 atomic add
        double* const p = gpo + k * fs + q;
        double* const n = gmo + k * fs + q;
        if (how == 2) {
            atomicAdd(p, vp);
            atomicAdd(n, vm);
        } else if (how == 1) {
            *p += vp;
            *n += vm;
        } else {
            *p = vp;
            *n = vm;
        }
    };
    auto emit = [&](int m, double vp, double vm) {
        if (m >= 0 && m < nd) {
            const long long q = base + (long long)m * stp;
            if (shared_cell(m)) put(q, vp, vm, 2);
            else if (!periodic && m == 0) put(q, vp + lo_p, vm + lo_m, 0);
            else put(q, vp, vm, periodic && m >= nd - G ? 1 : 0);
        } else if (m < 0) {
            if (!periodic) {
                lo_p += vp;
                lo_m += vm;
            } else {
                put(base + (long long)bc_map(m, nd, 1) * stp, vp, vm, periodic_split ? 2 : 0);
            }
        } else {
            put(base + (long long)bc_map(m, nd, bcd) * stp, vp, vm, periodic_split ? 2 : 1);
        }
    };
    double lamL = j0 >= 0 ? lam[k * fs + base + (long long)j0 * stp] : 0.0;
    for (int j = j0; j <= j1; ++j) {
        const double lamR = (j + 1 < nd) ? lam[k * fs + base + (long long)(j + 1) * stp] : 0.0;
        const double Fb = sc * (lamR - lamL);
        lamL = lamR;
        // the newest cell of each window receives its first contribution here
        weno_left_vjp<R, EMU>(gpw, a.eps_s, Fb, ap);           // cells j-G+1 .. j+G-1
        weno_right_vjp<R, EMU>(gmw + 1, a.eps_s, Fb, am + 1);  // cells j-G+2 .. j+G
        emit(j - G + 1, ap[0], am[0]);
#pragma unroll
        for (int i = 0; i < Wn - 1; ++i) {
            gpw[i] = gpw[i + 1];
            gmw[i] = gmw[i + 1];
            ap[i] = ap[i + 1];
            am[i] = am[i + 1];
        }
        if (j + 1 <= j1) gval(j + G + 1, gpw[Wn - 1], gmw[Wn - 1]);
    }
    // cells j1-G+2 .. j1+G: complete (last segment) or shared with the next one
#pragma unroll
    for (int i = 0; i < Wn - 1; ++i) emit(j1 - G + 2 + i, ap[i], am[i]);
}

// Fields between the x-fastest layout (x, then y, then z) and the x-slowest
// one used for the x pencils (y, then z, then x): plane by plane, 32 x 32
// tiles through shared memory, so both sides read and write coalesced rows.
struct FieldMove {
    const double* src[12];
    double* dst[12];
    int n;
};

// to_xslow: dst[(x nz + z) ny + y] = src[(z ny + y) nx + x]; otherwise the reverse
template <bool TO_XSLOW>
__global__ void __launch_bounds__(256) adj_transpose_kernel(FieldMove fm, int nx, int ny, int nz)
{
    __shared__ double t[32][33];
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32, z = blockIdx.z;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int f = 0; f < fm.n; ++f) {
        for (int j = ty; j < 32; j += 8) {
            if (TO_XSLOW) {
                const int x = x0 + tx, y = y0 + j;
                if (x < nx && y < ny) t[j][tx] = fm.src[f][((long long)z * ny + y) * nx + x];
            } else {
                const int y = y0 + tx, x = x0 + j;
                if (x < nx && y < ny) t[tx][j] = fm.src[f][((long long)x * nz + z) * ny + y];
            }
        }
        __syncthreads();
        for (int j = ty; j < 32; j += 8) {
            if (TO_XSLOW) {
                const int y = y0 + tx, x = x0 + j;
                if (x < nx && y < ny) fm.dst[f][((long long)x * nz + z) * ny + y] = t[tx][j];
            } else {
                const int x = x0 + tx, y = y0 + j;
                if (x < nx && y < ny) fm.dst[f][((long long)z * ny + y) * nx + x] = t[j][tx];
            }
        }
        __syncthreads();
    }
}

// V = sum over the active axes d of J_f_d(u)^T (gp_d + gm_d) + alpha_d (gp_d - gm_d)
// (gp_d, gm_d: 5 fields each at gp + 5 d fs); actmask bit d: axis d is active
__global__ void adj_flux_kernel(const double* u, const double* w, const double* gp, const double* gm, double* V,
                                const unsigned long long* rec, int stage, int actmask, long long fs, long long ncell,
                                double cs2)
{
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < ncell;
         q += (long long)gridDim.x * blockDim.x) {
        const double E = u[q], M[3] = {u[fs + q], u[2 * fs + q], u[3 * fs + q]}, Rr = u[4 * fs + q];
        const double p = w[q], v[3] = {w[fs + q], w[2 * fs + q], w[3 * fs + q]};
        const double h = E + p, ih = 1.0 / h;
        const double Q = fma(2.0, p, (1.0 - cs2) * E);
        const double iQ = 1.0 / Q;
        const double pE = (2.0 * cs2 * E - (1.0 - cs2) * p) * iQ;
        double pM[3];
        for (int j = 0; j < 3; ++j) pM[j] = -2.0 * cs2 * M[j] * iQ;
        double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (int d = 0; d < 3; ++d) {
            if (!(actmask & (1 << d))) continue;
            const double alpha = __longlong_as_double((long long)rec[3 * (stage - 1) + d]);
            const double* gpd = gp + 5LL * d * fs;
            const double* gmd = gm + 5LL * d * fs;
            double s[5], t[5];
#pragma unroll
            for (int f = 0; f < 5; ++f) {
                const double a = gpd[f * fs + q], b = gmd[f * fs + q];
                s[f] = a + b;
                t[f] = a - b;
            }
            const double vd = v[d];
            const double S = s[1] * M[0] + s[2] * M[1] + s[3] * M[2] + s[4] * Rr;
            const double vdE = -vd * (1.0 + pE) * ih;
            double ub[5];
            ub[0] = S * vdE + s[1 + d] * pE;
            for (int j = 0; j < 3; ++j) {
                const double vdM = ((j == d ? 1.0 : 0.0) - vd * pM[j]) * ih;
                ub[1 + j] = (j == d ? s[0] : 0.0) + s[1 + j] * vd + S * vdM + s[1 + d] * pM[j];
            }
            ub[4] = s[4] * vd;
#pragma unroll
            for (int f = 0; f < 5; ++f) acc[f] += fma(alpha, t[f], ub[f]);
        }
#pragma unroll
        for (int f = 0; f < 5; ++f) V[f * fs + q] = acc[f];
    }
}

// lam_s = cb lam + V (+ acc); acc = (reset ? 0 : acc) + ca lam
__global__ void adj_combine_kernel(const double* lam, const double* V, double* out, double* acc, double ca, double cb,
                                   int add_acc, int reset_acc, long long fs, long long ncell)
{
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < ncell;
         q += (long long)gridDim.x * blockDim.x)
        for (int f = 0; f < 5; ++f) {
            const long long i = f * fs + q;
            const double l = lam[i];
            double o = fma(cb, l, V[i]);
            if (add_acc) o += acc[i];
            out[i] = o;
            if (!add_acc) acc[i] = reset_acc ? ca * l : fma(ca, l, acc[i]);
        }
}

__global__ void record_kernel(const Ctl* c, unsigned long long* rec)
{
    for (int d = 0; d < 3; ++d) {
        rec[d] = c->a_cur[d];
        rec[3 + d] = c->a_s1[d];
        rec[6 + d] = c->a_s2[d];
    }
    rec[9] = (unsigned long long)__double_as_longlong(c->dt);
}

// ------------------------------------------------------------ eps_2
__global__ void eps2_partial_kernel(const double* u, long long fs, long long ncell, double cs2, double* part)
{
    double num = 0.0, den = 0.0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < ncell;
         q += (long long)gridDim.x * blockDim.x) {
        double p, vx, vy, vz, e;
        if (!con2prim(cs2, u[q], u[fs + q], u[2 * fs + q], u[3 * fs + q], p, vx, vy, vz, e)) {
            num = den = __longlong_as_double(0x7ff8000000000000LL);
            continue;
        }
        const double txx = fma(u[fs + q], vx, p), tyy = fma(u[2 * fs + q], vy, p);
        num += txx - tyy;
        den += txx + tyy;
    }
    __shared__ double sn[256], sd[256];
    sn[threadIdx.x] = num;
    sd[threadIdx.x] = den;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sn[threadIdx.x] += sn[threadIdx.x + o];
            sd[threadIdx.x] += sd[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = sn[0];
        part[2 * blockIdx.x + 1] = sd[0];
    }
}

__global__ void eps2_final_kernel(double* part, int nblocks)
{
    double n = 0.0, d = 0.0;
    for (int b = 0; b < nblocks; ++b) {
        n += part[2 * b];
        d += part[2 * b + 1];
    }
    part[0] = n;
    part[1] = d;
    part[2] = n / d;
}

// d eps_2 / d u at every cell (eps_2 = num/den): (dnum - eps2 dden) / den
__global__ void eps2_grad_kernel(const double* u, long long fs, long long ncell, double cs2, const double* sums,
                                 double* g, long long gs)
{
    const double den = sums[1], eps = sums[2];
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < ncell;
         q += (long long)gridDim.x * blockDim.x) {
        double p, vx, vy, vz, e;
        const double E = u[q], Mx = u[fs + q], My = u[2 * fs + q], Mz = u[3 * fs + q];
        con2prim(cs2, E, Mx, My, Mz, p, vx, vy, vz, e);
        const double h = E + p, ih = 1.0 / h;
        const double Q = fma(2.0, p, (1.0 - cs2) * E), iQ = 1.0 / Q;
        const double pE = (2.0 * cs2 * E - (1.0 - cs2) * p) * iQ;
        const double M[3] = {Mx, My, Mz};
        double pM[3];
        for (int j = 0; j < 3; ++j) pM[j] = -2.0 * cs2 * M[j] * iQ;
        // a = Mx vx, b = My vy, derivatives wrt (E, Mx, My, Mz)
        const double vxE = -vx * (1.0 + pE) * ih, vyE = -vy * (1.0 + pE) * ih;
        double ga[4], gb[4], gpp[4];
        ga[0] = Mx * vxE;
        gb[0] = My * vyE;
        gpp[0] = pE;
        for (int j = 0; j < 3; ++j) {
            const double vxM = ((j == 0 ? 1.0 : 0.0) - vx * pM[j]) * ih;
            const double vyM = ((j == 1 ? 1.0 : 0.0) - vy * pM[j]) * ih;
            ga[1 + j] = (j == 0 ? vx : 0.0) + Mx * vxM;
            gb[1 + j] = (j == 1 ? vy : 0.0) + My * vyM;
            gpp[1 + j] = pM[j];
        }
        for (int c = 0; c < 4; ++c) {
            const double dn = ga[c] - gb[c];
            const double dd = ga[c] + gb[c] + 2.0 * gpp[c];
            g[c * gs + q] = (dn - eps * dd) / den;
        }
        g[4 * gs + q] = 0.0;
    }
}

// Pencil kernel variants, all with the same bits: integer-pipe products
// (constants; + weights; + the reverse sweep's) and CTAs per SM.
using AdjPencilFn = void (*)(const AdjPencilArgs);
constexpr int kAdjPencilVariants = 6;
template <int R>
static AdjPencilFn adj_pencil_fn(int v)
{
    switch (v) {
    case 0: return adj_pencil_kernel<R, kEmuConst, 0>;
    case 2: return adj_pencil_kernel<R, kEmuConst | kEmuWeights | kEmuFace, 0>;
    case 3: return adj_pencil_kernel<R, kEmuConst | kEmuFace, 0>;
    case 4: return adj_pencil_kernel<R, kEmuConst | kEmuWeights | kEmuFace, 4>;
    case 5: return adj_pencil_kernel<R, kEmuConst, 4>;
    default: return adj_pencil_kernel<R, kEmuConst | kEmuWeights, 0>;
    }
}
// HYDRO_ADJ_PENCIL=<variant> picks one (for timing them); otherwise variant 1,
// the fastest at 96^3 (937 ms against 986 ms for the reverse sweep with the
// constants alone on the integer pipe, 1005 ms with every product there)
static int adj_pencil_variant()
{
    const char* e = getenv("HYDRO_ADJ_PENCIL");
    if (e && *e) {
        const int v = atoi(e);
        if (v >= 0 && v < kAdjPencilVariants) return v;
    }
    return 1;
}

}  // namespace hydro

// ------------------------------------------------------------------ host side
using namespace hydro;

static hydro_status afail(hydro_t* h, cudaError_t e, const char* where)
{
    return hydro_handle_fail(h, e == cudaErrorMemoryAllocation ? HYDRO_ERR_OOM : HYDRO_ERR_CUDA,
                             std::string(where) + ": " + cudaGetErrorString(e));
}
#define ACK(h, call, where)                                   \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return afail((h), e_, where);  \
    } while (0)

static int cells_blocks(long long n) { long long b = (n + 255) / 256; return (int)(b > 152 * 16 ? 152 * 16 : (b < 1 ? 1 : b)); }

// RK stage `stage` of step `step` with the recorded speeds and dt: input
// (u_in, w_in), step-start state u_n, output (u_out, w_out)
static StageArgs frozen_stage_at(const HandleView& v, AdjointWork* w, const double* u_in, const double* w_in,
                                 const double* u_n, double* u_out, double* w_out, int stage, int step)
{
    StageArgs a{};
    const int in = stage - 1;
    a.u_in = u_in;
    a.w_in = w_in;
    a.u_n = u_n;
    a.u_out = u_out;
    a.w_out = w_out;
    a.fs = w->fs;
    a.nx = v.cfg.n[0];
    a.ny = v.cfg.n[1];
    a.nz = v.cfg.n[2];
    a.zc = v.zc;
    a.zlo = 0;
    a.zhi = v.cfg.n[2];
    for (int d = 0; d < 3; ++d) {
        a.bc[d] = v.cfg.bc[d];
        a.act[d] = v.cfg.n[d] > 1;
        a.hdx[d] = 0.5 / v.cfg.dx[d];
    }
    a.cs2 = v.cfg.cs2;
    a.eps_s = v.cfg.weno_eps * (v.R == 3 ? SchemeConst<3>::eps_scale : SchemeConst<4>::eps_scale);
    static const double ca[3] = {0.0, 0.75, 1.0 / 3.0}, cb[3] = {1.0, 0.25, 2.0 / 3.0};
    a.ca = ca[in];
    a.cb = cb[in];
    a.alpha_in = w->rec + 10 * (long long)step + 3 * in;
    a.dt = reinterpret_cast<const double*>(w->rec + 10 * (long long)step + 9);
    a.alpha_out = w->ctl->a_next;
    a.status = &v.ctl->status;
    a.bad_cell = &v.ctl->bad_cell;
    a.fz = v.fz;
    a.fzs = v.fzs;
    a.fx = v.fx;
    a.fxs = v.fxs;
    a.fy = v.fy;
    a.fys = v.fys;
    return a;
}

// one frozen or recorded stage on the adjoint's buffers, with the handle's
// launch (face passes and combination, z pass and stage kernel, or fused)
static void forward_stage(const HandleView& v, const StageArgs& a, const dim3&)
{
    launch_stage_kernels(v.L, v.zc, a, v.sms, v.stream);
}

// segment storage: step i of the segment keeps its three stage inputs, each
// the 5 conserved fields followed by the 4 primitive fields (27 fields a step)
static double* seg_u(AdjointWork* w, int i, int k) { return w->SEG + w->fs * (27LL * i + 9LL * k); }
static double* seg_w(AdjointWork* w, int i, int k) { return w->SEG + w->fs * (27LL * i + 9LL * k + 5); }

static dim3 stage_grid(const HandleView& v)
{
    return dim3((v.cfg.n[0] + v.L.tx - 1) / v.L.tx, (v.cfg.n[1] + v.L.ty - 1) / v.L.ty, (v.cfg.n[2] + v.zc - 1) / v.zc);
}

extern "C" hydro_status hydro_forward_record(hydro_t* h, int32_t nsteps, int32_t ckpt_every)
{
    HandleView v;
    hydro_status s = hydro_handle_view(h, &v);
    if (s) return s;
    if (!v.loaded) return hydro_handle_fail(h, HYDRO_ERR_STATE, "no state loaded");
    if (v.cfg.split != 0)
        return hydro_handle_fail(h, HYDRO_ERR_INVALID_ARG, "the adjoint needs global Lax-Friedrichs splitting (split = 0)");
    if (v.cfg.nq > 1) return hydro_handle_fail(h, HYDRO_ERR_INVALID_ARG, "the adjoint supports one charge (nq <= 1)");
    if (v.cfg.charwise)
        return hydro_handle_fail(h, HYDRO_ERR_INVALID_ARG, "the adjoint differentiates component-wise WENO only");
    if (v.cfg.eos_mass != 0.0)
        return hydro_handle_fail(h, HYDRO_ERR_INVALID_ARG, "the adjoint differentiates the EOS p = cs2 e only");
    if (v.cfg.scheme == HYDRO_MUSTA_FORCE)
        return hydro_handle_fail(h, HYDRO_ERR_INVALID_ARG, "the adjoint differentiates the WENO schemes only");
    if (v.cfg.bc[2] == HYDRO_BC_HALO)
        return hydro_handle_fail(h, HYDRO_ERR_INVALID_ARG, "the adjoint runs on whole grids (no z halo)");
    if (nsteps < 1 || ckpt_every < 1) return hydro_handle_fail(h, HYDRO_ERR_INVALID_ARG, "need nsteps >= 1 and ckpt_every >= 1");
    AdjointWork* w = hydro_handle_adjoint(h, true);
    if (!w) return hydro_handle_fail(h, HYDRO_ERR_OOM, "host allocation failed");
    // (re)allocate the workspace for this length
    cudaStreamSynchronize(v.stream);
    cudaFree(w->buf);
    cudaFree(w->rec);
    cudaFree(w->ctl);
    w->buf = nullptr;
    w->rec = nullptr;
    w->ctl = nullptr;
    w->nsteps = nsteps;
    w->ckpt = ckpt_every;
    w->nckpt = (nsteps + ckpt_every - 1) / ckpt_every;
    w->fs = v.fs;
    const long long fs = v.fs;
    const long long nfields = 27 + 5 * 4 + 30 + 22 + 5LL * w->nckpt + 27LL * ckpt_every;
    ACK(h, cudaMalloc(&w->buf, sizeof(double) * (size_t)(fs * nfields)), "adjoint workspace");
    ACK(h, cudaMalloc(&w->rec, sizeof(unsigned long long) * 10 * (size_t)nsteps), "step record");
    ACK(h, cudaMalloc(&w->ctl, sizeof(Ctl)), "scratch control");
    double* p = w->buf;
    for (int i = 0; i < 3; ++i) {
        w->AU[i] = p;
        p += 5 * fs;
    }
    for (int i = 0; i < 3; ++i) {
        w->AW[i] = p;
        p += 4 * fs;
    }
    w->LAM = p; p += 5 * fs;
    w->OUT = p; p += 5 * fs;
    w->ACC = p; p += 5 * fs;
    w->V = p; p += 5 * fs;
    w->GP = p; p += 15 * fs;   // 5 fields per axis
    w->GM = p; p += 15 * fs;
    w->XT = p; p += 22 * fs;
    w->CK = p; p += 5 * fs * w->nckpt;
    w->SEG = p;
    // forward steps on the handle's own state, recording speeds and dt; the
    // stage-1/2 outputs go to the workspace
    double* U[3];
    double* Wp[3];
    set_t_end_kernel<<<1, 1, 0, v.stream>>>(v.ctl, -1.0);
    // U0/W0 are the handle's; stage outputs go to the workspace's AU1/AU2
    U[0] = v.U0;
    U[1] = w->AU[1];
    U[2] = w->AU[2];
    Wp[0] = v.W0;
    Wp[1] = w->AW[1];
    Wp[2] = w->AW[2];
    const dim3 grid = stage_grid(v);
    // the steps of the last segment keep their stage inputs in the segment
    // storage, as its recomputation would (the same operations on the same
    // operands, since the recorded speeds and steps are those used here), so
    // the reverse sweep starts without recomputing it
    const int last0 = (w->nckpt - 1) * ckpt_every;
    w->seg_kept = false;
    for (int n = 0; n < nsteps; ++n) {
        if (n % ckpt_every == 0)
            ACK(h, cudaMemcpyAsync(w->CK + 5 * fs * (n / ckpt_every), v.U0, sizeof(double) * 5 * fs,
                                   cudaMemcpyDeviceToDevice, v.stream), "checkpoint");
        const int i = n - last0;
        if (i == 0) {
            ACK(h, cudaMemcpyAsync(seg_u(w, 0, 0), v.U0, sizeof(double) * 5 * fs, cudaMemcpyDeviceToDevice, v.stream),
                "segment start");
            ACK(h, cudaMemcpyAsync(seg_w(w, 0, 0), v.W0, sizeof(double) * 4 * fs, cudaMemcpyDeviceToDevice, v.stream),
                "segment start");
        }
        step_begin_kernel<<<1, 1, 0, v.stream>>>(v.ctl, step_params(v.cfg));
        for (int st = 1; st <= 3; ++st) {
            StageArgs a{};
            const int in = st - 1;
            if (i >= 0) {
                const bool last = n == nsteps - 1;
                a.u_in = seg_u(w, i, in);
                a.w_in = seg_w(w, i, in);
                a.u_n = seg_u(w, i, 0);
                a.u_out = st < 3 ? seg_u(w, i, st) : (last ? U[0] : seg_u(w, i + 1, 0));
                a.w_out = st < 3 ? seg_w(w, i, st) : (last ? Wp[0] : seg_w(w, i + 1, 0));
            } else {
                a.u_in = U[in];
                a.w_in = Wp[in];
                a.u_n = U[0];
                a.u_out = st == 3 ? U[0] : U[st];
                a.w_out = st == 3 ? Wp[0] : Wp[st];
            }
            a.fs = fs;
            a.nx = v.cfg.n[0];
            a.ny = v.cfg.n[1];
            a.nz = v.cfg.n[2];
            a.zc = v.zc;
            a.zlo = 0;
            a.zhi = v.cfg.n[2];
            for (int d = 0; d < 3; ++d) {
                a.bc[d] = v.cfg.bc[d];
                a.act[d] = v.cfg.n[d] > 1;
                a.hdx[d] = 0.5 / v.cfg.dx[d];
            }
            a.cs2 = v.cfg.cs2;
            a.eps_s = v.cfg.weno_eps * (v.R == 3 ? SchemeConst<3>::eps_scale : SchemeConst<4>::eps_scale);
            static const double ca[3] = {0.0, 0.75, 1.0 / 3.0}, cb[3] = {1.0, 0.25, 2.0 / 3.0};
            a.ca = ca[in];
            a.cb = cb[in];
            a.alpha_in = st == 1 ? v.ctl->a_cur : (st == 2 ? v.ctl->a_s1 : v.ctl->a_s2);
            a.alpha_out = st == 1 ? v.ctl->a_s1 : (st == 2 ? v.ctl->a_s2 : v.ctl->a_next);
            a.dt = &v.ctl->dt;
            a.status = &v.ctl->status;
            a.bad_cell = &v.ctl->bad_cell;
            a.fz = v.fz;
            a.fzs = v.fzs;
            a.fx = v.fx;
            a.fxs = v.fxs;
            a.fy = v.fy;
            a.fys = v.fys;
            forward_stage(v, a, grid);
        }
        record_kernel<<<1, 1, 0, v.stream>>>(v.ctl, w->rec + 10 * (long long)n);
        step_end_kernel<<<1, 1, 0, v.stream>>>(v.ctl);
    }
    ACK(h, cudaGetLastError(), "recorded forward");
    w->seg_kept = true;
    return HYDRO_OK;
}

static hydro_status stage_adjoint(hydro_t* h, const HandleView& v, AdjointWork* w, const double* u, const double* ww,
                                  int stage, int step, const double* lam, double* out, int add_acc, int reset_acc)
{
    static const double ca[3] = {0.0, 0.75, 1.0 / 3.0}, cb[3] = {1.0, 0.25, 2.0 / 3.0};
    const long long fs = w->fs, nc = v.ncell;
    const int nx = v.cfg.n[0], ny = v.cfg.n[1], nz = v.cfg.n[2];
    const unsigned long long* rec = w->rec + 10 * (long long)step;
    AdjPencilArgs a{};
    a.rec = rec;
    a.fs = fs;
    a.stage = stage;
    a.cb = cb[stage - 1];
    a.eps_s = v.cfg.weno_eps * (v.R == 3 ? SchemeConst<3>::eps_scale : SchemeConst<4>::eps_scale);
    int actmask = 0;
    for (int d = 0; d < 3; ++d)
        if (v.cfg.n[d] > 1) actmask |= 1 << d;
    // one job per active axis, all in one launch: y and z pencils in the
    // state's own layout, x pencils in the x-slowest layout (dimensions ny,
    // nz, nx) swept along its slowest axis
    double* UT = w->XT;
    double* WT = UT + 5 * fs;
    double* LT = WT + 2 * fs;
    double* GPT = LT + 5 * fs;
    double* GMT = GPT + 5 * fs;
    const dim3 tg((nx + 31) / 32, (ny + 31) / 32, nz), tb(32, 8);
    a.njob = 0;
    long long threads = 0;
    for (int d = 0; d < 3; ++d) {
        if (!(actmask & (1 << d))) continue;
        AdjPencilJob& J = a.job[a.njob++];
        J.phys = d;
        J.bc = v.cfg.bc[d];
        J.hdx = 0.5 / v.cfg.dx[d];
        if (d == 0) {
            J.u = UT;
            J.w = WT;
            J.wv = 1;
            J.lam = LT;
            J.gpo = GPT;
            J.gmo = GMT;
            J.n[0] = ny;
            J.n[1] = nz;
            J.n[2] = nx;
            J.d = 2;
        } else {
            J.u = u;
            J.w = ww;
            J.wv = 1 + d;
            J.lam = lam;
            J.gpo = w->GP + 5LL * d * fs;
            J.gmo = w->GM + 5LL * d * fs;
            for (int e = 0; e < 3; ++e) J.n[e] = v.cfg.n[e];
            J.d = d;
        }
        // two segments per pencil where it is long enough for the shared cells
        // of the middle and of the periodic ends not to overlap
        J.nseg = v.cfg.n[d] >= 8 * v.R ? 2 : 1;
        J.count = 5LL * J.nseg * (nc / v.cfg.n[d]);
        threads += J.count;
    }
    // segmented jobs accumulate their shared cells with adds: zero those outputs
    for (int i = 0; i < a.njob; ++i)
        if (a.job[i].nseg == 2) {
            ACK(h, cudaMemsetAsync(a.job[i].gpo, 0, sizeof(double) * 5 * fs, v.stream), "clear adjoint outputs");
            ACK(h, cudaMemsetAsync(a.job[i].gmo, 0, sizeof(double) * 5 * fs, v.stream), "clear adjoint outputs");
        }
    if (actmask & 1) {
        FieldMove in{};
        for (int f = 0; f < 5; ++f) {
            in.src[f] = u + f * fs;
            in.dst[f] = UT + f * fs;
            in.src[7 + f] = lam + f * fs;
            in.dst[7 + f] = LT + f * fs;
        }
        in.src[5] = ww;            // p
        in.dst[5] = WT;
        in.src[6] = ww + fs;       // v_x
        in.dst[6] = WT + fs;
        in.n = 12;
        adj_transpose_kernel<true><<<tg, tb, 0, v.stream>>>(in, nx, ny, nz);
    }
    if (threads > 0) {
        const int blocks = (int)((threads + 127) / 128);
        const auto fn = v.R == 3 ? adj_pencil_fn<3>(adj_pencil_variant()) : adj_pencil_fn<4>(adj_pencil_variant());
        fn<<<blocks, 128, 0, v.stream>>>(a);
    }
    if (actmask & 1) {
        FieldMove out{};
        for (int f = 0; f < 5; ++f) {
            out.src[f] = GPT + f * fs;
            out.dst[f] = w->GP + f * fs;
            out.src[5 + f] = GMT + f * fs;
            out.dst[5 + f] = w->GM + f * fs;
        }
        out.n = 10;
        adj_transpose_kernel<false><<<tg, tb, 0, v.stream>>>(out, nx, ny, nz);
    }
    adj_flux_kernel<<<cells_blocks(nc), 256, 0, v.stream>>>(u, ww, w->GP, w->GM, w->V, rec, stage, actmask, fs, nc,
                                                             v.cfg.cs2);
    adj_combine_kernel<<<cells_blocks(nc), 256, 0, v.stream>>>(lam, w->V, out, w->ACC, ca[stage - 1], cb[stage - 1],
                                                               add_acc, reset_acc, fs, nc);
    ACK(h, cudaGetLastError(), "stage adjoint");
    return HYDRO_OK;
}

extern "C" hydro_status hydro_adjoint(hydro_t* h, const double* lambda_final, double* grad_u0, int64_t field_stride,
                                      int32_t mem)
{
    HandleView v;
    hydro_status s = hydro_handle_view(h, &v);
    if (s) return s;
    AdjointWork* w = hydro_handle_adjoint(h, false);
    if (!w || !w->buf) return hydro_handle_fail(h, HYDRO_ERR_STATE, "no recorded forward run (call hydro_forward_record)");
    if (!lambda_final || !grad_u0) return hydro_handle_fail(h, HYDRO_ERR_INVALID_ARG, "NULL pointer");
    if (field_stride < v.ncell) return hydro_handle_fail(h, HYDRO_ERR_INVALID_ARG, "field_stride smaller than the cell count");
    if (mem != HYDRO_MEM_HOST && mem != HYDRO_MEM_DEVICE) return hydro_handle_fail(h, HYDRO_ERR_INVALID_ARG, "mem must be 0 or 1");
    const long long fs = w->fs, nc = v.ncell;
    const cudaMemcpyKind kin = mem == HYDRO_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    const cudaMemcpyKind kout = mem == HYDRO_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    for (int f = 0; f < 5; ++f)
        ACK(h, cudaMemcpyAsync(w->LAM + f * fs, lambda_final + f * field_stride, sizeof(double) * nc, kin, v.stream),
            "load lambda");
    const dim3 grid = stage_grid(v);
    const int N = w->nsteps, C = w->ckpt;
    for (int seg = w->nckpt - 1; seg >= 0; --seg) {
        const int s0 = seg * C, s1 = (s0 + C < N) ? s0 + C : N;
        // the segment recomputed from its checkpoint with frozen stages; every
        // stage input is kept (the last step's third stage is not needed).
        // The last segment's are still there from the recorded forward until
        // another segment takes the storage.
        const bool kept = w->seg_kept && seg == w->nckpt - 1;
        if (!kept) {
            w->seg_kept = false;
            ACK(h, cudaMemcpyAsync(seg_u(w, 0, 0), w->CK + 5 * fs * seg, sizeof(double) * 5 * fs,
                                   cudaMemcpyDeviceToDevice, v.stream), "restore");
            prepare_kernel<<<cells_blocks(nc), 256, 0, v.stream>>>(seg_u(w, 0, 0), seg_w(w, 0, 0), fs, nc, v.cfg.cs2,
                                                                   w->ctl);
        }
        for (int n = s0; n < s1 && !kept; ++n) {
            const int i = n - s0;
            for (int st = 1; st <= 3; ++st) {
                if (st == 3 && n == s1 - 1) break;
                const StageArgs a = frozen_stage_at(v, w, seg_u(w, i, st - 1), seg_w(w, i, st - 1), seg_u(w, i, 0),
                                                    st < 3 ? seg_u(w, i, st) : seg_u(w, i + 1, 0),
                                                    st < 3 ? seg_w(w, i, st) : seg_w(w, i + 1, 0), st, n);
                forward_stage(v, a, grid);
            }
        }
        for (int n = s1 - 1; n >= s0; --n) {
            const int i = n - s0;
            // stage 3 (input u2): lam_u2 = 2/3 lam + J^T(2/3 dt lam); acc = 1/3 lam
            if ((s = stage_adjoint(h, v, w, seg_u(w, i, 2), seg_w(w, i, 2), 3, n, w->LAM, w->OUT, 0, 1))) return s;
            // stage 2 (input u1): lam_u1 = 1/4 lam_u2 + J^T(1/4 dt lam_u2); acc += 3/4 lam_u2
            if ((s = stage_adjoint(h, v, w, seg_u(w, i, 1), seg_w(w, i, 1), 2, n, w->OUT, w->LAM, 0, 0))) return s;
            // stage 1 (input u^n): lam_n = acc + lam_u1 + J^T(dt lam_u1)
            if ((s = stage_adjoint(h, v, w, seg_u(w, i, 0), seg_w(w, i, 0), 1, n, w->LAM, w->OUT, 1, 0))) return s;
            double* t = w->LAM;
            w->LAM = w->OUT;
            w->OUT = t;
        }
    }
    for (int f = 0; f < 5; ++f)
        ACK(h, cudaMemcpyAsync(grad_u0 + f * field_stride, w->LAM + f * fs, sizeof(double) * nc, kout, v.stream),
            "store gradient");
    ACK(h, cudaStreamSynchronize(v.stream), "synchronize");
    return HYDRO_OK;
}

extern "C" hydro_status hydro_recorded_steps(hydro_t* h, int32_t* nsteps, double* alpha, double* dt)
{
    HandleView v;
    hydro_status s = hydro_handle_view(h, &v);
    if (s) return s;
    AdjointWork* w = hydro_handle_adjoint(h, false);
    if (!w || !w->rec) return hydro_handle_fail(h, HYDRO_ERR_STATE, "no recorded forward run");
    if (nsteps) *nsteps = w->nsteps;
    if (alpha || dt) {
        std::vector<unsigned long long> r(10 * (size_t)w->nsteps);
        ACK(h, cudaMemcpyAsync(r.data(), w->rec, sizeof(unsigned long long) * r.size(), cudaMemcpyDeviceToHost, v.stream),
            "read record");
        ACK(h, cudaStreamSynchronize(v.stream), "synchronize");
        for (int n = 0; n < w->nsteps; ++n) {
            for (int i = 0; i < 9; ++i)
                if (alpha) memcpy(alpha + 9 * n + i, &r[10 * n + i], sizeof(double));
            if (dt) memcpy(dt + n, &r[10 * n + 9], sizeof(double));
        }
    }
    return HYDRO_OK;
}

extern "C" hydro_status hydro_eps2(hydro_t* h, const double* u, int64_t field_stride, int32_t mem, double* eps2,
                                   double* grad, int64_t grad_stride, int32_t grad_mem)
{
    HandleView v;
    hydro_status s = hydro_handle_view(h, &v);
    if (s) return s;
    if (!eps2) return hydro_handle_fail(h, HYDRO_ERR_INVALID_ARG, "eps2 is NULL");
    if (v.cfg.eos_mass != 0.0) return hydro_handle_fail(h, HYDRO_ERR_INVALID_ARG, "eps_2 is implemented for p = cs2 e only");
    const long long fs = v.fs, nc = v.ncell;
    if (u && field_stride < nc) return hydro_handle_fail(h, HYDRO_ERR_INVALID_ARG, "field_stride smaller than the cell count");
    if (grad && grad_stride < nc) return hydro_handle_fail(h, HYDRO_ERR_INVALID_ARG, "grad_stride smaller than the cell count");
    if (!u && !v.loaded) return hydro_handle_fail(h, HYDRO_ERR_STATE, "no state loaded");
    // scratch: one state, the gradient and the block partial sums (stream-ordered)
    double* scratch = nullptr;
    const int nb = 152 * 8;
    ACK(h, cudaMallocAsync(&scratch, sizeof(double) * (size_t)(10 * fs + 2 * nb + 8), v.stream), "eps2 scratch");
    const double* src = v.U0;
    if (u) {
        const cudaMemcpyKind k = mem == HYDRO_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
        for (int f = 0; f < 5; ++f)
            ACK(h, cudaMemcpyAsync(scratch + f * fs, u + f * field_stride, sizeof(double) * nc, k, v.stream), "copy");
        src = scratch;
    }
    double* part = scratch + 10 * fs;
    eps2_partial_kernel<<<nb, 256, 0, v.stream>>>(src, fs, nc, v.cfg.cs2, part);
    eps2_final_kernel<<<1, 1, 0, v.stream>>>(part, nb);
    double sums[3];
    ACK(h, cudaMemcpyAsync(sums, part, sizeof sums, cudaMemcpyDeviceToHost, v.stream), "read eps2");
    if (grad) {
        double* g = scratch + 5 * fs;
        eps2_grad_kernel<<<cells_blocks(nc), 256, 0, v.stream>>>(src, fs, nc, v.cfg.cs2, part, g, fs);
        const cudaMemcpyKind k = grad_mem == HYDRO_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
        for (int f = 0; f < 5; ++f)
            ACK(h, cudaMemcpyAsync(grad + f * grad_stride, g + f * fs, sizeof(double) * nc, k, v.stream), "copy grad");
    }
    ACK(h, cudaFreeAsync(scratch, v.stream), "free");
    ACK(h, cudaStreamSynchronize(v.stream), "synchronize");
    *eps2 = sums[2];
    if (!(sums[2] == sums[2])) return hydro_handle_fail(h, HYDRO_ERR_UNPHYSICAL, "eps2 of an unphysical state");
    return HYDRO_OK;
}
