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
// J_L^T mu is a sum over axes.  One thread per (axis, field, pencil segment)
// sweeps the segment's faces (adj_sweep, adj_weno.cuh): face adjoint
// F~bar_{j+1/2} = hdx (mu_{j+1} - mu_j), reverse-mode WENO of both biased
// reconstructions in their difference basis, with the differences and their
// adjoints carried from face to face, into the split-flux adjoints gbar+-;
// ghost-cell contributions fold back onto their source cells by the boundary
// rule, and the few cells two segments share are summed by two atomic adds
// into zeroed outputs; then one cell kernel applies, summed over the axes,
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

#include "adj_weno.cuh"
#include "hydro_common.cuh"

namespace hydro {

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
    constexpr int G = R;
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
    auto lam_at = [&](int m) { return (m >= 0 && m < nd) ? lam[k * fs + base + (long long)m * stp] : 0.0; };
    adj_sweep<R, EMU>(j0, j1, a.eps_s, sc, gval, lam_at, emit);
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
// the fastest at 96^3 (reverse sweep 830 ms, against 865 ms with the
// constants alone on the integer pipe, 927 ms with the constants and the
// reverse sweep's products, 1087 ms with every product there: 178 registers,
// two CTAs per SM instead of three)
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
    // (re)allocate the workspace for this length; a workspace of the same
    // length is reused (the forward overwrites every part of it that the
    // reverse sweep reads: checkpoints, the last segment, the step record)
    const long long fs = v.fs;
    const int nckpt = (nsteps + ckpt_every - 1) / ckpt_every;
    const long long nfields = 27 + 5 * 4 + 30 + 22 + 5LL * nckpt + 27LL * ckpt_every;
    if (!(w->buf && w->rec && w->ctl && w->nsteps == nsteps && w->ckpt == ckpt_every && w->fs == fs)) {
        cudaStreamSynchronize(v.stream);
        cudaFree(w->buf);
        cudaFree(w->rec);
        cudaFree(w->ctl);
        w->buf = nullptr;
        w->rec = nullptr;
        w->ctl = nullptr;
        w->nsteps = 0;
        ACK(h, cudaMalloc(&w->buf, sizeof(double) * (size_t)(fs * nfields)), "adjoint workspace");
        ACK(h, cudaMalloc(&w->rec, sizeof(unsigned long long) * 10 * (size_t)nsteps), "step record");
        ACK(h, cudaMalloc(&w->ctl, sizeof(Ctl)), "scratch control");
    }
    w->nsteps = nsteps;
    w->ckpt = ckpt_every;
    w->nckpt = nckpt;
    w->fs = fs;
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
