// stage_kernel.cuh -- one fused RK3 stage of the FD-WENO scheme
// (arXiv:1604.03360, Eq. 2 + Sec. 1.2 + the RK3 of Sec. 1) for sm_103a.
//
// One launch computes, for every interior cell,
//   L(u_s) = sum_d (F_d(j-1/2) - F_d(j+1/2)) / dx_d        (Eq. 2)
//   u_out  = ca * u_n + cb * (u_s + dt L(u_s))              (SSP-RK3 stage)
// then recovers the primitives of u_out (stored for the next stage) and
// reduces the largest characteristic speed per axis of u_out (the Lax-
// Friedrichs alpha of the next stage) with warp shuffles + one atomicMax per
// warp on the IEEE bit pattern (exact, order independent).
//
// Work decomposition: a CTA owns a TX x TY column tile and a chunk of z
// planes and sweeps along z.  Per plane:
//   1. each thread appends the split z-fluxes g = f_z +- alpha_z u of its own
//      column at plane p+G to a private ring (shared memory, 2G-1 planes) and
//      reconstructs the z-face p+1/2 from it (no barrier needed) -- or, in the
//      z-pass variants (ZEXT), nothing: zflux_kernel has written the z faces;
//   2. the CTA stages split x-fluxes of the tile rows plus G halo cells each
//      side, and split y-fluxes of the tile columns plus halo, in shared
//      memory (ghost cells come from the boundary rule by index mapping);
//   3. the CTA reconstructs all (TX+1) x TY x-faces and TX x (TY+1) y-faces:
//      one (face, field) item per thread at a time, or as pencil sweeps that
//      carry the stencil differences from face to face (kPencilSweep);
//   4. each thread combines the six face fluxes of its cell and finishes.
// Primitive variables (p, v) of the stage input come from the previous
// stage's epilogue, so no cell is recovered twice in a stage.
//
// Local Lax-Friedrichs variant (LLF): each face splits with its own speed,
// the largest |lambda| over the 2G cells of its two stencils, so cells are
// staged raw -- flux f, state u and that cell's speed s (kept from the
// previous stage's epilogue) -- and every face forms g+- = f +- alpha_face u
// itself.  The z ring then holds 2G planes and each z face is computed whole.
//
// Characteristic-wise variant (CHW, global LF): x/y cells are staged as in the
// component-wise scheme (g+ and g-), but every face is one work item that
// projects its 2G-cell window on the characteristic fields of the face state
// (char_weno.cuh), reconstructs them and maps the result back, all fields at
// once.  The z ring holds 2G planes of (u, p, v_z), from which the z faces
// form g+- themselves.
//
// TMA-staged variant (TMA, with ZEXT and the pencil sweep): the raw cells of
// each plane that step 2 stages -- u (5 fields) and p, v_x, v_y -- arrive in
// shared memory as one (TX + 8) x (TY + 2G) tile per field by tensor-map
// loads issued by one thread; the load of plane p+1 is issued as soon as
// plane p has been staged, so it overlaps the face work of plane p.  Step 2
// then reads in-grid cells from that tile and only cells outside the grid
// (boundary rule) from global memory.  The tile starts 4 cells left of the
// column tile (x * 8 bytes stays a multiple of 16 for WENO5 too).
#pragma once
#include "char_weno.cuh"
#include "hydro_math.cuh"
#include "tma_util.cuh"

namespace hydro {

struct StageArgs {
    const double* u_in;     // 5 fields: stage input u_s (stencil reads)
    const double* w_in;     // 4 fields: p, v_x, v_y, v_z of u_s
    const double* u_n;      // 5 fields: step-start state (ca != 0 only)
    double* u_out;          // 5 fields (may alias u_n: each thread reads then writes its own cell)
    double* w_out;          // 4 fields
    long long fs;           // field stride
    int nx, ny, nz;
    int zc;                 // z planes per CTA
    int bc[3];              // 0 outflow, 1 periodic
    int act[3];             // direction has more than one cell
    double hdx[3];          // 0.5 / dx_d (the 1/2 of the LF split folded in)
    double cs2;
    double eps_s;           // rescaled WENO epsilon
    double ca, cb;          // RK stage coefficients
    const unsigned long long* alpha_in;  // 3 speeds (IEEE bits) used for the split
    const double* dt;       // time step (device); <= 0: the stage does nothing
    unsigned long long* alpha_out;       // 3 speeds of u_out (atomicMax target)
    int* status;            // first error code
    long long* bad_cell;    // linear index of the first unphysical cell
    const double* s_in;     // local LF only: 3 fields, max |lambda| per axis of u_s
    double* s_out;          // local LF only: 3 fields, the same for u_out
    int limiter;            // MUSTA-FORCE only: MUSCL slope limiter (0 minmod, 1 MC, 2 van Leer, 3 superbee)
    int musta_k;            // MUSTA-FORCE only: number of MUSTA stages
    int zlo, zhi;           // planes computed: [zlo, zhi) of the nz stored (0, nz unless z halos are stored)
    double eos_m;           // EOS p = cs2 (e - eos_m n_1); 0: p = cs2 e
    double* fz;             // z-pass variants: z-face fluxes, field k face f (between planes zlo+f-1
    long long fzs;          // and zlo+f) at fz[k fzs + f nx ny + y nx + x], f = 0 .. zhi-zlo
    double* fx;             // three-pass variants: x-face fluxes, field k face f (between columns
    long long fxs;          // f-1 and f) of row (y, z) at fx[k fxs + ((z-zlo) ny + y)(nx+1) + f]
    double* fy;             // and y-face fluxes, face f between rows f-1 and f, at
    long long fys;          // fy[k fys + f nx (zhi-zlo) + (z-zlo) nx + x]
};

// boundary rule 0 outflow (copy edge cell), 1 periodic; 2 (z only) halo: the
// ghost planes are stored with the grid and filled from outside, so every
// index read is already inside the stored array
__device__ __forceinline__ int bc_map(int i, int n, int bc)
{
    if (i >= 0 && i < n) return i;
    if (bc == 2) return i;
    if (bc == 1) {
        i %= n;
        return i < 0 ? i + n : i;
    }
    return i < 0 ? 0 : n - 1;
}

// TMA-staged variants: halo width of the raw tile in x (even, >= G) and the
// raw fields per cell (u 5, then p, v_x, v_y)
constexpr int kTmaHalo = 4, kTmaRawFields = 8;

template <int R, int TX, int TY, bool LLF = false, int NF = 5, bool CHW = false, bool SWP = false,
          bool ZEXT = false, bool TMA = false>
struct StageSmem {
    static constexpr int G = R, S = 2 * R - 1, NT = TX * TY;
    // raw tile of the TMA variants, one (RW x RH) box per field
    static constexpr int RW = TX + 2 * kTmaHalo, RH = TY + 2 * R, RWH = RW * RH;
    static constexpr int RAW = TMA ? kTmaRawFields * RWH : 0;
    static constexpr int NV = LLF ? 2 * NF + 1 : 2 * NF;     // staged values per cell
    static constexpr int NRING = (LLF || CHW) ? 2 * R : 2 * R - 1;    // z planes kept per column
    // x rows of the staged split fluxes; the pencil sweep reads one row per
    // lane, so its pitch is odd (no shared-memory bank conflicts)
    static constexpr int GXW = TX + 2 * G + ((SWP && (TX + 2 * G) % 2 == 0) ? 1 : 0), GYH = TY + 2 * G;
    // z ring values per cell: characteristic-wise keeps (u, p, v_z) and forms
    // g+- when a face reads them (a smaller ring: two CTAs per SM at 16 x 8)
    static constexpr int NVR = CHW ? NF + 2 : NV;
    static constexpr int RING = ZEXT ? 0 : NRING * NVR * NT;   // z-pass variants keep no ring
    static constexpr int GX = NV * TY * GXW;
    static constexpr int GY = NV * GYH * TX;
    static constexpr int FX = NF * TY * (TX + 1);
    static constexpr int FY = NF * (TY + 1) * TX;
    static constexpr size_t bytes = sizeof(double) * (size_t)(RAW + RING + GX + GY + FX + FY);
    static_assert((RWH * sizeof(double)) % 128 == 0 || !TMA, "every field box of the raw tile stays 128-byte aligned");
};

// split fluxes g+- = f_d(u) +- alpha u (= 2 f^{+-}) of one cell along axis d
// (fields E, M_x, M_y, M_z, then the NF - 4 charges, each with flux R v_d)
// (explicitly rounded products and sums: no contraction into an FMA, so every
// kernel that forms these values gets the same bits)
template <int NF>
__device__ __forceinline__ void split_flux(int d, const double* u, const double w[4], double alpha, double* gp,
                                           double* gm)
{
    const double p = w[0], vd = w[1 + d];
    double f[NF];
    f[0] = u[1 + d];
#pragma unroll
    for (int k = 1; k < NF; ++k) f[k] = __dmul_rn(u[k], vd);
    f[1 + d] = __dadd_rn(f[1 + d], p);
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        gp[k] = fma(alpha, u[k], f[k]);
        gm[k] = fma(-alpha, u[k], f[k]);
    }
}

// physical flux f_d(u) of one cell along axis d
template <int NF>
__device__ __forceinline__ void raw_flux(int d, const double* u, const double w[4], double* f)
{
    const double vd = w[1 + d];
    f[0] = u[1 + d];
#pragma unroll
    for (int k = 1; k < NF; ++k) f[k] = u[k] * vd;
    f[1 + d] += w[0];
}

// physical flux f_d(u) of one cell along axis d with explicitly rounded
// operations (no FMA contraction), so that every kernel that forms the local
// Lax-Friedrichs stencils from raw cells -- the stage kernel's z ring and the
// local-LF z pass -- gets the same bits
template <int NF>
__device__ __forceinline__ void raw_flux_rn(int d, const double* u, const double w[4], double* f)
{
    const double vd = w[1 + d];
    f[0] = u[1 + d];
#pragma unroll
    for (int k = 1; k < NF; ++k) f[k] = __dmul_rn(u[k], vd);
    f[1 + d] = __dadd_rn(f[1 + d], w[0]);
}

// Local-LF face value (scaled by 2) from raw stencil data of one field over the
// 2G cells j-G+1 .. j+G of face j+1/2 (element stride st): alpha_face = max s,
// g+ = f + alpha u on the first 2G-1 cells, g- = f - alpha u on the last 2G-1.
template <int R, int EMU = 0>
__device__ __forceinline__ double llf_face(const double* f, const double* u, const double* s, int st, double eps_s)
{
    constexpr int W = 2 * R, S = 2 * R - 1;
    unsigned long long ab = (unsigned long long)__double_as_longlong(s[0]);
#pragma unroll
    for (int i = 1; i < W; ++i) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(s[i * st]);
        ab = b > ab ? b : ab;   // speeds are >= 0: integer order = value order
    }
    const double a = __longlong_as_double((long long)ab);
    double fv[W], uv[W], vp[S], vm[S];
#pragma unroll
    for (int i = 0; i < W; ++i) {
        fv[i] = f[i * st];
        uv[i] = u[i * st];
    }
#pragma unroll
    for (int i = 0; i < S; ++i) {
        vp[i] = fma(a, uv[i], fv[i]);
        vm[i] = fma(-a, uv[i + 1], fv[i + 1]);
    }
    double Np, Dp, Nm, Dm;
    weno_left<R, EMU>(vp, eps_s, Np, Dp);
    weno_right<R, EMU>(vm, eps_s, Nm, Dm);
    return face_sum(Np, Dp, vp[R - 1], Nm, Dm, vm[R - 1]);
}

// One work item: column tile (tile_x, tile_y) of TX x TY cells and z chunk chunk_z of the
// grid described by a.  All threads of the CTA call it with the same item.
// Face work of step 3 (component-wise, global LF): ILP = 1 or 2 takes one or
// two independent (face, field) items per thread and iteration; ILP =
// kPencilSweep has every lane sweep a run of consecutive faces of one pencil
// (axis, field, row or column), carrying the stencil differences from face to
// face (Diff5 / Diff7).
constexpr int kPencilSweep = 0;

template <int R> struct DiffOf;
template <> struct DiffOf<3> { using T = Diff5; };
template <> struct DiffOf<4> { using T = Diff7; };

template <int R, int EMU>
__device__ __forceinline__ void diffs_fresh(const double* v, double eps_s, typename DiffOf<R>::T& q)
{
    if constexpr (R == 3) weno5_diffs<EMU>(v, eps_s, q);
    else weno7_diffs<EMU>(v, eps_s, q);
}
template <int R, int EMU>
__device__ __forceinline__ void diffs_slide(const double* v, double eps_s, typename DiffOf<R>::T& q)
{
    if constexpr (R == 3) weno5_slide<EMU>(v, eps_s, q);
    else weno7_slide<EMU>(v, eps_s, q);
}
template <int R, int EMU>
__device__ __forceinline__ void diffs_slide_mirror(const double* m, double eps_s, typename DiffOf<R>::T& q)
{
    if constexpr (R == 3) weno5_slide_mirror<EMU>(m, eps_s, q);
    else weno7_slide_mirror<EMU>(m, eps_s, q);
}
template <int R, int EMU>
__device__ __forceinline__ void weno_core(const typename DiffOf<R>::T& q, double eps_s, double& M, double& D)
{
    if constexpr (R == 3) weno5_core<EMU>(q, M, D);
    else weno7_core<EMU>(q, M, D);
}

// EMU: which FP64 operations of the reconstructions run on the integer pipe
// instead (kEmu* mask, hydro_math.cuh); the result is bit-identical.  The
// products with constants go there by default when 8 warps share an SM (one
// 256-thread CTA, or two 128-thread WENO5 CTAs): the FP64 unit is the
// bottleneck and the issue slots are mostly idle.  With 4 warps per SM, and in
// the characteristic-wise kernels, the longer integer chains measured slower.
constexpr int default_emu(int R, int TX, int TY, bool LLF, int NF, bool CHW)
{
    return CHW ? 0 : ((TX * TY == 256 || (R == 3 && NF == 5 && !LLF)) ? kEmuConst : 0);
}

// ZEXT: the z-face fluxes come from zflux_kernel (global memory) instead of
// the per-column ring of this kernel.
template <int R, int TX, int TY, int ILP = 1, bool LLF = false, int NF = 5, bool CHW = false,
          int EMU = default_emu(R, TX, TY, LLF, NF, CHW), bool ZEXT = false, bool TMA = false>
__device__ __forceinline__ void stage_tile(const StageArgs& a, int tile_x, int tile_y, int chunk_z, double* smem,
                                           const TmaMaps* tm = nullptr, uint64_t* bar = nullptr)
{
    static_assert(!(LLF && CHW), "characteristic-wise WENO uses the global Lax-Friedrichs split");
    constexpr bool SWP = (ILP == kPencilSweep);
    static_assert(!(SWP && (LLF || CHW)), "the pencil sweep serves the component-wise global-LF scheme");
    static_assert((TX * TY) % 32 == 0, "whole warps");
    static_assert(!ZEXT || ((SWP || LLF) && NF == 5 && !CHW),
                  "the z pass serves the five-field pencil-sweep kernels and the five-field local-LF kernel");
    static_assert(!TMA || ZEXT, "the TMA-staged variants take their z faces from the z pass");
    using SM = StageSmem<R, TX, TY, LLF, NF, CHW, SWP, ZEXT, TMA>;
    constexpr int G = SM::G, S = SM::S, NT = SM::NT, NRING = SM::NRING, NVR = SM::NVR;
    constexpr int GXW = SM::GXW, GYH = SM::GYH;
    constexpr int RW = SM::RW, RWH = SM::RWH;
    double* raw = smem;
    double* ring = raw + SM::RAW;
    double* gx = ring + SM::RING;
    double* gy = gx + SM::GX;
    double* Fx = gy + SM::GY;
    double* Fy = Fx + SM::FX;

    const double dt = *a.dt;
    if (!(dt > 0.0)) return;
    double al[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) al[d] = __longlong_as_double((long long)a.alpha_in[d]);

    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    const int x0 = tile_x * TX, y0 = tile_y * TY;
    const int zb = a.zlo + chunk_z * a.zc, ze = min(zb + a.zc, a.zhi);
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int x = x0 + tx, y = y0 + ty;
    const bool own = (x < nx) && (y < ny);
    const int xs = bc_map(x, nx, a.bc[0]), ys = bc_map(y, ny, a.bc[1]);
    const long long fs = a.fs, plane = (long long)nx * ny;
    const bool zact = a.act[2] != 0;

    // TMA: one thread issues the raw-tile loads of a plane (u box and p, v_x,
    // v_y box) on the mbarrier; plane zb + i completes phase i
    constexpr uint32_t kRawBytes = (uint32_t)(sizeof(double) * kTmaRawFields * RWH);
    bool tma_dead = false;         // a wait ran out of time: stop waiting and issuing
    auto tma_issue = [&](int pz) {
        if constexpr (TMA) {
            fence_proxy_async();
            mbar_arrive_expect(bar, kRawBytes);
            tma_load_4d(raw, &tm->u, x0 - kTmaHalo, y0 - G, pz, 0, bar);
            tma_load_4d(raw + 5 * RWH, &tm->w, x0 - kTmaHalo, y0 - G, pz, 0, bar);
        }
    };
    if constexpr (TMA) {
        if (tid == 0 && zb < ze) tma_issue(zb);
    }

    auto load = [&](long long q, double* u, double w[4]) {
#pragma unroll
        for (int k = 0; k < NF; ++k) u[k] = __ldg(a.u_in + k * fs + q);
#pragma unroll
        for (int k = 0; k < 4; ++k) w[k] = __ldg(a.w_in + k * fs + q);
    };
    auto slot_of = [&](int m) { return (m + 4 * NRING) % NRING; };
    // ring slot layout: global LF g+ (5), g- (5); local LF f (5), u (5), s_z
    auto ingest = [&](int m) {
        const long long q = (long long)bc_map(m, nz, a.bc[2]) * plane + (long long)ys * nx + xs;
        double u[NF], w[4], gp[NF], gm[NF];
        load(q, u, w);
        double* r = ring + slot_of(m) * NVR * NT + tid;
        if constexpr (CHW) {
#pragma unroll
            for (int k = 0; k < NF; ++k) r[k * NT] = u[k];
            r[NF * NT] = w[0];
            r[(NF + 1) * NT] = w[3];
        } else if constexpr (LLF) {
            raw_flux_rn<NF>(2, u, w, gp);
#pragma unroll
            for (int k = 0; k < NF; ++k) {
                r[k * NT] = gp[k];
                r[(NF + k) * NT] = u[k];
            }
            r[2 * NF * NT] = __ldg(a.s_in + 2 * fs + q);
        } else {
            split_flux<NF>(2, u, w, al[2], gp, gm);
#pragma unroll
            for (int k = 0; k < NF; ++k) {
                r[k * NT] = gp[k];
                r[(NF + k) * NT] = gm[k];
            }
        }
    };
    // local LF: the whole z face m+1/2 of field k from planes m-G+1 .. m+G
    auto face_z_llf = [&](int m, int k) {
        double fv[2 * G], uv[2 * G], sv[2 * G];
#pragma unroll
        for (int i = 0; i < 2 * G; ++i) {
            const double* r = ring + slot_of(m - G + 1 + i) * NVR * NT + tid;
            fv[i] = r[k * NT];
            uv[i] = r[(NF + k) * NT];
            sv[i] = r[2 * NF * NT];
        }
        return llf_face<R, EMU>(fv, uv, sv, 1, a.eps_s);
    };
    // N/D of the left-biased (+) and right-biased (-) reconstructions of the
    // z-stencil centred on plane m, field k
    // (both stencils are centred on plane m: cp, cm are g+ and g- there)
    auto recon_z = [&](int m, int k, double& Np, double& Dp, double& cp, double& Nm, double& Dm, double& cm) {
        double vp[S], vm[S];
#pragma unroll
        for (int i = 0; i < S; ++i) {
            const double* r = ring + slot_of(m - G + 1 + i) * NVR * NT + tid;
            vp[i] = r[k * NT];
            vm[i] = r[(NF + k) * NT];
        }
        weno_left<R, EMU>(vp, a.eps_s, Np, Dp);
        weno_right<R, EMU>(vm, a.eps_s, Nm, Dm);
        cp = vp[G - 1];
        cm = vm[G - 1];
    };

    // characteristic-wise: the whole z face m+1/2 from planes m-G+1 .. m+G,
    // g+- = f_z +- alpha u formed from the ring's (u, p, v_z)
    auto face_z_chw = [&](int m, double* Fz) {
        double Fr[NF], ub[NF];
        auto rp = [&](int i) { return (const double*)(ring + slot_of(m - G + 1 + i) * NVR * NT + tid); };
        const double az = al[2];
        auto gval = [&](int i, int f, int s) {
            // volatile: reload per use rather than keep the window in registers
            const volatile double* r = rp(i);
            const double uf = r[rot_field(f, 2) * NT], vz = r[(NF + 1) * NT];
            const double fl = f == 0 ? r[rot_field(1, 2) * NT] : (f == 1 ? fma(uf, vz, r[NF * NT]) : uf * vz);
            return s == 0 ? fma(az, uf, fl) : fma(-az, uf, fl);
        };
#pragma unroll
        for (int f = 0; f < NF; ++f) ub[f] = 0.5 * (rp(G - 1)[rot_field(f, 2) * NT] + rp(G)[rot_field(f, 2) * NT]);
        const bool ok = char_face<R, NF, decltype(gval), EMU>(gval, ub, a.cs2, a.eps_s, Fr);
#pragma unroll
        for (int k = 0; k < NF; ++k) Fz[rot_field(k, 2)] = Fr[k];
        return ok;
    };
    bool face_ok = true;

    // columns outside the grid (ragged tiles) have no z-faces to compute: their
    // ring is private and nobody reads it
    const bool zwork = zact && own && !ZEXT;
    double hNp[NF], hDp[NF], hCp[NF], Fzm[NF], Fzp[NF];
#pragma unroll
    for (int k = 0; k < NF; ++k) { hNp[k] = 0.0; hDp[k] = 1.0; hCp[k] = 0.0; Fzm[k] = 0.0; Fzp[k] = 0.0; }
    if (zwork && LLF) {
        for (int m = zb - G; m <= zb + G - 1; ++m) ingest(m);
#pragma unroll
        for (int k = 0; k < NF; ++k) Fzm[k] = face_z_llf(zb - 1, k);
    } else if (zwork && CHW) {
        for (int m = zb - G; m <= zb + G - 1; ++m) ingest(m);
        face_ok &= face_z_chw(zb - 1, Fzm);
    } else if (zwork) {
        for (int m = zb - G; m <= zb + G - 2; ++m) ingest(m);
#pragma unroll
        for (int k = 0; k < NF; ++k) {
            double Nm, Dm, cm;
            recon_z(zb - 1, k, hNp[k], hDp[k], hCp[k], Nm, Dm, cm);
        }
        ingest(zb + G - 1);
#pragma unroll
        for (int k = 0; k < NF; ++k) {
            double Np, Dp, cp, Nm, Dm, cm;
            recon_z(zb, k, Np, Dp, cp, Nm, Dm, cm);
            Fzm[k] = face_sum(hNp[k], hDp[k], hCp[k], Nm, Dm, cm);
            hNp[k] = Np;
            hDp[k] = Dp;
            hCp[k] = cp;
        }
    }

    unsigned long long amax[3] = {0ull, 0ull, 0ull};
    // only the rows / columns of the tile inside the grid (plus halo) do work
    const int ncol = min(TX, nx - x0), nrow = min(TY, ny - y0);
    const int wx = ncol + 2 * G, hy = nrow + 2 * G;      // staged extents
    const int nfx = a.act[0] ? NF * nrow * (ncol + 1) : 0;
    const int nfy = a.act[1] ? NF * (nrow + 1) * ncol : 0;
    const int ngx = a.act[0] ? nrow * wx : 0;
    const int ngy = a.act[1] ? hy * ncol : 0;

    // Pencil-sweep schedule (SWP): pencils x (field, row) then y (field,
    // column), 32 per group, one per lane.  A group takes as many steps as its
    // longest pencil has faces; the (group, face) steps are dealt out to the
    // warps in contiguous runs, so every lane of a warp starts a new window at
    // the same step and the sweep never diverges.
    const int lane = tid & 31, warp = tid >> 5;
    constexpr int NW = NT / 32;
    const int npx = a.act[0] ? NF * nrow : 0, npy = a.act[1] ? NF * ncol : 0, npen = npx + npy;
    auto pen_faces = [&](int P) { return P < npx ? ncol + 1 : nrow + 1; };
    auto group_len = [&](int g) { return max(pen_faces(32 * g), pen_faces(min(32 * g + 31, npen - 1))); };
    int sw_g0 = 0, sw_f0 = 0, sw_u0 = 0, sw_u1 = 0;
    if constexpr (SWP) {
        const int ngrp = (npen + 31) / 32;
        int units = 0;
        for (int g = 0; g < ngrp; ++g) units += group_len(g);
        sw_u0 = units * warp / NW;
        sw_u1 = units * (warp + 1) / NW;
        sw_f0 = sw_u0;
        while (sw_g0 < ngrp && sw_f0 >= group_len(sw_g0)) sw_f0 -= group_len(sw_g0++);
    }

    for (int p = zb; p < ze; ++p) {
        // 1. z: ingest plane p+G, face p+1/2 = R+(p) + R-(p+1)
        if (zwork && LLF) {
            ingest(p + G);
#pragma unroll
            for (int k = 0; k < NF; ++k) Fzp[k] = face_z_llf(p, k);
        } else if (zwork && CHW) {
            ingest(p + G);
            face_ok &= face_z_chw(p, Fzp);
        } else if (zwork) {
            ingest(p + G);
#pragma unroll
            for (int k = 0; k < NF; ++k) {
                double Np, Dp, cp, Nm, Dm, cm;
                recon_z(p + 1, k, Np, Dp, cp, Nm, Dm, cm);
                Fzp[k] = face_sum(hNp[k], hDp[k], hCp[k], Nm, Dm, cm);
                hNp[k] = Np;
                hDp[k] = Dp;
                hCp[k] = cp;
            }
        }
        // 2. split x- and y-fluxes of plane p (tile + halo) into shared memory
        const long long qz = (long long)bc_map(p, nz, a.bc[2]) * plane;
        if constexpr (TMA) {
            if (!tma_dead && !mbar_wait(bar, (uint32_t)(p - zb) & 1u)) {
                tma_dead = true;
                atomicCAS(a.status, 0, 5);   // HYDRO_ERR_TIMEOUT
            }
        }
        // raw cell (lx, ly) of the TMA tile (u, then p, v_x, v_y)
        auto load_raw = [&](int lx, int ly, double* u, double w[4]) {
            const double* rp = raw + ly * RW + lx;
#pragma unroll
            for (int k = 0; k < NF; ++k) u[k] = rp[k * RWH];
#pragma unroll
            for (int k = 0; k < 3; ++k) w[k] = rp[(NF + k) * RWH];
            w[3] = 0.0;   // v_z: not used by the x and y split fluxes
        };
        for (int it = tid; it < ngx + ngy; it += NT) {
            double u[NF], w[4], gp[NF], gm[NF];
            if (it < ngx) {
                const int row = it / wx, col = it % wx;
                const int xr = x0 - G + col;
                if (TMA && xr >= 0 && xr < nx) {
                    load_raw(col + kTmaHalo - G, row + G, u, w);
                } else {
                    const int xx = bc_map(xr, nx, a.bc[0]), yy = bc_map(y0 + row, ny, a.bc[1]);
                    load(qz + (long long)yy * nx + xx, u, w);
                }
                if constexpr (LLF) {
                    const long long q =
                        qz + (long long)bc_map(y0 + row, ny, a.bc[1]) * nx + bc_map(x0 - G + col, nx, a.bc[0]);
                    raw_flux_rn<NF>(0, u, w, gp);
#pragma unroll
                    for (int k = 0; k < NF; ++k) {
                        gx[(k * TY + row) * GXW + col] = gp[k];
                        gx[((NF + k) * TY + row) * GXW + col] = u[k];
                    }
                    gx[(2 * NF * TY + row) * GXW + col] = __ldg(a.s_in + q);
                } else {
                    split_flux<NF>(0, u, w, al[0], gp, gm);
#pragma unroll
                    for (int k = 0; k < NF; ++k) {
                        gx[(k * TY + row) * GXW + col] = gp[k];
                        gx[((NF + k) * TY + row) * GXW + col] = gm[k];
                    }
                }
            } else {
                const int j = it - ngx, row = j / ncol, col = j % ncol;
                const int yr = y0 - G + row;
                const int xx = bc_map(x0 + col, nx, a.bc[0]), yy = bc_map(yr, ny, a.bc[1]);
                const long long q = qz + (long long)yy * nx + xx;
                if (TMA && yr >= 0 && yr < ny) load_raw(col + kTmaHalo, row, u, w);
                else load(q, u, w);
                if constexpr (LLF) {
                    raw_flux_rn<NF>(1, u, w, gp);
#pragma unroll
                    for (int k = 0; k < NF; ++k) {
                        gy[(k * GYH + row) * TX + col] = gp[k];
                        gy[((NF + k) * GYH + row) * TX + col] = u[k];
                    }
                    gy[(2 * NF * GYH + row) * TX + col] = __ldg(a.s_in + fs + q);
                } else {
                    split_flux<NF>(1, u, w, al[1], gp, gm);
#pragma unroll
                    for (int k = 0; k < NF; ++k) {
                        gy[(k * GYH + row) * TX + col] = gp[k];
                        gy[((NF + k) * GYH + row) * TX + col] = gm[k];
                    }
                }
            }
        }
        __syncthreads();
        if constexpr (TMA) {
            // plane p is staged: the raw tile is free for plane p+1
            if (tid == 0 && !tma_dead && p + 1 < ze) tma_issue(p + 1);
        }
        // 3. x- and y-faces, one (face, field) item per thread at a time (ILP
        //    items per iteration); every item is a stencil of S values with a
        //    stride in the staged arrays, so x and y items run the same code
        auto locate = [&](int it, const double*& pp, const double*& pm, int& st, double*& out) {
            if (it < nfx) {
                const int k = it / (nrow * (ncol + 1)), rr = it % (nrow * (ncol + 1));
                const int row = rr / (ncol + 1), f = rr % (ncol + 1);   // face f - 1/2 of the tile
                pp = gx + (k * TY + row) * GXW + f;
                pm = gx + ((NF + k) * TY + row) * GXW + f + 1;
                st = 1;
                out = Fx + (k * TY + row) * (TX + 1) + f;
            } else {
                const int j = it - nfx;
                const int k = j / ((nrow + 1) * ncol), rr = j % ((nrow + 1) * ncol);
                const int f = rr / ncol, col = rr % ncol;             // face f - 1/2 along y
                pp = gy + (k * GYH + f) * TX + col;
                pm = gy + ((NF + k) * GYH + f + 1) * TX + col;
                st = TX;
                out = Fy + (k * (TY + 1) + f) * TX + col;
            }
        };
        const int nitems = nfx + nfy;
        if constexpr (CHW) {
            // characteristic-wise: one face (all fields) per item
            const int nx_f = a.act[0] ? nrow * (ncol + 1) : 0;
            const int ny_f = a.act[1] ? (nrow + 1) * ncol : 0;
            for (int it = tid; it < nx_f + ny_f; it += NT) {
                double Fr[NF];
                int fo[NF];
                bool ok;
                if (it < nx_f) {
                    const int row = it / (ncol + 1), f = it % (ncol + 1);
                    const double* base = gx + row * GXW + f;
#pragma unroll
                    for (int m = 0; m < NF; ++m) fo[m] = rot_field(m, 0) * (TY * GXW);
                    constexpr int gmo = NF * TY * GXW;
                    auto gval = [&](int i, int m, int s) { return base[i + fo[m] + s * gmo]; };
                    double ub[NF];
                    const double q = 0.25 * rcp(al[0]);
#pragma unroll
                    for (int m = 0; m < NF; ++m)
                        ub[m] = ((gval(G - 1, m, 0) - gval(G - 1, m, 1)) + (gval(G, m, 0) - gval(G, m, 1))) * q;
                    ok = char_face<R, NF, decltype(gval), EMU>(gval, ub, a.cs2, a.eps_s, Fr);
#pragma unroll
                    for (int m = 0; m < NF; ++m) Fx[(rot_field(m, 0) * TY + row) * (TX + 1) + f] = Fr[m];
                } else {
                    const int j = it - nx_f, f = j / ncol, col = j % ncol;
                    const double* base = gy + f * TX + col;
#pragma unroll
                    for (int m = 0; m < NF; ++m) fo[m] = rot_field(m, 1) * (GYH * TX);
                    constexpr int gmo = NF * GYH * TX;
                    auto gval = [&](int i, int m, int s) { return base[i * TX + fo[m] + s * gmo]; };
                    double ub[NF];
                    const double q = 0.25 * rcp(al[1]);
#pragma unroll
                    for (int m = 0; m < NF; ++m)
                        ub[m] = ((gval(G - 1, m, 0) - gval(G - 1, m, 1)) + (gval(G, m, 0) - gval(G, m, 1))) * q;
                    ok = char_face<R, NF, decltype(gval), EMU>(gval, ub, a.cs2, a.eps_s, Fr);
#pragma unroll
                    for (int m = 0; m < NF; ++m) Fy[(rot_field(m, 1) * (TY + 1) + f) * TX + col] = Fr[m];
                }
                face_ok &= ok;
            }
        } else if constexpr (LLF) {
            // local LF: window of 2G raw cells starting at the same place as g+
            for (int it = tid; it < nitems; it += NT) {
                const double* pp;
                const double* pm;
                int st;
                double* out;
                locate(it, pp, pm, st, out);
                // pp points at f_k of the window start; u_k and s sit 5 and 10-k
                // field blocks further in the same staged array
                const int fb = (it < nfx) ? TY * GXW : GYH * TX;      // one field block
                const int k = (it < nfx) ? it / (nrow * (ncol + 1)) : (it - nfx) / ((nrow + 1) * ncol);
                *out = llf_face<R, EMU>(pp, pp + NF * fb, pp + (2 * NF - k) * fb, st, a.eps_s);
            }
        } else if constexpr (SWP) {
            using DF = typename DiffOf<R>::T;
            int g = sw_g0, f = sw_f0;
            for (int u = sw_u0; u < sw_u1; ++g, f = 0) {
                const int fe = min(group_len(g), f + (sw_u1 - u));
                const int P = 32 * g + lane;
                // this lane's pencil: staged g+ row (pp) and g- row (pm, one
                // cell further), element stride, output row; idle lanes read
                // the first staged row and store nothing
                const double* pp = gx;
                const double* pm = gx;
                int st = 1, nf = 1, ost = 1;
                double* out = nullptr;
                if (P < npx) {
                    const int k = P / nrow, row = P % nrow;
                    pp = gx + (k * TY + row) * GXW;
                    pm = gx + ((NF + k) * TY + row) * GXW + 1;
                    out = Fx + (k * TY + row) * (TX + 1);
                    nf = ncol + 1;
                } else if (P < npen) {
                    const int k = (P - npx) / ncol, col = (P - npx) % ncol;
                    pp = gy + k * GYH * TX + col;
                    pm = gy + ((NF + k) * GYH + 1) * TX + col;
                    st = TX;
                    out = Fy + k * (TY + 1) * TX + col;
                    ost = TX;
                    nf = nrow + 1;
                }
                DF qp, qm;
#pragma unroll 2
                for (int ff = f; ff < fe; ++ff) {
                    // lanes whose pencil is shorter than the group repeat its
                    // last face (in bounds) and store nothing
                    const int fc = min(ff, nf - 1);
                    double vp[S], vm[S];
#pragma unroll
                    for (int i = 0; i < S; ++i) {
                        vp[i] = pp[(fc + i) * st];
                        vm[i] = pm[(fc + S - 1 - i) * st];    // mirrored window of the right-biased stencil
                    }
                    if (ff == f) {
                        diffs_fresh<R, EMU>(vp, a.eps_s, qp);
                        diffs_fresh<R, EMU>(vm, a.eps_s, qm);
                    } else {
                        diffs_slide<R, EMU>(vp, a.eps_s, qp);
                        diffs_slide_mirror<R, EMU>(vm, a.eps_s, qm);
                    }
                    double Np, Dp, Nm, Dm;
                    weno_core<R, EMU>(qp, a.eps_s, Np, Dp);
                    weno_core<R, EMU>(qm, a.eps_s, Nm, Dm);
                    const double F = face_sum(Np, Dp, vp[G - 1], Nm, Dm, vm[G - 1]);
                    if (out && ff < nf) out[ff * ost] = F;
                }
                u += fe - f;
            }
        } else
        for (int it0 = tid; it0 < nitems; it0 += ILP * NT) {
            double vp[ILP][S], vm[ILP][S], F[ILP];
            double* out[ILP];
#pragma unroll
            for (int u = 0; u < ILP; ++u) {
                const int it = it0 + u * NT;
                const double* pp;
                const double* pm;
                int st;
                out[u] = nullptr;
                if (it < nitems) {
                    locate(it, pp, pm, st, out[u]);
#pragma unroll
                    for (int i = 0; i < S; ++i) {
                        vp[u][i] = pp[i * st];
                        vm[u][i] = pm[i * st];
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < S; ++i) vp[u][i] = vm[u][i] = 0.0;   // result discarded
                }
            }
#pragma unroll
            for (int u = 0; u < ILP; ++u) {
                double Np, Dp, Nm, Dm;
                weno_left<R, EMU>(vp[u], a.eps_s, Np, Dp);
                weno_right<R, EMU>(vm[u], a.eps_s, Nm, Dm);
                F[u] = face_sum(Np, Dp, vp[u][G - 1], Nm, Dm, vm[u][G - 1]);
            }
#pragma unroll
            for (int u = 0; u < ILP; ++u)
                if (out[u]) *out[u] = F[u];
        }
        __syncthreads();
        // 4. combine, RK update, primitives and speeds of the new state
        if constexpr (ZEXT) {
            // z faces p-1/2 and p+1/2 of this column, from the z pass (read here,
            // not before the x/y phase, so they hold no registers there)
            if (zact && own) {
                const double* fz = a.fz + (long long)(p - a.zlo) * plane + (long long)y * nx + x;
#pragma unroll
                for (int k = 0; k < NF; ++k) {
                    Fzm[k] = fz[k * a.fzs];
                    Fzp[k] = fz[k * a.fzs + plane];
                }
            }
        }
        if (own) {
            const long long q = (long long)p * plane + (long long)y * nx + x;
            double un[NF];
#pragma unroll
            for (int k = 0; k < NF; ++k) {
                double L = 0.0;
                if (a.act[0]) L = a.hdx[0] * (Fx[(k * TY + ty) * (TX + 1) + tx] - Fx[(k * TY + ty) * (TX + 1) + tx + 1]);
                if (a.act[1]) L = fma(a.hdx[1], Fy[(k * (TY + 1) + ty) * TX + tx] - Fy[(k * (TY + 1) + ty + 1) * TX + tx], L);
                if (zact) L = fma(a.hdx[2], Fzm[k] - Fzp[k], L);
                const double s = fma(dt, L, __ldg(a.u_in + k * fs + q));
                un[k] = (a.ca == 0.0) ? s : fma(a.ca, a.u_n[k * fs + q], a.cb * s);
                a.u_out[k * fs + q] = un[k];
            }
            double pr, vx, vy, vz, e, ks = a.cs2;
            bool okp;
            if (a.eos_m == 0.0) {
                okp = con2prim(a.cs2, un[0], un[1], un[2], un[3], pr, vx, vy, vz, e);
            } else {
                okp = con2prim_gas(a.cs2, a.eos_m, un[0], un[1], un[2], un[3], un[4], pr, vx, vy, vz, e);
                if (okp) ks = sound2_gas(a.cs2, pr, e);
            }
            if (okp) {
                a.w_out[q] = pr;
                a.w_out[fs + q] = vx;
                a.w_out[2 * fs + q] = vy;
                a.w_out[3 * fs + q] = vz;
                double sp[3];
                max_speeds(ks, vx, vy, vz, sp);
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const unsigned long long b = (unsigned long long)__double_as_longlong(sp[d]);
                    amax[d] = b > amax[d] ? b : amax[d];
                    if constexpr (LLF) a.s_out[d * fs + q] = sp[d];
                }
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k) a.w_out[k * fs + q] = 0.0;
                if constexpr (LLF)
                    for (int d = 0; d < 3; ++d) a.s_out[d * fs + q] = 0.0;
                if (atomicCAS(a.status, 0, 4) == 0) *a.bad_cell = q;
            }
        }
#pragma unroll
        for (int k = 0; k < NF; ++k) Fzm[k] = Fzp[k];
    }
    if constexpr (TMA) {
        // a wait ran out of time: give the copy still in flight one more
        // bounded wait before the CTA's shared memory goes away
        if (tma_dead && ze > zb) mbar_wait(bar, (uint32_t)(ze - 1 - zb) & 1u);
    }
    if constexpr (CHW) {
        // a face state that is not physical (only possible next to an
        // unphysical cell): report it like one
        if (!face_ok && atomicCAS(a.status, 0, 4) == 0) *a.bad_cell = (long long)zb * plane + (long long)ys * nx + xs;
    }
    // speeds: warp max, one atomic per warp and axis
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        unsigned long long v = amax[d];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
            v = w > v ? w : v;
        }
        if ((tid & 31) == 0 && v) atomicMax(a.alpha_out + d, v);
    }
}

// MINB > 0: at least that many CTAs per SM (the compiler caps the registers)
template <int R, int TX, int TY, int ILP = 1, bool LLF = false, int NF = 5, bool CHW = false,
          int EMU = default_emu(R, TX, TY, LLF, NF, CHW), bool ZEXT = false, int MINB = 0>
__global__ void __launch_bounds__(TX * TY, (MINB > 0 ? MINB : (TX * TY <= 128 && R == 3 && NF == 5 && !CHW ? 2 : 1)))
    stage_kernel(const StageArgs a)
{
    extern __shared__ __align__(16) double smem[];
    stage_tile<R, TX, TY, ILP, LLF, NF, CHW, EMU, ZEXT>(a, blockIdx.x, blockIdx.y, blockIdx.z, smem);
}

// TMA-staged stage kernel (z faces from the z pass): the tensor maps of the
// stage input arrive as a kernel parameter; one mbarrier per CTA
template <int R, int TX, int TY, int EMU, int MINB>
__global__ void __launch_bounds__(TX * TY, MINB) stage_kernel_tma(const StageArgs a, const __grid_constant__ TmaMaps tm)
{
    extern __shared__ __align__(16) double smem[];
    __shared__ __align__(8) uint64_t bar;
    // the raw tile starts on a 128-byte boundary (the launch adds 128 bytes)
    double* base = smem + ((128u - (smem_addr(smem) & 127u)) & 127u) / sizeof(double);
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    stage_tile<R, TX, TY, kPencilSweep, false, 5, false, EMU, true, true>(a, blockIdx.x, blockIdx.y, blockIdx.z, base,
                                                                           &tm, &bar);
}

// z pass of a stage (ZEXT variants): the z-face fluxes of the five fields,
// each thread sweeping one (x, y, field) pencil over a chunk of faces
// with the stencil differences carried from face to face -- the same
// operations on the same operands as the ring of the fused kernel, so the same
// bits.  A CTA is 32 consecutive columns of the plane (flat index y nx + x,
// so rows of any width fill whole warps; one warp per field); grid
// (ceil(nx ny / 32), face chunks).  Face f lies between planes
// zlo+f-1 and zlo+f (f = 0 .. zhi-zlo); its left-biased stencil is centred
// on plane zlo+f-1, its right-biased one on plane zlo+f.
constexpr int kZFaces = 64, kZPassThreads = 160;
// A pass over nf faces cuts each pencil into c chunks of equal length
// ceil(nf / c) (every chunk non-empty); which faces a thread computes changes
// nothing in them (each face is the same operations on the same operands).
__host__ __device__ inline int chunk_len(int nf, int c) { return (nf + c - 1) / c; }
// c with chunks of about kZFaces faces (work-lists of uneven grids)
__host__ __device__ inline int face_chunks(int nf)
{
    const int c = (nf + kZFaces / 2) / kZFaces;
    const int len = chunk_len(nf, c < 1 ? 1 : c);
    return (nf + len - 1) / len;
}
// integer-pipe products of the z pass of the fused launches (measured fastest:
// WENO5 all three kinds, WENO7 without the face products; the WENO7 passes of
// the three-pass launch are fastest with all three)
constexpr int kZPassEmu5 = kEmuConst | kEmuWeights | kEmuFace, kZPassEmu7 = kEmuConst | kEmuWeights;

// one pass item along axis AX: pencil block cb (32 consecutive pencils), face
// chunk fch of clen faces (clen <= 0: chunks of equal length, gridDim.y of
// them), of the grid described by a; the CTA's five warps are the five
// fields.  Pencils and outputs:
//   AX = 2 (z pass): pencil = column y nx + x of the plane; faces f = 0 ..
//      zhi-zlo between stored planes zlo+f-1 and zlo+f; out fz[k fzs + f nx ny + pencil];
//   AX = 1 (y pass): pencil = (z-zlo) nx + x; faces f = 0 .. ny between rows
//      f-1 and f; out fy[k fys + f nx nzi + pencil] (nzi = zhi - zlo);
//   AX = 0 (x pass): pencil = (z-zlo) ny + y; faces f = 0 .. nx between
//      columns f-1 and f; out fx[k fxs + pencil (nx+1) + f].
// Consecutive lanes take consecutive pencils, so the z and y passes read and
// write coalesced rows; the x pass reads rows a row apart (each lane's next
// cells hit the same L1 sectors) and writes its faces contiguously per row.
template <int R, int EMU, int AX>
__device__ __forceinline__ void axis_flux_item(const StageArgs& a, long long cb, int fch, int clen)
{
    constexpr int G = R, S = 2 * R - 1;
    using DF = typename DiffOf<R>::T;
    if (!(*a.dt > 0.0)) return;
    const int k = threadIdx.x >> 5;
    const long long plane = (long long)a.nx * a.ny;
    const int nzi = a.zhi - a.zlo;
    const long long npen = AX == 2 ? plane : (AX == 1 ? (long long)a.nx * nzi : (long long)a.ny * nzi);
    const long long pen = cb * 32 + (threadIdx.x & 31);
    if (pen >= npen) return;                     // no barriers below
    const int nax = AX == 2 ? nzi : (AX == 1 ? a.ny : a.nx);     // cells along the pencil (interior)
    if (clen <= 0) clen = chunk_len(nax + 1, (int)gridDim.y);
    const int f0 = fch * clen, f1 = min(f0 + clen, nax + 1);
    if (f0 >= f1) return;
    const double al = __longlong_as_double((long long)a.alpha_in[AX]);
    // first cell of the pencil and the step between its cells
    long long base, step;
    int lo, ncell_ax, bcax;
    if constexpr (AX == 2) {
        base = pen;
        step = plane;
        lo = a.zlo;
        ncell_ax = a.nz;
        bcax = a.bc[2];
    } else if constexpr (AX == 1) {
        base = (long long)(a.zlo + pen / a.nx) * plane + pen % a.nx;
        step = a.nx;
        lo = 0;
        ncell_ax = a.ny;
        bcax = a.bc[1];
    } else {
        base = (long long)(a.zlo + pen / a.ny) * plane + (pen % a.ny) * a.nx;
        step = 1;
        lo = 0;
        ncell_ax = a.nx;
        bcax = a.bc[0];
    }
    // split fluxes g+- = f_AX +- alpha u of field k at (stored) position m
    // along the pencil (as split_flux)
    auto split_at = [&](int m, double& gp, double& gm) {
        const long long q = base + (long long)bc_map(m, ncell_ax, bcax) * step;
        const double uk = __ldg(a.u_in + k * a.fs + q);
        double f;
        if (k == 0) {
            f = __ldg(a.u_in + (1 + AX) * a.fs + q);
        } else {
            f = __dmul_rn(uk, __ldg(a.w_in + (1 + AX) * a.fs + q));
            if (k == 1 + AX) f = __dadd_rn(f, __ldg(a.w_in + q));
        }
        gp = fma(al, uk, f);
        gm = fma(-al, uk, f);
    };
    // windows of face p+1/2 (p = lo+f-1): wp = g+ at p-G+1 .. p+G-1,
    // wm = g- at p-G+2 .. p+G; gl = g+ of the newest cell p+G
    double wp[S], wm[S], gl = 0.0;
    const int p0 = lo + f0 - 1;
#pragma unroll
    for (int i = 0; i < 2 * G; ++i) {
        double gp, gm;
        split_at(p0 - G + 1 + i, gp, gm);
        if (i < S) wp[i] = gp;
        if (i > 0) wm[i - 1] = gm;
        gl = gp;
    }
    DF qp, qm;
    double* out;
    long long ostep;
    if constexpr (AX == 2) {
        out = a.fz + k * a.fzs + pen;
        ostep = plane;
    } else if constexpr (AX == 1) {
        out = a.fy + k * a.fys + pen;
        ostep = (long long)a.nx * nzi;
    } else {
        out = a.fx + k * a.fxs + pen * (a.nx + 1);
        ostep = 1;
    }
    for (int f = f0; f < f1; ++f) {
        double mm[S];
#pragma unroll
        for (int i = 0; i < S; ++i) mm[i] = wm[S - 1 - i];
        if (f == f0) {
            diffs_fresh<R, EMU>(wp, a.eps_s, qp);
            diffs_fresh<R, EMU>(mm, a.eps_s, qm);
        } else {
            diffs_slide<R, EMU>(wp, a.eps_s, qp);
            diffs_slide_mirror<R, EMU>(mm, a.eps_s, qm);
        }
        double Np, Dp, Nm, Dm;
        weno_core<R, EMU>(qp, a.eps_s, Np, Dp);
        weno_core<R, EMU>(qm, a.eps_s, Nm, Dm);
        out[(long long)f * ostep] = face_sum<EMU>(Np, Dp, wp[G - 1], Nm, Dm, wm[G - 1]);
        if (f + 1 < f1) {
            // next face: the window moves by one cell
#pragma unroll
            for (int i = 0; i < S - 1; ++i) {
                wp[i] = wp[i + 1];
                wm[i] = wm[i + 1];
            }
            wp[S - 1] = gl;
            double gm;
            split_at(lo + f + G, gl, gm);
            wm[S - 1] = gm;
        }
    }
}

template <int R, int EMU>
__device__ __forceinline__ void zflux_item(const StageArgs& a, long long cb, int zch, int clen)
{
    axis_flux_item<R, EMU, 2>(a, cb, zch, clen);
}

// (3 CTAs per SM for WENO7, 4 for WENO5: 15 and 20 warps)
template <int R, int EMU>
__global__ void __launch_bounds__(kZPassThreads, R == 4 ? 3 : 4) zflux_kernel(const StageArgs a)
{
    zflux_item<R, EMU>(a, blockIdx.x, blockIdx.y, 0);
}

// x and y passes of the three-pass variants (same CTA and occupancy as the z
// pass); MINB > 0 asks for that many CTAs per SM instead.  NF > 5 (several
// charges): one warp per field, NF warps per CTA.
template <int R, int EMU, int AX, int MINB = 0, int NF = 5>
__global__ void __launch_bounds__(32 * NF, MINB > 0 ? MINB : (R == 4 ? 3 : 4)) axis_flux_kernel(const StageArgs a)
{
    axis_flux_item<R, EMU, AX>(a, blockIdx.x, blockIdx.y, 0);
}

// pencil blocks of a pass along axis AX
inline long long pass_blocks(int AX, int nx, int ny, int nzi)
{
    const long long npen = AX == 2 ? (long long)nx * ny : (AX == 1 ? (long long)nx * nzi : (long long)ny * nzi);
    return (npen + 31) / 32;
}

// Three-pass variants: the rest of the stage once the x, y and z passes have
// written every face flux -- per cell the flux differences (Eq. 2), the RK
// combination, the primitives and the speeds of the new state, with the same
// operations in the same order as step 4 of stage_tile (component-wise, global
// or local Lax-Friedrichs, NF = 4 + number of charges fields), so the same
// bits.  Grid-stride over the interior cells, x fastest.
//
// combine_cells does cells i0, i0 + step, ... < i1 (flat index over the
// interior cells, x fastest) and the speed reduction of the calling warps;
// every thread of a warp must call it.  (Templates only so that every
// translation unit including this header can share one definition.)
template <int NF = 5, bool LLF = false>
__device__ __forceinline__ void combine_cells(const StageArgs& a, long long i0, long long i1, long long step)
{
    const double dt = *a.dt;
    if (!(dt > 0.0)) return;
    const int nx = a.nx, ny = a.ny, nzi = a.zhi - a.zlo;
    const long long plane = (long long)nx * ny, fs = a.fs;
    const long long yrow = (long long)nx * nzi;           // one y-face row of the fy buffer
    const bool ax0 = a.act[0] != 0, ax1 = a.act[1] != 0, ax2 = a.act[2] != 0;
    unsigned long long amax[3] = {0ull, 0ull, 0ull};
    for (long long i = i0; i < i1; i += step) {
        const int x = (int)(i % nx);
        const long long r = i / nx;
        const int y = (int)(r % ny), zi = (int)(r / ny);
        const long long q = (long long)(a.zlo + zi) * plane + (long long)y * nx + x;
        double un[NF];
#pragma unroll
        for (int k = 0; k < NF; ++k) {
            double L = 0.0;
            if (ax0) {
                const double* fx = a.fx + k * a.fxs + ((long long)zi * ny + y) * (nx + 1) + x;
                L = a.hdx[0] * (fx[0] - fx[1]);
            }
            if (ax1) {
                const double* fy = a.fy + k * a.fys + (long long)y * yrow + (long long)zi * nx + x;
                L = fma(a.hdx[1], fy[0] - fy[yrow], L);
            }
            if (ax2) {
                const double* fz = a.fz + k * a.fzs + (long long)zi * plane + (long long)y * nx + x;
                L = fma(a.hdx[2], fz[0] - fz[plane], L);
            }
            const double s = fma(dt, L, __ldg(a.u_in + k * fs + q));
            un[k] = (a.ca == 0.0) ? s : fma(a.ca, a.u_n[k * fs + q], a.cb * s);
            a.u_out[k * fs + q] = un[k];
        }
        double pr, vx, vy, vz, e, ks = a.cs2;
        bool okp;
        if (a.eos_m == 0.0) {
            okp = con2prim(a.cs2, un[0], un[1], un[2], un[3], pr, vx, vy, vz, e);
        } else {
            okp = con2prim_gas(a.cs2, a.eos_m, un[0], un[1], un[2], un[3], un[4], pr, vx, vy, vz, e);
            if (okp) ks = sound2_gas(a.cs2, pr, e);
        }
        if (okp) {
            a.w_out[q] = pr;
            a.w_out[fs + q] = vx;
            a.w_out[2 * fs + q] = vy;
            a.w_out[3 * fs + q] = vz;
            double sp[3];
            max_speeds(ks, vx, vy, vz, sp);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const unsigned long long b = (unsigned long long)__double_as_longlong(sp[d]);
                amax[d] = b > amax[d] ? b : amax[d];
                if constexpr (LLF) a.s_out[d * fs + q] = sp[d];
            }
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) a.w_out[k * fs + q] = 0.0;
            if constexpr (LLF)
                for (int d = 0; d < 3; ++d) a.s_out[d * fs + q] = 0.0;
            if (atomicCAS(a.status, 0, 4) == 0) *a.bad_cell = q;
        }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        unsigned long long v = amax[d];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
            v = w > v ? w : v;
        }
        if ((threadIdx.x & 31) == 0 && v) atomicMax(a.alpha_out + d, v);
    }
}

template <int NF = 5, bool LLF = false>
__global__ void __launch_bounds__(256) stage_combine_kernel(const StageArgs a)
{
    const long long ncell = (long long)a.nx * a.ny * (a.zhi - a.zlo);
    combine_cells<NF, LLF>(a, blockIdx.x * (long long)blockDim.x + threadIdx.x, ncell,
                           (long long)gridDim.x * blockDim.x);
}

// z pass of a local Lax-Friedrichs stage: the z-face fluxes of the five
// fields, each thread sweeping one (x, y, field) pencil over kZFaces faces.
// Face p+1/2 splits with the largest z speed over its 2G cells p-G+1 .. p+G,
// so its stencils cannot carry differences from the previous face; the
// thread keeps the raw window (flux f_z, state u, speed s_z of those 2G
// planes) in registers, moves it by one plane per face and evaluates the face
// exactly as the local-LF z ring of the stage kernel does (llf_face on the
// same values), so both give the same bits.  Same grid and CTA as zflux_kernel.
// The same along any axis AX (pencils, faces and outputs as in
// axis_flux_item): the raw window holds the flux f_AX, the state and the AX
// speed of 2G cells, formed as the stage kernel's local-LF staging does.
template <int R, int EMU, int AX>
__device__ __forceinline__ void axis_flux_llf_item(const StageArgs& a, long long cb, int fch, int clen)
{
    constexpr int G = R, W = 2 * R;
    if (!(*a.dt > 0.0)) return;
    const int k = threadIdx.x >> 5;
    const long long plane = (long long)a.nx * a.ny;
    const int nzi = a.zhi - a.zlo;
    const long long npen = AX == 2 ? plane : (AX == 1 ? (long long)a.nx * nzi : (long long)a.ny * nzi);
    const long long pen = cb * 32 + (threadIdx.x & 31);
    if (pen >= npen) return;                     // no barriers below
    const int nax = AX == 2 ? nzi : (AX == 1 ? a.ny : a.nx);
    if (clen <= 0) clen = chunk_len(nax + 1, (int)gridDim.y);
    const int f0 = fch * clen, f1 = min(f0 + clen, nax + 1);
    if (f0 >= f1) return;
    long long base, step;
    int lo, ncell_ax, bcax;
    if constexpr (AX == 2) {
        base = pen;
        step = plane;
        lo = a.zlo;
        ncell_ax = a.nz;
        bcax = a.bc[2];
    } else if constexpr (AX == 1) {
        base = (long long)(a.zlo + pen / a.nx) * plane + pen % a.nx;
        step = a.nx;
        lo = 0;
        ncell_ax = a.ny;
        bcax = a.bc[1];
    } else {
        base = (long long)(a.zlo + pen / a.ny) * plane + (pen % a.ny) * a.nx;
        step = 1;
        lo = 0;
        ncell_ax = a.nx;
        bcax = a.bc[0];
    }
    // raw flux, state and speed of field k at (stored) position m (as raw_flux_rn)
    auto raw_at = [&](int m, double& fv, double& uv, double& sv) {
        const long long q = base + (long long)bc_map(m, ncell_ax, bcax) * step;
        const double uk = __ldg(a.u_in + k * a.fs + q);
        double f;
        if (k == 0) {
            f = __ldg(a.u_in + (1 + AX) * a.fs + q);
        } else {
            f = __dmul_rn(uk, __ldg(a.w_in + (1 + AX) * a.fs + q));
            if (k == 1 + AX) f = __dadd_rn(f, __ldg(a.w_in + q));
        }
        fv = f;
        uv = uk;
        sv = __ldg(a.s_in + AX * a.fs + q);
    };
    // window of face p+1/2 (p = lo+f-1): cells p-G+1 .. p+G
    double fw[W], uw[W], sw[W];
    const int p0 = lo + f0 - 1;
#pragma unroll
    for (int i = 0; i < W; ++i) raw_at(p0 - G + 1 + i, fw[i], uw[i], sw[i]);
    double* out;
    long long ostep;
    if constexpr (AX == 2) {
        out = a.fz + k * a.fzs + pen;
        ostep = plane;
    } else if constexpr (AX == 1) {
        out = a.fy + k * a.fys + pen;
        ostep = (long long)a.nx * nzi;
    } else {
        out = a.fx + k * a.fxs + pen * (a.nx + 1);
        ostep = 1;
    }
    for (int f = f0; f < f1; ++f) {
        out[(long long)f * ostep] = llf_face<R, EMU>(fw, uw, sw, 1, a.eps_s);
        if (f + 1 < f1) {
#pragma unroll
            for (int i = 0; i < W - 1; ++i) {
                fw[i] = fw[i + 1];
                uw[i] = uw[i + 1];
                sw[i] = sw[i + 1];
            }
            raw_at(lo + f + G, fw[W - 1], uw[W - 1], sw[W - 1]);
        }
    }
}

template <int R, int EMU>
__device__ __forceinline__ void zflux_llf_item(const StageArgs& a, long long cb, int zch, int clen)
{
    axis_flux_llf_item<R, EMU, 2>(a, cb, zch, clen);
}

template <int R, int EMU>
__global__ void __launch_bounds__(kZPassThreads, R == 4 ? 3 : 4) zflux_llf_kernel(const StageArgs a)
{
    zflux_llf_item<R, EMU>(a, blockIdx.x, blockIdx.y, 0);
}

// x and y passes of the local-LF three-pass variants (AX = 2: a z pass of NF
// warps, for several charges)
template <int R, int EMU, int AX, int MINB = 0, int NF = 5>
__global__ void __launch_bounds__(32 * NF, MINB > 0 ? MINB : (R == 4 ? 3 : 4)) axis_flux_llf_kernel(const StageArgs a)
{
    axis_flux_llf_item<R, EMU, AX>(a, blockIdx.x, blockIdx.y, 0);
}

}  // namespace hydro
