// hydro_kernels.cu -- the stage kernel instantiations and the bookkeeping
// kernels of the step driver.
#include <cstdlib>
#include "hydro_common.cuh"
#include "musta_kernel.cuh"

namespace hydro {

__global__ void step_begin_kernel(Ctl* c, StepParams sp)
{
    double amax = 0.0;
    for (int d = 0; d < 3; ++d)
        if (sp.actmask & (1 << d)) amax = fmax(amax, __longlong_as_double((long long)c->a_cur[d]));
    double dt = sp.dt_fixed > 0.0 ? sp.dt_fixed : sp.cfl * sp.mindx / amax;
    if (c->t_end >= 0.0 && c->t + dt > c->t_end) dt = c->t_end - c->t;
    if (!(dt > 0.0)) dt = 0.0;
    c->dt = dt;
    for (int d = 0; d < 3; ++d) {
        c->a_s1[d] = 0ull;
        c->a_s2[d] = 0ull;
        c->a_next[d] = 0ull;
    }
}

__global__ void step_end_kernel(Ctl* c)
{
    if (c->dt > 0.0) {
        for (int d = 0; d < 3; ++d) c->a_cur[d] = c->a_next[d];
        c->t += c->dt;
        c->last_dt = c->dt;
        c->step += 1;
    }
}

__global__ void set_t_end_kernel(Ctl* c, double t_end) { c->t_end = t_end; }

__global__ void halo_replicate_kernel(FieldList fl, long long plane, long long src, long long dst, int G)
{
    const long long tot = (long long)fl.n * G * plane;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
        const long long c = i % plane, r = i / plane;
        const int g = (int)(r % G), f = (int)(r / G);
        fl.f[f][dst + g * plane + c] = fl.f[f][src + c];
    }
}

__global__ void reset_ctl_kernel(Ctl* c, double t)
{
    for (int d = 0; d < 3; ++d) {
        c->a_cur[d] = c->a_s1[d] = c->a_s2[d] = c->a_next[d] = 0ull;
    }
    c->dt = 0.0;
    c->t = t;
    c->t_end = -1.0;
    c->last_dt = 0.0;
    c->step = 0;
    c->bad_cell = -1;
    c->status = 0;
}

__global__ void run_status_kernel(const Ctl* c, RunStatus* r, int item)
{
    if (c->status && !r->status) {
        r->status = c->status;
        r->bad_cell = c->bad_cell;
        r->item = item;
    }
}

__global__ void prepare_kernel(const double* u, double* w, long long fs, long long n, double cs2, Ctl* c, double* s,
                               double eos_m)
{
    unsigned long long am[3] = {0ull, 0ull, 0ull};
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        double pr, vx, vy, vz, e, ks;
        if (recover(cs2, eos_m, u, fs, q, pr, vx, vy, vz, e, ks)) {
            w[q] = pr;
            w[fs + q] = vx;
            w[2 * fs + q] = vy;
            w[3 * fs + q] = vz;
            double sp[3];
            max_speeds(ks, vx, vy, vz, sp);
            for (int d = 0; d < 3; ++d) {
                const unsigned long long b = (unsigned long long)__double_as_longlong(sp[d]);
                am[d] = b > am[d] ? b : am[d];
                if (s) s[d * fs + q] = sp[d];
            }
        } else {
            for (int k = 0; k < 4; ++k) w[k * fs + q] = 0.0;
            if (s)
                for (int d = 0; d < 3; ++d) s[d * fs + q] = 0.0;
            if (atomicCAS(&c->status, 0, (int)HYDRO_ERR_UNPHYSICAL) == 0) c->bad_cell = q;
        }
    }
    for (int d = 0; d < 3; ++d) {
        unsigned long long v = am[d];
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long x = __shfl_xor_sync(0xffffffffu, v, o);
            v = x > v ? x : v;
        }
        if ((threadIdx.x & 31) == 0 && v) atomicMax(&c->a_cur[d], v);
    }
}

__global__ void prim2con_kernel(const double* wp, long long ws, double* u, long long fs, long long n, double cs2,
                                Ctl* c, int nf, double eos_m)
{
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const double e = wp[q], vx = wp[ws + q], vy = wp[2 * ws + q], vz = wp[3 * ws + q], nn = wp[4 * ws + q];
        const double v2 = fma(vx, vx, fma(vy, vy, vz * vz));
        if (!(e > 0.0) || !(v2 < 1.0) || (eos_m != 0.0 && !(e > eos_m * nn && nn >= 0.0))) {
            if (atomicCAS(&c->status, 0, (int)HYDRO_ERR_UNPHYSICAL) == 0) c->bad_cell = q;
        }
        const double p = eos_m == 0.0 ? cs2 * e : cs2 * (e - eos_m * nn);
        const double g2 = 1.0 / (1.0 - v2);
        const double W = (e + p) * g2;
        u[q] = W - p;
        u[fs + q] = W * vx;
        u[2 * fs + q] = W * vy;
        u[3 * fs + q] = W * vz;
        u[4 * fs + q] = nn * sqrt(g2);
        for (int k = 5; k < nf; ++k) u[k * fs + q] = wp[k * ws + q] * sqrt(g2);   // further charges
    }
}

__global__ void state_to_prim_kernel(const double* u, long long fs, double* out, long long os, long long n,
                                     double cs2, int nf, double eos_m)
{
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        double pr, vx, vy, vz, e, ks;
        if (recover(cs2, eos_m, u, fs, q, pr, vx, vy, vz, e, ks)) {
            const double v2 = fma(vx, vx, fma(vy, vy, vz * vz));
            out[q] = e;
            out[os + q] = vx;
            out[2 * os + q] = vy;
            out[3 * os + q] = vz;
            for (int k = 4; k < nf; ++k) out[k * os + q] = u[k * fs + q] * sqrt(1.0 - v2);
        } else {
            for (int k = 0; k < nf; ++k) out[k * os + q] = __longlong_as_double(0x7ff8000000000000LL);
        }
    }
}

template <int R, int TX, int TY, int ILP = 1, bool LLF = false, int NF = 5,
          int EMU = default_emu(R, TX, TY, LLF, NF, false), bool ZEXT = false, int ZEMU = EMU, int MINB = 0>
static cudaError_t info_for(StageLaunch* out)
{
    auto fn = stage_kernel<R, TX, TY, ILP, LLF, NF, false, EMU, ZEXT, MINB>;
    out->fn = fn;
    out->zfn = nullptr;
    if constexpr (ZEXT) out->zfn = LLF ? zflux_llf_kernel<R, ZEMU> : zflux_kernel<R, ZEMU>;
    out->smem = StageSmem<R, TX, TY, LLF, NF, false, ILP == kPencilSweep, ZEXT>::bytes;
    out->tx = TX;
    out->ty = TY;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)out->smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&out->ctas_per_sm, fn, TX * TY, out->smem);
}

// three-pass stage: x, y and z passes, then the per-cell combination (LLF:
// local Lax-Friedrichs passes, and the combination also stores the speeds)
template <int R, int ZEMU, bool LLF = false, int MINB = 0, int XMINB = MINB, int NF = 5>
static cudaError_t info_for_three(StageLaunch* out)
{
    out->fn = stage_combine_kernel<NF, LLF>;
    out->pass_threads = 32 * NF;
    if constexpr (NF > 5) {
        // several charges: one warp per field, MINB CTAs per SM
        if constexpr (LLF) {
            out->xfn = axis_flux_llf_kernel<R, ZEMU, 0, MINB, NF>;
            out->yfn = axis_flux_llf_kernel<R, ZEMU, 1, MINB, NF>;
            out->zfn = axis_flux_llf_kernel<R, ZEMU, 2, MINB, NF>;
        } else {
            out->xfn = axis_flux_kernel<R, ZEMU, 0, MINB, NF>;
            out->yfn = axis_flux_kernel<R, ZEMU, 1, MINB, NF>;
            out->zfn = axis_flux_kernel<R, ZEMU, 2, MINB, NF>;
        }
    } else if constexpr (LLF) {
        out->xfn = axis_flux_llf_kernel<R, ZEMU, 0>;
        out->yfn = axis_flux_llf_kernel<R, ZEMU, 1>;
        out->zfn = zflux_llf_kernel<R, ZEMU>;
    } else if constexpr (MINB > 0) {
        out->xfn = axis_flux_kernel<R, ZEMU, 0, XMINB>;
        out->yfn = axis_flux_kernel<R, ZEMU, 1, MINB>;
        out->zfn = axis_flux_kernel<R, ZEMU, 2, MINB>;
    } else {
        out->xfn = axis_flux_kernel<R, ZEMU, 0>;
        out->yfn = axis_flux_kernel<R, ZEMU, 1>;
        out->zfn = zflux_kernel<R, ZEMU>;
    }
    out->combine = true;
    out->smem = 0;
    out->tx = 16;
    out->ty = 16;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&out->ctas_per_sm, stage_combine_kernel<NF, LLF>, 256, 0);
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// the driver's tensor-map encoder, looked up once (null if unavailable)
static EncodeTiledFn encode_tiled_fn()
{
    static EncodeTiledFn fn = []() -> EncodeTiledFn {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

// TMA-staged stage kernel (with the z pass) for a TX x TY tile; the encoder
// is looked up here, outside any stream capture
template <int R, int TX, int TY, int EMU, int ZEMU, int MINB>
static cudaError_t info_for_tma(StageLaunch* out)
{
    if (!encode_tiled_fn()) return cudaErrorNotSupported;
    auto fn = stage_kernel_tma<R, TX, TY, EMU, MINB>;
    out->fn = nullptr;
    out->fn_tma = fn;
    out->zfn = zflux_kernel<R, ZEMU>;
    using SM = StageSmem<R, TX, TY, false, 5, false, true, true, true>;
    out->smem = SM::bytes + 128;   // room to start the raw tile on a 128-byte boundary
    out->tx = TX;
    out->ty = TY;
    out->tma_rw = SM::RW;
    out->tma_rh = SM::RH;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)out->smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&out->ctas_per_sm, fn, TX * TY, out->smem);
}

// Face chunks of a pass over nf faces: equal chunks of about kZFaces faces
// (measured at 256^3 against 1, 2, 5 and 8 chunks: within 0.1% of the best
// for WENO7 and the best for WENO5; at 96^3 the equal halves take the stage
// from 1.85 to 1.62 ms against a 64 + 33 split).  HYDRO_PASS_FACES=<faces per
// chunk> overrides it, for timing.
int pass_chunks(int nf)
{
    static const int forced = [] {
        const char* e = getenv("HYDRO_PASS_FACES");
        return e && *e ? atoi(e) : 0;
    }();
    if (forced > 0) {
        const int c = (nf + forced - 1) / forced;
        return (nf + chunk_len(nf, c) - 1) / chunk_len(nf, c);
    }
    return face_chunks(nf);
}

cudaError_t launch_stage_kernels(const StageLaunch& L, int zc, const StageArgs& a, int sms, cudaStream_t s)
{
    const int nzi = a.zhi - a.zlo;
    if (L.combine) {
        // three-pass stage: every face flux by its axis pass, then the per-cell combination
        void (*fns[3])(StageArgs) = {L.xfn, L.yfn, L.zfn};
        const int nfa[3] = {a.nx + 1, a.ny + 1, nzi + 1};
        for (int d = 0; d < 3; ++d) {
            if (!a.act[d]) continue;
            if (L.face_per_thread) {
                // one thread per face of the axis
                const long long nfaces = (long long)nfa[d] * (d == 0 ? (long long)a.ny * nzi
                                                                      : (d == 1 ? (long long)a.nx * nzi
                                                                                : (long long)a.nx * a.ny));
                const long long nb = (nfaces + L.pass_threads - 1) / L.pass_threads;
                fns[d]<<<(unsigned)nb, L.pass_threads, L.pass_smem, s>>>(a);
                continue;
            }
            const long long pb = pass_blocks(d, a.nx, a.ny, nzi);
            fns[d]<<<dim3((unsigned)pb, (unsigned)pass_chunks(nfa[d])), L.pass_threads, 0, s>>>(a);
        }
        const long long cells = (long long)a.nx * a.ny * nzi;
        const long long want = (cells + 255) / 256, cap = (long long)sms * 8;
        L.fn<<<(unsigned)(want < cap ? want : cap), 256, 0, s>>>(a);
        return cudaSuccess;
    }
    if (L.zfn && a.act[2]) {
        const long long pb = zpass_blocks(a.nx, a.ny);
        const dim3 zg((unsigned)pb, (unsigned)pass_chunks(nzi + 1));
        L.zfn<<<zg, kZPassThreads, 0, s>>>(a);
    }
    const dim3 grid((a.nx + L.tx - 1) / L.tx, (a.ny + L.ty - 1) / L.ty, (nzi + zc - 1) / zc);
    if (L.fn_tma) {
        // tensor maps of this stage's input (host-side encoding, no GPU work)
        TmaMaps m;
        const cudaError_t e = encode_stage_maps(L, a.u_in, a.w_in, a.nx, a.ny, a.nz, a.fs, &m);
        if (e != cudaSuccess) return e;
        L.fn_tma<<<grid, L.tx * L.ty, L.smem, s>>>(a, m);
        return cudaSuccess;
    }
    L.fn<<<grid, L.tx * L.ty, L.smem, s>>>(a);
    return cudaSuccess;
}

cudaError_t encode_stage_maps(const StageLaunch& L, const double* u, const double* w, int nx, int ny, int nz,
                              long long fs, TmaMaps* out)
{
    if (!L.fn_tma || !tma_layout_ok(nx, ny)) return cudaErrorNotSupported;
    EncodeTiledFn enc = encode_tiled_fn();
    if (!enc) return cudaErrorNotSupported;
    // (x, y, z, field), x fastest; strides of y, z and field in bytes
    const cuuint64_t gdim_u[4] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz, 5};
    const cuuint64_t gdim_w[4] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz, 4};
    const cuuint64_t gstr[3] = {(cuuint64_t)nx * 8, (cuuint64_t)nx * ny * 8, (cuuint64_t)fs * 8};
    const cuuint32_t box_u[4] = {(cuuint32_t)L.tma_rw, (cuuint32_t)L.tma_rh, 1, 5};
    const cuuint32_t box_w[4] = {(cuuint32_t)L.tma_rw, (cuuint32_t)L.tma_rh, 1, 3};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = enc(&out->u, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, (void*)u, gdim_u, gstr, box_u, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    r = enc(&out->w, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, (void*)w, gdim_w, gstr, box_w, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// WENO5: 0 16x16 (1 CTA of 8 warps per SM), 1 16x8 (2 CTAs of 4 warps),
//        2 32x8, 3 16x16 with two face items per iteration, pencil sweeps on
//        4 16x16 (all products on the FP64 unit) and 5 16x8, 6 the 16x16
//        pencil sweep, 7 and 8 the same with the z pass.
// WENO7: 0 16x16 (8 warps, 221 KB shared memory), 1 16x8 (4 warps), 2 16x16
//        with two face items per iteration, pencil sweeps on 3 16x16 (all
//        products on the FP64 unit) and 4 16x8, 5 the 16x16 pencil sweep,
//        6 and 7 the same with the z pass; 8 and 9 as 7 with the weight
//        products (9: also the face products) on the integer pipe.
// With the z pass, 16x8 tiles without and with TMA staging of the raw cells
// (same occupancy, for comparison) and the 16x16 tile with TMA staging (its
// raw tile leaves room for one CTA per SM): WENO5 9, 10, 11; WENO7 10, 11, 12.
// Three-pass (x, y and z passes, then the per-cell combination): WENO5 12,
// WENO7 13 (passes at four / three CTAs per SM); WENO5 13, 14 with the
// passes at five and six CTAs per SM, WENO7 14, 15 at four and five, and 16
// at five with the face products of the passes on the integer pipe too, 17
// with the x pass at four and the y and z passes at five.
// (Passes with only the weight products, or only their squares, on the
// integer pipe measured 6-10 % slower: the passes are bound by FP64 issue.)
// Variants 4 (WENO5) and 3 (WENO7) keep every product on the FP64 unit (the
// bitwise reference); the others take the default of default_emu.  WENO5 7, 8 /
// WENO7 6, 7: the 16x16 pencil sweep with the z faces from a separate z pass
// (zflux_kernel: long z pencils at 15-20 warps per SM, carried differences;
// the stage kernel then keeps no z ring), with one stage CTA per SM or two
// (8 / 16 warps; the compiler caps the registers at 128).  The z pass, and
// with 16 warps the WENO5 stage kernel, also take the weight products on the
// integer pipe: with that many warps the longer integer chains are hidden.
// Local LF (raw staging, 2G-plane ring): WENO5 0 16x16 and 1 16x8; WENO7 0
// 16x8 (16x16 would need 247 KB of shared memory).  With the local-LF z pass
// (zflux_llf_kernel, no ring): WENO5 2 16x16 (two CTAs per SM) and 3 16x8
// (four), WENO7 1 16x16 and 2 16x8.
// Several charges (nq = 2, 3): 0 the 16x8 stage kernel, 1 three-pass (one
// warp per field in the passes; the default).
// the launch a grid gets before any tuning: the fastest on the 256^3 workload
// (the three-pass variant, for component-wise WENO with global or local LF; a
// handle that cannot run it keeps the fused one)
int default_launch_variant(int R, int split, int nq, int charw)
{
    if (charw) return (R == 3 || R == 4) && split == 0 ? char_default_variant(R, nq) : 0;   // face passes
    if (R == 2) return 0;
    if (nq > 1) return 1;               // several charges, three-pass
    if (split) return R == 3 ? 4 : 3;   // local LF, three-pass
    return R == 3 ? 12 : 16;            // three-pass (WENO7: passes at five CTAs per SM, face
                                        // products on the integer pipe too)
}

int fused_launch_variant(int R, int split, int nq, int charw)
{
    if (charw || R == 2 || split || nq > 1) return 0;
    return R == 3 ? 6 : 5;
}

int batch_variant_count(int R, int split)
{
    if (split == 1) return R == 3 ? 2 : 1;
    return R == 3 ? 10 : 9;   // the last is the three-pass variant
}

int launch_variant_count(int R, int split, int nq, int charw)
{
    if (charw) return (R == 3 || R == 4) && split == 0 ? char_variant_count(R, nq) : 0;
    if (R == 2) return (split == 0 && nq <= 1) ? 2 : 0;
    if (nq > 1) return 2;
    if (split == 1) return R == 3 ? 5 : 4;
    return R == 3 ? 15 : 18;
}

// several charges: v 0 the 16x8 stage kernel, 1 three-pass (passes of NF
// warps: WENO5 at three CTAs per SM, 21 warps for NF = 7; WENO7 at four with
// the weight and face products on the integer pipe as in its default)
template <int NF>
static cudaError_t charges_variant(int R, int split, int v, StageLaunch* out)
{
    if (v == 1) {
        if (R == 3)
            return split ? info_for_three<3, kZPassEmu5, true, 3, 3, NF>(out)
                         : info_for_three<3, kZPassEmu5, false, 3, 3, NF>(out);
        return split ? info_for_three<4, kZPassEmu7, true, 4, 4, NF>(out)
                     : info_for_three<4, kEmuConst | kEmuWeights | kEmuFace, false, 4, 4, NF>(out);
    }
    if (v != 0) return cudaErrorInvalidValue;
    if (R == 3) return split ? info_for<3, 16, 8, 1, true, NF>(out) : info_for<3, 16, 8, 1, false, NF>(out);
    return split ? info_for<4, 16, 8, 1, true, NF>(out) : info_for<4, 16, 8, 1, false, NF>(out);
}

template <int TX, int TY>
static cudaError_t musta_info_for(StageLaunch* out)
{
    out->fn = musta_stage_kernel<TX, TY>;
    out->zfn = nullptr;
    out->smem = MustaSmem<TX, TY>::bytes;
    out->tx = TX;
    out->ty = TY;
    cudaError_t e = cudaFuncSetAttribute(musta_stage_kernel<TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)out->smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&out->ctas_per_sm, musta_stage_kernel<TX, TY>, TX * TY,
                                                         out->smem);
}

// R == 2 denotes MUSTA-FORCE + MUSCL (two ghost cells): 16x16 and 16x8 tiles.
cudaError_t stage_launch_variant(int R, int split, int nq, int v, StageLaunch* out, int charw)
{
    if (charw) return split == 0 ? char_launch_variant(R, nq, v, out) : cudaErrorInvalidValue;
    if (R == 2) {
        if (split != 0 || nq > 1) return cudaErrorInvalidValue;
        if (v == 0) return musta_info_for<16, 16>(out);
        if (v == 1) return musta_info_for<16, 8>(out);
        return cudaErrorInvalidValue;
    }
    if (nq > 1) {
        if (nq == 2) return charges_variant<6>(R, split, v, out);
        if (nq == 3) return charges_variant<7>(R, split, v, out);
        return cudaErrorInvalidValue;
    }
    if (split == 1) {
        if (R == 3 && v == 0) return info_for<3, 16, 16, 1, true>(out);
        if (R == 3 && v == 1) return info_for<3, 16, 8, 1, true>(out);
        if (R == 3 && v == 2) return info_for<3, 16, 16, 1, true, 5, kEmuConst, true, kZPassEmu5, 2>(out);
        if (R == 3 && v == 3) return info_for<3, 16, 8, 1, true, 5, kEmuConst, true, kZPassEmu5, 4>(out);
        if (R == 4 && v == 0) return info_for<4, 16, 8, 1, true>(out);
        if (R == 4 && v == 1) return info_for<4, 16, 16, 1, true, 5, kEmuConst, true, kZPassEmu7, 2>(out);
        if (R == 4 && v == 2) return info_for<4, 16, 8, 1, true, 5, kEmuConst, true, kZPassEmu7, 4>(out);
        if (R == 3 && v == 4) return info_for_three<3, kZPassEmu5, true>(out);
        if (R == 4 && v == 3) return info_for_three<4, kZPassEmu7, true>(out);
        return cudaErrorInvalidValue;
    }
    if (R == 3) {
        if (v == 0) return info_for<3, 16, 16>(out);
        if (v == 1) return info_for<3, 16, 8>(out);
        if (v == 2) return info_for<3, 32, 8>(out);
        if (v == 3) return info_for<3, 16, 16, 2>(out);
        if (v == 4) return info_for<3, 16, 16, kPencilSweep, false, 5, 0>(out);
        if (v == 5) return info_for<3, 16, 8, kPencilSweep>(out);
        if (v == 6) return info_for<3, 16, 16, kPencilSweep>(out);
        if (v == 7) return info_for<3, 16, 16, kPencilSweep, false, 5, kEmuConst, true, kZPassEmu5>(out);
        if (v == 8) return info_for<3, 16, 16, kPencilSweep, false, 5, kEmuConst | kEmuWeights, true, kZPassEmu5, 2>(out);
        if (v == 9) return info_for<3, 16, 8, kPencilSweep, false, 5, kEmuConst | kEmuWeights, true, kZPassEmu5, 4>(out);
        if (v == 10) return info_for_tma<3, 16, 8, kEmuConst | kEmuWeights, kZPassEmu5, 4>(out);
        if (v == 11) return info_for_tma<3, 16, 16, kEmuConst | kEmuWeights, kZPassEmu5, 1>(out);
        if (v == 12) return info_for_three<3, kZPassEmu5>(out);
        if (v == 13) return info_for_three<3, kZPassEmu5, false, 5>(out);
        if (v == 14) return info_for_three<3, kZPassEmu5, false, 6>(out);

    }
    if (R == 4) {
        if (v == 0) return info_for<4, 16, 16>(out);
        if (v == 1) return info_for<4, 16, 8>(out);
        if (v == 2) return info_for<4, 16, 16, 2>(out);
        if (v == 3) return info_for<4, 16, 16, kPencilSweep, false, 5, 0>(out);
        if (v == 4) return info_for<4, 16, 8, kPencilSweep>(out);
        if (v == 5) return info_for<4, 16, 16, kPencilSweep>(out);
        if (v == 6) return info_for<4, 16, 16, kPencilSweep, false, 5, kEmuConst, true, kZPassEmu7>(out);
        if (v == 7) return info_for<4, 16, 16, kPencilSweep, false, 5, kEmuConst, true, kZPassEmu7, 2>(out);
        if (v == 8) return info_for<4, 16, 16, kPencilSweep, false, 5, kEmuConst | kEmuWeights, true, kZPassEmu7, 2>(out);
        if (v == 9)
            return info_for<4, 16, 16, kPencilSweep, false, 5, kEmuConst | kEmuWeights | kEmuFace, true, kZPassEmu7, 2>(out);
        if (v == 10) return info_for<4, 16, 8, kPencilSweep, false, 5, kEmuConst, true, kZPassEmu7, 3>(out);
        if (v == 11) return info_for_tma<4, 16, 8, kEmuConst, kZPassEmu7, 3>(out);
        if (v == 12) return info_for_tma<4, 16, 16, kEmuConst, kZPassEmu7, 1>(out);
        if (v == 13) return info_for_three<4, kZPassEmu7>(out);
        if (v == 14) return info_for_three<4, kZPassEmu7, false, 4>(out);
        if (v == 15) return info_for_three<4, kZPassEmu7, false, 5>(out);
        if (v == 16) return info_for_three<4, kEmuConst | kEmuWeights | kEmuFace, false, 5>(out);
        if (v == 17) return info_for_three<4, kZPassEmu7, false, 5, 4>(out);
    }
    return cudaErrorInvalidValue;
}

std::string check_config(const hydro_config* c)
{
    if (!c) return "config is NULL";
    if (c->scheme != HYDRO_WENO5 && c->scheme != HYDRO_WENO7 && c->scheme != HYDRO_MUSTA_FORCE)
        return "scheme must be 5, 7 (WENO) or 2 (MUSTA-FORCE)";
    const int G = c->scheme == HYDRO_WENO5 ? 3 : (c->scheme == HYDRO_WENO7 ? 4 : 2);
    if (c->scheme == HYDRO_MUSTA_FORCE) {
        if (c->limiter < 0 || c->limiter > 3) return "limiter must be 0 (minmod), 1 (MC), 2 (van Leer) or 3 (superbee)";
        if (c->musta_stages < 0 || c->musta_stages > 8) return "musta_stages must be 0 (default 2) .. 8";
        if (c->split != 0) return "MUSTA-FORCE has no flux splitting (split must be 0)";
        if (c->nq > 1) return "MUSTA-FORCE supports one charge (nq <= 1)";
    }
    for (int d = 0; d < 3; ++d) {
        if (c->n[d] < 1) return "grid size must be >= 1";
        if (!(c->dx[d] > 0.0) || !std::isfinite(c->dx[d])) return "dx must be positive and finite";
        if (c->bc[d] != HYDRO_BC_OUTFLOW && c->bc[d] != HYDRO_BC_PERIODIC && !(d == 2 && c->bc[d] == HYDRO_BC_HALO))
            return "bc must be 0 (outflow) or 1 (periodic); 2 (halo) on z only";
        if (c->n[d] > 1 && c->bc[d] == HYDRO_BC_PERIODIC && c->n[d] < G) return "periodic axis shorter than the stencil";
    }
    if (c->bc[2] == HYDRO_BC_HALO && c->n[2] < G) return "a halo slab needs nz >= the stencil half-width r";
    if ((long long)c->n[0] * c->n[1] > (1LL << 40) || c->n[0] > (1 << 28) || c->n[1] > 65535 * 8 ||
        c->n[2] > (1 << 28))
        return "grid too large";
    if (!(c->cs2 > 0.0 && c->cs2 < 1.0)) return "cs2 must lie in (0, 1)";
    // the one-reciprocal WENO face form keeps every product of smoothness
    // terms a normal number for eps in this range (hydro_math.cuh face_sum)
    if (!(c->weno_eps >= 1e-40 && c->weno_eps <= 1e30)) return "weno_eps must lie in [1e-40, 1e30]";
    if (!(c->dt_fixed > 0.0) && !(c->cfl > 0.0)) return "need cfl > 0 or dt_fixed > 0";
    if (c->split != 0 && c->split != 1) return "split must be 0 (global) or 1 (local Lax-Friedrichs)";
    if (c->nq < 0 || c->nq > 3) return "nq (number of charges) must be 0..3";
    if (c->charwise != 0 && c->charwise != 1) return "charwise must be 0 (component-wise) or 1 (characteristic-wise)";
    if (!(c->eos_mass >= 0.0) || !std::isfinite(c->eos_mass)) return "eos_mass must be >= 0 and finite";
    if (c->eos_mass > 0.0 && (c->scheme == HYDRO_MUSTA_FORCE || c->charwise))
        return "the general EOS (eos_mass > 0) runs component-wise WENO only";
    if (c->charwise && (c->scheme == HYDRO_MUSTA_FORCE || c->split != 0))
        return "characteristic-wise reconstruction needs WENO with global Lax-Friedrichs splitting (split = 0)";
    return std::string();
}

}  // namespace hydro
