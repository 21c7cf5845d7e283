// hydro_api.cu -- the C ABI of include/hydro.h for one grid: buffers, the
// device control block, the captured per-step CUDA graph and the copies.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <utility>
#include <vector>
#include <new>
#include <string>

#include "hydro_common.cuh"

using namespace hydro;

struct hydro_s {
    hydro_config cfg;
    int R = 3;
    int dev = 0;
    int sms = 0;
    cudaStream_t stream = nullptr;   // caller's stream
    cudaStream_t cap = nullptr;      // private stream used only for graph capture
    long long ncell = 0, fs = 0;
    double* buf = nullptr;
    double* U[3] = {nullptr, nullptr, nullptr};
    double* W[3] = {nullptr, nullptr, nullptr};
    double* S[3] = {nullptr, nullptr, nullptr};   // per-axis speeds (local LF only)
    double* fz = nullptr;            // z-face fluxes of the z-pass variants (5 fields of nz+1 planes)
    long long fzs = 0;
    double* fx = nullptr;            // x- and y-face fluxes of the three-pass variants (global LF)
    long long fxs = 0;
    double* fy = nullptr;
    long long fys = 0;
    Ctl* ctl = nullptr;
    Ctl* hctl = nullptr;             // pinned mirror for read-back
    cudaGraphExec_t exec = nullptr;
    StageLaunch L{};
    int variant = 0;
    int zc = 0;
    int nf = 5;                      // state fields: E, M, and nq >= 1 charges
    // z halo storage (bc[2] == HYDRO_BC_HALO, a slab of a larger grid): nz_alloc
    // stored planes, interior [zlo, zhi), interior data starts `off` doubles
    // into every field; otherwise nz_alloc = n[2], zlo = 0, off = 0
    int nz_alloc = 0, zlo = 0, zhi = 0, G = 3;
    long long off = 0;
    bool have_state = false;
    AdjointWork* adj = nullptr;      // reverse-mode workspace (hydro_adjoint.cu)
    // hydro_run_many: staging states (two in, one out), copy streams, events
    // and the first-error record over the items (allocated on first use)
    double* io_buf = nullptr;
    RunStatus* run_st = nullptr;
    RunStatus* hrun_st = nullptr;
    cudaStream_t s_in = nullptr, s_out = nullptr;
    cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_used[2] = {nullptr, nullptr};
    cudaEvent_t ev_out_ready = nullptr, ev_out_free = nullptr;
    std::string err;
};

static thread_local std::string g_create_err;

static hydro_status fail(hydro_t* h, hydro_status s, const std::string& msg)
{
    if (h) h->err = msg;
    else g_create_err = msg;
    return s;
}

static hydro_status cuda_fail(hydro_t* h, cudaError_t e, const char* where)
{
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(h, e == cudaErrorMemoryAllocation ? HYDRO_ERR_OOM : HYDRO_ERR_CUDA, m);
}

#define CK(h, call, where)                                       \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, where); \
    } while (0)

static StageArgs stage_args(hydro_t* h, int stage)
{
    StageArgs a{};
    const int in = stage - 1;                       // U0 -> U1 -> U2 -> U0
    a.u_in = h->U[in];
    a.w_in = h->W[in];
    a.u_n = h->U[0];
    a.u_out = stage == 3 ? h->U[0] : h->U[stage];
    a.w_out = stage == 3 ? h->W[0] : h->W[stage];
    a.fs = h->fs;
    a.nx = h->cfg.n[0];
    a.ny = h->cfg.n[1];
    a.nz = h->nz_alloc;
    a.zc = h->zc;
    a.zlo = h->zlo;
    a.zhi = h->zhi;
    for (int d = 0; d < 3; ++d) {
        a.bc[d] = h->cfg.bc[d];
        a.act[d] = axis_active(h->cfg, d);
        a.hdx[d] = 0.5 / h->cfg.dx[d];
    }
    a.cs2 = h->cfg.cs2;
    a.eps_s = h->cfg.weno_eps * (h->R == 3 ? SchemeConst<3>::eps_scale : SchemeConst<4>::eps_scale);
    static const double ca[3] = {0.0, 0.75, 1.0 / 3.0}, cb[3] = {1.0, 0.25, 2.0 / 3.0};
    a.ca = ca[in];
    a.cb = cb[in];
    a.alpha_in = stage == 1 ? h->ctl->a_cur : (stage == 2 ? h->ctl->a_s1 : h->ctl->a_s2);
    a.alpha_out = stage == 1 ? h->ctl->a_s1 : (stage == 2 ? h->ctl->a_s2 : h->ctl->a_next);
    a.dt = &h->ctl->dt;
    a.status = &h->ctl->status;
    a.bad_cell = &h->ctl->bad_cell;
    a.s_in = h->S[in];
    a.s_out = stage == 3 ? h->S[0] : h->S[stage];
    a.limiter = h->cfg.limiter;
    a.musta_k = musta_stages_of(h->cfg);
    a.eos_m = h->cfg.eos_mass;
    a.fz = h->fz;
    a.fzs = h->fzs;
    a.fx = h->fx;
    a.fxs = h->fxs;
    a.fy = h->fy;
    a.fys = h->fys;
    return a;
}

// a launch this handle can run: z-pass variants need the z-face buffer and a
// row count that fits the z pass's grid
static bool launch_fits(const hydro_t* h, const StageLaunch& L)
{
    if (L.fn_tma && !tma_layout_ok(h->cfg.n[0], h->cfg.n[1])) return false;
    if (L.combine) {
        const int nzi = h->zhi - h->zlo;
        if (!h->fx || !h->fy || pass_blocks(0, h->cfg.n[0], h->cfg.n[1], nzi) > 0x7fffffffLL ||
            pass_blocks(1, h->cfg.n[0], h->cfg.n[1], nzi) > 0x7fffffffLL)
            return false;
        // one thread per face: every axis's face count must fit the grid
        if (L.face_per_thread && (long long)(h->cfg.n[0] + 1) * (h->cfg.n[1] + 1) * (nzi + 1) / L.pass_threads >
                                     0x7fffffffLL)
            return false;
    }
    return !L.zfn || (h->fz && zpass_blocks(h->cfg.n[0], h->cfg.n[1]) <= 0x7fffffffLL);
}

// one RK3 stage: the z pass first (z-pass variants, z active), then the stage
// kernel.  Returns an error only when a TMA-staged launch cannot build its
// tensor maps (nothing is launched then); launch errors come from
// cudaGetLastError as usual.
static cudaError_t launch_stage(const hydro_t* h, const StageLaunch& L, int zc, const StageArgs& a, cudaStream_t s)
{
    return launch_stage_kernels(L, zc, a, h->sms, s);
}

static cudaError_t enqueue_step(hydro_t* h, cudaStream_t s)
{
    step_begin_kernel<<<1, 1, 0, s>>>(h->ctl, step_params(h->cfg));
    for (int st = 1; st <= 3; ++st) {
        const cudaError_t e = launch_stage(h, h->L, h->zc, stage_args(h, st), s);
        if (e != cudaSuccess) return e;
    }
    step_end_kernel<<<1, 1, 0, s>>>(h->ctl);
    return cudaGetLastError();
}

static hydro_status build_graph(hydro_t* h)
{
    if (h->exec) return HYDRO_OK;
    cudaGraph_t g = nullptr;
    CK(h, cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal), "capture begin");
    cudaError_t e1 = enqueue_step(h, h->cap);
    cudaError_t e2 = cudaStreamEndCapture(h->cap, &g);
    if (e1 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(h, e1, "capture step");
    }
    CK(h, e2, "capture end");
    cudaError_t e3 = cudaGraphInstantiate(&h->exec, g, 0);
    cudaGraphDestroy(g);
    CK(h, e3, "graph instantiate");
    return HYDRO_OK;
}

namespace hydro {
hydro_status hydro_handle_view(hydro_t* h, HandleView* v)
{
    if (!h || !v) return HYDRO_ERR_INVALID_ARG;
    v->loaded = h->have_state;
    v->cfg = h->cfg;
    v->R = h->R;
    v->stream = h->stream;
    v->ncell = h->ncell;
    v->fs = h->fs;
    v->U0 = h->U[0] + h->off;
    v->W0 = h->W[0] + h->off;
    v->ctl = h->ctl;
    v->L = h->L;
    v->zc = h->zc;
    v->fz = nullptr;
    v->fzs = 0;
    v->fx = v->fy = nullptr;
    v->fxs = v->fys = 0;
    v->sms = h->sms;
    if (h->L.zfn && h->fz && !h->L.fn_tma && (!h->L.combine || (h->fx && h->fy)) && h->cfg.bc[2] != HYDRO_BC_HALO) {
        // the adjoint's recorded forward runs the handle's z-pass or three-pass
        // launch on its own state buffers, with the handle's face buffers as scratch
        v->fz = h->fz;
        v->fzs = h->fzs;
        v->fx = h->fx;
        v->fxs = h->fxs;
        v->fy = h->fy;
        v->fys = h->fys;
    } else if (h->L.zfn || h->L.fn_tma) {
        // otherwise the fastest variant that needs no z-face buffer
        cudaError_t e = stage_launch_variant(h->R, h->cfg.split, h->cfg.nq,
                                             fused_launch_variant(h->R, h->cfg.split, h->cfg.nq, h->cfg.charwise), &v->L,
                                             h->cfg.charwise);
        if (e != cudaSuccess) return cuda_fail(h, e, "stage kernel setup");
        v->zc = pick_zc(h->cfg.n[0], h->cfg.n[1], h->cfg.n[2], v->L, h->sms);
    }
    return HYDRO_OK;
}

AdjointWork* hydro_handle_adjoint(hydro_t* h, bool create)
{
    if (!h) return nullptr;
    if (!h->adj && create) h->adj = new (std::nothrow) AdjointWork();
    return h->adj;
}

hydro_status hydro_handle_fail(hydro_t* h, hydro_status s, const std::string& m) { return fail(h, s, m); }
}  // namespace hydro

static int blocks_for(long long n) { long long b = (n + 255) / 256; return (int)(b > 152 * 16 ? 152 * 16 : (b < 1 ? 1 : b)); }

extern "C" {

const char* hydro_version(void) { return "hydro-gb300 1.0 (sm_103a, FP64 WENO5/7 + SSP-RK3)"; }

hydro_status hydro_create(const hydro_config* cfg, void* stream, hydro_t** out)
{
    if (!out) return fail(nullptr, HYDRO_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    const std::string why = check_config(cfg);
    if (!why.empty()) return fail(nullptr, HYDRO_ERR_INVALID_ARG, why);
    hydro_t* h = new (std::nothrow) hydro_t();
    if (!h) return fail(nullptr, HYDRO_ERR_OOM, "host allocation failed");
    h->cfg = *cfg;
    h->R = scheme_R(cfg->scheme);
    h->stream = (cudaStream_t)stream;
    cudaError_t e;
    auto bail = [&](hydro_status s) {
        g_create_err = h->err;
        hydro_destroy(h);
        return s;
    };
    if ((e = cudaGetDevice(&h->dev)) != cudaSuccess) return bail(cuda_fail(h, e, "cudaGetDevice"));
    if ((e = cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->dev)) != cudaSuccess)
        return bail(cuda_fail(h, e, "device attribute"));
    h->nf = state_fields(*cfg);
    h->variant = fused_launch_variant(h->R, cfg->split, cfg->nq, cfg->charwise);
    if ((e = stage_launch_variant(h->R, cfg->split, cfg->nq, h->variant, &h->L, cfg->charwise)) != cudaSuccess)
        return bail(cuda_fail(h, e, "stage kernel setup"));
    h->G = h->R;
    h->ncell = (long long)cfg->n[0] * cfg->n[1] * cfg->n[2];
    const bool halo = cfg->bc[2] == HYDRO_BC_HALO;
    h->nz_alloc = cfg->n[2] + (halo ? 2 * h->G : 0);
    h->zlo = halo ? h->G : 0;
    h->zhi = h->zlo + cfg->n[2];
    h->off = (long long)h->zlo * cfg->n[0] * cfg->n[1];
    const long long nalloc = (long long)cfg->n[0] * cfg->n[1] * h->nz_alloc;
    h->fs = (nalloc + 31) / 32 * 32;   // 256-byte aligned fields
    h->zc = pick_zc(cfg->n[0], cfg->n[1], cfg->n[2], h->L, h->sms);
    // U0..U2 (nf fields each), W0..W2 (4 each), speeds S0..S2 (3 each, local LF)
    const int nf = h->nf;
    const int nfields = 3 * nf + 12 + (cfg->split ? 9 : 0);
    const size_t bytes = sizeof(double) * (size_t)h->fs * nfields;
    if ((e = cudaMalloc(&h->buf, bytes)) != cudaSuccess) return bail(cuda_fail(h, e, "state buffers"));
    for (int i = 0; i < 3; ++i) {
        h->U[i] = h->buf + (size_t)h->fs * nf * i;
        h->W[i] = h->buf + (size_t)h->fs * (3 * nf + 4 * i);
        if (cfg->split) h->S[i] = h->buf + (size_t)h->fs * (3 * nf + 12 + 3 * i);
    }
    if ((e = cudaMemsetAsync(h->buf, 0, bytes, h->stream)) != cudaSuccess) return bail(cuda_fail(h, e, "memset"));
    if (zpass_capable(*cfg, h->R)) {
        // z-face fluxes for the z-pass variants: nf fields of nz+1 face planes
        h->fzs = ((long long)cfg->n[0] * cfg->n[1] * (cfg->n[2] + 1) + 31) / 32 * 32;
        if ((e = cudaMalloc(&h->fz, sizeof(double) * (size_t)h->fzs * nf)) != cudaSuccess)
            return bail(cuda_fail(h, e, "z-face buffer"));
        {
            // x- and y-face fluxes for the three-pass variants
            const long long nzi = cfg->n[2];
            h->fxs = ((long long)(cfg->n[0] + 1) * cfg->n[1] * nzi + 31) / 32 * 32;
            h->fys = ((long long)cfg->n[0] * (cfg->n[1] + 1) * nzi + 31) / 32 * 32;
            if ((e = cudaMalloc(&h->fx, sizeof(double) * (size_t)h->fxs * nf)) != cudaSuccess)
                return bail(cuda_fail(h, e, "x-face buffer"));
            if ((e = cudaMalloc(&h->fy, sizeof(double) * (size_t)h->fys * nf)) != cudaSuccess)
                return bail(cuda_fail(h, e, "y-face buffer"));
        }
    }
    {
        // the variant new grids start on (it may need the z-face buffer)
        const int dv = default_launch_variant(h->R, cfg->split, cfg->nq, cfg->charwise);
        StageLaunch L{};
        if (dv != h->variant && stage_launch_variant(h->R, cfg->split, cfg->nq, dv, &L, cfg->charwise) == cudaSuccess &&
            launch_fits(h, L)) {
            h->variant = dv;
            h->L = L;
            h->zc = pick_zc(cfg->n[0], cfg->n[1], cfg->n[2], L, h->sms);
        }
    }
    if ((e = cudaMalloc(&h->ctl, sizeof(Ctl))) != cudaSuccess) return bail(cuda_fail(h, e, "control block"));
    if ((e = cudaMallocHost(&h->hctl, sizeof(Ctl))) != cudaSuccess) return bail(cuda_fail(h, e, "pinned control"));
    if ((e = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking)) != cudaSuccess)
        return bail(cuda_fail(h, e, "capture stream"));
    reset_ctl_kernel<<<1, 1, 0, h->stream>>>(h->ctl, 0.0);
    if ((e = cudaGetLastError()) != cudaSuccess) return bail(cuda_fail(h, e, "reset"));
    hydro_status s = build_graph(h);
    if (s != HYDRO_OK) return bail(s);
    *out = h;
    return HYDRO_OK;
}

hydro_status hydro_destroy(hydro_t* h)
{
    if (!h) return HYDRO_OK;
    if (h->stream || h->buf) cudaStreamSynchronize(h->stream);
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->cap) cudaStreamDestroy(h->cap);
    if (h->buf) cudaFree(h->buf);
    if (h->fz) cudaFree(h->fz);
    if (h->fx) cudaFree(h->fx);
    if (h->fy) cudaFree(h->fy);
    if (h->ctl) cudaFree(h->ctl);
    if (h->hctl) cudaFreeHost(h->hctl);
    if (h->adj) {
        cudaFree(h->adj->buf);
        cudaFree(h->adj->rec);
        cudaFree(h->adj->ctl);
        delete h->adj;
    }
    if (h->s_in) cudaStreamSynchronize(h->s_in);
    if (h->s_out) cudaStreamSynchronize(h->s_out);
    if (h->io_buf) cudaFree(h->io_buf);
    if (h->run_st) cudaFree(h->run_st);
    if (h->hrun_st) cudaFreeHost(h->hrun_st);
    for (cudaEvent_t ev : {h->ev_in[0], h->ev_in[1], h->ev_used[0], h->ev_used[1], h->ev_out_ready, h->ev_out_free})
        if (ev) cudaEventDestroy(ev);
    if (h->s_in) cudaStreamDestroy(h->s_in);
    if (h->s_out) cudaStreamDestroy(h->s_out);
    delete h;
    return HYDRO_OK;
}

const char* hydro_last_error(hydro_t* h) { return h ? h->err.c_str() : g_create_err.c_str(); }

static hydro_status copy_fields(hydro_t* h, double* dst, long long dstride, const double* src, long long sstride,
                                int nf, cudaMemcpyKind kind)
{
    for (int f = 0; f < nf; ++f)
        CK(h, cudaMemcpyAsync(dst + f * dstride, src + f * sstride, sizeof(double) * h->ncell, kind, h->stream),
           "copy");
    return HYDRO_OK;
}

static hydro_status check_io(hydro_t* h, const void* p, int64_t stride, int32_t mem)
{
    if (!h) return HYDRO_ERR_INVALID_ARG;
    if (!p) return fail(h, HYDRO_ERR_INVALID_ARG, "NULL data pointer");
    if (stride < h->ncell) return fail(h, HYDRO_ERR_INVALID_ARG, "field_stride smaller than the cell count");
    if (mem != HYDRO_MEM_HOST && mem != HYDRO_MEM_DEVICE) return fail(h, HYDRO_ERR_INVALID_ARG, "mem must be 0 or 1");
    return HYDRO_OK;
}

static hydro_status after_load(hydro_t* h, double t)
{
    reset_ctl_kernel<<<1, 1, 0, h->stream>>>(h->ctl, t);
    prepare_kernel<<<blocks_for(h->ncell), 256, 0, h->stream>>>(h->U[0] + h->off, h->W[0] + h->off, h->fs, h->ncell,
                                                                 h->cfg.cs2, h->ctl, h->S[0] ? h->S[0] + h->off : nullptr,
                                                                 h->cfg.eos_mass);
    CK(h, cudaGetLastError(), "prepare");
    h->have_state = true;
    return HYDRO_OK;
}

hydro_status hydro_set_state(hydro_t* h, const double* u, int64_t field_stride, int32_t mem, double t)
{
    hydro_status s = check_io(h, u, field_stride, mem);
    if (s) return s;
    s = copy_fields(h, h->U[0] + h->off, h->fs, u, field_stride, h->nf,
                    mem == HYDRO_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice);
    if (s) return s;
    return after_load(h, t);
}

hydro_status hydro_set_primitive(hydro_t* h, const double* w, int64_t field_stride, int32_t mem, double t)
{
    hydro_status s = check_io(h, w, field_stride, mem);
    if (s) return s;
    const double* src = w;
    long long ss = field_stride;
    if (mem == HYDRO_MEM_HOST) {   // stage through U1 (scratch between steps)
        s = copy_fields(h, h->U[1] + h->off, h->fs, w, field_stride, h->nf, cudaMemcpyHostToDevice);
        if (s) return s;
        src = h->U[1] + h->off;
        ss = h->fs;
    }
    reset_ctl_kernel<<<1, 1, 0, h->stream>>>(h->ctl, t);
    prim2con_kernel<<<blocks_for(h->ncell), 256, 0, h->stream>>>(src, ss, h->U[0] + h->off, h->fs, h->ncell, h->cfg.cs2,
                                                                  h->ctl, h->nf, h->cfg.eos_mass);
    CK(h, cudaGetLastError(), "prim2con");
    prepare_kernel<<<blocks_for(h->ncell), 256, 0, h->stream>>>(h->U[0] + h->off, h->W[0] + h->off, h->fs, h->ncell,
                                                                 h->cfg.cs2, h->ctl, h->S[0] ? h->S[0] + h->off : nullptr,
                                                                 h->cfg.eos_mass);
    CK(h, cudaGetLastError(), "prepare");
    h->have_state = true;
    return HYDRO_OK;
}

hydro_status hydro_step(hydro_t* h, int32_t nsteps, double t_end)
{
    if (!h) return HYDRO_ERR_INVALID_ARG;
    if (h->cfg.bc[2] == HYDRO_BC_HALO) return fail(h, HYDRO_ERR_INVALID_ARG, "a halo slab steps through hydro_stage");
    if (nsteps < 0) return fail(h, HYDRO_ERR_INVALID_ARG, "nsteps < 0");
    if (!h->have_state) return fail(h, HYDRO_ERR_STATE, "no state loaded");
    set_t_end_kernel<<<1, 1, 0, h->stream>>>(h->ctl, t_end);
    CK(h, cudaGetLastError(), "set t_end");
    for (int i = 0; i < nsteps; ++i) CK(h, cudaGraphLaunch(h->exec, h->stream), "graph launch");
    return HYDRO_OK;
}

hydro_status hydro_profile_step(hydro_t* h, int32_t nsteps, double t_end, double kernel_ms[5])
{
    if (!h || !kernel_ms) return HYDRO_ERR_INVALID_ARG;
    if (h->cfg.bc[2] == HYDRO_BC_HALO) return fail(h, HYDRO_ERR_INVALID_ARG, "a halo slab steps through hydro_stage");
    if (nsteps < 0) return fail(h, HYDRO_ERR_INVALID_ARG, "nsteps < 0");
    if (!h->have_state) return fail(h, HYDRO_ERR_STATE, "no state loaded");
    for (int i = 0; i < 5; ++i) kernel_ms[i] = 0.0;
    cudaEvent_t ev[6];
    for (int i = 0; i < 6; ++i) CK(h, cudaEventCreate(&ev[i]), "event create");
    hydro_status st = HYDRO_OK;
    set_t_end_kernel<<<1, 1, 0, h->stream>>>(h->ctl, t_end);
    for (int s = 0; s < nsteps && st == HYDRO_OK; ++s) {
        cudaEventRecord(ev[0], h->stream);
        step_begin_kernel<<<1, 1, 0, h->stream>>>(h->ctl, step_params(h->cfg));
        cudaEventRecord(ev[1], h->stream);
        cudaError_t el = cudaSuccess;
        for (int k = 1; k <= 3; ++k) {
            const cudaError_t e1 = launch_stage(h, h->L, h->zc, stage_args(h, k), h->stream);
            if (el == cudaSuccess) el = e1;
            cudaEventRecord(ev[1 + k], h->stream);
        }
        step_end_kernel<<<1, 1, 0, h->stream>>>(h->ctl);
        cudaEventRecord(ev[5], h->stream);
        cudaError_t e = cudaEventSynchronize(ev[5]);
        if (e == cudaSuccess) e = el;
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) {
            st = cuda_fail(h, e, "profiled step");
            break;
        }
        for (int i = 0; i < 5; ++i) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
            kernel_ms[i] += ms;
        }
    }
    for (int i = 0; i < 6; ++i) cudaEventDestroy(ev[i]);
    return st;
}

// ---- z-slab domain decomposition ---------------------------------------

static bool is_halo(const hydro_t* h) { return h->cfg.bc[2] == HYDRO_BC_HALO; }

// the exchanged fields of one level, in pack order: u (nf), w (4), speeds (3, local LF)
static int level_fields(hydro_t* h, int level, double* f[16])
{
    int n = 0;
    for (int k = 0; k < h->nf; ++k) f[n++] = h->U[level] + (size_t)h->fs * k;
    for (int k = 0; k < 4; ++k) f[n++] = h->W[level] + (size_t)h->fs * k;
    if (h->cfg.split)
        for (int k = 0; k < 3; ++k) f[n++] = h->S[level] + (size_t)h->fs * k;
    return n;
}

int64_t hydro_halo_doubles(hydro_t* h)
{
    if (!h || !is_halo(h)) return 0;
    double* f[16];
    return (int64_t)level_fields(h, 0, f) * h->G * h->cfg.n[0] * h->cfg.n[1];
}

static hydro_status halo_args(hydro_t* h, int level, int side, int mem, const void* buf)
{
    if (!h) return HYDRO_ERR_INVALID_ARG;
    if (!is_halo(h)) return fail(h, HYDRO_ERR_INVALID_ARG, "not a halo (bc[2] = HYDRO_BC_HALO) handle");
    if (level < 0 || level > 2 || side < 0 || side > 1) return fail(h, HYDRO_ERR_INVALID_ARG, "level must be 0..2, side 0..1");
    if (mem != HYDRO_MEM_HOST && mem != HYDRO_MEM_DEVICE) return fail(h, HYDRO_ERR_INVALID_ARG, "bad mem");
    if (!buf) return fail(h, HYDRO_ERR_INVALID_ARG, "buffer is NULL");
    return HYDRO_OK;
}

// pack: interior planes next to `side` -> buf; unpack: buf -> ghost planes on `side`
static hydro_status halo_copy(hydro_t* h, int level, int side, double* out, const double* in, int mem, bool pack)
{
    const long long plane = (long long)h->cfg.n[0] * h->cfg.n[1], blk = (long long)h->G * plane;
    const int z0 = pack ? (side ? h->zhi - h->G : h->zlo) : (side ? h->zhi : 0);
    double* f[16];
    const int n = level_fields(h, level, f);
    const cudaMemcpyKind kind = mem == HYDRO_MEM_DEVICE ? cudaMemcpyDeviceToDevice
                                                        : (pack ? cudaMemcpyDeviceToHost : cudaMemcpyHostToDevice);
    for (int k = 0; k < n; ++k) {
        double* dst = pack ? out + k * blk : f[k] + z0 * plane;
        const double* src = pack ? f[k] + z0 * plane : in + k * blk;
        CK(h, cudaMemcpyAsync(dst, src, sizeof(double) * blk, kind, h->stream), "halo copy");
    }
    if (mem == HYDRO_MEM_HOST) CK(h, cudaStreamSynchronize(h->stream), "synchronize");
    return HYDRO_OK;
}

hydro_status hydro_halo_pack(hydro_t* h, int32_t level, int32_t side, double* buf, int32_t mem)
{
    hydro_status s = halo_args(h, level, side, mem, buf);
    return s ? s : halo_copy(h, level, side, buf, nullptr, mem, true);
}

hydro_status hydro_halo_unpack(hydro_t* h, int32_t level, int32_t side, const double* buf, int32_t mem)
{
    hydro_status s = halo_args(h, level, side, mem, buf);
    return s ? s : halo_copy(h, level, side, nullptr, buf, mem, false);
}

hydro_status hydro_halo_fill_outflow(hydro_t* h, int32_t level, int32_t side)
{
    hydro_status s = halo_args(h, level, side, HYDRO_MEM_DEVICE, h);
    if (s) return s;
    FieldList fl{};
    fl.n = level_fields(h, level, fl.f);
    const long long plane = (long long)h->cfg.n[0] * h->cfg.n[1];
    const long long src = (long long)(side ? h->zhi - 1 : h->zlo) * plane;
    const long long dst = (long long)(side ? h->zhi : 0) * plane;
    halo_replicate_kernel<<<blocks_for((long long)fl.n * h->G * plane), 256, 0, h->stream>>>(fl, plane, src, dst, h->G);
    CK(h, cudaGetLastError(), "halo fill");
    return HYDRO_OK;
}

hydro_status hydro_stage(hydro_t* h, int32_t which, double t_end)
{
    if (!h) return HYDRO_ERR_INVALID_ARG;
    if (!is_halo(h)) return fail(h, HYDRO_ERR_INVALID_ARG, "hydro_stage drives halo (bc[2] = HYDRO_BC_HALO) handles only");
    if (which < 0 || which > 4) return fail(h, HYDRO_ERR_INVALID_ARG, "which must be 0..4");
    if (!h->have_state) return fail(h, HYDRO_ERR_STATE, "no state loaded");
    if (which == 0) {
        set_t_end_kernel<<<1, 1, 0, h->stream>>>(h->ctl, t_end);
        step_begin_kernel<<<1, 1, 0, h->stream>>>(h->ctl, step_params(h->cfg));
    } else if (which == 4) {
        step_end_kernel<<<1, 1, 0, h->stream>>>(h->ctl);
    } else {
        CK(h, launch_stage(h, h->L, h->zc, stage_args(h, which), h->stream), "stage launch");
    }
    CK(h, cudaGetLastError(), "stage launch");
    return HYDRO_OK;
}

hydro_status hydro_speed_slot(hydro_t* h, int32_t slot, int32_t io, double* speeds, int32_t mem)
{
    if (!h) return HYDRO_ERR_INVALID_ARG;
    if (slot < 0 || slot > 3 || (io != 0 && io != 1) || !speeds ||
        (mem != HYDRO_MEM_HOST && mem != HYDRO_MEM_DEVICE))
        return fail(h, HYDRO_ERR_INVALID_ARG, "bad speed-slot arguments");
    unsigned long long* p = slot == 0 ? h->ctl->a_cur : slot == 1 ? h->ctl->a_s1 : slot == 2 ? h->ctl->a_s2 : h->ctl->a_next;
    // the slot holds the IEEE bits of non-negative doubles (ordered like the values)
    const cudaMemcpyKind kind = mem == HYDRO_MEM_DEVICE ? cudaMemcpyDeviceToDevice
                                                        : (io ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost);
    if (io) CK(h, cudaMemcpyAsync(p, speeds, 3 * sizeof(double), kind, h->stream), "speed slot write");
    else CK(h, cudaMemcpyAsync(speeds, p, 3 * sizeof(double), kind, h->stream), "speed slot read");
    if (mem == HYDRO_MEM_HOST) CK(h, cudaStreamSynchronize(h->stream), "synchronize");
    return HYDRO_OK;
}

__global__ void set_dt_kernel(Ctl* c, double dt) { c->dt = dt; }

static hydro_status apply_launch(hydro_t* h, int variant, int zc)
{
    StageLaunch L{};
    cudaError_t e = stage_launch_variant(h->R, h->cfg.split, h->cfg.nq, variant, &L, h->cfg.charwise);
    if (e == cudaErrorInvalidValue) return fail(h, HYDRO_ERR_INVALID_ARG, "no such launch variant");
    CK(h, e, "stage kernel setup");
    if (!launch_fits(h, L))
        return fail(h, HYDRO_ERR_INVALID_ARG,
                    "launch variant does not fit this grid (TMA-staged variants need an even nx)");
    CK(h, cudaStreamSynchronize(h->stream), "synchronize");
    if (h->exec) {
        cudaGraphExecDestroy(h->exec);
        h->exec = nullptr;
    }
    h->L = L;
    h->variant = variant;
    h->zc = zc > 0 ? (zc < h->cfg.n[2] ? zc : h->cfg.n[2]) : pick_zc(h->cfg.n[0], h->cfg.n[1], h->cfg.n[2], L, h->sms);
    return build_graph(h);
}

static std::string tune_key(const hydro_t* h)
{
    char b[96];
    snprintf(b, sizeof b, "%d %d %d %d", h->R * 10 + h->cfg.split + 100 * h->cfg.nq + 1000 * h->cfg.charwise,
             h->cfg.n[0], h->cfg.n[1], h->cfg.n[2]);
    return b;
}

static bool tune_cache_lookup(const hydro_t* h, int* variant, int* zc)
{
    const char* path = getenv("HYDRO_TUNE_CACHE");
    if (!path || !*path) return false;
    FILE* f = fopen(path, "r");
    if (!f) return false;
    const std::string key = tune_key(h);
    char line[256];
    bool found = false;
    while (fgets(line, sizeof line, f)) {
        int R, nx, ny, nz, v, z;
        if (sscanf(line, "%d %d %d %d %d %d", &R, &nx, &ny, &nz, &v, &z) == 6) {
            char k[96];
            snprintf(k, sizeof k, "%d %d %d %d", R, nx, ny, nz);
            if (key == k) {
                *variant = v;
                *zc = z;
                found = true;   // the last matching line wins
            }
        }
    }
    fclose(f);
    return found;
}

static void tune_cache_store(const hydro_t* h, int variant, int zc)
{
    const char* path = getenv("HYDRO_TUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d %d\n", tune_key(h).c_str(), variant, zc);
    fclose(f);
}

extern "C" int32_t hydro_launch_variants(int32_t scheme, int32_t split, int32_t nq)
{
    if (split != 0 && split != 1) return 0;
    if (nq < 0 || nq > 3) return 0;
    if (scheme == HYDRO_WENO5 || scheme == HYDRO_WENO7 || scheme == HYDRO_MUSTA_FORCE)
        return launch_variant_count(scheme_R(scheme), split, nq);
    return 0;
}

extern "C" int32_t hydro_launch_variants_cfg(const hydro_config* cfg)
{
    if (!check_config(cfg).empty()) return 0;
    return launch_variant_count(scheme_R(cfg->scheme), cfg->split, cfg->nq, cfg->charwise);
}

extern "C" int32_t hydro_kernels_per_step(hydro_t* h)
{
    if (!h) return 0;
    const bool zpass = h->L.zfn && axis_active(h->cfg, 2);
    int per_stage = 1 + (zpass ? 1 : 0);
    if (h->L.combine) per_stage += (axis_active(h->cfg, 0) ? 1 : 0) + (axis_active(h->cfg, 1) ? 1 : 0);
    return 2 + 3 * per_stage;
}

extern "C" hydro_status hydro_set_launch(hydro_t* h, int32_t variant, int32_t zc)
{
    if (!h) return HYDRO_ERR_INVALID_ARG;
    if (variant < 0 || variant >= hydro_launch_variants_cfg(&h->cfg))
        return fail(h, HYDRO_ERR_INVALID_ARG, "no such launch variant");
    return apply_launch(h, variant, zc);
}

extern "C" hydro_status hydro_get_launch(hydro_t* h, int32_t* variant, int32_t* tile_x, int32_t* tile_y, int32_t* zc)
{
    if (!h) return HYDRO_ERR_INVALID_ARG;
    if (variant) *variant = h->variant;
    if (tile_x) *tile_x = h->L.tx;
    if (tile_y) *tile_y = h->L.ty;
    if (zc) *zc = h->zc;
    return HYDRO_OK;
}

extern "C" hydro_status hydro_autotune(hydro_t* h, double* best_ms)
{
    if (!h) return HYDRO_ERR_INVALID_ARG;
    if (h->cfg.bc[2] == HYDRO_BC_HALO) return fail(h, HYDRO_ERR_INVALID_ARG, "hydro_autotune runs whole grids (no z halo)");
    if (!h->have_state) return fail(h, HYDRO_ERR_STATE, "no state loaded");
    int cv = 0, cz = 0;
    if (tune_cache_lookup(h, &cv, &cz) && cv >= 0 && cv < hydro_launch_variants_cfg(&h->cfg)) {
        if (best_ms) *best_ms = -1.0;
        return apply_launch(h, cv, cz);
    }
    cudaEvent_t e0, e1;
    CK(h, cudaEventCreate(&e0), "event");
    CK(h, cudaEventCreate(&e1), "event");
    double best = 1e300;
    int bv = h->variant, bz = h->zc;
    hydro_status st = HYDRO_OK;
    const int nz = h->cfg.n[2];
    // a positive dt makes the stage kernel run; it only writes stage-1 scratch
    set_dt_kernel<<<1, 1, 0, h->stream>>>(h->ctl, 1e-300);
    for (int v = 0; v < hydro_launch_variants_cfg(&h->cfg) && st == HYDRO_OK; ++v) {
        StageLaunch L{};
        if (stage_launch_variant(h->R, h->cfg.split, h->cfg.nq, v, &L, h->cfg.charwise) != cudaSuccess) continue;
        if (!launch_fits(h, L)) continue;
        // z chunks: balanced splits ceil(nz/k) and a fixed ladder; time the five
        // the wave-count model likes best
        std::vector<int> zs;
        if (L.combine) {
            zs.push_back(nz);     // three-pass launches have no z chunks: one trial
        } else {
            for (int k = 1; k <= 64; ++k) zs.push_back((nz + k - 1) / k);
            for (int z : {8, 12, 16, 24, 32, 48, 64}) zs.push_back(z);
        }
        std::vector<std::pair<double, int>> scored;
        const long long tiles = (long long)((h->cfg.n[0] + L.tx - 1) / L.tx) * ((h->cfg.n[1] + L.ty - 1) / L.ty);
        const long long conc = (long long)h->sms * (L.ctas_per_sm > 0 ? L.ctas_per_sm : 1);
        for (int z : zs) {
            if (z < 1 || z > nz || (z < 8 && nz >= 8)) continue;
            bool dup = false;
            for (auto& q : scored) dup |= (q.second == z);
            if (dup) continue;
            const long long ctas = tiles * ((nz + z - 1) / z);
            const double cost = (double)((ctas + conc - 1) / conc) * (z + zc_prologue(L));
            scored.push_back({cost, z});
        }
        std::sort(scored.begin(), scored.end());
        if (scored.size() > 5) scored.resize(5);
        for (auto& cz : scored) {
            const int zc = cz.second;
            h->L = L;
            h->zc = zc;
            const StageArgs a = stage_args(h, 1);
            cudaError_t el = launch_stage(h, L, zc, a, h->stream);   // warm-up
            cudaEventRecord(e0, h->stream);
            if (el == cudaSuccess) el = launch_stage(h, L, zc, a, h->stream);
            cudaEventRecord(e1, h->stream);
            cudaError_t e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = el;
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e != cudaSuccess) {
                st = cuda_fail(h, e, "autotune");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                bv = v;
                bz = zc;
            }
        }
    }
    set_dt_kernel<<<1, 1, 0, h->stream>>>(h->ctl, 0.0);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != HYDRO_OK) return st;
    if (best_ms) *best_ms = best;
    tune_cache_store(h, bv, bz);
    return apply_launch(h, bv, bz);
}

static hydro_status read_ctl(hydro_t* h)
{
    CK(h, cudaMemcpyAsync(h->hctl, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->stream), "read control");
    CK(h, cudaStreamSynchronize(h->stream), "synchronize");
    if (h->hctl->status == HYDRO_ERR_TIMEOUT)
        return fail(h, HYDRO_ERR_TIMEOUT, "a stage kernel's wait for its TMA tile load ran out of time; results are invalid");
    if (h->hctl->status) {
        char b[160];
        snprintf(b, sizeof b, "unphysical state (E <= 0, |M| >= E or NaN) first seen at cell %lld",
                 (long long)h->hctl->bad_cell);
        return fail(h, HYDRO_ERR_UNPHYSICAL, b);
    }
    return HYDRO_OK;
}

hydro_status hydro_sync(hydro_t* h)
{
    if (!h) return HYDRO_ERR_INVALID_ARG;
    return read_ctl(h);
}

// staging buffers, copy streams and events of hydro_run_many
static hydro_status run_many_setup(hydro_t* h)
{
    if (h->io_buf) return HYDRO_OK;
    const size_t state = sizeof(double) * (size_t)h->fs * h->nf;
    CK(h, cudaMalloc(&h->io_buf, 3 * state), "staging buffers");
    CK(h, cudaMalloc(&h->run_st, sizeof(RunStatus)), "run status");
    CK(h, cudaMallocHost(&h->hrun_st, sizeof(RunStatus)), "pinned run status");
    CK(h, cudaStreamCreateWithFlags(&h->s_in, cudaStreamNonBlocking), "copy-in stream");
    CK(h, cudaStreamCreateWithFlags(&h->s_out, cudaStreamNonBlocking), "copy-out stream");
    for (cudaEvent_t* ev : {&h->ev_in[0], &h->ev_in[1], &h->ev_used[0], &h->ev_used[1], &h->ev_out_ready, &h->ev_out_free})
        CK(h, cudaEventCreateWithFlags(ev, cudaEventDisableTiming), "event");
    return HYDRO_OK;
}

hydro_status hydro_run_many(hydro_t* h, int32_t n_items, const double* const* u_in, double* const* u_out,
                            int64_t field_stride, int32_t nsteps, double t0, double t_end)
{
    if (!h) return HYDRO_ERR_INVALID_ARG;
    if (h->cfg.bc[2] == HYDRO_BC_HALO) return fail(h, HYDRO_ERR_INVALID_ARG, "a halo slab steps through hydro_stage");
    if (n_items < 0 || nsteps < 0) return fail(h, HYDRO_ERR_INVALID_ARG, "n_items and nsteps must be >= 0");
    if (n_items == 0) return HYDRO_OK;
    if (!u_in || !u_out) return fail(h, HYDRO_ERR_INVALID_ARG, "NULL item list");
    if (field_stride < h->ncell) return fail(h, HYDRO_ERR_INVALID_ARG, "field_stride smaller than the cell count");
    for (int i = 0; i < n_items; ++i)
        if (!u_in[i] || !u_out[i]) return fail(h, HYDRO_ERR_INVALID_ARG, "NULL data pointer in the item list");
    hydro_status st = run_many_setup(h);
    if (st) return st;
    const size_t fbytes = sizeof(double) * (size_t)h->ncell;
    const size_t sbytes = sizeof(double) * (size_t)h->fs * h->nf;     // one whole state, padding included
    double* const stage_in[2] = {h->io_buf, h->io_buf + (size_t)h->fs * h->nf};
    double* const stage_out = h->io_buf + 2 * (size_t)h->fs * h->nf;
    cudaStream_t s = h->stream;
    CK(h, cudaMemsetAsync(h->run_st, 0, sizeof(RunStatus), s), "run status");
    auto copy_in = [&](int i, int b) -> hydro_status {
        for (int f = 0; f < h->nf; ++f)
            CK(h, cudaMemcpyAsync(stage_in[b] + (size_t)f * h->fs, u_in[i] + (size_t)f * field_stride, fbytes,
                                  cudaMemcpyHostToDevice, h->s_in), "copy in");
        CK(h, cudaEventRecord(h->ev_in[b], h->s_in), "event");
        return HYDRO_OK;
    };
    // the copy-in stream starts after everything already queued on the handle's stream
    CK(h, cudaEventRecord(h->ev_used[1], s), "event");
    CK(h, cudaStreamWaitEvent(h->s_in, h->ev_used[1], 0), "wait");
    CK(h, cudaStreamWaitEvent(h->s_out, h->ev_used[1], 0), "wait");
    if ((st = copy_in(0, 0))) return st;
    for (int i = 0; i < n_items; ++i) {
        const int b = i & 1;
        if (i + 1 < n_items) {
            // prefetch item i+1 into the buffer item i-1 came through, once the
            // state has taken it
            CK(h, cudaStreamWaitEvent(h->s_in, h->ev_used[b ^ 1], 0), "wait");
            if ((st = copy_in(i + 1, b ^ 1))) return st;
        }
        CK(h, cudaStreamWaitEvent(s, h->ev_in[b], 0), "wait");
        CK(h, cudaMemcpyAsync(h->U[0], stage_in[b], sbytes, cudaMemcpyDeviceToDevice, s), "load item");
        CK(h, cudaEventRecord(h->ev_used[b], s), "event");
        if ((st = after_load(h, t0))) return st;
        set_t_end_kernel<<<1, 1, 0, s>>>(h->ctl, t_end);
        CK(h, cudaGetLastError(), "set t_end");
        for (int k = 0; k < nsteps; ++k) CK(h, cudaGraphLaunch(h->exec, s), "graph launch");
        run_status_kernel<<<1, 1, 0, s>>>(h->ctl, h->run_st, i);
        CK(h, cudaGetLastError(), "run status");
        // result out through the staging buffer, once item i-1's copy-out is done
        CK(h, cudaStreamWaitEvent(s, h->ev_out_free, 0), "wait");
        CK(h, cudaMemcpyAsync(stage_out, h->U[0], sbytes, cudaMemcpyDeviceToDevice, s), "store item");
        CK(h, cudaEventRecord(h->ev_out_ready, s), "event");
        CK(h, cudaStreamWaitEvent(h->s_out, h->ev_out_ready, 0), "wait");
        for (int f = 0; f < h->nf; ++f)
            CK(h, cudaMemcpyAsync(u_out[i] + (size_t)f * field_stride, stage_out + (size_t)f * h->fs, fbytes,
                                  cudaMemcpyDeviceToHost, h->s_out), "copy out");
        CK(h, cudaEventRecord(h->ev_out_free, h->s_out), "event");
    }
    CK(h, cudaMemcpyAsync(h->hrun_st, h->run_st, sizeof(RunStatus), cudaMemcpyDeviceToHost, s), "read run status");
    CK(h, cudaStreamSynchronize(h->s_out), "synchronize");
    CK(h, cudaStreamSynchronize(h->s_in), "synchronize");
    CK(h, cudaStreamSynchronize(s), "synchronize");
    if (h->hrun_st->status == HYDRO_ERR_TIMEOUT)
        return fail(h, HYDRO_ERR_TIMEOUT, "a stage kernel's wait for its TMA tile load ran out of time; results are invalid");
    if (h->hrun_st->status) {
        char msg[200];
        snprintf(msg, sizeof msg, "unphysical state (E <= 0, |M| >= E or NaN) in item %d, first seen at cell %lld",
                 h->hrun_st->item, (long long)h->hrun_st->bad_cell);
        return fail(h, HYDRO_ERR_UNPHYSICAL, msg);
    }
    return HYDRO_OK;
}

hydro_status hydro_get_state(hydro_t* h, double* u, int64_t field_stride, int32_t mem, double* t, int64_t* step)
{
    hydro_status s = check_io(h, u, field_stride, mem);
    if (s) return s;
    s = copy_fields(h, u, field_stride, h->U[0] + h->off, h->fs, h->nf,
                    mem == HYDRO_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice);
    if (s) return s;
    s = read_ctl(h);
    if (t) *t = h->hctl->t;
    if (step) *step = h->hctl->step;
    return s;
}

hydro_status hydro_get_primitive(hydro_t* h, double* w, int64_t field_stride, int32_t mem)
{
    hydro_status s = check_io(h, w, field_stride, mem);
    if (s) return s;
    state_to_prim_kernel<<<blocks_for(h->ncell), 256, 0, h->stream>>>(h->U[0] + h->off, h->fs, h->U[1] + h->off,
                                                                      h->fs, h->ncell, h->cfg.cs2, h->nf,
                                                                      h->cfg.eos_mass);
    CK(h, cudaGetLastError(), "state_to_prim");
    s = copy_fields(h, w, field_stride, h->U[1] + h->off, h->fs, h->nf,
                    mem == HYDRO_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice);
    if (s) return s;
    return read_ctl(h);
}

hydro_status hydro_get_speeds(hydro_t* h, double alpha[3], double* last_dt)
{
    if (!h) return HYDRO_ERR_INVALID_ARG;
    hydro_status s = read_ctl(h);
    if (alpha)
        for (int d = 0; d < 3; ++d) {
            unsigned long long b = h->hctl->a_cur[d];
            double v;
            memcpy(&v, &b, sizeof v);
            alpha[d] = v;
        }
    if (last_dt) *last_dt = h->hctl->last_dt;
    return s;
}

const double* hydro_state_device_ptr(hydro_t* h) { return h ? h->U[0] + h->off : nullptr; }
int64_t hydro_field_stride(hydro_t* h) { return h ? h->fs : 0; }

}  // extern "C"
