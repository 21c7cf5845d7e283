// hydro_batch.cu -- event-by-event ensembles: many independent grids of
// uneven size advanced together (the paper's motivation, Sec. 1: event-by-
// event simulations of flow fluctuations).
//
// Every RK3 stage of all events is ONE persistent launch: sms x (CTAs per SM)
// CTAs pop (event, tile x, tile y, z chunk) items from a precomputed work-list
// with one atomicAdd each and run the same per-item stage code as the single-
// grid kernel.  Each event keeps its own buffers, Lax-Friedrichs speeds and
// time step.  A step (per-event step-begin, three persistent stages, per-event
// step-end) is captured once as a CUDA graph and replayed.  The work-list
// counters are plain atomics; no CTA ever waits for another.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "hydro_common.cuh"

namespace hydro {

struct BatchEvent {
    double* U[3];
    double* W[3];
    double* S[3];             // per-axis speeds (local LF only)
    double* fz;               // z-face fluxes (z-pass variants): 5 fields of nz + 1 face planes
    long long fzs;
    double* fx;               // x- and y-face fluxes (three-pass variants), layouts as in StageArgs
    long long fxs;
    double* fy;
    long long fys;
    long long fs, ncell;
    int n[3], bc[3], act[3];
    double hdx[3];
    double cs2, eps_s;
    StepParams sp;
    Ctl* ctl;
};

struct BatchArgs {
    const BatchEvent* ev;
    const int4* items;        // (event, tile x, tile y, z chunk)
    int n_items;
    const int4* zitems;       // z pass: (event, column block of 32, unused, face chunk)
    const int4* xitems;       // three-pass variants: x and y passes (event, pencil block, unused, face
    const int4* yitems;       // chunk) and the combination (event, block of kCombineCells cells)
    const int4* citems;
    unsigned int* counter;    // this stage's work-list counter (zeroed by step-begin)
    int stage;                // 1, 2, 3
    int zc;
};

__device__ __forceinline__ StageArgs batch_stage_args(const BatchEvent& E, int stage, int zc)
{
    StageArgs a{};
    const int in = stage - 1;
    a.u_in = E.U[in];
    a.w_in = E.W[in];
    a.u_n = E.U[0];
    a.u_out = stage == 3 ? E.U[0] : E.U[stage];
    a.w_out = stage == 3 ? E.W[0] : E.W[stage];
    a.fs = E.fs;
    a.nx = E.n[0];
    a.ny = E.n[1];
    a.nz = E.n[2];
    a.zc = zc;
    a.zlo = 0;
    a.zhi = E.n[2];
    for (int d = 0; d < 3; ++d) {
        a.bc[d] = E.bc[d];
        a.act[d] = E.act[d];
        a.hdx[d] = E.hdx[d];
    }
    a.cs2 = E.cs2;
    a.eps_s = E.eps_s;
    a.ca = stage == 1 ? 0.0 : (stage == 2 ? 0.75 : 1.0 / 3.0);
    a.cb = stage == 1 ? 1.0 : (stage == 2 ? 0.25 : 2.0 / 3.0);
    a.alpha_in = stage == 1 ? E.ctl->a_cur : (stage == 2 ? E.ctl->a_s1 : E.ctl->a_s2);
    a.alpha_out = stage == 1 ? E.ctl->a_s1 : (stage == 2 ? E.ctl->a_s2 : E.ctl->a_next);
    a.dt = &E.ctl->dt;
    a.status = &E.ctl->status;
    a.bad_cell = &E.ctl->bad_cell;
    a.s_in = E.S[in];
    a.s_out = stage == 3 ? E.S[0] : E.S[stage];
    a.fz = E.fz;
    a.fzs = E.fzs;
    a.fx = E.fx;
    a.fxs = E.fxs;
    a.fy = E.fy;
    a.fys = E.fys;
    return a;
}

template <int R, int TX, int TY, int ILP = 1, bool LLF = false, int EMU = default_emu(R, TX, TY, LLF, 5, false),
          bool ZEXT = false, int MINB = 0>
__global__ void __launch_bounds__(TX * TY, (MINB > 0 ? MINB : (TX * TY <= 128 && R == 3 ? 2 : 1)))
    batch_stage_kernel(const BatchArgs b)
{
    extern __shared__ __align__(16) double smem[];
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(b.counter, 1u);
        __syncthreads();
        const int it = s_item;
        __syncthreads();   // everyone has read s_item before thread 0 overwrites it
        if (it >= b.n_items) break;
        const int4 w = b.items[it];
        const StageArgs a = batch_stage_args(b.ev[w.x], b.stage, b.zc);
        stage_tile<R, TX, TY, ILP, LLF, 5, false, EMU, ZEXT>(a, w.y, w.z, w.w, smem);
    }
}

// z pass of all events (z-pass variants): one CTA per z item
template <int R, int EMU>
__global__ void __launch_bounds__(kZPassThreads, R == 4 ? 3 : 4) batch_zflux_kernel(const BatchArgs b)
{
    const int4 w = b.zitems[blockIdx.x];
    const StageArgs a = batch_stage_args(b.ev[w.x], b.stage, b.zc);
    zflux_item<R, EMU>(a, w.y, w.w, w.z);
}

// three-pass variants: x and y passes of all events (one CTA per item) and the
// combination (one CTA per block of kCombineCells cells of one event)
template <int R, int EMU, int AX>
__global__ void __launch_bounds__(kZPassThreads, R == 4 ? 3 : 4) batch_axis_flux_kernel(const BatchArgs b)
{
    const int4 w = (AX == 0 ? b.xitems : b.yitems)[blockIdx.x];
    const StageArgs a = batch_stage_args(b.ev[w.x], b.stage, b.zc);
    axis_flux_item<R, EMU, AX>(a, w.y, w.w, w.z);
}

constexpr int kCombineCells = 2048;

template <int NF = 5>
__global__ void __launch_bounds__(256) batch_combine_kernel(const BatchArgs b)
{
    const int4 w = b.citems[blockIdx.x];
    const BatchEvent& E = b.ev[w.x];
    const StageArgs a = batch_stage_args(E, b.stage, b.zc);
    const long long c0 = (long long)w.y * kCombineCells;
    const long long c1 = c0 + kCombineCells < E.ncell ? c0 + kCombineCells : E.ncell;
    combine_cells<NF>(a, c0 + threadIdx.x, c1, blockDim.x);
}

__global__ void batch_step_begin_kernel(const BatchEvent* ev, int n, unsigned int* counters)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e == 0) counters[0] = counters[1] = counters[2] = 0u;
    if (e >= n) return;
    Ctl* c = ev[e].ctl;
    const StepParams sp = ev[e].sp;
    double amax = 0.0;
    for (int d = 0; d < 3; ++d)
        if (sp.actmask & (1 << d)) amax = fmax(amax, __longlong_as_double((long long)c->a_cur[d]));
    double dt = sp.dt_fixed > 0.0 ? sp.dt_fixed : sp.cfl * sp.mindx / amax;
    if (c->t_end >= 0.0 && c->t + dt > c->t_end) dt = c->t_end - c->t;
    if (!(dt > 0.0)) dt = 0.0;
    c->dt = dt;
    for (int d = 0; d < 3; ++d) c->a_s1[d] = c->a_s2[d] = c->a_next[d] = 0ull;
}

__global__ void batch_step_end_kernel(const BatchEvent* ev, int n)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    Ctl* c = ev[e].ctl;
    if (c->dt > 0.0) {
        for (int d = 0; d < 3; ++d) c->a_cur[d] = c->a_next[d];
        c->t += c->dt;
        c->last_dt = c->dt;
        c->step += 1;
    }
}

struct BatchLaunch {
    void (*fn)(BatchArgs);
    size_t smem;
    int tx, ty, ctas_per_sm;
    void (*zfn)(BatchArgs) = nullptr;   // z pass before fn (z-pass variants)
    void (*xfn)(BatchArgs) = nullptr;   // three-pass variants: x and y passes, fn is the combination
    void (*yfn)(BatchArgs) = nullptr;
    bool combine = false;
};

template <int R, int ZEMU>
static cudaError_t batch_info_for_three(BatchLaunch* out)
{
    out->fn = batch_combine_kernel<5>;
    out->xfn = batch_axis_flux_kernel<R, ZEMU, 0>;
    out->yfn = batch_axis_flux_kernel<R, ZEMU, 1>;
    out->zfn = batch_zflux_kernel<R, ZEMU>;
    out->combine = true;
    out->smem = 0;
    out->tx = 16;
    out->ty = 16;
    out->ctas_per_sm = 1;
    return cudaSuccess;
}

template <int R, int TX, int TY, int ILP = 1, bool LLF = false, int EMU = default_emu(R, TX, TY, LLF, 5, false),
          bool ZEXT = false, int ZEMU = EMU, int MINB = 0>
static cudaError_t batch_info_for(BatchLaunch* out)
{
    auto fn = batch_stage_kernel<R, TX, TY, ILP, LLF, EMU, ZEXT, MINB>;
    out->fn = fn;
    out->zfn = nullptr;
    if constexpr (ZEXT) out->zfn = batch_zflux_kernel<R, ZEMU>;
    out->smem = StageSmem<R, TX, TY, LLF, 5, false, ILP == kPencilSweep, ZEXT>::bytes;
    out->tx = TX;
    out->ty = TY;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)out->smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&out->ctas_per_sm, fn, TX * TY, out->smem);
}

// same tile shapes as the single-grid kernel (variant numbering matches)
static cudaError_t batch_launch_variant(int R, int split, int v, BatchLaunch* out)
{
    if (split == 1) {
        if (R == 3 && v == 0) return batch_info_for<3, 16, 16, 1, true>(out);
        if (R == 3 && v == 1) return batch_info_for<3, 16, 8, 1, true>(out);
        if (R == 4 && v == 0) return batch_info_for<4, 16, 8, 1, true>(out);
        return cudaErrorInvalidValue;
    }
    if (R == 3) {
        if (v == 0) return batch_info_for<3, 16, 16>(out);
        if (v == 1) return batch_info_for<3, 16, 8>(out);
        if (v == 2) return batch_info_for<3, 32, 8>(out);
        if (v == 3) return batch_info_for<3, 16, 16, 2>(out);
        if (v == 4) return batch_info_for<3, 16, 16, kPencilSweep, false, 0>(out);
        if (v == 5) return batch_info_for<3, 16, 8, kPencilSweep>(out);
        if (v == 6) return batch_info_for<3, 16, 16, kPencilSweep>(out);
        if (v == 7) return batch_info_for<3, 16, 16, kPencilSweep, false, kEmuConst, true, kZPassEmu5>(out);
        if (v == 8)
            return batch_info_for<3, 16, 16, kPencilSweep, false, kEmuConst | kEmuWeights, true, kZPassEmu5, 2>(out);
        if (v == 9) return batch_info_for_three<3, kZPassEmu5>(out);
    }
    if (R == 4) {
        if (v == 0) return batch_info_for<4, 16, 16>(out);
        if (v == 1) return batch_info_for<4, 16, 8>(out);
        if (v == 2) return batch_info_for<4, 16, 16, 2>(out);
        if (v == 3) return batch_info_for<4, 16, 16, kPencilSweep, false, 0>(out);
        if (v == 4) return batch_info_for<4, 16, 8, kPencilSweep>(out);
        if (v == 5) return batch_info_for<4, 16, 16, kPencilSweep>(out);
        if (v == 6) return batch_info_for<4, 16, 16, kPencilSweep, false, kEmuConst, true, kZPassEmu7>(out);
        if (v == 7) return batch_info_for<4, 16, 16, kPencilSweep, false, kEmuConst, true, kZPassEmu7, 2>(out);
        if (v == 8) return batch_info_for_three<4, kZPassEmu7>(out);
    }
    return cudaErrorInvalidValue;
}

}  // namespace hydro

using namespace hydro;

struct hydro_batch_s {
    int n_events = 0;
    int R = 3;
    int dev = 0, sms = 0;
    cudaStream_t stream = nullptr, cap = nullptr;
    std::vector<hydro_config> cfg;
    std::vector<BatchEvent> ev;      // host copy
    BatchEvent* d_ev = nullptr;
    double* buf = nullptr;
    Ctl* ctl = nullptr;              // n_events control blocks
    Ctl* hctl = nullptr;             // pinned mirror
    unsigned int* counters = nullptr;
    int4* d_items = nullptr;
    int n_items = 0;
    int4* d_zitems = nullptr;        // z-pass items (z-pass variants)
    int n_zitems = 0;
    int4* d_xitems = nullptr;        // three-pass variants: x-, y-pass and combination items
    int n_xitems = 0;
    int4* d_yitems = nullptr;
    int n_yitems = 0;
    int4* d_citems = nullptr;
    int n_citems = 0;
    BatchLaunch L{};
    int variant = 0, zc = 16;
    cudaGraphExec_t exec = nullptr;
    std::vector<char> loaded;
    std::string err;
};

static thread_local std::string g_batch_create_err;

static hydro_status bfail(hydro_batch_t* b, hydro_status s, const std::string& m)
{
    if (b) b->err = m;
    else g_batch_create_err = m;
    return s;
}

static hydro_status bcuda(hydro_batch_t* b, cudaError_t e, const char* where)
{
    return bfail(b, e == cudaErrorMemoryAllocation ? HYDRO_ERR_OOM : HYDRO_ERR_CUDA,
                 std::string(where) + ": " + cudaGetErrorString(e));
}

#define BCK(b, call, where)                                    \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return bcuda((b), e_, where);   \
    } while (0)

// work-list: every (tile, chunk) of every event, largest events first
static hydro_status build_items(hydro_batch_t* b)
{
    std::vector<int> order(b->n_events);
    for (int e = 0; e < b->n_events; ++e) order[e] = e;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->ev[x].ncell > b->ev[y].ncell; });
    std::vector<int4> items;
    for (int e : order) {
        const int* n = b->ev[e].n;
        const int gx = (n[0] + b->L.tx - 1) / b->L.tx, gy = (n[1] + b->L.ty - 1) / b->L.ty;
        const int gz = (n[2] + b->zc - 1) / b->zc;
        for (int z = 0; z < gz; ++z)
            for (int y = 0; y < gy; ++y)
                for (int x = 0; x < gx; ++x) items.push_back(make_int4(e, x, y, z));
    }
    if (b->d_items) {
        cudaFree(b->d_items);
        b->d_items = nullptr;
    }
    b->n_items = (int)items.size();
    BCK(b, cudaMalloc(&b->d_items, sizeof(int4) * items.size()), "work-list");
    BCK(b, cudaMemcpy(b->d_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice), "work-list copy");
    // z-pass items: (event, block of 32 consecutive columns of the plane,
    // faces per chunk, chunk) of every event with an active z axis
    if (b->d_zitems) {
        cudaFree(b->d_zitems);
        b->d_zitems = nullptr;
    }
    b->n_zitems = 0;
    if (b->L.zfn) {
        std::vector<int4> zi;
        for (int e : order) {
            const int* n = b->ev[e].n;
            if (!b->ev[e].act[2]) continue;
            const long long gc = zpass_blocks(n[0], n[1]);
            const int gz = face_chunks(n[2] + 1), len = chunk_len(n[2] + 1, gz);
            if (gc > 0x7fffffffLL) return bfail(b, HYDRO_ERR_INVALID_ARG, "event too large for the z pass");
            for (int z = 0; z < gz; ++z)
                for (long long c = 0; c < gc; ++c) zi.push_back(make_int4(e, (int)c, len, z));
        }
        b->n_zitems = (int)zi.size();
        if (!zi.empty()) {
            BCK(b, cudaMalloc(&b->d_zitems, sizeof(int4) * zi.size()), "z work-list");
            BCK(b, cudaMemcpy(b->d_zitems, zi.data(), sizeof(int4) * zi.size(), cudaMemcpyHostToDevice),
                "z work-list copy");
        }
    }
    // three-pass variants: x- and y-pass items (event, pencil block, faces per
    // chunk, chunk) of the events with that axis active, and the combination items
    // (event, block of kCombineCells cells)
    int4** dl[3] = {&b->d_xitems, &b->d_yitems, &b->d_citems};
    int* nl[3] = {&b->n_xitems, &b->n_yitems, &b->n_citems};
    for (int i = 0; i < 3; ++i) {
        if (*dl[i]) cudaFree(*dl[i]);
        *dl[i] = nullptr;
        *nl[i] = 0;
    }
    if (b->L.combine) {
        std::vector<int4> li[3];
        for (int e : order) {
            const BatchEvent& E = b->ev[e];
            for (int ax = 0; ax < 2; ++ax) {
                if (!E.act[ax]) continue;
                const long long gc = pass_blocks(ax, E.n[0], E.n[1], E.n[2]);
                if (gc > 0x7fffffffLL) return bfail(b, HYDRO_ERR_INVALID_ARG, "event too large for the face passes");
                const int gf = face_chunks(E.n[ax] + 1), len = chunk_len(E.n[ax] + 1, gf);
                for (int f = 0; f < gf; ++f)
                    for (long long c = 0; c < gc; ++c) li[ax].push_back(make_int4(e, (int)c, len, f));
            }
            const long long nb = (E.ncell + kCombineCells - 1) / kCombineCells;
            for (long long c = 0; c < nb; ++c) li[2].push_back(make_int4(e, (int)c, 0, 0));
        }
        for (int i = 0; i < 3; ++i) {
            *nl[i] = (int)li[i].size();
            if (li[i].empty()) continue;
            BCK(b, cudaMalloc(dl[i], sizeof(int4) * li[i].size()), "pass work-list");
            BCK(b, cudaMemcpy(*dl[i], li[i].data(), sizeof(int4) * li[i].size(), cudaMemcpyHostToDevice),
                "pass work-list copy");
        }
    }
    return HYDRO_OK;
}

static BatchArgs batch_args(const hydro_batch_t* b, int stage)
{
    BatchArgs a;
    a.ev = b->d_ev;
    a.items = b->d_items;
    a.n_items = b->n_items;
    a.zitems = b->d_zitems;
    a.xitems = b->d_xitems;
    a.yitems = b->d_yitems;
    a.citems = b->d_citems;
    a.counter = b->counters + (stage - 1);
    a.stage = stage;
    a.zc = b->zc;
    return a;
}

// one stage of all events: the z pass (z-pass variants), then the persistent stage kernel
static void launch_batch_stage(const hydro_batch_t* b, const BatchArgs& a, cudaStream_t s)
{
    if (b->L.combine) {
        if (b->n_xitems > 0) b->L.xfn<<<b->n_xitems, kZPassThreads, 0, s>>>(a);
        if (b->n_yitems > 0) b->L.yfn<<<b->n_yitems, kZPassThreads, 0, s>>>(a);
        if (b->n_zitems > 0) b->L.zfn<<<b->n_zitems, kZPassThreads, 0, s>>>(a);
        if (b->n_citems > 0) b->L.fn<<<b->n_citems, 256, 0, s>>>(a);
        return;
    }
    if (b->L.zfn && b->n_zitems > 0) b->L.zfn<<<b->n_zitems, kZPassThreads, 0, s>>>(a);
    const int grid = b->sms * (b->L.ctas_per_sm > 0 ? b->L.ctas_per_sm : 1);
    b->L.fn<<<grid, b->L.tx * b->L.ty, b->L.smem, s>>>(a);
}

static cudaError_t enqueue_batch_step(hydro_batch_t* b, cudaStream_t s, cudaEvent_t* marks)
{
    const int eb = (b->n_events + 127) / 128;
    if (marks) cudaEventRecord(marks[0], s);
    batch_step_begin_kernel<<<eb, 128, 0, s>>>(b->d_ev, b->n_events, b->counters);
    if (marks) cudaEventRecord(marks[1], s);
    for (int k = 1; k <= 3; ++k) {
        launch_batch_stage(b, batch_args(b, k), s);
        if (marks) cudaEventRecord(marks[1 + k], s);
    }
    batch_step_end_kernel<<<eb, 128, 0, s>>>(b->d_ev, b->n_events);
    if (marks) cudaEventRecord(marks[5], s);
    return cudaGetLastError();
}

static hydro_status batch_graph(hydro_batch_t* b)
{
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    cudaGraph_t g = nullptr;
    BCK(b, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "capture begin");
    cudaError_t e1 = enqueue_batch_step(b, b->cap, nullptr);
    cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);
    if (e1 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bcuda(b, e1, "capture step");
    }
    BCK(b, e2, "capture end");
    cudaError_t e3 = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    BCK(b, e3, "graph instantiate");
    return HYDRO_OK;
}

static int batch_default_zc(const hydro_batch_t* b)
{
    // aim for at least ~8 items per resident CTA with chunks of >= 16 planes
    long long tiles = 0, cells = 0;
    for (const auto& E : b->ev) {
        tiles += (long long)((E.n[0] + b->L.tx - 1) / b->L.tx) * ((E.n[1] + b->L.ty - 1) / b->L.ty);
        cells += E.ncell;
    }
    const long long conc = (long long)b->sms * (b->L.ctas_per_sm > 0 ? b->L.ctas_per_sm : 1);
    long long mean_nz = cells / (tiles * b->L.tx * b->L.ty > 0 ? tiles * b->L.tx * b->L.ty : 1);
    int zc = 64;
    while (zc > 16 && tiles * ((mean_nz + zc - 1) / zc) < 8 * conc) zc /= 2;
    return zc;
}

static hydro_status apply_batch_launch(hydro_batch_t* b, int variant, int zc)
{
    BatchLaunch L{};
    cudaError_t e = batch_launch_variant(b->R, b->cfg[0].split, variant, &L);
    if (e == cudaErrorInvalidValue) return bfail(b, HYDRO_ERR_INVALID_ARG, "no such launch variant");
    BCK(b, e, "batch kernel setup");
    BCK(b, cudaStreamSynchronize(b->stream), "synchronize");
    b->L = L;
    b->variant = variant;
    b->zc = zc > 0 ? zc : batch_default_zc(b);
    hydro_status s = build_items(b);
    if (s) return s;
    return batch_graph(b);
}

extern "C" {

hydro_status hydro_batch_destroy(hydro_batch_t* b)
{
    if (!b) return HYDRO_OK;
    if (b->buf || b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->cap) cudaStreamDestroy(b->cap);
    cudaFree(b->buf);
    cudaFree(b->ctl);
    cudaFree(b->d_ev);
    cudaFree(b->counters);
    cudaFree(b->d_items);
    cudaFree(b->d_zitems);
    cudaFree(b->d_xitems);
    cudaFree(b->d_yitems);
    cudaFree(b->d_citems);
    if (b->hctl) cudaFreeHost(b->hctl);
    delete b;
    return HYDRO_OK;
}

hydro_status hydro_batch_create(const hydro_config* cfgs, int32_t n_events, void* stream, hydro_batch_t** out)
{
    if (!out) return bfail(nullptr, HYDRO_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!cfgs || n_events < 1) return bfail(nullptr, HYDRO_ERR_INVALID_ARG, "need at least one event config");
    for (int e = 0; e < n_events; ++e) {
        const std::string why = check_config(&cfgs[e]);
        if (!why.empty()) return bfail(nullptr, HYDRO_ERR_INVALID_ARG, "event " + std::to_string(e) + ": " + why);
        if (cfgs[e].bc[2] == HYDRO_BC_HALO)
            return bfail(nullptr, HYDRO_ERR_INVALID_ARG, "batch events are whole grids (no z halo)");
        if (cfgs[e].scheme == HYDRO_MUSTA_FORCE)
            return bfail(nullptr, HYDRO_ERR_INVALID_ARG, "the batched path runs the WENO schemes only");
        if (cfgs[e].nq > 1)
            return bfail(nullptr, HYDRO_ERR_INVALID_ARG, "the batched path supports one charge (nq <= 1)");
        if (cfgs[e].charwise)
            return bfail(nullptr, HYDRO_ERR_INVALID_ARG, "the batched path runs component-wise WENO only");
        if (cfgs[e].eos_mass != 0.0)
            return bfail(nullptr, HYDRO_ERR_INVALID_ARG, "the batched path runs the EOS p = cs2 e only (eos_mass = 0)");
        if (cfgs[e].scheme != cfgs[0].scheme || cfgs[e].split != cfgs[0].split)
            return bfail(nullptr, HYDRO_ERR_INVALID_ARG, "all events of a batch must use the same scheme and splitting");
    }
    hydro_batch_t* b = new (std::nothrow) hydro_batch_t();
    if (!b) return bfail(nullptr, HYDRO_ERR_OOM, "host allocation failed");
    auto bail = [&](hydro_status s) {
        g_batch_create_err = b->err;
        hydro_batch_destroy(b);
        return s;
    };
    b->n_events = n_events;
    b->R = cfgs[0].scheme == HYDRO_WENO5 ? 3 : 4;
    b->stream = (cudaStream_t)stream;
    b->cfg.assign(cfgs, cfgs + n_events);
    b->loaded.assign(n_events, 0);
    cudaError_t e;
    if ((e = cudaGetDevice(&b->dev)) != cudaSuccess) return bail(bcuda(b, e, "cudaGetDevice"));
    if ((e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->dev)) != cudaSuccess)
        return bail(bcuda(b, e, "device attribute"));
    b->ev.resize(n_events);
    long long total = 0;
    for (int i = 0; i < n_events; ++i) {
        const long long nc = (long long)cfgs[i].n[0] * cfgs[i].n[1] * cfgs[i].n[2];
        b->ev[i].ncell = nc;
        b->ev[i].fs = (nc + 31) / 32 * 32;
        total += (cfgs[0].split ? 36 : 27) * b->ev[i].fs;
        // z-face fluxes for the z-pass variants (global Lax-Friedrichs)
        b->ev[i].fzs = cfgs[0].split ? 0 : ((long long)cfgs[i].n[0] * cfgs[i].n[1] * (cfgs[i].n[2] + 1) + 31) / 32 * 32;
        // x- and y-face fluxes for the three-pass variants (global Lax-Friedrichs)
        b->ev[i].fxs = cfgs[0].split ? 0 : ((long long)(cfgs[i].n[0] + 1) * cfgs[i].n[1] * cfgs[i].n[2] + 31) / 32 * 32;
        b->ev[i].fys = cfgs[0].split ? 0 : ((long long)cfgs[i].n[0] * (cfgs[i].n[1] + 1) * cfgs[i].n[2] + 31) / 32 * 32;
        total += 5 * (b->ev[i].fzs + b->ev[i].fxs + b->ev[i].fys);
    }
    if ((e = cudaMalloc(&b->buf, sizeof(double) * (size_t)total)) != cudaSuccess) return bail(bcuda(b, e, "event buffers"));
    if ((e = cudaMalloc(&b->ctl, sizeof(Ctl) * n_events)) != cudaSuccess) return bail(bcuda(b, e, "control blocks"));
    if ((e = cudaMallocHost(&b->hctl, sizeof(Ctl) * n_events)) != cudaSuccess) return bail(bcuda(b, e, "pinned control"));
    if ((e = cudaMalloc(&b->counters, sizeof(unsigned int) * 4)) != cudaSuccess) return bail(bcuda(b, e, "counters"));
    if ((e = cudaMalloc(&b->d_ev, sizeof(BatchEvent) * n_events)) != cudaSuccess) return bail(bcuda(b, e, "events"));
    long long off = 0;
    for (int i = 0; i < n_events; ++i) {
        BatchEvent& E = b->ev[i];
        const hydro_config& c = cfgs[i];
        for (int k = 0; k < 3; ++k) {
            E.U[k] = b->buf + off + E.fs * 5 * k;
            E.W[k] = b->buf + off + E.fs * (15 + 4 * k);
            E.S[k] = c.split ? b->buf + off + E.fs * (27 + 3 * k) : nullptr;
        }
        off += (c.split ? 36 : 27) * E.fs;
        E.fz = E.fzs ? b->buf + off : nullptr;
        off += 5 * E.fzs;
        E.fx = E.fxs ? b->buf + off : nullptr;
        off += 5 * E.fxs;
        E.fy = E.fys ? b->buf + off : nullptr;
        off += 5 * E.fys;
        for (int d = 0; d < 3; ++d) {
            E.n[d] = c.n[d];
            E.bc[d] = c.bc[d];
            E.act[d] = c.n[d] > 1;
            E.hdx[d] = 0.5 / c.dx[d];
        }
        E.cs2 = c.cs2;
        E.eps_s = c.weno_eps * (b->R == 3 ? SchemeConst<3>::eps_scale : SchemeConst<4>::eps_scale);
        E.sp = step_params(c);
        E.ctl = b->ctl + i;
    }
    if ((e = cudaMemcpyAsync(b->d_ev, b->ev.data(), sizeof(BatchEvent) * n_events, cudaMemcpyHostToDevice, b->stream)) !=
        cudaSuccess)
        return bail(bcuda(b, e, "event table"));
    if ((e = cudaMemsetAsync(b->buf, 0, sizeof(double) * (size_t)total, b->stream)) != cudaSuccess)
        return bail(bcuda(b, e, "memset"));
    for (int i = 0; i < n_events; ++i) reset_ctl_kernel<<<1, 1, 0, b->stream>>>(b->ctl + i, 0.0);
    if ((e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking)) != cudaSuccess)
        return bail(bcuda(b, e, "capture stream"));
    hydro_status s = apply_batch_launch(b, fused_launch_variant(b->R, b->cfg[0].split, 1, 0), 0);
    if (s) return bail(s);
    *out = b;
    return HYDRO_OK;
}

const char* hydro_batch_last_error(hydro_batch_t* b) { return b ? b->err.c_str() : g_batch_create_err.c_str(); }

static hydro_status bcheck_io(hydro_batch_t* b, int32_t e, const void* p, int64_t stride, int32_t mem)
{
    if (!b) return HYDRO_ERR_INVALID_ARG;
    if (e < 0 || e >= b->n_events) return bfail(b, HYDRO_ERR_INVALID_ARG, "event index out of range");
    if (!p) return bfail(b, HYDRO_ERR_INVALID_ARG, "NULL data pointer");
    if (stride < b->ev[e].ncell) return bfail(b, HYDRO_ERR_INVALID_ARG, "field_stride smaller than the cell count");
    if (mem != HYDRO_MEM_HOST && mem != HYDRO_MEM_DEVICE) return bfail(b, HYDRO_ERR_INVALID_ARG, "mem must be 0 or 1");
    return HYDRO_OK;
}

static int bblocks(long long n) { long long k = (n + 255) / 256; return (int)(k > 152 * 16 ? 152 * 16 : (k < 1 ? 1 : k)); }

hydro_status hydro_batch_set_state(hydro_batch_t* b, int32_t e, const double* u, int64_t field_stride, int32_t mem,
                                   double t)
{
    hydro_status s = bcheck_io(b, e, u, field_stride, mem);
    if (s) return s;
    const BatchEvent& E = b->ev[e];
    const cudaMemcpyKind k = mem == HYDRO_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    for (int f = 0; f < 5; ++f)
        BCK(b, cudaMemcpyAsync(E.U[0] + f * E.fs, u + f * field_stride, sizeof(double) * E.ncell, k, b->stream), "copy");
    reset_ctl_kernel<<<1, 1, 0, b->stream>>>(E.ctl, t);
    prepare_kernel<<<bblocks(E.ncell), 256, 0, b->stream>>>(E.U[0], E.W[0], E.fs, E.ncell, E.cs2, E.ctl, E.S[0]);
    BCK(b, cudaGetLastError(), "prepare");
    b->loaded[e] = 1;
    return HYDRO_OK;
}

hydro_status hydro_batch_set_primitive(hydro_batch_t* b, int32_t e, const double* w, int64_t field_stride,
                                       int32_t mem, double t)
{
    hydro_status s = bcheck_io(b, e, w, field_stride, mem);
    if (s) return s;
    const BatchEvent& E = b->ev[e];
    const double* src = w;
    long long ss = field_stride;
    if (mem == HYDRO_MEM_HOST) {
        for (int f = 0; f < 5; ++f)
            BCK(b, cudaMemcpyAsync(E.U[1] + f * E.fs, w + f * field_stride, sizeof(double) * E.ncell,
                                   cudaMemcpyHostToDevice, b->stream), "copy");
        src = E.U[1];
        ss = E.fs;
    }
    reset_ctl_kernel<<<1, 1, 0, b->stream>>>(E.ctl, t);
    prim2con_kernel<<<bblocks(E.ncell), 256, 0, b->stream>>>(src, ss, E.U[0], E.fs, E.ncell, E.cs2, E.ctl, 5);
    prepare_kernel<<<bblocks(E.ncell), 256, 0, b->stream>>>(E.U[0], E.W[0], E.fs, E.ncell, E.cs2, E.ctl, E.S[0]);
    BCK(b, cudaGetLastError(), "prim2con");
    b->loaded[e] = 1;
    return HYDRO_OK;
}

static hydro_status all_loaded(hydro_batch_t* b)
{
    for (int e = 0; e < b->n_events; ++e)
        if (!b->loaded[e]) return bfail(b, HYDRO_ERR_STATE, "event " + std::to_string(e) + " has no state");
    return HYDRO_OK;
}

hydro_status hydro_batch_step(hydro_batch_t* b, int32_t nsteps)
{
    if (!b) return HYDRO_ERR_INVALID_ARG;
    if (nsteps < 0) return bfail(b, HYDRO_ERR_INVALID_ARG, "nsteps < 0");
    hydro_status s = all_loaded(b);
    if (s) return s;
    for (int i = 0; i < nsteps; ++i) BCK(b, cudaGraphLaunch(b->exec, b->stream), "graph launch");
    return HYDRO_OK;
}

hydro_status hydro_batch_profile_step(hydro_batch_t* b, int32_t nsteps, double kernel_ms[5])
{
    if (!b || !kernel_ms) return HYDRO_ERR_INVALID_ARG;
    hydro_status s = all_loaded(b);
    if (s) return s;
    for (int i = 0; i < 5; ++i) kernel_ms[i] = 0.0;
    cudaEvent_t ev[6];
    for (int i = 0; i < 6; ++i) BCK(b, cudaEventCreate(&ev[i]), "event");
    hydro_status st = HYDRO_OK;
    for (int n = 0; n < nsteps && st == HYDRO_OK; ++n) {
        cudaError_t e = enqueue_batch_step(b, b->stream, ev);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[5]);
        if (e != cudaSuccess) {
            st = bcuda(b, e, "profiled step");
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

static hydro_status batch_read_ctl(hydro_batch_t* b)
{
    BCK(b, cudaMemcpyAsync(b->hctl, b->ctl, sizeof(Ctl) * b->n_events, cudaMemcpyDeviceToHost, b->stream), "read control");
    BCK(b, cudaStreamSynchronize(b->stream), "synchronize");
    for (int e = 0; e < b->n_events; ++e)
        if (b->hctl[e].status) {
            char m[200];
            snprintf(m, sizeof m, "event %d: unphysical state (E <= 0, |M| >= E or NaN) first seen at cell %lld", e,
                     (long long)b->hctl[e].bad_cell);
            return bfail(b, HYDRO_ERR_UNPHYSICAL, m);
        }
    return HYDRO_OK;
}

hydro_status hydro_batch_sync(hydro_batch_t* b)
{
    if (!b) return HYDRO_ERR_INVALID_ARG;
    return batch_read_ctl(b);
}

hydro_status hydro_batch_get_state(hydro_batch_t* b, int32_t e, double* u, int64_t field_stride, int32_t mem, double* t,
                                   int64_t* step)
{
    hydro_status s = bcheck_io(b, e, u, field_stride, mem);
    if (s) return s;
    const BatchEvent& E = b->ev[e];
    const cudaMemcpyKind k = mem == HYDRO_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    for (int f = 0; f < 5; ++f)
        BCK(b, cudaMemcpyAsync(u + f * field_stride, E.U[0] + f * E.fs, sizeof(double) * E.ncell, k, b->stream), "copy");
    s = batch_read_ctl(b);
    if (t) *t = b->hctl[e].t;
    if (step) *step = b->hctl[e].step;
    return s;
}

int32_t hydro_batch_size(hydro_batch_t* b) { return b ? b->n_events : 0; }

int32_t hydro_batch_kernels_per_step(hydro_batch_t* b)
{
    if (!b) return 0;
    if (b->L.combine) return 2 + 3 * (1 + (b->n_xitems > 0) + (b->n_yitems > 0) + (b->n_zitems > 0));
    return 2 + 3 * ((b->L.zfn && b->n_zitems > 0) ? 2 : 1);
}

hydro_status hydro_batch_set_launch(hydro_batch_t* b, int32_t variant, int32_t zc)
{
    if (!b) return HYDRO_ERR_INVALID_ARG;
    if (variant < 0 || variant >= batch_variant_count(b->R, b->cfg[0].split))
        return bfail(b, HYDRO_ERR_INVALID_ARG, "no such launch variant");
    return apply_batch_launch(b, variant, zc);
}

hydro_status hydro_batch_get_launch(hydro_batch_t* b, int32_t* variant, int32_t* tile_x, int32_t* tile_y, int32_t* zc,
                                    int32_t* n_items)
{
    if (!b) return HYDRO_ERR_INVALID_ARG;
    if (variant) *variant = b->variant;
    if (tile_x) *tile_x = b->L.tx;
    if (tile_y) *tile_y = b->L.ty;
    if (zc) *zc = b->zc;
    if (n_items) *n_items = b->n_items;
    return HYDRO_OK;
}

// Time one stage-1 launch per candidate (tile shape x z chunk) and keep the
// fastest.  Stage 1 only writes scratch (its output state and speed slots),
// so the events' states, speeds and times are unchanged by tuning.
hydro_status hydro_batch_autotune(hydro_batch_t* b, double* best_ms)
{
    if (!b) return HYDRO_ERR_INVALID_ARG;
    hydro_status s = all_loaded(b);
    if (s) return s;
    static const int zcs[] = {16, 32, 64};
    double best = 1e300;
    int bv = b->variant, bz = b->zc;
    cudaEvent_t e0, e1;
    BCK(b, cudaEventCreate(&e0), "event");
    BCK(b, cudaEventCreate(&e1), "event");
    const int eb = (b->n_events + 127) / 128;
    for (int v = 0; v < batch_variant_count(b->R, b->cfg[0].split) && s == HYDRO_OK; ++v)
        for (int zc : zcs) {
            s = apply_batch_launch(b, v, zc);
            if (s) break;
            if (b->L.combine && zc != zcs[0]) continue;   // three-pass launches have no z chunks
            const BatchArgs a = batch_args(b, 1);
            float ms = 0.f;
            for (int rep = 0; rep < 2; ++rep) {   // warm-up, then timed
                batch_step_begin_kernel<<<eb, 128, 0, b->stream>>>(b->d_ev, b->n_events, b->counters);
                cudaEventRecord(e0, b->stream);
                launch_batch_stage(b, a, b->stream);
                cudaEventRecord(e1, b->stream);
            }
            cudaError_t e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e != cudaSuccess) {
                s = bcuda(b, e, "autotune");
                break;
            }
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                bv = v;
                bz = zc;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s) return s;
    if (best_ms) *best_ms = best;
    return apply_batch_launch(b, bv, bz);
}

}  // extern "C"
