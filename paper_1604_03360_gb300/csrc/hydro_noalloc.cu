// hydro_noalloc.cu -- hydro_step_noalloc: RK3 steps of one grid that allocate
// no device memory.
//
// Some callers cannot call cudaMalloc: applications whose device memory is
// owned by their own pool allocator and must not change behind its back, or
// loops with a fixed, preallocated footprint where cudaMalloc's implicit
// synchronisation and failure modes are not acceptable.  For them this entry
// point keeps every intermediate buffer (the two intermediate RK states, the
// primitives of three states and the control block) in one file-scope device
// array that exists from the moment the library is loaded until the process
// exits, on every GPU that loads the library.  The caller passes the input and
// output states; nothing is allocated or freed per call.
//
// Consequences, stated for users:
//  * the array is shared by all calls in the process: calls whose GPU work
//    overlaps (for example on two streams at once) race on it -- serialise them;
//  * it keeps the previous call's contents; every call resets the control
//    block and overwrites each scratch field before reading it;
//  * grids whose field stride exceeds HYDRO_NOALLOC_MAX_CELLS are rejected.
#include <mutex>

#include "hydro_common.cuh"

namespace {

constexpr long long kMaxCells = HYDRO_NOALLOC_MAX_CELLS;
// 32 doubles (256 bytes) for the control block, then 22 fields of
// kMaxCells doubles: U1, U2 (5 each) and W0, W1, W2 (4 each).
constexpr long long kCtlDoubles = 32;
constexpr long long kScratchDoubles = kCtlDoubles + 22 * kMaxCells;
static_assert(sizeof(hydro::Ctl) <= kCtlDoubles * sizeof(double), "control block does not fit");

static __device__ __align__(256) double g_scratch[kScratchDoubles];

struct DeviceSetup {
    bool ready = false;
    double* scratch = nullptr;     // device address of g_scratch on this device
    hydro::StageLaunch L[2];       // WENO5, WENO7
};
constexpr int kMaxDevices = 64;
DeviceSetup g_setup[kMaxDevices];
std::mutex g_mutex;

// Once per device, with that device current: resolve the device address of
// the scratch array (the host-side symbol is only a stand-in) and configure
// the stage kernels.
hydro_status setup_device(int dev, DeviceSetup** out, std::string& err)
{
    if (dev < 0 || dev >= kMaxDevices) {
        err = "device ordinal out of range";
        return HYDRO_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    DeviceSetup& s = g_setup[dev];
    if (!s.ready) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return HYDRO_ERR_CUDA;
        }
        for (int i = 0; i < 2; ++i) {
            e = hydro::stage_launch_info(i == 0 ? 3 : 4, &s.L[i]);
            if (e != cudaSuccess) {
                err = std::string("stage kernel setup: ") + cudaGetErrorString(e);
                return HYDRO_ERR_CUDA;
            }
        }
        s.scratch = static_cast<double*>(p);
        s.ready = true;
    }
    *out = &s;
    return HYDRO_OK;
}

thread_local std::string g_err;

hydro_status fail(hydro_status s, const std::string& m)
{
    g_err = m;
    return s;
}

}  // namespace

extern "C" const char* hydro_noalloc_last_error(void) { return g_err.c_str(); }

extern "C" hydro_status hydro_step_noalloc(const hydro_config* cfg, const double* u_in, double* u_out,
                                           int64_t field_stride, double t0, int32_t nsteps, double t_end,
                                           void* stream, double* t_out)
{
    using namespace hydro;
    g_err.clear();
    const std::string why = check_config(cfg);
    if (!why.empty()) return fail(HYDRO_ERR_INVALID_ARG, why);
    if (cfg->split != 0) return fail(HYDRO_ERR_INVALID_ARG, "hydro_step_noalloc supports global splitting only");
    if (cfg->nq > 1) return fail(HYDRO_ERR_INVALID_ARG, "hydro_step_noalloc supports one charge (nq <= 1)");
    if (cfg->charwise) return fail(HYDRO_ERR_INVALID_ARG, "hydro_step_noalloc runs component-wise WENO only");
    if (cfg->eos_mass != 0.0) return fail(HYDRO_ERR_INVALID_ARG, "hydro_step_noalloc runs the EOS p = cs2 e only");
    if (cfg->bc[2] == HYDRO_BC_HALO) return fail(HYDRO_ERR_INVALID_ARG, "hydro_step_noalloc runs whole grids (no z halo)");
    if (cfg->scheme == HYDRO_MUSTA_FORCE) return fail(HYDRO_ERR_INVALID_ARG, "hydro_step_noalloc runs the WENO schemes only");
    if (!u_in || !u_out) return fail(HYDRO_ERR_INVALID_ARG, "NULL state pointer");
    if (nsteps < 0) return fail(HYDRO_ERR_INVALID_ARG, "nsteps < 0");
    const long long ncell = (long long)cfg->n[0] * cfg->n[1] * cfg->n[2];
    if (field_stride < ncell) return fail(HYDRO_ERR_INVALID_ARG, "field_stride smaller than the cell count");
    if (field_stride > kMaxCells)
        return fail(HYDRO_ERR_INVALID_ARG, "field_stride " + std::to_string((long long)field_stride) +
                                               " exceeds the no-allocation limit of " +
                                               std::to_string(kMaxCells) + " cells");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(HYDRO_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    DeviceSetup* ds = nullptr;
    std::string err;
    hydro_status st = setup_device(dev, &ds, err);
    if (st != HYDRO_OK) return fail(st, err);
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail(HYDRO_ERR_CUDA, std::string("device attribute: ") + cudaGetErrorString(e));

    cudaStream_t s = (cudaStream_t)stream;
    const long long fs = field_stride;
    Ctl* ctl = reinterpret_cast<Ctl*>(ds->scratch);
    double* base = ds->scratch + kCtlDoubles;
    double* U[3] = {u_out, base, base + 5 * fs};
    double* W[3] = {base + 10 * fs, base + 14 * fs, base + 18 * fs};
    const StageLaunch& L = ds->L[cfg->scheme == HYDRO_WENO5 ? 0 : 1];
    const int R = cfg->scheme == HYDRO_WENO5 ? 3 : 4;
    const int zc = pick_zc(cfg->n[0], cfg->n[1], cfg->n[2], L, sms);

    if (u_out != u_in) {
        e = cudaMemcpyAsync(u_out, u_in, sizeof(double) * (size_t)(4 * fs + ncell), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return fail(HYDRO_ERR_CUDA, std::string("copy: ") + cudaGetErrorString(e));
    }
    // every call starts from a clean control block; the scratch fields are
    // written before they are read (W0 here, U1/W1 by stage 1, U2/W2 by stage 2)
    reset_ctl_kernel<<<1, 1, 0, s>>>(ctl, t0);
    long long nb = (ncell + 255) / 256;
    if (nb > 152LL * 16) nb = 152LL * 16;
    prepare_kernel<<<(int)(nb < 1 ? 1 : nb), 256, 0, s>>>(U[0], W[0], fs, ncell, cfg->cs2, ctl);
    set_t_end_kernel<<<1, 1, 0, s>>>(ctl, t_end);

    const dim3 grid((cfg->n[0] + L.tx - 1) / L.tx, (cfg->n[1] + L.ty - 1) / L.ty, (cfg->n[2] + zc - 1) / zc);
    static const double ca[3] = {0.0, 0.75, 1.0 / 3.0}, cb[3] = {1.0, 0.25, 2.0 / 3.0};
    for (int n = 0; n < nsteps; ++n) {
        step_begin_kernel<<<1, 1, 0, s>>>(ctl, step_params(*cfg));
        for (int k = 1; k <= 3; ++k) {
            StageArgs a{};
            a.u_in = U[k - 1];
            a.w_in = W[k - 1];
            a.u_n = U[0];
            a.u_out = k == 3 ? U[0] : U[k];
            a.w_out = k == 3 ? W[0] : W[k];
            a.fs = fs;
            a.nx = cfg->n[0];
            a.ny = cfg->n[1];
            a.nz = cfg->n[2];
            a.zc = zc;
            a.zlo = 0;
            a.zhi = cfg->n[2];
            for (int d = 0; d < 3; ++d) {
                a.bc[d] = cfg->bc[d];
                a.act[d] = cfg->n[d] > 1;
                a.hdx[d] = 0.5 / cfg->dx[d];
            }
            a.cs2 = cfg->cs2;
            a.eps_s = cfg->weno_eps * (R == 3 ? SchemeConst<3>::eps_scale : SchemeConst<4>::eps_scale);
            a.ca = ca[k - 1];
            a.cb = cb[k - 1];
            a.alpha_in = k == 1 ? ctl->a_cur : (k == 2 ? ctl->a_s1 : ctl->a_s2);
            a.alpha_out = k == 1 ? ctl->a_s1 : (k == 2 ? ctl->a_s2 : ctl->a_next);
            a.dt = &ctl->dt;
            a.status = &ctl->status;
            a.bad_cell = &ctl->bad_cell;
            L.fn<<<grid, L.tx * L.ty, L.smem, s>>>(a);
        }
        step_end_kernel<<<1, 1, 0, s>>>(ctl);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(HYDRO_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    if (t_out) {
        Ctl h;
        e = cudaMemcpyAsync(&h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return fail(HYDRO_ERR_CUDA, std::string("read back: ") + cudaGetErrorString(e));
        *t_out = h.t;
        if (h.status)
            return fail(HYDRO_ERR_UNPHYSICAL, "unphysical state (E <= 0, |M| >= E or NaN) at cell " +
                                                  std::to_string(h.bad_cell));
    }
    return HYDRO_OK;
}
