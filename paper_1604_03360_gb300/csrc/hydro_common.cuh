// hydro_common.cuh -- host/device pieces shared by the library's translation
// units: the device control block, small bookkeeping kernels and launch
// helpers.
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <string>

#include "../../include/hydro.h"
#include "stage_kernel.cuh"

namespace hydro {

// Device-resident control block of one grid (or one event of a batch).
// Speeds are stored as IEEE bit patterns so atomicMax on them is exact.
struct Ctl {
    unsigned long long a_cur[3];   // speeds of the current state u^n
    unsigned long long a_s1[3];    // speeds of the stage-1 output
    unsigned long long a_s2[3];    // speeds of the stage-2 output
    unsigned long long a_next[3];  // speeds of the stage-3 output
    double dt;                     // step being taken (0: nothing to do)
    double t;                      // simulation time
    double t_end;                  // < 0: unlimited
    double last_dt;
    long long step;
    long long bad_cell;
    int status;
    int pad_;
};

// first error over the items of hydro_run_many
struct RunStatus {
    long long bad_cell;
    int status;
    int item;
};

struct StepParams {
    double cfl, dt_fixed, mindx;
    int actmask;                   // bit d: axis d takes part in dt
};

// dt from the speeds of u^n, clipped to t_end; zero the accumulation slots.
__global__ void step_begin_kernel(Ctl* c, StepParams sp);
// commit the step: speeds of u^{n+1} become current, advance t.
__global__ void step_end_kernel(Ctl* c);
__global__ void set_t_end_kernel(Ctl* c, double t_end);
// ghost planes of a z-slab (outflow end of the grid): for every listed field,
// planes dst .. dst + G - 1 (offsets in doubles / plane) become copies of the
// plane at offset src
struct FieldList {
    double* f[16];
    int n;
};
__global__ void halo_replicate_kernel(FieldList fl, long long plane, long long src, long long dst, int G);
__global__ void reset_ctl_kernel(Ctl* c, double t);
// keep the first error of item `item` (hydro_run_many)
__global__ void run_status_kernel(const Ctl* c, RunStatus* r, int item);
// primitives and speeds of a state (after set_state)
// (and, if s != nullptr, the per-axis speeds of every cell: 3 fields)
// eos_m: mass of the EOS p = cs2 (e - eos_m n_1) (0: p = cs2 e)
__global__ void prepare_kernel(const double* u, double* w, long long fs, long long n, double cs2, Ctl* c,
                               double* s = nullptr, double eos_m = 0.0);
// primitives (e, v, n) -> conserved
__global__ void prim2con_kernel(const double* wp, long long ws, double* u, long long fs, long long n, double cs2,
                                Ctl* c, int nf, double eos_m = 0.0);
// conserved -> (e, v, n)
__global__ void state_to_prim_kernel(const double* u, long long fs, double* out, long long os, long long n,
                                     double cs2, int nf, double eos_m = 0.0);
// conserved -> (p, v, e) and the squared sound speed for either EOS
__device__ __forceinline__ bool recover(double cs2, double eos_m, const double* u, long long fs, long long q,
                                        double& p, double& vx, double& vy, double& vz, double& e, double& ks)
{
    ks = cs2;
    if (eos_m == 0.0) return con2prim(cs2, u[q], u[fs + q], u[2 * fs + q], u[3 * fs + q], p, vx, vy, vz, e);
    if (!con2prim_gas(cs2, eos_m, u[q], u[fs + q], u[2 * fs + q], u[3 * fs + q], u[4 * fs + q], p, vx, vy, vz, e))
        return false;
    ks = sound2_gas(cs2, p, e);
    return true;
}

// an axis takes part in the scheme if it has more than one cell; a z axis
// with stored halos (a slab of a larger grid) always does
inline bool axis_active(const hydro_config& cfg, int d)
{
    return cfg.n[d] > 1 || (d == 2 && cfg.bc[2] == HYDRO_BC_HALO);
}

inline StepParams step_params(const hydro_config& cfg)
{
    StepParams sp;
    sp.cfl = cfg.cfl;
    sp.dt_fixed = cfg.dt_fixed;
    int mask = 0;
    for (int d = 0; d < 3; ++d)
        if (axis_active(cfg, d)) mask |= 1 << d;
    if (!mask) mask = 7;
    double m = INFINITY;
    for (int d = 0; d < 3; ++d)
        if (mask & (1 << d)) m = fmin(m, cfg.dx[d]);
    sp.mindx = m;
    sp.actmask = mask;
    return sp;
}

// validate a config; returns an empty string when it is usable
std::string check_config(const hydro_config* c);

// stage kernel dispatch for a scheme (R = 3 or 4) and a tile shape
struct StageLaunch {
    void (*fn)(StageArgs);
    size_t smem;
    int tx, ty;
    int ctas_per_sm;
    void (*zfn)(StageArgs) = nullptr;   // z pass launched before fn (ZEXT variants), else null
    // TMA-staged variants: the stage kernel takes the stage input's tensor
    // maps (fn is then null); raw tile box of tma_rw x tma_rh cells
    void (*fn_tma)(StageArgs, TmaMaps) = nullptr;
    int tma_rw = 0, tma_rh = 0;
    // three-pass variants: x and y passes (like the z pass) write every face
    // flux, then fn is the per-cell combination kernel, launched grid-stride
    void (*xfn)(StageArgs) = nullptr;
    void (*yfn)(StageArgs) = nullptr;
    bool combine = false;
    int pass_threads = kZPassThreads;   // threads per pass CTA: one warp per field
    // characteristic-wise passes: one thread per face (grid over the faces of
    // the axis), pass_smem bytes of shared memory per CTA
    bool face_per_thread = false;
    size_t pass_smem = 0;
};
// tensor maps of the stage input (u: 5 fields, w: p, v_x, v_y of 4) for a
// TMA-staged launch; cudaErrorNotSupported where the layout does not allow
// them (x rows must be a multiple of 16 bytes: nx even)
cudaError_t encode_stage_maps(const StageLaunch& L, const double* u, const double* w, int nx, int ny, int nz,
                              long long fs, TmaMaps* out);
inline bool tma_layout_ok(int nx, int ny) { return nx % 2 == 0 && nx >= 2 && ny >= 1; }
// face chunks of a pass over nf faces
int pass_chunks(int nf);
// the launches of one RK3 stage of the grid described by a (z planes zlo ..
// zhi): face passes and the combination for a three-pass launch, else the z
// pass if any and the stage kernel; zc planes per stage-kernel CTA.  Returns
// an error only when a TMA-staged launch cannot build its tensor maps.
cudaError_t launch_stage_kernels(const StageLaunch& L, int zc, const StageArgs& a, int sms, cudaStream_t s);
// CTAs per face chunk of a z pass: 32 consecutive columns of the plane each
inline long long zpass_blocks(int nx, int ny) { return ((long long)nx * ny + 31) / 32; }
// Tile shapes compiled per scheme and splitting (index 0 is the default);
// stage_launch_variant returns cudaErrorInvalidValue for a variant that does
// not exist.  split: 0 global, 1 local Lax-Friedrichs.
// nq: number of charges (state fields = 4 + nq).
// charw: characteristic-wise reconstruction (hydro_char.cu; split must be 0).
int launch_variant_count(int R, int split, int nq, int charw = 0);
int default_launch_variant(int R, int split, int nq, int charw = 0);
// the fastest variant that keeps the z faces in the stage kernel (no z pass):
// for launch paths without a z-flux buffer (adjoint, no-alloc)
int fused_launch_variant(int R, int split, int nq, int charw = 0);
// variants that the batched (persistent) kernel also has
int batch_variant_count(int R, int split);
cudaError_t stage_launch_variant(int R, int split, int nq, int v, StageLaunch* out, int charw = 0);
int char_variant_count(int R, int nq);
int char_default_variant(int R, int nq);
cudaError_t char_launch_variant(int R, int nq, int v, StageLaunch* out);
inline cudaError_t stage_launch_info(int R, StageLaunch* out)
{
    return stage_launch_variant(R, 0, 1, fused_launch_variant(R, 0, 1), out);
}
inline int state_fields(const hydro_config& c) { return 4 + (c.nq > 1 ? c.nq : 1); }
// configurations with z-pass and three-pass launch variants (WENO with global
// or local LF, up to three charges; characteristic-wise with global LF)
inline bool zpass_capable(const hydro_config& c, int R)
{
    return (R == 3 || R == 4) && (c.split == 0 || c.split == 1) && c.nq <= 3 && (c.charwise == 0 || c.split == 0);
}
// internal scheme code: 3 WENO5, 4 WENO7, 2 MUSTA-FORCE (the ghost width)
inline int scheme_R(int scheme) { return scheme == HYDRO_WENO5 ? 3 : (scheme == HYDRO_WENO7 ? 4 : 2); }
inline int musta_stages_of(const hydro_config& c) { return c.musta_stages > 0 ? c.musta_stages : 2; }

// per-chunk cost of a stage CTA in planes: the z ring's warm-up (2G-1 planes
// ingested, one z stencil) for the fused kernels, next to nothing for the
// z-pass variants (no ring)
inline double zc_prologue(const StageLaunch& L) { return L.zfn ? 0.25 : 1.5; }

inline int pick_zc(int nx, int ny, int nz, const StageLaunch& L, int sms)
{
    const long long tiles = (long long)((nx + L.tx - 1) / L.tx) * ((ny + L.ty - 1) / L.ty);
    const long long conc = (long long)sms * (L.ctas_per_sm > 0 ? L.ctas_per_sm : 1);
    static const int cand[] = {8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512};
    int best = nz;
    double best_cost = 1e300;
    for (int zc : cand) {
        if (zc > nz && zc != cand[0]) break;
        const int z = zc < nz ? zc : nz;
        const long long ctas = tiles * ((nz + z - 1) / z);
        const long long waves = (ctas + conc - 1) / conc;
        const double cost = (double)waves * (z + zc_prologue(L));
        if (cost < best_cost * 0.999) {
            best_cost = cost;
            best = z;
        }
    }
    return best;
}

// The adjoint workspace lives beside the handle; hydro_api.cu owns the handle.
struct AdjointWork {
    int nsteps = 0, ckpt = 0, nckpt = 0;
    long long fs = 0;
    double* buf = nullptr;                 // all states below
    double *AU[3], *AW[3], *LAM, *OUT, *ACC, *V, *GP, *GM, *CK, *SEG;
    double* XT = nullptr;                  // x pencils in the x-slowest layout: u 5, p and v_x 2,
                                           // lambda 5, gbar+ 5, gbar- 5 (22 fields)
    bool seg_kept = false;                 // SEG holds the last segment's stage inputs
    unsigned long long* rec = nullptr;     // nsteps x 10
    Ctl* ctl = nullptr;                    // scratch control block (speed sinks)
};

// Interface to the handle (defined in hydro_api.cu).
struct HandleView {
    bool loaded;
    hydro_config cfg;
    int R;
    cudaStream_t stream;
    long long ncell, fs;
    double *U0, *W0;
    Ctl* ctl;
    StageLaunch L;                 // stage launch for the adjoint's own buffers: the
    int zc;                        // handle's z-pass launch (z faces in fz) or a fused one
    double* fz;                    // the handle's face buffers (null with a fused launch;
    long long fzs;                 // fx, fy only with a three-pass launch)
    double* fx;
    long long fxs;
    double* fy;
    long long fys;
    int sms;
};
hydro_status hydro_handle_view(hydro_t* h, HandleView* v);
AdjointWork* hydro_handle_adjoint(hydro_t* h, bool create);
hydro_status hydro_handle_fail(hydro_t* h, hydro_status s, const std::string& m);


}  // namespace hydro
