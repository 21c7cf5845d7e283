// char_pass.cuh -- characteristic-wise face passes: the faces of one axis as
// a pass of their own, one thread per face (Sec. 1.2 applied to the
// characteristic fields of the flux Jacobian at each face; see char_weno.cuh).
//
// A characteristic-wise face projects its window on the basis of its own face
// state, so nothing carries from one face to the next and a face is the
// natural unit of work.  The pass writes the face fluxes of all fields in the
// layout of the component-wise passes (fx, fy, fz of StageArgs), and
// stage_combine_kernel finishes the stage exactly as it does for them.
//
// Per face (window cells j-r+1 .. j+r along the axis):
//   1. face state: the mean of the conserved states of cells j and j+1 (all
//      three axes alike), and its characteristic basis (char_setup);
//   2. + side: for cells j-r+1 .. j+r-1 the split flux g+ = f + alpha u
//      (explicitly rounded, as every other kernel forms it), projected on the
//      characteristic fields; the NF x (2r-1) projected values go to the
//      thread's own slice of shared memory, then each field is reconstructed
//      from it (WENO, left-biased);
//   3. - side: the same with g- on cells j-r+2 .. j+r (right-biased), and the
//      face value of each characteristic field;
//   4. back-projection and the store of the NF face fluxes.
// Consecutive threads take consecutive entries of the face buffer, so every
// load of a window cell and every store is a coalesced row.  No barriers: a
// thread's shared memory is its own.
#pragma once
#include "char_weno.cuh"
#include "stage_kernel.cuh"

namespace hydro {

constexpr int kCharPassThreads = 128;

// shared memory of one pass CTA: NF x (2r-1) doubles per thread
template <int R, int NF>
constexpr size_t char_pass_smem() { return sizeof(double) * (size_t)NF * (2 * R - 1) * kCharPassThreads; }

// faces of a pass along AX over interior planes zlo .. zhi
__host__ __device__ inline long long char_pass_faces(int AX, int nx, int ny, int nzi)
{
    if (AX == 0) return (long long)(nx + 1) * ny * nzi;
    if (AX == 1) return (long long)nx * (ny + 1) * nzi;
    return (long long)nx * ny * (nzi + 1);
}

template <int R, int NF, int AX, int EMU, int MINB>
__global__ void __launch_bounds__(kCharPassThreads, MINB) charw_pass_kernel(const StageArgs a)
{
    constexpr int G = R, S = 2 * R - 1, NT = kCharPassThreads;
    extern __shared__ double cp_smem[];
    if (!(*a.dt > 0.0)) return;
    const int nx = a.nx, ny = a.ny, nzi = a.zhi - a.zlo;
    const long long plane = (long long)nx * ny;
    const long long fi = (long long)blockIdx.x * NT + threadIdx.x;
    if (fi >= char_pass_faces(AX, nx, ny, nzi)) return;       // no barriers below
    // face f (between cells lo+f-1 and lo+f along AX) of the pencil that starts
    // at base and steps by step; out: this face's entry of field 0
    long long base, step;
    int f, lo, ncell, bcax;
    double* out;
    long long ofs;
    if constexpr (AX == 0) {
        const long long row = fi / (nx + 1);
        f = (int)(fi - row * (nx + 1));
        base = (long long)(a.zlo + row / ny) * plane + (row % ny) * nx;
        step = 1;
        lo = 0;
        ncell = nx;
        bcax = a.bc[0];
        out = a.fx + fi;
        ofs = a.fxs;
    } else if constexpr (AX == 1) {
        const long long span = (long long)nx * nzi;
        f = (int)(fi / span);
        const long long r = fi - f * span;
        base = (long long)(a.zlo + r / nx) * plane + r % nx;
        step = nx;
        lo = 0;
        ncell = ny;
        bcax = a.bc[1];
        out = a.fy + fi;
        ofs = a.fys;
    } else {
        f = (int)(fi / plane);
        base = fi - f * plane;
        step = plane;
        lo = a.zlo;
        ncell = a.nz;
        bcax = a.bc[2];
        out = a.fz + fi;
        ofs = a.fzs;
    }
    const int p0 = lo + f - G;                     // window cell 0
    auto cell = [&](int i) { return base + (long long)bc_map(p0 + i, ncell, bcax) * step; };
    int mf[NF];                                    // memory field of rotated field m
#pragma unroll
    for (int m = 0; m < NF; ++m) mf[m] = rot_field(m, AX);

    // 1. face state and basis
    CharBasis<NF> B;
    bool ok;
    {
        const long long qa = cell(G - 1), qb = cell(G);
        double ub[NF];
#pragma unroll
        for (int m = 0; m < NF; ++m) ub[m] = 0.5 * (__ldg(a.u_in + mf[m] * a.fs + qa) + __ldg(a.u_in + mf[m] * a.fs + qb));
        ok = char_setup<NF>(ub, a.cs2, B);
    }
    if (!ok) {
        // a face state that is not physical (only next to an unphysical
        // cell): no flux, reported like an unphysical cell
#pragma unroll
        for (int m = 0; m < NF; ++m) out[m * ofs] = 0.0;
        if (atomicCAS(a.status, 0, 4) == 0) *a.bad_cell = cell(G - 1);
        return;
    }
    const double al = __longlong_as_double((long long)a.alpha_in[AX]);
    double* win = cp_smem + threadIdx.x;           // win[(m S + i) NT]: projected value of field m, cell i
    // rotated split flux g+ (s = +1) or g- (s = -1) of window cell i, projected
    auto project_cell = [&](int i, double sgn, int slot) {
        const long long q = cell(i);
        double u[NF];
#pragma unroll
        for (int m = 0; m < NF; ++m) u[m] = __ldg(a.u_in + mf[m] * a.fs + q);
        const double vd = __ldg(a.w_in + (1 + AX) * a.fs + q);
        const double pr = __ldg(a.w_in + q);
        const double sa = sgn * al;
        double g[NF];
        g[0] = fma(sa, u[0], u[1]);                               // f_E = M_d
        g[1] = fma(sa, u[1], __dadd_rn(__dmul_rn(u[1], vd), pr));  // f = M_d v_d + p
#pragma unroll
        for (int m = 2; m < NF; ++m) g[m] = fma(sa, u[m], __dmul_rn(u[m], vd));
        double c[NF];
        char_project<NF>(B, [&](int m) { return g[m]; }, c);
#pragma unroll
        for (int m = 0; m < NF; ++m) win[(m * S + slot) * NT] = c[m];
    };

    // 2. + side: cells 0 .. S-1, left-biased
    double Np[NF], Dp[NF], Cp[NF];
    // (unrolling these two loops, or 255 registers at two CTAs per SM, measured
    // the same: the pass is bound by the FP64 pipe)
#pragma unroll 1
    for (int i = 0; i < S; ++i) project_cell(i, 1.0, i);
#pragma unroll
    for (int m = 0; m < NF; ++m) {
        double v[S];
#pragma unroll
        for (int i = 0; i < S; ++i) v[i] = win[(m * S + i) * NT];
        weno_left<R, EMU>(v, a.eps_s, Np[m], Dp[m]);
        Cp[m] = v[G - 1];
    }
    // 3. - side: cells 1 .. S, right-biased
#pragma unroll 1
    for (int i = 0; i < S; ++i) project_cell(i + 1, -1.0, i);
    double Fc[NF];
#pragma unroll
    for (int m = 0; m < NF; ++m) {
        double v[S];
#pragma unroll
        for (int i = 0; i < S; ++i) v[i] = win[(m * S + i) * NT];
        double Nm, Dm;
        weno_right<R, EMU>(v, a.eps_s, Nm, Dm);
        Fc[m] = face_sum<EMU>(Np[m], Dp[m], Cp[m], Nm, Dm, v[G - 1]);
    }
    // 4. back to conserved fluxes
    double F[NF];
    char_back<NF>(B, Fc, F);
#pragma unroll
    for (int m = 0; m < NF; ++m) out[mf[m] * ofs] = F[m];
}

}  // namespace hydro
