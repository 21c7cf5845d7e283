// musta_kernel.cuh -- one fused RK3 stage of the second-order MUSTA-FORCE +
// MUSCL scheme (arXiv:1604.03360, Sec. 1.1) for sm_103a.
//
// Face flux: the state is reconstructed linearly in each cell, component-wise
// on the conserved variables, with a limited slope (minmod, MC, van Leer or
// superbee); an unphysical reconstructed state falls back to the cell value.
// MUSTA then runs K stages of the centred FORCE flux on the two local states,
//   F = (F_LF + F_LW) / 2,  F_LF = (f_L + f_R)/2 - (u_R - u_L) / (2 r),
//   F_LW = f(u_LW),  u_LW = (u_L + u_R)/2 - r (f_R - f_L) / 2,
// with the local ratio r = dt/dx = 0.9 / max|lambda| over the local states,
// advancing the local states between stages as a predictor
// (u_L -= r (F - f_L), u_R -= r (f_R - F)).  If u_LW is unphysical the stage
// flux is F_LF; if a predicted state is unphysical the iteration stops.
//
// Work decomposition as the WENO stage kernel, with G = 2: a per-column ring
// of 4 z-planes of the state; the tile's state plus a 2-cell halo staged in
// shared memory; one item per face (all five fields at once); the same fused
// RK combine, primitive recovery and speed reduction.
#pragma once
#include "stage_kernel.cuh"

namespace hydro {

__device__ __forceinline__ double mm2(double a, double b)
{
    if (a * b <= 0.0) return 0.0;
    return fabs(a) < fabs(b) ? a : b;
}

// limited slope from backward / forward differences a, b
__device__ __forceinline__ double muscl_slope(int kind, double a, double b)
{
    if (a * b <= 0.0) return 0.0;
    if (kind == 0) return mm2(a, b);
    if (kind == 1) return mm2(mm2(2.0 * a, 0.5 * (a + b)), 2.0 * b);
    if (kind == 2) return 2.0 * a * b * rcp(a + b);
    const double s1 = mm2(2.0 * a, b), s2 = mm2(a, 2.0 * b);
    return fabs(s1) > fabs(s2) ? s1 : s2;
}

// max |lambda_+-| along d for primitives (p, v) (see max_speeds)
__device__ __forceinline__ double max_speed_d(double k, int d, const double w[4])
{
    const double v2 = fma(w[1], w[1], fma(w[2], w[2], w[3] * w[3]));
    const double one_kv2 = fma(-k, v2, 1.0);
    const double vd = w[1 + d];
    const double rad = k * (1.0 - v2) * fma(-(1.0 - k) * vd, vd, one_kv2);
    return fma(fabs(vd), 1.0 - k, sqrt(rad)) * rcp(one_kv2);
}

__device__ __forceinline__ bool prim_of(double k, const double u[5], double w[4])
{
    double e;
    return con2prim(k, u[0], u[1], u[2], u[3], w[0], w[1], w[2], w[3], e);
}

// MUSTA-FORCE flux along d; false if the initial local states are unphysical
__device__ __forceinline__ bool musta_flux(double k, int d, int K, const double* uL0, const double* uR0, double F[5])
{
    double uL[5], uR[5], wL[4], wR[4], fL[5], fR[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        uL[i] = uL0[i];
        uR[i] = uR0[i];
    }
    if (!prim_of(k, uL, wL) || !prim_of(k, uR, wR)) return false;
    for (int l = 1; l <= K; ++l) {
        raw_flux<5>(d, uL, wL, fL);
        raw_flux<5>(d, uR, wR, fR);
        const double S = fmax(max_speed_d(k, d, wL), max_speed_d(k, d, wR));
        const double r = 0.9 * rcp(S), ir = S * (1.0 / 0.9);
        double uLW[5], wLW[4], fLW[5], Flf[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            Flf[i] = fma(-0.5 * ir, uR[i] - uL[i], 0.5 * (fL[i] + fR[i]));
            uLW[i] = fma(-0.5 * r, fR[i] - fL[i], 0.5 * (uL[i] + uR[i]));
        }
        if (prim_of(k, uLW, wLW)) {
            raw_flux<5>(d, uLW, wLW, fLW);
#pragma unroll
            for (int i = 0; i < 5; ++i) F[i] = 0.5 * (Flf[i] + fLW[i]);
        } else {
#pragma unroll
            for (int i = 0; i < 5; ++i) F[i] = Flf[i];
        }
        if (l == K) break;
        double nL[5], nR[5], vL[4], vR[4];
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            nL[i] = fma(-r, F[i] - fL[i], uL[i]);
            nR[i] = fma(-r, fR[i] - F[i], uR[i]);
        }
        if (!prim_of(k, nL, vL) || !prim_of(k, nR, vR)) break;
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            uL[i] = nL[i];
            uR[i] = nR[i];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            wL[i] = vL[i];
            wR[i] = vR[i];
        }
    }
    return true;
}

// MUSCL states at face j+1/2 from cells j-1 .. j+2 (pointer at cell j-1,
// element stride st, field stride fsd), then the MUSTA-FORCE flux
__device__ __forceinline__ bool muscl_musta_face(double k, int d, int K, int lim, const double* v, int st, int fsd,
                                                 double F[5])
{
    double uL[5], uR[5], c0[5], c1[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const double* q = v + i * fsd;
        const double a = q[0], b = q[st], c = q[2 * st], e = q[3 * st];
        const double sl = muscl_slope(lim, b - a, c - b), sr = muscl_slope(lim, c - b, e - c);
        c0[i] = b;
        c1[i] = c;
        uL[i] = fma(0.5, sl, b);
        uR[i] = fma(-0.5, sr, c);
    }
    double w[4];
    if (!prim_of(k, uL, w))
#pragma unroll
        for (int i = 0; i < 5; ++i) uL[i] = c0[i];
    if (!prim_of(k, uR, w))
#pragma unroll
        for (int i = 0; i < 5; ++i) uR[i] = c1[i];
    return musta_flux(k, d, K, uL, uR, F);
}

template <int TX, int TY>
struct MustaSmem {
    static constexpr int G = 2, NT = TX * TY, NRING = 4;
    static constexpr int GXW = TX + 2 * G, GYH = TY + 2 * G;
    static constexpr int RING = NRING * 5 * NT;
    static constexpr int GX = 5 * TY * GXW;
    static constexpr int GY = 5 * GYH * TX;
    static constexpr int FX = 5 * TY * (TX + 1);
    static constexpr int FY = 5 * (TY + 1) * TX;
    static constexpr size_t bytes = sizeof(double) * (size_t)(RING + GX + GY + FX + FY);
};

template <int TX, int TY>
__device__ __forceinline__ void musta_tile(const StageArgs& a, int tile_x, int tile_y, int chunk_z, double* smem)
{
    using SM = MustaSmem<TX, TY>;
    constexpr int G = SM::G, NT = SM::NT, NRING = SM::NRING, GXW = SM::GXW, GYH = SM::GYH;
    double* ring = smem;
    double* ux = ring + SM::RING;
    double* uy = ux + SM::GX;
    double* Fx = uy + SM::GY;
    double* Fy = Fx + SM::FX;

    const double dt = *a.dt;
    if (!(dt > 0.0)) return;
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    const int x0 = tile_x * TX, y0 = tile_y * TY;
    const int zb = a.zlo + chunk_z * a.zc, ze = min(zb + a.zc, a.zhi);
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int x = x0 + tx, y = y0 + ty;
    const bool own = (x < nx) && (y < ny);
    const int xs = bc_map(x, nx, a.bc[0]), ys = bc_map(y, ny, a.bc[1]);
    const long long fs = a.fs, plane = (long long)nx * ny;
    const bool zwork = a.act[2] != 0 && own;
    const double k = a.cs2;
    const double idx[3] = {2.0 * a.hdx[0], 2.0 * a.hdx[1], 2.0 * a.hdx[2]};   // 1 / dx

    auto slot_of = [&](int m) { return (m + 4 * NRING) % NRING; };
    auto ingest = [&](int m) {
        const long long q = (long long)bc_map(m, nz, a.bc[2]) * plane + (long long)ys * nx + xs;
        double* r = ring + slot_of(m) * 5 * NT + tid;
#pragma unroll
        for (int i = 0; i < 5; ++i) r[i * NT] = __ldg(a.u_in + i * fs + q);
    };
    auto face_z = [&](int m, double F[5]) {   // face m+1/2 from planes m-1 .. m+2
        double v[5 * 4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const double* r = ring + slot_of(m - 1 + j) * 5 * NT + tid;
#pragma unroll
            for (int i = 0; i < 5; ++i) v[i * 4 + j] = r[i * NT];
        }
        if (!muscl_musta_face(k, 2, a.musta_k, a.limiter, v, 1, 4, F))
            if (atomicCAS(a.status, 0, 4) == 0) *a.bad_cell = -1;
    };

    double Fzm[5], Fzp[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) Fzm[i] = Fzp[i] = 0.0;
    if (zwork) {
        for (int m = zb - G; m <= zb + 1; ++m) ingest(m);
        face_z(zb - 1, Fzm);
    }
    unsigned long long amax[3] = {0ull, 0ull, 0ull};
    const int ncol = min(TX, nx - x0), nrow = min(TY, ny - y0);
    const int wx = ncol + 2 * G, hy = nrow + 2 * G;
    const int nfx = a.act[0] ? nrow * (ncol + 1) : 0;
    const int nfy = a.act[1] ? (nrow + 1) * ncol : 0;
    const int ngx = a.act[0] ? nrow * wx : 0;
    const int ngy = a.act[1] ? hy * ncol : 0;

    for (int p = zb; p < ze; ++p) {
        if (zwork) {
            ingest(p + G);
            face_z(p, Fzp);
        }
        const long long qz = (long long)bc_map(p, nz, a.bc[2]) * plane;
        for (int it = tid; it < ngx + ngy; it += NT) {
            if (it < ngx) {
                const int row = it / wx, col = it % wx;
                const long long q = qz + (long long)bc_map(y0 + row, ny, a.bc[1]) * nx + bc_map(x0 - G + col, nx, a.bc[0]);
#pragma unroll
                for (int i = 0; i < 5; ++i) ux[(i * TY + row) * GXW + col] = __ldg(a.u_in + i * fs + q);
            } else {
                const int j = it - ngx, row = j / ncol, col = j % ncol;
                const long long q = qz + (long long)bc_map(y0 - G + row, ny, a.bc[1]) * nx + bc_map(x0 + col, nx, a.bc[0]);
#pragma unroll
                for (int i = 0; i < 5; ++i) uy[(i * GYH + row) * TX + col] = __ldg(a.u_in + i * fs + q);
            }
        }
        __syncthreads();
        for (int it = tid; it < nfx + nfy; it += NT) {
            double F[5];
            bool ok;
            if (it < nfx) {
                const int row = it / (ncol + 1), f = it % (ncol + 1);   // face f - 1/2: cells f-2 .. f+1
                ok = muscl_musta_face(k, 0, a.musta_k, a.limiter, ux + row * GXW + f, 1, TY * GXW, F);
#pragma unroll
                for (int i = 0; i < 5; ++i) Fx[(i * TY + row) * (TX + 1) + f] = F[i];
            } else {
                const int j = it - nfx, f = j / ncol, col = j % ncol;
                ok = muscl_musta_face(k, 1, a.musta_k, a.limiter, uy + f * TX + col, TX, GYH * TX, F);
#pragma unroll
                for (int i = 0; i < 5; ++i) Fy[(i * (TY + 1) + f) * TX + col] = F[i];
            }
            if (!ok && atomicCAS(a.status, 0, 4) == 0) *a.bad_cell = -1;
        }
        __syncthreads();
        if (own) {
            const long long q = (long long)p * plane + (long long)y * nx + x;
            double un[5];
#pragma unroll
            for (int i = 0; i < 5; ++i) {
                double L = 0.0;
                if (a.act[0]) L = idx[0] * (Fx[(i * TY + ty) * (TX + 1) + tx] - Fx[(i * TY + ty) * (TX + 1) + tx + 1]);
                if (a.act[1]) L = fma(idx[1], Fy[(i * (TY + 1) + ty) * TX + tx] - Fy[(i * (TY + 1) + ty + 1) * TX + tx], L);
                if (a.act[2]) L = fma(idx[2], Fzm[i] - Fzp[i], L);
                const double s = fma(dt, L, __ldg(a.u_in + i * fs + q));
                un[i] = (a.ca == 0.0) ? s : fma(a.ca, a.u_n[i * fs + q], a.cb * s);
                a.u_out[i * fs + q] = un[i];
            }
            double pr, vx, vy, vz, e;
            if (con2prim(k, un[0], un[1], un[2], un[3], pr, vx, vy, vz, e)) {
                a.w_out[q] = pr;
                a.w_out[fs + q] = vx;
                a.w_out[2 * fs + q] = vy;
                a.w_out[3 * fs + q] = vz;
                double sp[3];
                max_speeds(k, vx, vy, vz, sp);
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const unsigned long long b = (unsigned long long)__double_as_longlong(sp[d]);
                    amax[d] = b > amax[d] ? b : amax[d];
                }
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i) a.w_out[i * fs + q] = 0.0;
                if (atomicCAS(a.status, 0, 4) == 0) *a.bad_cell = q;
            }
        }
#pragma unroll
        for (int i = 0; i < 5; ++i) Fzm[i] = Fzp[i];
    }
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

template <int TX, int TY>
__global__ void __launch_bounds__(TX * TY) musta_stage_kernel(const StageArgs a)
{
    extern __shared__ __align__(16) double smem[];
    musta_tile<TX, TY>(a, blockIdx.x, blockIdx.y, blockIdx.z, smem);
}

}  // namespace hydro
