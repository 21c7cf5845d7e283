// char_weno.cuh -- characteristic-wise FD-WENO face flux (Sec. 1.2 applied to
// the characteristic fields of the flux Jacobian instead of the components
// of u) for the fused stage kernel.
//
// At the face j+1/2 along axis d the split fluxes g+- = f_d +- alpha u of the
// 2r cells j-r+1 .. j+r are projected on the characteristic fields of the
// face state, reconstructed field by field, and mapped back:
//     F = R_d  WENO( L_d g )      with  L_d = R_d^{-1}
// The face state is the mean of the conserved states of cells j and j+1
// (recovered as (g+ - g-) / (2 alpha)).  Its right eigenvectors are the
// changes of u for a unit change of e along a sound wave (eigenvalues
// lambda_-+), of one transverse velocity (shear waves) or of one charge
// density (both with eigenvalue v_d).
//
// GB300 form: no matrix is built.  R_d = J R_w, where J = du/dw is the
// linearised primitive -> conserved map at the face state and R_w holds the
// eigenvectors in primitive variables (sparse: the shear and charge columns
// are unit vectors, the sound columns (1, X, Y_t1, Y_t2, N_q)).  So
//   L_d g = R_w^{-1} (J^{-1} g):  J^{-1} g is the linearised primitive
//   recovery (differentiating k e^2 + (1-k) E e - (E^2 - M^2) = 0,
//   v = M / (E + k e), n = R / gamma), and R_w^{-1} needs one 2x2 inverse;
//   R_d c = J (R_w c).
// About 26 FP64 operations per projected vector (NF = 5) and 30 for the
// back-projection, with 9 reciprocals and 3 square roots of setup per face.
// Fields are handled in the face's own frame: (E, M_d, M_t1, M_t2, R...),
// t1 = (d+1)%3, t2 = (d+2)%3; the caller maps them to memory.  Staged x/y
// faces read g+- from shared memory and recover the face state as
// (g+ - g-) / (2 alpha); z faces read a per-column ring of (u, p, v_z) and
// form g+- and the face state from it.
#pragma once
#include "hydro_math.cuh"

namespace hydro {

// memory field index of rotated field k along axis d
__device__ __forceinline__ int rot_field(int k, int d)
{
    if (k == 0 || k >= 4) return k;
    const int a = d + k - 1;   // k = 1 -> d, 2 -> d+1, 3 -> d+2 (mod 3)
    return 1 + (a >= 3 ? a - 3 : a);
}

// The characteristic basis of one face state (rotated fields): what the
// projection L_d g and the back-projection R_d c need.
template <int NF>
struct CharBasis {
    static constexpr int NQ = NF - 4, NQ1 = NQ > 0 ? NQ : 1;
    double k;                        // cs2
    double vn, v1, v2;               // face-state velocity (normal, two transverse)
    double ig, g2, gam, K;           // 1/gamma, gamma^2, gamma, (e + p) gamma^2
    double nq[NQ1];                  // charge densities n_q = R_q / gamma
    double X[2], Y1[2], Y2[2];       // sound eigenvectors in primitive variables (de = 1)
    double Nw[2][NQ1];
    double iX, A0, A1;               // the 2 x 2 inverse on (de, dv_n)
    double aE, aN, a1, a2, iEp;      // linearised primitive recovery
};

// Basis at the rotated face state ub.  Returns false if the face state is
// not physical.
template <int NF>
__device__ __forceinline__ bool char_setup(const double* ub, double k, CharBasis<NF>& B)
{
    constexpr int NQ = NF - 4;
    double pr, e;
    if (!con2prim(k, ub[0], ub[1], ub[2], ub[3], pr, B.vn, B.v1, B.v2, e)) return false;
    B.k = k;
    const double vn = B.vn, v1 = B.v1, v2 = B.v2;
    const double vsq = fma(vn, vn, fma(v1, v1, v2 * v2));
    const double om = 1.0 - vsq;
    B.ig = sqrt(om);                 // 1 / gamma
    B.g2 = rcp(om);                  // gamma^2
    B.gam = B.ig * B.g2;             // gamma
    B.K = (1.0 + k) * e * B.g2;      // (e + p) gamma^2
    const double K = B.K, g2 = B.g2;
#pragma unroll
    for (int q = 0; q < NQ; ++q) B.nq[q] = ub[4 + q] * B.ig;

    // sound speeds and the primitive-space sound eigenvectors (de = 1):
    //    dv_d = k (1 - lam v_d) / (K (lam - v_d)), dv_t = -lam k v_t / (K (lam - v_d)),
    //    dn_q = n_q (dv_d / (lam - v_d) - gamma^2 v.dv)
    const double root = sqrt(k * om * fma(-k, vsq - vn * vn, fma(-vn, vn, 1.0)));
    const double iden = rcp(fma(-k, vsq, 1.0));
    const double b0 = vn * (1.0 - k);
    const double lam[2] = {(b0 - root) * iden, (b0 + root) * iden};
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const double dl = lam[s] - vn;
        const double D = rcp(K * dl);
        B.X[s] = k * fma(-lam[s], vn, 1.0) * D;
        const double ly = -lam[s] * k * D;
        B.Y1[s] = ly * v1;
        B.Y2[s] = ly * v2;
        const double vdv = fma(vn, B.X[s], fma(v1, B.Y1[s], v2 * B.Y2[s]));
        const double a = fma(B.X[s], K * D, -g2 * vdv);    // 1 / (lam - v_d) = K D
#pragma unroll
        for (int q = 0; q < NQ; ++q) B.Nw[s][q] = B.nq[q] * a;
    }
    B.iX = rcp(B.X[1] - B.X[0]);
    B.A0 = B.X[1] * B.iX;
    B.A1 = B.X[0] * B.iX;

    // linearised primitive recovery at the face state
    const double Dn = rcp(fma(2.0 * k, e, (1.0 - k) * ub[0]));
    B.aE = fma(-(1.0 - k), e, 2.0 * ub[0]) * Dn;
    const double m2 = -2.0 * Dn;
    B.aN = m2 * ub[1];
    B.a1 = m2 * ub[2];
    B.a2 = m2 * ub[3];
    B.iEp = rcp(fma(k, e, ub[0]));
    return true;
}

// Characteristic fields c = L_d g of one rotated split-flux vector, read
// through g(m) (m = 0 .. NF-1).
template <int NF, class GA>
__device__ __forceinline__ void char_project(const CharBasis<NF>& B, GA g, double* c)
{
    constexpr int NQ = NF - 4;
    const double k = B.k;
    const double gE = g(0), gN = g(1), g1 = g(2), g2v = g(3);
    const double de = fma(B.aE, gE, fma(B.aN, gN, fma(B.a1, g1, B.a2 * g2v)));
    const double t = fma(k, de, gE);
    const double dvn = fma(-B.vn, t, gN) * B.iEp;
    const double dv1 = fma(-B.v1, t, g1) * B.iEp;
    const double dv2 = fma(-B.v2, t, g2v) * B.iEp;
    const double cm = fma(B.A0, de, -B.iX * dvn);
    const double cp = fma(B.iX, dvn, -B.A1 * de);
    c[0] = cm;
    c[1] = cp;
    c[2] = fma(-B.Y1[1], cp, fma(-B.Y1[0], cm, dv1));
    c[3] = fma(-B.Y2[1], cp, fma(-B.Y2[0], cm, dv2));
    if constexpr (NQ > 0) {
        const double vdv = fma(B.vn, dvn, fma(B.v1, dv1, B.v2 * dv2));
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const double dn = fma(g(4 + q), B.ig, -B.nq[q] * B.g2 * vdv);
            c[4 + q] = fma(-B.Nw[1][q], cp, fma(-B.Nw[0][q], cm, dn));
        }
    }
}

// Back to conserved fluxes: dw = R_w Fc, F = J dw (rotated fields).
template <int NF>
__device__ __forceinline__ void char_back(const CharBasis<NF>& B, const double* Fc, double* F)
{
    constexpr int NQ = NF - 4;
    const double k = B.k, K = B.K;
    const double de = Fc[0] + Fc[1];
    const double dvn = fma(B.X[1], Fc[1], B.X[0] * Fc[0]);
    const double dv1 = fma(B.Y1[1], Fc[1], fma(B.Y1[0], Fc[0], Fc[2]));
    const double dv2 = fma(B.Y2[1], Fc[1], fma(B.Y2[0], Fc[0], Fc[3]));
    const double vdv = fma(B.vn, dvn, fma(B.v1, dv1, B.v2 * dv2));
    const double Q = B.g2 * fma(2.0 * K, vdv, (1.0 + k) * de);
    F[0] = fma(-k, de, Q);
    F[1] = fma(Q, B.vn, K * dvn);
    F[2] = fma(Q, B.v1, K * dv1);
    F[3] = fma(Q, B.v2, K * dv2);
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const double dn = fma(B.Nw[1][q], Fc[1], fma(B.Nw[0][q], Fc[0], Fc[4 + q]));
        F[4 + q] = B.gam * fma(B.nq[q] * B.g2, vdv, dn);
    }
}

// Characteristic-wise face flux (scaled like g: 2 F).  gval(i, m, s) returns
// rotated field m of the split flux g+ (s = 0) or g- (s = 1) of window cell i
// (i = 0 .. 2r-1, cell j-r+1+i); ub holds the rotated face state, the mean of
// the conserved states of window cells r-1 and r.  Returns false (F = 0) if
// the face state is not physical.
template <int R, int NF, class GV, int EMU = 0>
__device__ __forceinline__ bool char_face(GV gval, const double* ub, double k, double eps_s, double* F)
{
    constexpr int S = 2 * R - 1;
    CharBasis<NF> B;
    if (!char_setup<NF>(ub, k, B)) {
#pragma unroll
        for (int m = 0; m < NF; ++m) F[m] = 0.0;
        return false;
    }
    // reconstruct: + side from cells 0 .. S-1, - side from cells 1 .. S
    double Np[NF], Dp[NF], Cp[NF], Fc[NF];
    {
        double v[NF][S];
#pragma unroll
        for (int i = 0; i < S; ++i) {
            double c[NF];
            char_project<NF>(B, [&](int m) { return gval(i, m, 0); }, c);
#pragma unroll
            for (int m = 0; m < NF; ++m) v[m][i] = c[m];
        }
#pragma unroll
        for (int m = 0; m < NF; ++m) {
            weno_left<R, EMU>(v[m], eps_s, Np[m], Dp[m]);
            Cp[m] = v[m][R - 1];
        }
    }
    {
        double v[NF][S];
#pragma unroll
        for (int i = 0; i < S; ++i) {
            double c[NF];
            char_project<NF>(B, [&](int m) { return gval(i + 1, m, 1); }, c);
#pragma unroll
            for (int m = 0; m < NF; ++m) v[m][i] = c[m];
        }
#pragma unroll
        for (int m = 0; m < NF; ++m) {
            double Nm, Dm;
            weno_right<R, EMU>(v[m], eps_s, Nm, Dm);
            Fc[m] = face_sum(Np[m], Dp[m], Cp[m], Nm, Dm, v[m][R - 1]);
        }
    }
    char_back<NF>(B, Fc, F);
    return true;
}

}  // namespace hydro
