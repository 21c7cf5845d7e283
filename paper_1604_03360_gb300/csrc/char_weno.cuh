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

// Characteristic-wise face flux (scaled like g: 2 F).  gval(i, m, s) returns
// rotated field m of the split flux g+ (s = 0) or g- (s = 1) of window cell i
// (i = 0 .. 2r-1, cell j-r+1+i); ub holds the rotated face state, the mean of
// the conserved states of window cells r-1 and r.  Returns false (F = 0) if
// the face state is not physical.
template <int R, int NF, class GV, int EMU = 0>
__device__ __forceinline__ bool char_face(GV gval, const double* ub, double k, double eps_s, double* F)
{
    constexpr int S = 2 * R - 1, NQ = NF - 4;
    double pr, vn, v1, v2, e;
    if (!con2prim(k, ub[0], ub[1], ub[2], ub[3], pr, vn, v1, v2, e)) {
#pragma unroll
        for (int m = 0; m < NF; ++m) F[m] = 0.0;
        return false;
    }
    const double vsq = fma(vn, vn, fma(v1, v1, v2 * v2));
    const double om = 1.0 - vsq;
    const double ig = sqrt(om);          // 1 / gamma
    const double g2 = rcp(om);           // gamma^2
    const double gam = ig * g2;          // gamma
    const double K = (1.0 + k) * e * g2; // (e + p) gamma^2
    double nq[NQ > 0 ? NQ : 1];
#pragma unroll
    for (int q = 0; q < NQ; ++q) nq[q] = ub[4 + q] * ig;

    // 2. sound speeds and the primitive-space sound eigenvectors (de = 1):
    //    dv_d = k (1 - lam v_d) / (K (lam - v_d)), dv_t = -lam k v_t / (K (lam - v_d)),
    //    dn_q = n_q (dv_d / (lam - v_d) - gamma^2 v.dv)
    const double root = sqrt(k * om * fma(-k, vsq - vn * vn, fma(-vn, vn, 1.0)));
    const double iden = rcp(fma(-k, vsq, 1.0));
    const double b0 = vn * (1.0 - k);
    const double lam[2] = {(b0 - root) * iden, (b0 + root) * iden};
    double X[2], Y1[2], Y2[2], Nw[2][NQ > 0 ? NQ : 1];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const double dl = lam[s] - vn;
        const double D = rcp(K * dl);
        X[s] = k * fma(-lam[s], vn, 1.0) * D;
        const double ly = -lam[s] * k * D;
        Y1[s] = ly * v1;
        Y2[s] = ly * v2;
        const double vdv = fma(vn, X[s], fma(v1, Y1[s], v2 * Y2[s]));
        const double a = fma(X[s], K * D, -g2 * vdv);    // 1 / (lam - v_d) = K D
#pragma unroll
        for (int q = 0; q < NQ; ++q) Nw[s][q] = nq[q] * a;
    }
    const double iX = rcp(X[1] - X[0]);
    const double A0 = X[1] * iX, A1 = X[0] * iX;

    // 3. linearised primitive recovery at the face state
    const double Dn = rcp(fma(2.0 * k, e, (1.0 - k) * ub[0]));
    const double aE = fma(-(1.0 - k), e, 2.0 * ub[0]) * Dn;
    const double m2 = -2.0 * Dn;
    const double aN = m2 * ub[1], a1 = m2 * ub[2], a2 = m2 * ub[3];
    const double iEp = rcp(fma(k, e, ub[0]));

    // characteristic fields of the split-flux vector g+ (s = 0) or g- (s = 1) of cell i
    auto project = [&](int i, int s, double* c) {
        const double gE = gval(i, 0, s), gN = gval(i, 1, s), g1 = gval(i, 2, s), g2v = gval(i, 3, s);
        const double de = fma(aE, gE, fma(aN, gN, fma(a1, g1, a2 * g2v)));
        const double t = fma(k, de, gE);
        const double dvn = fma(-vn, t, gN) * iEp;
        const double dv1 = fma(-v1, t, g1) * iEp;
        const double dv2 = fma(-v2, t, g2v) * iEp;
        const double cm = fma(A0, de, -iX * dvn);
        const double cp = fma(iX, dvn, -A1 * de);
        c[0] = cm;
        c[1] = cp;
        c[2] = fma(-Y1[1], cp, fma(-Y1[0], cm, dv1));
        c[3] = fma(-Y2[1], cp, fma(-Y2[0], cm, dv2));
        if constexpr (NQ > 0) {
            const double vdv = fma(vn, dvn, fma(v1, dv1, v2 * dv2));
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const double dn = fma(gval(i, 4 + q, s), ig, -nq[q] * g2 * vdv);
                c[4 + q] = fma(-Nw[1][q], cp, fma(-Nw[0][q], cm, dn));
            }
        }
    };

    // 4. reconstruct: + side from cells 0 .. S-1, - side from cells 1 .. S
    double Np[NF], Dp[NF], Cp[NF], Fc[NF];
    {
        double v[NF][S];
#pragma unroll
        for (int i = 0; i < S; ++i) {
            double c[NF];
            project(i, 0, c);
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
            project(i + 1, 1, c);
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

    // 5. back to conserved fluxes: dw = R_w Fc, F = J dw
    const double de = Fc[0] + Fc[1];
    const double dvn = fma(X[1], Fc[1], X[0] * Fc[0]);
    const double dv1 = fma(Y1[1], Fc[1], fma(Y1[0], Fc[0], Fc[2]));
    const double dv2 = fma(Y2[1], Fc[1], fma(Y2[0], Fc[0], Fc[3]));
    const double vdv = fma(vn, dvn, fma(v1, dv1, v2 * dv2));
    const double Q = g2 * fma(2.0 * K, vdv, (1.0 + k) * de);
    F[0] = fma(-k, de, Q);
    F[1] = fma(Q, vn, K * dvn);
    F[2] = fma(Q, v1, K * dv1);
    F[3] = fma(Q, v2, K * dv2);
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const double dn = fma(Nw[1][q], Fc[1], fma(Nw[0][q], Fc[0], Fc[4 + q]));
        F[4 + q] = gam * fma(nq[q] * g2, vdv, dn);
    }
    return true;
}

}  // namespace hydro
