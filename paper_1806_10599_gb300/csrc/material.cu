// Per-voxel constitutive update P, K = dP/dF (Eqs. constitutive, P_dif) and
// the fatigue-indicator accumulators (Sect. 3.3).
//
// St.Venant-Kirchhoff: E = (F^T F - I)/2, S = C:E, P = F S,
//   K_ijkl = delta_ik S_lj + F_ip C_pjln F_kn.
// FCC crystal plasticity (12 {111}<110> systems, flow rule of Eq. gamma_dot
// with a constant resistance tau0 and an Armstrong-Frederick backstress):
//   Fp^-1 = Fp^-1_n (I - sum_a dg_a S0_a), Fe = F Fp^-1, Ce = Fe^T Fe,
//   S = C : (Ce - I)/2, tau_a = (Ce S) : S0_a,
//   chi_a = (chi_n,a + c dg_a) / (1 + d |dg_a|),
//   r_a = dg_a - dt gdot0 h((tau_a - chi_a)/tau0),  h(x) = |x|^p sign(x),
// solved for dg by Newton, then
//   P = Fe S Fp^-T and K by implicit differentiation of r(dg, F) = 0.
// The local Newton starts from the slip increments of the previous global
// Newton iterate when there is one (else from 0) and takes its steps with the
// per-grain small-elastic-strain Jacobian, solved as a 5x5 system on the
// deviatoric strains (cp_correction_lowrank); the residual is always exact,
// so it converges to the same root.  The exact 12x12 Jacobian is assembled
// once, at the root, for the tangent (LU with partial pivoting).  If the fast
// iteration fails, the return map restarts from dg = 0 with exact Newton
// steps (12x12 LU with partial pivoting) -- the fallback; a handle can also
// ask for that exact iteration alone (gff_set_return_map).
// Everything is FP64.  One thread per voxel.
#include <cmath>

#include "gff_internal.cuh"

namespace gff {
namespace {

constexpr int TPB = 128;

// ---------------------------------------------------------------- small dense helpers (row-major 3x3)
template <typename T> __device__ __forceinline__ void mm(const T* a, const T* b, T* c) {  // c = a b
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) c[3 * i + j] = a[3 * i] * b[j] + a[3 * i + 1] * b[3 + j] + a[3 * i + 2] * b[6 + j];
}
template <typename T> __device__ __forceinline__ void mtm(const T* a, const T* b, T* c) {  // c = a^T b
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) c[3 * i + j] = a[i] * b[j] + a[3 + i] * b[3 + j] + a[6 + i] * b[6 + j];
}
template <typename T> __device__ __forceinline__ void mmt(const T* a, const T* b, T* c) {  // c = a b^T
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            c[3 * i + j] = a[3 * i] * b[3 * j] + a[3 * i + 1] * b[3 * j + 1] + a[3 * i + 2] * b[3 * j + 2];
}
__device__ __forceinline__ double ddot9(const double* a, const double* b) {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 9; ++k) s = fma(a[k], b[k], s);
    return s;
}
// S = C : E (C has minor symmetries; stored in TC, used in T)
template <typename T, typename TC>
__device__ __forceinline__ void c_ddot(const TC* __restrict__ C, const T* E, T* S) {
#pragma unroll
    for (int ij = 0; ij < 9; ++ij) {
        const TC* Cr = C + 9 * ij;
        T s = (T)0;
#pragma unroll
        for (int kl = 0; kl < 9; ++kl) s = fma((T)__ldg(Cr + kl), E[kl], s);
        S[ij] = s;
    }
}

__device__ __forceinline__ double ipow(double a, int p) {  // a >= 0, p >= 0
    double r = 1.0, b = a;
    while (p) {
        if (p & 1) r *= b;
        b *= b;
        p >>= 1;
    }
    return r;
}

template <typename T> __device__ __forceinline__ T sgn(T v) { return (T)((v > (T)0) - (v < (T)0)); }

struct CPOut {
    double P[9];
    double Fpi[9];
    double chi[12];
    double dg[12];
    double tau[12];
    bool ok;
    bool fallback;  // the small-strain iteration failed; the exact Newton from zero ran
    int iters;      // local Newton iterations in FP64, both tries
    int iters32;    // FP32 pre-iterations
};

// LU with partial pivoting of an NN x NN row-major matrix, in place.
template <int NN, typename T>
__device__ bool lu_factor(T* a, int* piv) {
    for (int k = 0; k < NN; ++k) {
        int p = k;
        T m = fabs(a[k * NN + k]);
        for (int i = k + 1; i < NN; ++i) {
            const T v = fabs(a[i * NN + k]);
            if (v > m) {
                m = v;
                p = i;
            }
        }
        piv[k] = p;
        if (m == (T)0) return false;
        if (p != k)
            for (int j = 0; j < NN; ++j) {
                const T t = a[k * NN + j];
                a[k * NN + j] = a[p * NN + j];
                a[p * NN + j] = t;
            }
        const T inv = (T)1 / a[k * NN + k];
        for (int i = k + 1; i < NN; ++i) {
            const T l = a[i * NN + k] * inv;
            a[i * NN + k] = l;
            for (int j = k + 1; j < NN; ++j) a[i * NN + j] = fma(-l, a[k * NN + j], a[i * NN + j]);
        }
    }
    return true;
}
template <int NN, typename T>
__device__ void lu_solve(const T* a, const int* piv, T* b) {
    for (int k = 0; k < NN; ++k) {
        const int p = piv[k];
        if (p != k) {
            const T t = b[k];
            b[k] = b[p];
            b[p] = t;
        }
    }
    for (int i = 1; i < NN; ++i) {
        T s = b[i];
        for (int j = 0; j < i; ++j) s = fma(-a[i * NN + j], b[j], s);
        b[i] = s;
    }
    for (int i = NN - 1; i >= 0; --i) {
        T s = b[i];
        for (int j = i + 1; j < NN; ++j) s = fma(-a[i * NN + j], b[j], s);
        b[i] = s / a[i * NN + i];
    }
}

// Elastic state for slip increments dg: Fpi, Fe, Ce, S, M = Ce S, tau.
template <typename T> struct ElStateT {
    T Fpi[9], Fe[9], Ce[9], S[9], M[9], tau[12];
};
using ElState = ElStateT<double>;

// Uses the grain's slip planes (three systems per normal m_p) and the Voigt
// stiffness: Lp = sum_p (sum_(a in p) dg_a s_a) (x) m_p, tau_a = s_a . (M m_p),
// Ce and S computed as the symmetric tensors they are.
__device__ void elastic_state(const double* F, const double* A, const double* dg, const double* __restrict__ geo,
                              ElState& st) {
    const double* sd = geo + GEO_DIR;
    const double* mn = geo + GEO_NRM;
    const double* C6 = geo + GEO_C6;
    double Lp[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) Lp[k] = 0.0;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        double v[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) v[j] = fma(dg[3 * p + i], __ldg(sd + 3 * (3 * p + i) + j), v[j]);
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = 0; k < 3; ++k) Lp[3 * j + k] = fma(v[j], __ldg(mn + 3 * p + k), Lp[3 * j + k]);
    }
    double IL[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) IL[k] = ((k % 4) == 0 ? 1.0 : 0.0) - Lp[k];
    mm(A, IL, st.Fpi);
    mm(F, st.Fpi, st.Fe);
    // Ce = Fe^T Fe (symmetric)
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            const double c = st.Fe[i] * st.Fe[j] + st.Fe[3 + i] * st.Fe[3 + j] + st.Fe[6 + i] * st.Fe[6 + j];
            st.Ce[3 * i + j] = c;
            st.Ce[3 * j + i] = c;
        }
    // S = C : E, E = (Ce - I) / 2, in Voigt form (engineering shears)
    const double e[6] = {0.5 * (st.Ce[0] - 1.0), 0.5 * (st.Ce[4] - 1.0), 0.5 * (st.Ce[8] - 1.0),
                         st.Ce[5], st.Ce[2], st.Ce[1]};
    double sv[6];
#pragma unroll
    for (int I = 0; I < 6; ++I) {
        double t = 0.0;
#pragma unroll
        for (int J = 0; J < 6; ++J) t = fma(__ldg(C6 + 6 * I + J), e[J], t);
        sv[I] = t;
    }
    st.S[0] = sv[0], st.S[4] = sv[1], st.S[8] = sv[2];
    st.S[5] = st.S[7] = sv[3];
    st.S[2] = st.S[6] = sv[4];
    st.S[1] = st.S[3] = sv[5];
    mm(st.Ce, st.S, st.M);
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const double m0 = __ldg(mn + 3 * p), m1 = __ldg(mn + 3 * p + 1), m2 = __ldg(mn + 3 * p + 2);
        double Mm[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) Mm[j] = st.M[3 * j] * m0 + st.M[3 * j + 1] * m1 + st.M[3 * j + 2] * m2;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const double* s = sd + 3 * (3 * p + i);
            st.tau[3 * p + i] = __ldg(s) * Mm[0] + __ldg(s + 1) * Mm[1] + __ldg(s + 2) * Mm[2];
        }
    }
}

// Derivatives with respect to dg_b at fixed F:
//   dFpi_b = -A S0_b, dFe_b = F dFpi_b, dCe_b = dFe_b^T Fe + Fe^T dFe_b,
//   dS_b = C : dCe_b / 2.
template <typename T>
__device__ void dstate_ddg(const T* F, const T* A, const T* __restrict__ S0_b, const T* __restrict__ C,
                           const ElStateT<T>& st, T* dFpi, T* dFe, T* dCe, T* dS) {
    T Sb[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) Sb[k] = __ldg(S0_b + k);
    mm(A, Sb, dFpi);
#pragma unroll
    for (int k = 0; k < 9; ++k) dFpi[k] = -dFpi[k];
    mm(F, dFpi, dFe);
    T t1[9];
    mtm(dFe, st.Fe, t1);
    T hE[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            dCe[3 * i + j] = t1[3 * i + j] + t1[3 * j + i];  // Fe^T dFe = (dFe^T Fe)^T
            hE[3 * i + j] = (T)0.5 * dCe[3 * i + j];
        }
    c_ddot(C, hE, dS);
}

// Residual r_a(dg) and the quantities the Jacobians need; returns max |r_a|.
// iden[a] = 1 / (1 + d |dg_a|), the backstress denominator, kept for the correction.
__device__ double cp_residual(const double* F, const double* A, const double* chin, const double* dg,
                              const double* __restrict__ geo, const CPParamsDev& pr, double coef, int p, ElState& st,
                              double* chi, double* dh, double* r, double* iden) {
    elastic_state(F, A, dg, geo, st);
    // the twelve denominators 1 + d |dg_a| inverted with one FP64 division
    // (simultaneous inversion: prefix products, one reciprocal of the last,
    // back-substitution), unless their product leaves the finite range
    double den[NSLIP], pre[NSLIP];
#pragma unroll
    for (int a = 0; a < NSLIP; ++a) {
        den[a] = fma(pr.d, fabs(dg[a]), 1.0);
        pre[a] = a ? pre[a - 1] * den[a] : den[a];
    }
    if (pre[NSLIP - 1] < 1e300) {
        double inv = 1.0 / pre[NSLIP - 1];
#pragma unroll
        for (int a = NSLIP - 1; a > 0; --a) {
            iden[a] = inv * pre[a - 1];
            inv *= den[a];
        }
        iden[0] = inv;
    } else {
        for (int a = 0; a < NSLIP; ++a) iden[a] = 1.0 / den[a];
    }
    const double pd = (double)p;
    double rmax = 0.0;
#pragma unroll
    for (int a = 0; a < NSLIP; ++a) {
        chi[a] = (chin[a] + pr.c * dg[a]) * iden[a];
        const double x = (st.tau[a] - chi[a]) * pr.itau0;
        const double ax = fabs(x);
        const double axp1 = ipow(ax, p - 1);
        dh[a] = pd * axp1;
        r[a] = dg[a] - coef * copysign(axp1 * ax, x);
        rmax = fmax(rmax, fabs(r[a]));
    }
    return rmax;
}

// Exact Jacobian dr_a/ddg_b at the state st, in precision T (S0 and C given in T).
template <typename T>
__device__ void cp_jacobian_exact(const T* F, const T* A, const T* dg, const T* __restrict__ S0,
                                  const T* __restrict__ C, const CPParamsDev& pr, double coef,
                                  const ElStateT<T>& st, const T* chi, const T* dh, T* J) {
    const T cg = (T)(coef / pr.tau0), c = (T)pr.c, d = (T)pr.d;
    for (int b = 0; b < NSLIP; ++b) {
        T dFpi[9], dFe[9], dCe[9], dS[9], dM[9], t1[9];
        dstate_ddg(F, A, S0 + 9 * b, C, st, dFpi, dFe, dCe, dS);
        mm(dCe, st.S, dM);
        mm(st.Ce, dS, t1);
#pragma unroll
        for (int k = 0; k < 9; ++k) dM[k] += t1[k];
        for (int a = 0; a < NSLIP; ++a) {
            T dtau = (T)0;
#pragma unroll
            for (int k = 0; k < 9; ++k) dtau = fma(dM[k], __ldg(S0 + 9 * a + k), dtau);
            T v = -cg * dh[a] * dtau;
            if (a == b) {
                const T den = (T)1 + d * fabs(dg[a]);
                const T dchi = (c - d * sgn(dg[a]) * chi[a]) / den;
                v += (T)1 + cg * dh[a] * dchi;
            }
            J[a * NSLIP + b] = v;
        }
    }
}

// Newton correction with the small-elastic-strain Jacobian.  At Ce ~ I and
// S << C, dtau_a/ddg_b ~ -H_ab with the per-grain constant
// H_ab = S0_a : C : sym(S0_b), so J = D + F H with the diagonals
// D_a = 1 + f_a dchi_a >= 1 and F_a = f_a = (coef/tau0) h'_a >= 0.  The
// symmetric traceless sym(S0_a) live in the 5-dimensional deviatoric space:
// with an orthonormal basis e_i of it, sym(S0_a) = sum_i P_ia e_i and
// H = P^T C5 P, C5_ij = e_i : C : e_j.  J x = r is then solved through the
// 5 x 5 SPD system (C5^-1 + P G P^T) u = P D^-1 r, G = D^-1 F, and
// x = D^-1 (r - F P^T u) -- the same correction as a 12 x 12 solve with J,
// at a fraction of the work and registers.  PC holds P [5][12] then C5^-1
// [5][5] for the grain.  The correction only steers the iteration: the FP64
// residual decides convergence.
template <typename TJ>
__device__ __forceinline__ bool cp_correction_lowrank(const double* __restrict__ PC, const double* dg,
                                                      const CPParamsDev& pr, double coef, const double* chi,
                                                      const double* dh, const double* iden, const double* r,
                                                      double* x) {
    const TJ cg = (TJ)(coef * pr.itau0), c = (TJ)pr.c, d = (TJ)pr.d;
    TJ A[15], b[5];  // packed lower triangle of C5^-1 + P G P^T, and P D^-1 r
    {
        int k = 0;
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            b[i] = (TJ)0;
#pragma unroll
            for (int j = 0; j <= i; ++j) A[k++] = (TJ)__ldg(PC + 60 + 5 * i + j);
        }
    }
    TJ f[NSLIP], Di[NSLIP];
#pragma unroll
    for (int a = 0; a < NSLIP; ++a) {
        f[a] = cg * (TJ)dh[a];
        const TJ dga = (TJ)dg[a];
        const TJ dchi = (c - d * sgn(dga) * (TJ)chi[a]) * (TJ)iden[a];
        // the correction only steers the iteration: an FP32 reciprocal is accurate enough
        Di[a] = (TJ)__frcp_rn((float)((TJ)1 + f[a] * dchi));
        const TJ ga = f[a] * Di[a], ra = (TJ)r[a] * Di[a];
        TJ p[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) p[i] = (TJ)__ldg(PC + 12 * i + a);
        int k = 0;
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            b[i] = fma(ra, p[i], b[i]);
#pragma unroll
            for (int j = 0; j <= i; ++j) A[k] = fma(ga * p[i], p[j], A[k]), ++k;
        }
    }
    // A = L diag(q) L^T (no pivoting: A is SPD)
    TJ L[5][5], q[5], iq[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        TJ s = A[j * (j + 1) / 2 + j];
#pragma unroll
        for (int k = 0; k < j; ++k) s -= L[j][k] * L[j][k] * q[k];
        if (!(s > (TJ)0)) return false;
        q[j] = s;
        const TJ inv = (TJ)1 / s;
        iq[j] = inv;
#pragma unroll
        for (int i = j + 1; i < 5; ++i) {
            TJ t = A[i * (i + 1) / 2 + j];
#pragma unroll
            for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k] * q[k];
            L[i][j] = t * inv;
        }
    }
    TJ u[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        TJ t = b[i];
#pragma unroll
        for (int k = 0; k < i; ++k) t -= L[i][k] * u[k];
        u[i] = t;
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) u[i] *= iq[i];
#pragma unroll
    for (int i = 4; i >= 0; --i) {
#pragma unroll
        for (int k = i + 1; k < 5; ++k) u[i] -= L[k][i] * u[k];
    }
#pragma unroll
    for (int a = 0; a < NSLIP; ++a) {
        TJ t = (TJ)0;
#pragma unroll
        for (int i = 0; i < 5; ++i) t = fma((TJ)__ldg(PC + 12 * i + a), u[i], t);
        x[a] = (double)(Di[a] * ((TJ)r[a] - f[a] * t));
    }
    return true;
}

// ---------------------------------------------------------------- FP32 pre-iteration
// The same iteration as the FP64 one (exact residual, small-elastic-strain
// corrections), in FP32.  With f = F - I, a = Fp^-1_n - I and G = Fe - I all
// small, the elastic state is formed from them directly --
//   Fp^-1 - I = a - Lp - a Lp,  G = (Fp^-1 - I) + f + f (Fp^-1 - I),
//   E = (G + G^T + G^T G) / 2,  M = Ce S = S + 2 E S --
// so FP32 keeps its relative accuracy on E instead of losing it in Ce - I.
// It stops at FP32 resolution (or when it stalls); the FP64 iteration then
// starts from its iterate.  It only steers: the FP64 residual decides
// convergence, so the root does not change.
__device__ __forceinline__ float ipowf_n(float a, int p) {  // a >= 0, p >= 0
    float r = 1.f, b = a;
    while (p) {
        if (p & 1) r *= b;
        b *= b;
        p >>= 1;
    }
    return r;
}

__device__ void elastic_tau_f32(const float* f, const float* a, const float* dg, const float* __restrict__ g,
                                float* tau) {
    const float* sd = g + G32_DIR;
    const float* mn = g + G32_NRM;
    const float* C6 = g + G32_C6;
    float Lp[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) Lp[k] = 0.f;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        float v[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) v[j] = fmaf(dg[3 * p + i], __ldg(sd + 3 * (3 * p + i) + j), v[j]);
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = 0; k < 3; ++k) Lp[3 * j + k] = fmaf(v[j], __ldg(mn + 3 * p + k), Lp[3 * j + k]);
    }
    float aL[9], q[9], fq[9], G[9], GtG[9];
    mm(a, Lp, aL);
#pragma unroll
    for (int k = 0; k < 9; ++k) q[k] = a[k] - Lp[k] - aL[k];  // Fp^-1 - I
    mm(f, q, fq);
#pragma unroll
    for (int k = 0; k < 9; ++k) G[k] = q[k] + f[k] + fq[k];  // Fe - I
    mtm(G, G, GtG);
    float E[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) E[3 * i + j] = 0.5f * (G[3 * i + j] + G[3 * j + i] + GtG[3 * i + j]);
    const float e[6] = {E[0], E[4], E[8], 2.f * E[5], 2.f * E[2], 2.f * E[1]};  // Voigt, engineering shears
    float sv[6];
#pragma unroll
    for (int I = 0; I < 6; ++I) {
        float t = 0.f;
#pragma unroll
        for (int J = 0; J < 6; ++J) t = fmaf(__ldg(C6 + 6 * I + J), e[J], t);
        sv[I] = t;
    }
    float S[9];
    S[0] = sv[0], S[4] = sv[1], S[8] = sv[2];
    S[5] = S[7] = sv[3];
    S[2] = S[6] = sv[4];
    S[1] = S[3] = sv[5];
    float ES[9], M[9];
    mm(E, S, ES);
#pragma unroll
    for (int k = 0; k < 9; ++k) M[k] = fmaf(2.f, ES[k], S[k]);
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const float m0 = __ldg(mn + 3 * p), m1 = __ldg(mn + 3 * p + 1), m2 = __ldg(mn + 3 * p + 2);
        float Mm[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) Mm[j] = M[3 * j] * m0 + M[3 * j + 1] * m1 + M[3 * j + 2] * m2;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float* sv3 = sd + 3 * (3 * p + i);
            tau[3 * p + i] = __ldg(sv3) * Mm[0] + __ldg(sv3 + 1) * Mm[1] + __ldg(sv3 + 2) * Mm[2];
        }
    }
}

struct F32Consts {
    float cf, c, d, it0;
    int p;
};

__device__ float cp_residual_f32(const float* f, const float* a, const float* chn, const float* dg,
                                 const float* __restrict__ g, const F32Consts& k, float* chi, float* dh, float* r,
                                 float* iden) {
    float tau[NSLIP];
    elastic_tau_f32(f, a, dg, g, tau);
    float rmax = 0.f;
    for (int s = 0; s < NSLIP; ++s) {
        const float id = 1.f / (1.f + k.d * fabsf(dg[s]));
        iden[s] = id;
        chi[s] = (chn[s] + k.c * dg[s]) * id;
        const float x = (tau[s] - chi[s]) * k.it0;
        const float ax = fabsf(x);
        const float axp1 = ipowf_n(ax, k.p - 1);
        dh[s] = (float)k.p * axp1;
        r[s] = dg[s] - k.cf * sgn(x) * axp1 * ax;
        rmax = fmaxf(rmax, fabsf(r[s]));
    }
    return rmax;
}

// The small-elastic-strain correction (as cp_correction_lowrank) in FP32 throughout.
__device__ bool cp_correction_f32(const float* __restrict__ PC, const float* dg, const F32Consts& k, const float* chi,
                                  const float* dh, const float* iden, const float* r, float* x) {
    float A[15], b[5];
    {
        int q = 0;
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            b[i] = 0.f;
#pragma unroll
            for (int j = 0; j <= i; ++j) A[q++] = __ldg(PC + 60 + 5 * i + j);
        }
    }
    float fa[NSLIP], Di[NSLIP];
#pragma unroll
    for (int s = 0; s < NSLIP; ++s) {
        fa[s] = k.cf * k.it0 * dh[s];
        const float dchi = (k.c - k.d * sgn(dg[s]) * chi[s]) * iden[s];
        Di[s] = 1.f / (1.f + fa[s] * dchi);
        const float ga = fa[s] * Di[s], ra = r[s] * Di[s];
        float pp[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) pp[i] = __ldg(PC + 12 * i + s);
        int q = 0;
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            b[i] = fmaf(ra, pp[i], b[i]);
#pragma unroll
            for (int j = 0; j <= i; ++j) A[q] = fmaf(ga * pp[i], pp[j], A[q]), ++q;
        }
    }
    float L[5][5], qd[5], iq[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        float t = A[j * (j + 1) / 2 + j];
#pragma unroll
        for (int m = 0; m < j; ++m) t -= L[j][m] * L[j][m] * qd[m];
        if (!(t > 0.f)) return false;
        qd[j] = t;
        iq[j] = 1.f / t;
#pragma unroll
        for (int i = j + 1; i < 5; ++i) {
            float u = A[i * (i + 1) / 2 + j];
#pragma unroll
            for (int m = 0; m < j; ++m) u -= L[i][m] * L[j][m] * qd[m];
            L[i][j] = u * iq[j];
        }
    }
    float u[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        float t = b[i];
#pragma unroll
        for (int m = 0; m < i; ++m) t -= L[i][m] * u[m];
        u[i] = t;
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) u[i] *= iq[i];
#pragma unroll
    for (int i = 4; i >= 0; --i) {
#pragma unroll
        for (int m = i + 1; m < 5; ++m) u[i] -= L[m][i] * u[m];
    }
#pragma unroll
    for (int s = 0; s < NSLIP; ++s) {
        float t = 0.f;
#pragma unroll
        for (int i = 0; i < 5; ++i) t = fmaf(__ldg(PC + 12 * i + s), u[i], t);
        x[s] = Di[s] * (r[s] - fa[s] * t);
    }
    return true;
}

// FP32 iteration from dg (in/out, FP64 storage); false (dg untouched) if it
// breaks down before reaching FP32 resolution or stalling.  Not inlined: the
// compiler contracts FP32 multiply-adds per inlined copy, and the one-handle
// and the batched constitutive kernels must iterate to the same bits (the
// FP64 iteration that follows stops at its tolerance, so a last-bit change of
// its start would show up at that tolerance).
__device__ __noinline__ bool cp_presolve_f32(const double* F, const double* A, const double* chin, const float* __restrict__ g,
                                const CPParamsDev& pr, double coef, double* dg64, int* iters) {
    float f[9], a[9], chn[NSLIP], dg[NSLIP], chi[NSLIP], dh[NSLIP], r[NSLIP], iden[NSLIP], x[NSLIP];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const double I = (k % 4) == 0 ? 1.0 : 0.0;
        f[k] = (float)(F[k] - I);
        a[k] = (float)(A[k] - I);
    }
    for (int s = 0; s < NSLIP; ++s) {
        chn[s] = (float)chin[s];
        dg[s] = (float)dg64[s];
    }
    F32Consts k;
    k.cf = (float)coef;
    k.c = (float)pr.c;
    k.d = (float)pr.d;
    k.it0 = (float)pr.itau0;
    k.p = (int)pr.p;
    float prev = 3.0e38f;
    constexpr int MAXIT = 30;
    for (int it = 0; it < MAXIT; ++it) {
        const float rmax = cp_residual_f32(f, a, chn, dg, g, k, chi, dh, r, iden);
        *iters = it;
        if (!(rmax < 1e30f)) return false;
        float dgmax = 0.f;
        for (int s = 0; s < NSLIP; ++s) dgmax = fmaxf(dgmax, fabsf(dg[s]));
        // FP32 resolution of this residual is a few 1e-6 of the slips; stalling there (or
        // slower than halving after a few steps) ends the pre-iteration
        if (rmax <= 1e-5f * dgmax || (it > 3 && rmax > 0.5f * prev)) {
            for (int s = 0; s < NSLIP; ++s) dg64[s] = (double)dg[s];
            return true;
        }
        prev = rmax;
        if (!cp_correction_f32(g + G32_PC, dg, k, chi, dh, iden, r, x)) return false;
        for (int s = 0; s < NSLIP; ++s) dg[s] -= x[s];
    }
    return false;
}

// Local Newton on dg from the given start.  lowrank: corrections from the
// small-elastic-strain Jacobian in precision TJ; otherwise the exact
// Jacobian with pivoting in FP64.
template <typename TJ>
__device__ bool cp_local_solve(const double* F, const double* A, const double* chin, const double* __restrict__ S0,
                               const double* __restrict__ C, const double* __restrict__ PC, const CPParamsDev& pr,
                               double coef, int p, bool lowrank, int maxit, double* dg, ElState& st, double* chi,
                               double* dh, int* iters) {
    for (int it = 0; it <= maxit; ++it) {
        double r[NSLIP];
        double iden[NSLIP];
        const double rmax = cp_residual(F, A, chin, dg, S0, pr, coef, p, st, chi, dh, r, iden);
        *iters = it;
        if (rmax <= pr.rtol) return true;
        if (it == maxit || !(rmax < 1e300)) return false;
        if (lowrank) {
            double x[NSLIP];
            if (!cp_correction_lowrank<TJ>(PC, dg, pr, coef, chi, dh, iden, r, x)) return false;
            for (int a = 0; a < NSLIP; ++a) dg[a] -= x[a];
        } else {
            double J[NSLIP * NSLIP];
            int piv[NSLIP];
            cp_jacobian_exact<double>(F, A, dg, S0, C, pr, coef, st, chi, dh, J);
            if (!lu_factor<NSLIP>(J, piv)) return false;
            lu_solve<NSLIP>(J, piv, r);
            for (int a = 0; a < NSLIP; ++a) dg[a] -= r[a];
        }
    }
    return false;
}

// Consistent tangent K = dP/dF at the converged return map, in precision T
// (the grain's S0 and C given in T, so no conversions in the loops):
//   K = dP/dF|_dg + (dP/ddg) (ddg/dF),  J ddg/dF = (coef/g) h' dtau/dF|_dg.
template <typename T>
__device__ __forceinline__ bool cp_tangent_core(const T* F, const T* A, const T* dg, const T* __restrict__ S0,
                                                const T* __restrict__ C, const CPParamsDev& pr, double coef,
                                                const ElStateT<T>& st, const T* chi, const T* dh, T* K) {
    T J[NSLIP * NSLIP];
    int piv[NSLIP];
    const T cg = (T)(coef / pr.tau0);
    T FeS[9];
    mm(st.Fe, st.S, FeS);
    // column b of the exact Jacobian dr_a/ddg_b (as cp_jacobian_exact) and dP/ddg_b (12 x 9) from
    // one derivative of the elastic state per slip system
    T dPb[NSLIP * 9];
    {
        const T cc = (T)pr.c, d = (T)pr.d;
        for (int b = 0; b < NSLIP; ++b) {
            T dFpi[9], dFe[9], dCe[9], dS[9], t1[9], t2[9], t3[9], t4[9];
            dstate_ddg(F, A, S0 + 9 * b, C, st, dFpi, dFe, dCe, dS);
            {
                T dM[9];
                mm(dCe, st.S, dM);
                mm(st.Ce, dS, t1);
#pragma unroll
                for (int k = 0; k < 9; ++k) dM[k] += t1[k];
                for (int a = 0; a < NSLIP; ++a) {
                    T dtau = (T)0;
#pragma unroll
                    for (int k = 0; k < 9; ++k) dtau = fma(dM[k], __ldg(S0 + 9 * a + k), dtau);
                    T v = -cg * dh[a] * dtau;
                    if (a == b) {
                        const T den = (T)1 + d * fabs(dg[a]);
                        const T dchi = (cc - d * sgn(dg[a]) * chi[a]) / den;
                        v += (T)1 + cg * dh[a] * dchi;
                    }
                    J[a * NSLIP + b] = v;
                }
            }
            mm(dFe, st.S, t1);
            mmt(t1, st.Fpi, t2);  // dFe S Fpi^T
            mm(st.Fe, dS, t1);
            mmt(t1, st.Fpi, t3);  // Fe dS Fpi^T
            mmt(FeS, dFpi, t4);   // Fe S dFpi^T
#pragma unroll
            for (int k = 0; k < 9; ++k) dPb[9 * b + k] = t2[k] + t3[k] + t4[k];
        }
    }
    if (!lu_factor<NSLIP>(J, piv)) return false;
    T SFt[9];
    mmt(st.S, st.Fpi, SFt);  // S Fpi^T
    for (int kl = 0; kl < 9; ++kl) {
        const int k = kl / 3, l = kl % 3;
        // dFe = E_kl Fpi: row k equals row l of Fpi
        T dFe[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) dFe[q] = (T)0;
        dFe[3 * k] = st.Fpi[3 * l];
        dFe[3 * k + 1] = st.Fpi[3 * l + 1];
        dFe[3 * k + 2] = st.Fpi[3 * l + 2];
        T t1[9], t2[9], dCe[9], hE[9], dS[9];
        mtm(dFe, st.Fe, t1);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                dCe[3 * i + j] = t1[3 * i + j] + t1[3 * j + i];
                hE[3 * i + j] = (T)0.5 * dCe[3 * i + j];
            }
        c_ddot(C, hE, dS);
        // dP at fixed dg = dFe S Fpi^T + Fe dS Fpi^T
        T dP[9], t3[9];
        mm(dFe, SFt, dP);
        mm(st.Fe, dS, t3);
        mmt(t3, st.Fpi, t1);
#pragma unroll
        for (int q = 0; q < 9; ++q) dP[q] += t1[q];
        // dtau_a = (dCe S + Ce dS) : S0_a ; J ddg = (coef/g) h'_a dtau_a
        T dM[9];
        mm(dCe, st.S, dM);
        mm(st.Ce, dS, t2);
#pragma unroll
        for (int q = 0; q < 9; ++q) dM[q] += t2[q];
        T rhs[NSLIP];
        for (int a = 0; a < NSLIP; ++a) {
            T dtau = (T)0;
#pragma unroll
            for (int q = 0; q < 9; ++q) dtau = fma(dM[q], __ldg(S0 + 9 * a + q), dtau);
            rhs[a] = cg * dh[a] * dtau;
        }
        lu_solve<NSLIP>(J, piv, rhs);
        for (int b = 0; b < NSLIP; ++b)
#pragma unroll
            for (int q = 0; q < 9; ++q) dP[q] = fma(dPb[9 * b + q], rhs[b], dP[q]);
#pragma unroll
        for (int q = 0; q < 9; ++q) K[9 * q + kl] = dP[q];
    }
    return true;
}

// The tangent from the FP64 state of the converged return map, computed in T.
template <typename T>
__device__ bool cp_tangent(const double* Fd, const double* Ad, const double* dgd, const T* __restrict__ S0,
                           const T* __restrict__ C, const CPParamsDev& pr, double coef, const ElState& sd,
                           const double* chid, const double* dhd, T* K) {
    T F[9], A[9], dg[NSLIP], chi[NSLIP], dh[NSLIP];
    ElStateT<T> st;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        F[k] = (T)Fd[k];
        A[k] = (T)Ad[k];
        st.Fpi[k] = (T)sd.Fpi[k];
        st.Fe[k] = (T)sd.Fe[k];
        st.Ce[k] = (T)sd.Ce[k];
        st.S[k] = (T)sd.S[k];
        st.M[k] = (T)sd.M[k];
    }
    for (int a = 0; a < NSLIP; ++a) {
        dg[a] = (T)dgd[a];
        chi[a] = (T)chid[a];
        dh[a] = (T)dhd[a];
        st.tau[a] = (T)sd.tau[a];
    }
    return cp_tangent_core<T>(F, A, dg, S0, C, pr, coef, st, chi, dh, K);
}

// The elastic state at slips dg in FP32, in the displacement-gradient form of the
// FP32 pre-iteration (f = F - I, a = Fp^-1_n - I; Fp^-1 - I = a - Lp - a Lp,
// Fe - I = G = q + f + f q, E = (G + G^T + G^T G)/2, Ce = I + 2E, M = S + 2 E S), so
// that the small parts of Fe, Ce and the stresses keep FP32 relative precision.
__device__ void elastic_state_f32(const float* f, const float* a, const float* dg, const float* __restrict__ g,
                                  ElStateT<float>& st) {
    const float* sd = g + G32_DIR;
    const float* mn = g + G32_NRM;
    const float* C6 = g + G32_C6;
    float Lp[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) Lp[k] = 0.f;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        float v[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) v[j] = fmaf(dg[3 * p + i], __ldg(sd + 3 * (3 * p + i) + j), v[j]);
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = 0; k < 3; ++k) Lp[3 * j + k] = fmaf(v[j], __ldg(mn + 3 * p + k), Lp[3 * j + k]);
    }
    float aL[9], q[9], fq[9], G[9], GtG[9];
    mm(a, Lp, aL);
#pragma unroll
    for (int k = 0; k < 9; ++k) q[k] = a[k] - Lp[k] - aL[k];
    mm(f, q, fq);
#pragma unroll
    for (int k = 0; k < 9; ++k) G[k] = q[k] + f[k] + fq[k];
    mtm(G, G, GtG);
    float E[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) E[3 * i + j] = 0.5f * (G[3 * i + j] + G[3 * j + i] + GtG[3 * i + j]);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const float I = (k % 4) == 0 ? 1.f : 0.f;
        st.Fpi[k] = I + q[k];
        st.Fe[k] = I + G[k];
        st.Ce[k] = I + 2.f * E[k];
    }
    const float e[6] = {E[0], E[4], E[8], 2.f * E[5], 2.f * E[2], 2.f * E[1]};  // Voigt, engineering shears
    float sv[6];
#pragma unroll
    for (int I = 0; I < 6; ++I) {
        float t = 0.f;
#pragma unroll
        for (int J = 0; J < 6; ++J) t = fmaf(__ldg(C6 + 6 * I + J), e[J], t);
        sv[I] = t;
    }
    st.S[0] = sv[0], st.S[4] = sv[1], st.S[8] = sv[2];
    st.S[5] = st.S[7] = sv[3];
    st.S[2] = st.S[6] = sv[4];
    st.S[1] = st.S[3] = sv[5];
    float ES[9];
    mm(E, st.S, ES);
#pragma unroll
    for (int k = 0; k < 9; ++k) st.M[k] = fmaf(2.f, ES[k], st.S[k]);
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const float m0 = __ldg(mn + 3 * p), m1 = __ldg(mn + 3 * p + 1), m2 = __ldg(mn + 3 * p + 2);
        float Mm[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) Mm[j] = st.M[3 * j] * m0 + st.M[3 * j + 1] * m1 + st.M[3 * j + 2] * m2;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float* sv3 = sd + 3 * (3 * p + i);
            st.tau[3 * p + i] = __ldg(sv3) * Mm[0] + __ldg(sv3 + 1) * Mm[1] + __ldg(sv3 + 2) * Mm[2];
        }
    }
}

// The FP32 tangent of mixed precision at the stored slips, written to Kg[(9q + kl) ldk]:
//   K = dP/dF|_dg + (dP/ddg) X,   J X = R,   R_a,kl = (coef/tau0) h'_a dtau_a/dF_kl|_dg,
// with the elastic state, backstress and flow-rule derivative formed in FP32 from the
// displacement-gradient form (elastic_state_f32), dP/ddg exact, and J the small-elastic-
// strain Jacobian D + F P^T C5 P of the return map's corrections, solved for the nine
// columns through one 5 x 5 LDL^T factorisation (cp_correction_f32 for one right-hand
// side).  Against the exact Jacobian this drops terms of the order of the elastic strain
// (~1e-3) from the plastic part of K, below the CG tolerance the tangent serves; it keeps
// no 12 x 12 matrix, so the tangent stays in registers.  Not inlined, so that the
// one-handle and the batched kernels compute the same bits.
__device__ __noinline__ bool cp_tangent_f32(const double* Fd, const double* Ad, const double* chind, const double* dgd,
                                            double dt, const float* __restrict__ g, const CPParamsDev& pr,
                                            float* __restrict__ Kg, long long ldk) {
    float F[9], A[9], dg[NSLIP], chi[NSLIP], dh[NSLIP];
    ElStateT<float> st;
    {
        float f[9], a[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const double I = (k % 4) == 0 ? 1.0 : 0.0;
            f[k] = (float)(Fd[k] - I);
            a[k] = (float)(Ad[k] - I);
            F[k] = (float)Fd[k];
            A[k] = (float)Ad[k];
        }
        for (int s = 0; s < NSLIP; ++s) dg[s] = (float)dgd[s];
        elastic_state_f32(f, a, dg, g, st);
    }
    const float c = (float)pr.c, d = (float)pr.d, it0 = (float)pr.itau0, cg = (float)(dt * pr.gdot0 / pr.tau0);
    const int p = (int)pr.p;
    const float* __restrict__ S0 = g + G32_S0;
    const float* __restrict__ C = g + G32_C;
    const float* __restrict__ PC = g + G32_PC;  // P [5][12], then C5^-1 [5][5]
    float fa[NSLIP], Di[NSLIP];
    float A5[15];
    {
        int q = 0;
#pragma unroll
        for (int i = 0; i < 5; ++i)
#pragma unroll
            for (int j = 0; j <= i; ++j) A5[q++] = __ldg(PC + 60 + 5 * i + j);
    }
    for (int s = 0; s < NSLIP; ++s) {
        const float id = 1.f / (1.f + d * fabsf(dg[s]));
        chi[s] = ((float)chind[s] + c * dg[s]) * id;
        const float x = (st.tau[s] - chi[s]) * it0;
        dh[s] = (float)p * ipowf_n(fabsf(x), p - 1);
        fa[s] = cg * dh[s];
        const float dchi = (c - d * sgn(dg[s]) * chi[s]) * id;
        Di[s] = 1.f / (1.f + fa[s] * dchi);
        const float ga = fa[s] * Di[s];
        int q = 0;
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            const float pi = __ldg(PC + 12 * i + s);
#pragma unroll
            for (int j = 0; j <= i; ++j) A5[q] = fmaf(ga * pi, __ldg(PC + 12 * j + s), A5[q]), ++q;
        }
    }
    // A5 = L diag(qd) L^T
    float L[5][5], iq[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        float t = A5[j * (j + 1) / 2 + j];
#pragma unroll
        for (int m = 0; m < j; ++m) t -= L[j][m] * L[j][m] / iq[m];
        if (!(t > 0.f)) return false;
        iq[j] = 1.f / t;
#pragma unroll
        for (int i = j + 1; i < 5; ++i) {
            float u = A5[i * (i + 1) / 2 + j];
#pragma unroll
            for (int m = 0; m < j; ++m) u -= L[i][m] * L[j][m] / iq[m];
            L[i][j] = u * iq[j];
        }
    }
    float FeS[9], SFt[9];
    mm(st.Fe, st.S, FeS);
    mmt(st.S, st.Fpi, SFt);  // S Fpi^T
    // dP/ddg_b (12 x 9)
    float dPb[NSLIP * 9];
    for (int b = 0; b < NSLIP; ++b) {
        float dFpi[9], dFe[9], dCe[9], dS[9], t1[9], t2[9], t3[9], t4[9];
        dstate_ddg(F, A, S0 + 9 * b, C, st, dFpi, dFe, dCe, dS);
        mm(dFe, st.S, t1);
        mmt(t1, st.Fpi, t2);  // dFe S Fpi^T
        mm(st.Fe, dS, t1);
        mmt(t1, st.Fpi, t3);  // Fe dS Fpi^T
        mmt(FeS, dFpi, t4);   // Fe S dFpi^T
#pragma unroll
        for (int k = 0; k < 9; ++k) dPb[9 * b + k] = t2[k] + t3[k] + t4[k];
    }
    for (int kl = 0; kl < 9; ++kl) {
        const int k = kl / 3, l = kl % 3;
        float dFe[9];  // dFe = E_kl Fpi: row k equals row l of Fpi
#pragma unroll
        for (int q = 0; q < 9; ++q) dFe[q] = 0.f;
        dFe[3 * k] = st.Fpi[3 * l];
        dFe[3 * k + 1] = st.Fpi[3 * l + 1];
        dFe[3 * k + 2] = st.Fpi[3 * l + 2];
        float t1[9], t2[9], dCe[9], hE[9], dS[9];
        mtm(dFe, st.Fe, t1);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                dCe[3 * i + j] = t1[3 * i + j] + t1[3 * j + i];
                hE[3 * i + j] = 0.5f * dCe[3 * i + j];
            }
        c_ddot(C, hE, dS);
        float dP[9], t3[9], dM[9];
        mm(dFe, SFt, dP);  // dP at fixed dg = dFe S Fpi^T + Fe dS Fpi^T
        mm(st.Fe, dS, t3);
        mmt(t3, st.Fpi, t1);
#pragma unroll
        for (int q = 0; q < 9; ++q) dP[q] += t1[q];
        mm(dCe, st.S, dM);  // dM = dCe S + Ce dS
        mm(st.Ce, dS, t2);
#pragma unroll
        for (int q = 0; q < 9; ++q) dM[q] += t2[q];
        // J x = R_kl through the 5 x 5 system
        float r[NSLIP], u[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        for (int a = 0; a < NSLIP; ++a) {
            float dtau = 0.f;
#pragma unroll
            for (int q = 0; q < 9; ++q) dtau = fmaf(dM[q], __ldg(S0 + 9 * a + q), dtau);
            r[a] = fa[a] * dtau;
            const float ra = r[a] * Di[a];
#pragma unroll
            for (int i = 0; i < 5; ++i) u[i] = fmaf(ra, __ldg(PC + 12 * i + a), u[i]);
        }
#pragma unroll
        for (int i = 0; i < 5; ++i)
#pragma unroll
            for (int m = 0; m < i; ++m) u[i] -= L[i][m] * u[m];
#pragma unroll
        for (int i = 0; i < 5; ++i) u[i] *= iq[i];
#pragma unroll
        for (int i = 4; i >= 0; --i)
#pragma unroll
            for (int m = i + 1; m < 5; ++m) u[i] -= L[m][i] * u[m];
        for (int b = 0; b < NSLIP; ++b) {
            float t = 0.f;
#pragma unroll
            for (int i = 0; i < 5; ++i) t = fmaf(__ldg(PC + 12 * i + b), u[i], t);
            const float xb = Di[b] * (r[b] - fa[b] * t);
#pragma unroll
            for (int q = 0; q < 9; ++q) dP[q] = fmaf(dPb[9 * b + q], xb, dP[q]);
        }
#pragma unroll
        for (int q = 0; q < 9; ++q) Kg[(9 * q + kl) * ldk] = dP[q];
    }
    return true;
}

// Return map (FP64) and, when K is not null, the tangent in precision T.
template <typename T>
__device__ void cp_update(const double* F, const double* A, const double* chin, double dt,
                          const double* __restrict__ S0, const double* __restrict__ C, const double* __restrict__ H,
                          const T* __restrict__ S0t, const T* __restrict__ Ct, const CPParamsDev& pr,
                          const double* dg0 /* 12 or null */, T* K /* 81 or null */, CPOut& out,
                          bool exact_only = false, const float* __restrict__ g32 = nullptr) {
    const double coef = dt * pr.gdot0;
    const int p = (int)pr.p;
    double dg[NSLIP], dh[NSLIP], chi[NSLIP];
    ElState st;
    for (int a = 0; a < NSLIP; ++a) dg[a] = dg0 ? dg0[a] : 0.0;
    out.iters32 = 0;
    if (g32 && !exact_only) {  // FP32 pre-iteration (g32: the grain's FP32 data)
        double dgs[NSLIP];
        for (int a = 0; a < NSLIP; ++a) dgs[a] = dg[a];
        int it32 = 0;
        if (cp_presolve_f32(F, A, chin, g32, pr, coef, dgs, &it32))
            for (int a = 0; a < NSLIP; ++a) dg[a] = dgs[a];
        out.iters32 = it32;
    }
    // FP64 corrections: J is ill-conditioned (cond ~ 1e8 and more) once slip
    // systems are active, beyond what an FP32 solve can steer
    int it1 = 0, it2 = 0;
    bool conv = false;
    if (!exact_only) conv = cp_local_solve<double>(F, A, chin, S0, C, H, pr, coef, p, true, 60, dg, st, chi, dh, &it1);
    out.fallback = !conv;
    if (!conv) {  // fall back: exact Newton from dg = 0
        for (int a = 0; a < NSLIP; ++a) dg[a] = 0.0;
        conv = cp_local_solve<double>(F, A, chin, S0, C, H, pr, coef, p, false, 300, dg, st, chi, dh, &it2);
    }
    out.iters = it1 + it2;
    out.ok = conv;
    double FeS[9];
    mm(st.Fe, st.S, FeS);
    mmt(FeS, st.Fpi, out.P);  // P = Fe S Fpi^T
#pragma unroll
    for (int k = 0; k < 9; ++k) out.Fpi[k] = st.Fpi[k];
    for (int a = 0; a < NSLIP; ++a) {
        out.chi[a] = chi[a];
        out.dg[a] = dg[a];
        out.tau[a] = st.tau[a];
    }
    if (K && conv) out.ok = cp_tangent<T>(F, A, dg, S0t, Ct, pr, coef, st, chi, dh, K);
}

__device__ void svk_update(const double* F, const double* __restrict__ C, double* P, double* K) {
    double E[9], S[9];
    mtm(F, F, E);
#pragma unroll
    for (int k = 0; k < 9; ++k) E[k] = 0.5 * (E[k] - ((k % 4) == 0 ? 1.0 : 0.0));
    c_ddot(C, E, S);
    mm(F, S, P);
    if (!K) return;
    // K_ijkl = delta_ik S_lj + sum_p F_ip (sum_n C_pjln F_kn)
    for (int j = 0; j < 3; ++j)
        for (int l = 0; l < 3; ++l) {
            double h[9];  // h[p][k] = sum_n C_pjln F_kn
#pragma unroll
            for (int pp = 0; pp < 3; ++pp)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const double* Cr = C + 27 * pp + 9 * j + 3 * l;  // C_{p j l n}
                    h[3 * pp + k] = __ldg(Cr) * F[3 * k] + __ldg(Cr + 1) * F[3 * k + 1] + __ldg(Cr + 2) * F[3 * k + 2];
                }
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    double v = F[3 * i] * h[k] + F[3 * i + 1] * h[3 + k] + F[3 * i + 2] * h[6 + k];
                    if (i == k) v += S[3 * l + j];
                    K[9 * (3 * i + j) + (3 * k + l)] = v;
                }
        }
}

// ---- Appendix A: umat outputs (Cauchy stress sigma, Jaumann-rate tangent C^ab)
// to P = J sigma F^-T (Eq. fPK) and K = dP/dF:
//   d tau_ip/d F_kl = J C_ipkm Fi_lm + 1/2 delta_ik (Fi tau)_lp - 1/2 Fi_li tau_kp
//                     + 1/2 delta_pk (tau Fi^T)_il - 1/2 Fi_lp tau_ik,
//   K_ijkl = d tau_ip/d F_kl Fi_jp - (tau Fi^T)_il Fi_jk,
// tau = J sigma, Fi = F^-1.  Cab(q) returns C^ab at index q = 9 (3i+j) + 3k + l;
// K is written column by column through Kout(q, value).
__device__ __forceinline__ double det3(const double* F) {
    return F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) + F[2] * (F[3] * F[7] - F[4] * F[6]);
}
__device__ __forceinline__ void inv3(const double* F, double J, double* Fi) {
    const double r = 1.0 / J;
    Fi[0] = (F[4] * F[8] - F[5] * F[7]) * r;
    Fi[1] = (F[2] * F[7] - F[1] * F[8]) * r;
    Fi[2] = (F[1] * F[5] - F[2] * F[4]) * r;
    Fi[3] = (F[5] * F[6] - F[3] * F[8]) * r;
    Fi[4] = (F[0] * F[8] - F[2] * F[6]) * r;
    Fi[5] = (F[2] * F[3] - F[0] * F[5]) * r;
    Fi[6] = (F[3] * F[7] - F[4] * F[6]) * r;
    Fi[7] = (F[1] * F[6] - F[0] * F[7]) * r;
    Fi[8] = (F[0] * F[4] - F[1] * F[3]) * r;
}

template <typename CA, typename KO>
__device__ __forceinline__ void umat_to_PK(const double* F, const double* sig, CA Cab, double* P, KO Kout) {
    const double J = det3(F);
    double Fi[9], tau[9], A[9], B[9];
    inv3(F, J, Fi);
#pragma unroll
    for (int q = 0; q < 9; ++q) tau[q] = J * sig[q];
    mm(Fi, tau, A);   // A_lp = Fi_lm tau_mp
    mmt(tau, Fi, B);  // B_il = tau_im Fi_lm
    mmt(tau, Fi, P);  // P_ij = tau_ip Fi_jp
    for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) {
            double dt[9];  // d tau_ip / d F_kl
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int p = 0; p < 3; ++p) {
                    double c = 0.0;
#pragma unroll
                    for (int m = 0; m < 3; ++m) c = fma(Cab(9 * (3 * i + p) + 3 * k + m), Fi[3 * l + m], c);
                    double v = J * c - 0.5 * Fi[3 * l + i] * tau[3 * k + p] - 0.5 * Fi[3 * l + p] * tau[3 * i + k];
                    if (i == k) v += 0.5 * A[3 * l + p];
                    if (p == k) v += 0.5 * B[3 * i + l];
                    dt[3 * i + p] = v;
                }
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const double v = dt[3 * i] * Fi[3 * j] + dt[3 * i + 1] * Fi[3 * j + 1] + dt[3 * i + 2] * Fi[3 * j + 2] -
                                     B[3 * i + l] * Fi[3 * j + k];
                    Kout(9 * (3 * i + j) + 3 * k + l, v);
                }
        }
}

// Compressible neo-Hookean solid in umat form: tau = mu (b - I) + lam ln(J) I,
// sigma = tau / J and J C^ab_ijkl = mu/2 (d_ik b_jl + d_il b_jk + b_ik d_jl + b_il d_jk) + lam d_ij d_kl.
__device__ __forceinline__ void neohooke_umat(const double* F, double lam, double mu, double* sig, double* b, double& J) {
    J = det3(F);
    mmt(F, F, b);  // b = F F^T
    const double lnJ = log(J), iJ = 1.0 / J;
#pragma unroll
    for (int q = 0; q < 9; ++q) sig[q] = (mu * (b[q] - ((q % 4) == 0 ? 1.0 : 0.0)) + ((q % 4) == 0 ? lam * lnJ : 0.0)) * iJ;
}
__device__ __forceinline__ double neohooke_Cab(int q, const double* b, double lam, double mu, double iJ) {
    const int i = q / 27, j = (q / 9) % 3, k = (q / 3) % 3, l = q % 3;
    double v = 0.0;
    if (i == k) v += b[3 * j + l];
    if (i == l) v += b[3 * j + k];
    if (j == l) v += b[3 * i + k];
    if (j == k) v += b[3 * i + l];
    v *= 0.5 * mu;
    if (i == j && k == l) v += lam;
    return v * iJ;
}

__global__ void __launch_bounds__(TPB) k_umat_convert(long long n, const double* __restrict__ F,
                                                      const double* __restrict__ sig, const double* __restrict__ Cab,
                                                      double* __restrict__ P, double* __restrict__ K) {
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    double f[9], s9[9], p9[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        f[q] = F[q * n + v];
        s9[q] = sig[q * n + v];
    }
    umat_to_PK(f, s9, [&](int q) { return __ldg(Cab + q * n + v); }, p9, [&](int q, double x) { K[q * n + v] = x; });
#pragma unroll
    for (int q = 0; q < 9; ++q) P[q * n + v] = p9[q];
}

struct ConstArgs {
    const double* F;
    const int* gid;
    const double* C;
    const double* S0;
    const float* G32;  // [ngrains][G32_STRIDE]: S0 and C in FP32 for the FP32 tangent
    const double* H;  // [ngrains][144]: P [5][12], C5^-1 [5][5] of the small-strain Jacobian (cp_correction_lowrank)
    int warm;         // 1: start the local Newton from dg (previous iterate)
    const int* warm_dev;  // device flag (may be null): when set, start warm as well
    int exact;        // 1: skip the small-strain iteration, exact Newton from dg = 0 only
    int small;        // 1: small-strain variant, F holds the strain: P = C : F (Cauchy stress), K = C
    int f32first;     // 1: FP32 pre-iteration of the return map
    double rtol;      // return-map tolerance (return_map_tol)
    const int* gkind;
    const double* gprm;  // [ngrains][5]: gdot0, p, tau0, c, d
    const double* Fpi_n;
    const double* chi_n;
    double dt;
    double* P;
    double* K;    // FP64 tangent (null: not written)
    float* K32;   // FP32 tangent (null: not written)
    double* Fpi_t;
    double* chi_t;
    double* dg;
    double* tau;
    int* flag;
    int* stats;  // [2] (may be null): voxels whose return map fell back, local Newton iterations
    long long N;
    const int* skip;  // batched launches: RVE left alone when *skip != 0
};

// F32T: the crystal-plasticity tangent is computed in FP32 and only K32 is
// written (mixed precision); otherwise the tangent is FP64, written to K and,
// when K32 is set, also rounded into K32.
// The tangent alone, at the slips dg of the last return map (stored by a
// PART_P launch): the elastic state and the residual terms are rebuilt at dg
// -- the same function of the same values, so K equals what the return map's
// own tangent would have been, bit for bit.
template <typename T>
__device__ bool cp_tangent_at(const double* F, const double* A, const double* chin, const double* dg, double dt,
                              const double* __restrict__ geo, const T* __restrict__ S0t, const T* __restrict__ Ct,
                              const CPParamsDev& pr, T* K) {
    const double coef = dt * pr.gdot0;
    ElState st;
    double chi[NSLIP], dh[NSLIP], r[NSLIP], iden[NSLIP];
    cp_residual(F, A, chin, dg, geo, pr, coef, (int)pr.p, st, chi, dh, r, iden);
    return cp_tangent<T>(F, A, dg, S0t, Ct, pr, coef, st, chi, dh, K);
}

// PART_ALL: return map, P and the tangent; PART_P: return map and P (K left as
// it was); PART_K: the tangent at the stored slips (P and the trial state
// left as they were).
enum { PART_ALL = 0, PART_P = 1, PART_K = 2 };

template <bool F32T, int PART>
__device__ __forceinline__ void constitutive_voxel(const ConstArgs& a, const long long v) {
    const long long N = a.N;
    const int gi = a.gid[v];
    const int kind = a.gkind[gi];
    const double* C = a.C + 81LL * gi;
    double F[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) F[k] = a.F[k * N + v];
    int n_fb = 0, n_it = 0;
    if (kind == GFF_MAT_CP_FCC) {
        double A[9], chin[12];
#pragma unroll
        for (int k = 0; k < 9; ++k) A[k] = a.Fpi_n[k * N + v];
        for (int s = 0; s < NSLIP; ++s) chin[s] = a.chi_n[s * N + v];
        CPParamsDev pr;
        const double* gp = a.gprm + 5LL * gi;
        pr.gdot0 = gp[0];
        pr.p = gp[1];
        pr.tau0 = gp[2];
        pr.c = gp[3];
        pr.d = gp[4];
        pr.itau0 = 1.0 / pr.tau0;
        pr.rtol = a.rtol;
        const double* geo = a.S0 + (long long)GEO_STRIDE * gi;
        const float* g32 = a.G32 + (long long)G32_STRIDE * gi;
        if (PART == PART_K) {
            double dg[12];
            for (int s = 0; s < NSLIP; ++s) dg[s] = a.dg[s * N + v];
            bool ok;
            if (F32T) {
                ok = cp_tangent_f32(F, A, chin, dg, a.dt, g32, pr, a.K32 + v, N);
            } else {
                double K[81];
                ok = cp_tangent_at<double>(F, A, chin, dg, a.dt, geo, geo + GEO_S0, C, pr, K);
#pragma unroll
                for (int k = 0; k < 81; ++k) a.K[k * N + v] = K[k];
                if (a.K32) {
#pragma unroll
                    for (int k = 0; k < 81; ++k) a.K32[k * N + v] = (float)K[k];
                }
            }
            if (!ok) atomicAdd(a.flag, 1);
            return;
        }
        double dg0[12];
        const bool warm = a.warm || (a.warm_dev && *a.warm_dev);
        if (warm)
            for (int s2 = 0; s2 < NSLIP; ++s2) dg0[s2] = a.dg[s2 * N + v];
        CPOut o;
        if (PART == PART_P) {
            cp_update<double>(F, A, chin, a.dt, geo, C, a.H + 144LL * gi, geo + GEO_S0, C, pr, warm ? dg0 : nullptr,
                              (double*)nullptr, o, a.exact != 0, a.f32first ? g32 : nullptr);
        } else if (F32T) {  // the return map, then the tangent as a tangent-only launch forms it
            cp_update<float>(F, A, chin, a.dt, geo, C, a.H + 144LL * gi, g32 + G32_S0, g32 + G32_C, pr,
                             warm ? dg0 : nullptr, (float*)nullptr, o, a.exact != 0, a.f32first ? g32 : nullptr);
            if (o.ok) o.ok = cp_tangent_f32(F, A, chin, o.dg, a.dt, g32, pr, a.K32 + v, N);
        } else {
            double K[81];
            cp_update<double>(F, A, chin, a.dt, geo, C, a.H + 144LL * gi, geo + GEO_S0, C, pr, warm ? dg0 : nullptr,
                              K, o, a.exact != 0, a.f32first ? g32 : nullptr);
#pragma unroll
            for (int k = 0; k < 81; ++k) a.K[k * N + v] = K[k];
            if (a.K32) {
#pragma unroll
                for (int k = 0; k < 81; ++k) a.K32[k * N + v] = (float)K[k];
            }
        }
        if (!o.ok) atomicAdd(a.flag, 1);
        n_fb = o.fallback ? 1 : 0;
        n_it = o.iters;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            a.P[k * N + v] = o.P[k];
            a.Fpi_t[k * N + v] = o.Fpi[k];
        }
        for (int s = 0; s < NSLIP; ++s) {
            a.chi_t[s * N + v] = o.chi[s];
            a.dg[s * N + v] = o.dg[s];
            a.tau[s * N + v] = o.tau[s];
        }
    } else {
        double P[9], K[81];
        if (a.small) {  // linear elasticity at small strain: sigma = C : eps, tangent C
            c_ddot(C, F, P);
#pragma unroll
            for (int q = 0; q < 81; ++q) K[q] = __ldg(C + q);
        } else if (kind == GFF_MAT_NEOHOOKE) {  // through the umat interface (Appendix A)
            const double lam = __ldg(C + 4), mu = __ldg(C + 10);  // C_1122, C_1212 of the isotropic C
            double sg[9], b[9], J;
            neohooke_umat(F, lam, mu, sg, b, J);
            const double iJ = 1.0 / J;
            umat_to_PK(F, sg, [&](int q) { return neohooke_Cab(q, b, lam, mu, iJ); }, P,
                       [&](int q, double x) { K[q] = x; });
        } else {
            svk_update(F, C, P, K);
        }
        if (PART != PART_K) {
#pragma unroll
            for (int k = 0; k < 9; ++k) a.P[k * N + v] = P[k];
#pragma unroll
            for (int k = 0; k < 9; ++k) a.Fpi_t[k * N + v] = a.Fpi_n[k * N + v];
            for (int s = 0; s < NSLIP; ++s) {
                a.chi_t[s * N + v] = a.chi_n[s * N + v];
                a.dg[s * N + v] = 0.0;
                a.tau[s * N + v] = 0.0;
            }
        }
        if (PART != PART_P) {
            if (!F32T) {
#pragma unroll
                for (int k = 0; k < 81; ++k) a.K[k * N + v] = K[k];
            }
            if (a.K32) {
#pragma unroll
                for (int k = 0; k < 81; ++k) a.K32[k * N + v] = (float)K[k];
            }
        }
    }
    if (PART != PART_K && a.stats) {  // one atomic per warp
        const unsigned m = __activemask();
        const int sfb = __reduce_add_sync(m, n_fb), sit = __reduce_add_sync(m, n_it);
        if ((int)(threadIdx.x & 31) == __ffs(m) - 1) {
            if (sfb) atomicAdd(a.stats, sfb);
            atomicAdd(a.stats + 1, sit);
        }
    }
}

template <bool F32T, int PART>
__global__ void __launch_bounds__(TPB) k_constitutive(ConstArgs a) {
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= a.N) return;
    constitutive_voxel<F32T, PART>(a, v);
}

// one launch over the voxels of several RVEs: RVE r owns blocks [start[r], start[r+1])
template <bool F32T, int PART>
__global__ void __launch_bounds__(TPB) k_constitutive_batch(const ConstArgs* __restrict__ args,
                                                            const int* __restrict__ start, int n) {
    int r = 0;
    while (r + 1 < n && __ldg(start + r + 1) <= (int)blockIdx.x) ++r;
    const ConstArgs& a = args[r];
    if (a.skip && *a.skip) return;
    const long long v = (long long)(blockIdx.x - start[r]) * blockDim.x + threadIdx.x;
    if (v >= a.N) return;
    constitutive_voxel<F32T, PART>(a, v);
}

// ---------------------------------------------------------------- fatigue indicator parameters
struct FipArgs {
    const int* gid;
    const int* gkind;
    const double* S0;
    const double* nrm;
    const double* dg;
    const double* tau;
    const double* F;
    const double* P;
    double* acc;  // [NACC][N]
    long long N;
};

__global__ void __launch_bounds__(TPB) k_fip_accumulate(FipArgs a) {
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= a.N) return;
    const long long N = a.N;
    const int gi = a.gid[v];
    if (a.gkind[gi] != GFF_MAT_CP_FCC) return;
    const double* S0 = a.S0 + (long long)GEO_STRIDE * gi;
    const double* nr = a.nrm + 36LL * gi;
    double dDp[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) dDp[k] = 0.0;
    for (int s = 0; s < NSLIP; ++s) {
        const double d = a.dg[s * N + v];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) dDp[3 * i + j] += d * 0.5 * (S0[9 * s + 3 * i + j] + S0[9 * s + 3 * j + i]);
    }
    double* acc = a.acc;
    acc[v] += sqrt(2.0 / 3.0 * ddot9(dDp, dDp));
    double F[9], P[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        F[k] = a.F[k * N + v];
        P[k] = a.P[k * N + v];
    }
    const double J = F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
                     F[2] * (F[3] * F[7] - F[4] * F[6]);
    double sig[9];
    mmt(P, F, sig);
#pragma unroll
    for (int k = 0; k < 9; ++k) sig[k] /= J;
    for (int s = 0; s < NSLIP; ++s) {
        const double d = a.dg[s * N + v];
        acc[(1 + s) * N + v] += a.tau[s * N + v] * d;
        const double gm = acc[(13 + s) * N + v] + d;
        acc[(13 + s) * N + v] = gm;
        acc[(25 + s) * N + v] = fmin(acc[(25 + s) * N + v], gm);
        acc[(37 + s) * N + v] = fmax(acc[(37 + s) * N + v], gm);
        const double m0 = nr[3 * s], m1 = nr[3 * s + 1], m2 = nr[3 * s + 2];
        const double sn = m0 * (sig[0] * m0 + sig[1] * m1 + sig[2] * m2) + m1 * (sig[3] * m0 + sig[4] * m1 + sig[5] * m2) +
                          m2 * (sig[6] * m0 + sig[7] * m1 + sig[8] * m2);
        acc[(49 + s) * N + v] = fmax(acc[(49 + s) * N + v], sn);
    }
}

__global__ void __launch_bounds__(TPB) k_fip_reset(double* acc, long long N) {
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N) return;
    acc[v] = 0.0;
    for (int s = 0; s < NSLIP; ++s) {
        acc[(1 + s) * N + v] = 0.0;
        const double gm = acc[(13 + s) * N + v];
        acc[(25 + s) * N + v] = gm;
        acc[(37 + s) * N + v] = gm;
        acc[(49 + s) * N + v] = -INFINITY;
    }
}

// per-grain sums: out[g][0] = count, [1] = pcyc, [2..13] = W, [14..25] = dgamma, [26..37] = sn
constexpr int GSUM = 38;
__global__ void __launch_bounds__(TPB) k_grain_sums(const int* gid, const int* gkind, const double* acc, long long N,
                                                    double* out) {
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N) return;
    const int gi = gid[v];
    if (gkind[gi] != GFF_MAT_CP_FCC) return;
    double* o = out + (long long)GSUM * gi;
    atomicAdd(o, 1.0);
    atomicAdd(o + 1, acc[v]);
    for (int s = 0; s < NSLIP; ++s) {
        atomicAdd(o + 2 + s, acc[(1 + s) * N + v]);
        atomicAdd(o + 14 + s, acc[(37 + s) * N + v] - acc[(25 + s) * N + v]);
        atomicAdd(o + 26 + s, acc[(49 + s) * N + v]);
    }
}

__global__ void k_grain_final(const double* sums, int ngrains, double fs_k, double fs_sy, double* pc, double* w,
                              double* fs) {
    const int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= ngrains) return;
    const double* o = sums + (long long)GSUM * gi;
    const double n = o[0];
    if (n <= 0.0) {
        pc[gi] = 0.0;
        fs[gi] = 0.0;
        for (int s = 0; s < NSLIP; ++s) w[NSLIP * gi + s] = 0.0;
        return;
    }
    pc[gi] = o[1] / n;
    double best = -INFINITY;
    for (int s = 0; s < NSLIP; ++s) {
        w[NSLIP * gi + s] = o[2 + s] / n;
        const double v = 0.5 * (o[14 + s] / n) * (1.0 + fs_k * (o[26 + s] / n) / fs_sy);
        best = fmax(best, v);
    }
    fs[gi] = best;
}

// ---- band-averaged dissipated energy (Eq. Wmax).  Bands of width w parallel to
// each of a grain's four slip planes: the band index of a voxel for plane p is
// floor(s / w + 1/2), s = (x - x_ref) . m_p with the minimum-image offset of the
// voxel centre from the grain's reference voxel (its lowest voxel index), which
// sits in the middle of band 0.
__global__ void __launch_bounds__(TPB) k_band_ref(const int* __restrict__ gid, long long N, int* __restrict__ ref) {
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N) return;
    atomicMin(ref + gid[v], (int)v);
}

__device__ __forceinline__ int min_image(int i, int r, int n) {
    int d = i - r;
    if (d < 0) d += n;
    return 2 * d >= n ? d - n : d;
}

struct BandArgs {
    const int* gid;
    const int* gkind;
    const double* nrm;  // [ngrains][12][3] sample-frame normals; plane p is system 3p's
    const double* w;    // [12][N] W_cyc per system
    const int* ref;
    int nx, ny, nz, NB;
    double hx, hy, hz, width;
    long long N;
    double* sums;  // [ngrains][4][NB][4]: voxel count, then the three systems' W sums
};

__global__ void __launch_bounds__(TPB) k_band_sums(BandArgs a) {
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= a.N) return;
    const int gi = a.gid[v];
    if (a.gkind[gi] != GFF_MAT_CP_FCC) return;
    const int ix = (int)(v % a.nx), iy = (int)((v / a.nx) % a.ny), iz = (int)(v / ((long long)a.nx * a.ny));
    const int r = a.ref[gi];
    const int rx = r % a.nx, ry = (r / a.nx) % a.ny, rz = r / (a.nx * a.ny);
    const double dx = min_image(ix, rx, a.nx) * a.hx, dy = min_image(iy, ry, a.ny) * a.hy,
                 dz = min_image(iz, rz, a.nz) * a.hz;
    const double* nr = a.nrm + 36LL * gi;
    for (int p = 0; p < 4; ++p) {
        const double* m = nr + 9 * p;  // system 3p
        const double sc = dx * m[0] + dy * m[1] + dz * m[2];
        const int jo = (int)floor(sc / a.width + 0.5) + a.NB / 2;
        if (jo < 0 || jo >= a.NB) continue;  // the host sizes NB so that this never happens
        double* o = a.sums + 4 * ((4LL * gi + p) * a.NB + jo);
        atomicAdd(o, 1.0);
        for (int k = 0; k < 3; ++k) atomicAdd(o + 1 + k, a.w[(3 * p + k) * a.N + v]);
    }
}

// out[g] = the largest band average over the grain's planes, bands and systems (0 without bands)
__global__ void k_band_final(const double* __restrict__ sums, int ngrains, int NB, double* __restrict__ out) {
    const int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= ngrains) return;
    double best = -INFINITY;
    bool any = false;
    for (long long b = 4LL * gi * NB; b < 4LL * (gi + 1) * NB; ++b) {
        const double* o = sums + 4 * b;
        if (o[0] <= 0.0) continue;
        any = true;
        for (int k = 0; k < 3; ++k) best = fmax(best, o[1 + k] / o[0]);
    }
    out[gi] = any ? best : 0.0;
}

}  // namespace

cudaError_t launch_umat_convert(long long n, const double* F, const double* sigma, const double* Cab, double* P,
                                double* K, cudaStream_t st) {
    k_umat_convert<<<(unsigned)((n + TPB - 1) / TPB), TPB, 0, st>>>(n, F, sigma, Cab, P, K);
    return cudaGetLastError();
}

// Band-averaged W_cyc per grain into out[ngrains] (device); scratch holds
// ngrains ints + 16 NB ngrains doubles (band_scratch_bytes).
size_t band_scratch_bytes(int ngrains, int NB) {
    return ((size_t)ngrains * sizeof(int) + 255) / 256 * 256 + (size_t)ngrains * 16 * NB * sizeof(double);
}

cudaError_t launch_band_fips(gff_handle* h, double width, int NB, void* scratch, double* out) {
    const int ng = h->ngrains;
    int* ref = static_cast<int*>(scratch);
    double* sums = reinterpret_cast<double*>(static_cast<unsigned char*>(scratch) +
                                             ((size_t)ng * sizeof(int) + 255) / 256 * 256);
    cudaError_t e = cudaMemsetAsync(ref, 0x7f, (size_t)ng * sizeof(int), h->stream);  // large positive ints
    if (e == cudaSuccess) e = cudaMemsetAsync(sums, 0, (size_t)ng * 16 * NB * sizeof(double), h->stream);
    if (e != cudaSuccess) return e;
    const int blocks = (int)((h->N + TPB - 1) / TPB);
    k_band_ref<<<blocks, TPB, 0, h->stream>>>(h->d_gid, h->N, ref);
    BandArgs a;
    a.gid = h->d_gid;
    a.gkind = h->d_gkind;
    a.nrm = h->d_nrm;
    a.w = h->d_acc + h->N;
    a.ref = ref;
    a.nx = h->grid.nx;
    a.ny = h->grid.ny;
    a.nz = h->grid.nz;
    a.NB = NB;
    a.hx = h->grid.L[0] / h->grid.nx;
    a.hy = h->grid.L[1] / h->grid.ny;
    a.hz = h->grid.L[2] / h->grid.nz;
    a.width = width;
    a.N = h->N;
    a.sums = sums;
    k_band_sums<<<blocks, TPB, 0, h->stream>>>(a);
    k_band_final<<<(ng + 127) / 128, 128, 0, h->stream>>>(sums, ng, NB, out);
    return cudaGetLastError();
}

// Loads every constitutive kernel now (with lazy module loading the first launch of
// each would otherwise pay for it inside the caller's first increment).
cudaError_t preload_constitutive() {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, k_constitutive<true, PART_ALL>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_constitutive<true, PART_P>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_constitutive<true, PART_K>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_constitutive<false, PART_ALL>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_constitutive<false, PART_P>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_constitutive<false, PART_K>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_constitutive_batch<true, PART_P>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_constitutive_batch<true, PART_K>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_constitutive_batch<false, PART_P>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_constitutive_batch<false, PART_K>);
    return e;
}

// the return-map mode's FP32 pre-iteration for this handle (gff_set_return_map)
int f32_first(const gff_handle* h) {
    return h->cp_f32_first == 1 || (h->cp_f32_first == 2 && h->opt.precision == GFF_PREC_MIXED) ? 1 : 0;
}

cudaError_t launch_constitutive(gff_handle* h, const double* F, double dt, int tangent, bool warm, int part) {
    ConstArgs a;
    a.F = F;
    a.gid = h->d_gid;
    a.C = h->d_C;
    a.S0 = h->d_S0;
    a.G32 = h->d_geo32;
    a.H = h->d_nrm + 41LL * h->ngrains;
    a.warm = warm ? 1 : 0;
    a.warm_dev = nullptr;
    a.exact = h->cp_exact_only;
    a.small = h->small_strain;
    a.f32first = f32_first(h);
    a.rtol = return_map_tol(h->opt.newton_tol);
    a.gkind = h->d_gkind;
    a.gprm = h->d_nrm + 36LL * h->ngrains;  // parameters stored after the normals
    a.Fpi_n = h->d_Fpi;
    a.chi_n = h->d_chi;
    a.dt = dt;
    a.P = h->d_P;
    a.K = tangent == TANGENT_F32 ? nullptr : h->d_K;
    a.K32 = tangent == TANGENT_F64 ? nullptr : h->d_K32;
    a.Fpi_t = h->d_Fpi_t;
    a.chi_t = h->d_chi_t;
    a.dg = h->d_dg;
    a.tau = h->d_tau;
    a.flag = h->d_flag;
    a.stats = h->d_flag + 4;
    a.N = h->N;
    a.skip = nullptr;
    const int blocks = (int)((h->N + TPB - 1) / TPB);
    const bool f32 = tangent == TANGENT_F32;
    switch (part) {
        case CONST_P:
            if (f32) k_constitutive<true, PART_P><<<blocks, TPB, 0, h->stream>>>(a);
            else k_constitutive<false, PART_P><<<blocks, TPB, 0, h->stream>>>(a);
            break;
        case CONST_K:
            if (f32) k_constitutive<true, PART_K><<<blocks, TPB, 0, h->stream>>>(a);
            else k_constitutive<false, PART_K><<<blocks, TPB, 0, h->stream>>>(a);
            break;
        default:
            if (f32) k_constitutive<true, PART_ALL><<<blocks, TPB, 0, h->stream>>>(a);
            else k_constitutive<false, PART_ALL><<<blocks, TPB, 0, h->stream>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t upload_constitutive_batch(gff_handle* const* hs, int n, double dt, int tangent, const bool* warm,
                                      const int* warm_dev, const int* skip_dev, int* cpflag_dev, void* scratch_dev,
                                      int* blocks_out, cudaStream_t st) {
    ConstArgs args[MAX_BATCH];
    int start[MAX_BATCH + 1];
    start[0] = 0;
    for (int r = 0; r < n; ++r) {
        gff_handle* h = hs[r];
        ConstArgs& a = args[r];
        a.F = h->d_Fk;
        a.gid = h->d_gid;
        a.C = h->d_C;
        a.S0 = h->d_S0;
        a.G32 = h->d_geo32;
        a.H = h->d_nrm + 41LL * h->ngrains;
        a.warm = warm[r] ? 1 : 0;
        a.warm_dev = warm_dev ? warm_dev + r : nullptr;
        a.exact = h->cp_exact_only;
        a.small = h->small_strain;
        a.f32first = f32_first(h);
        a.rtol = return_map_tol(h->opt.newton_tol);
        a.gkind = h->d_gkind;
        a.gprm = h->d_nrm + 36LL * h->ngrains;
        a.Fpi_n = h->d_Fpi;
        a.chi_n = h->d_chi;
        a.dt = dt;
        a.P = h->d_P;
        a.K = tangent == TANGENT_F32 ? nullptr : h->d_K;
        a.K32 = tangent == TANGENT_F64 ? nullptr : h->d_K32;
        a.Fpi_t = h->d_Fpi_t;
        a.chi_t = h->d_chi_t;
        a.dg = h->d_dg;
        a.tau = h->d_tau;
        a.flag = cpflag_dev + r;
        a.stats = nullptr;
        a.N = h->N;
        a.skip = skip_dev + 2 * r;
        start[r + 1] = start[r] + (int)((h->N + TPB - 1) / TPB);
    }
    unsigned char* d = static_cast<unsigned char*>(scratch_dev);
    cudaError_t e = cudaMemcpyAsync(d, args, sizeof(ConstArgs) * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d + sizeof(ConstArgs) * MAX_BATCH, start, sizeof(int) * (n + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host arrays above go out of scope
    *blocks_out = start[n];
    return e;
}

cudaError_t launch_constitutive_batch_uploaded(const void* scratch_dev, int n, int blocks, int tangent, int part,
                                               cudaStream_t st) {
    const unsigned char* d = static_cast<const unsigned char*>(scratch_dev);
    const ConstArgs* dargs = reinterpret_cast<const ConstArgs*>(d);
    const int* dstart = reinterpret_cast<const int*>(d + sizeof(ConstArgs) * MAX_BATCH);
    const bool f32 = tangent == TANGENT_F32;
    switch (part) {
        case CONST_P:
            if (f32) k_constitutive_batch<true, PART_P><<<blocks, TPB, 0, st>>>(dargs, dstart, n);
            else k_constitutive_batch<false, PART_P><<<blocks, TPB, 0, st>>>(dargs, dstart, n);
            break;
        case CONST_K:
            if (f32) k_constitutive_batch<true, PART_K><<<blocks, TPB, 0, st>>>(dargs, dstart, n);
            else k_constitutive_batch<false, PART_K><<<blocks, TPB, 0, st>>>(dargs, dstart, n);
            break;
        default:
            if (f32) k_constitutive_batch<true, PART_ALL><<<blocks, TPB, 0, st>>>(dargs, dstart, n);
            else k_constitutive_batch<false, PART_ALL><<<blocks, TPB, 0, st>>>(dargs, dstart, n);
    }
    return cudaGetLastError();
}

size_t constitutive_batch_scratch_bytes() { return sizeof(ConstArgs) * MAX_BATCH + sizeof(int) * (MAX_BATCH + 1); }

cudaError_t launch_fip_accumulate(gff_handle* h) {
    FipArgs a;
    a.gid = h->d_gid;
    a.gkind = h->d_gkind;
    a.S0 = h->d_S0;
    a.nrm = h->d_nrm;
    a.dg = h->d_dg;
    a.tau = h->d_tau;
    a.F = h->d_F;
    a.P = h->d_P;
    a.acc = h->d_acc;
    a.N = h->N;
    const int blocks = (int)((h->N + TPB - 1) / TPB);
    k_fip_accumulate<<<blocks, TPB, 0, h->stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_fip_reset(gff_handle* h) {
    const int blocks = (int)((h->N + TPB - 1) / TPB);
    k_fip_reset<<<blocks, TPB, 0, h->stream>>>(h->d_acc, h->N);
    return cudaGetLastError();
}

// pc[ngrains], w[ngrains*12], fs[ngrains] are device arrays; scratch holds GSUM*ngrains doubles
cudaError_t launch_grain_fips(gff_handle* h, double* pc, double* w, double* fs) {
    double* sums = pc + h->ngrains * 14;  // caller provides room after the outputs
    cudaError_t e = cudaMemsetAsync(sums, 0, sizeof(double) * GSUM * h->ngrains, h->stream);
    if (e != cudaSuccess) return e;
    const int blocks = (int)((h->N + TPB - 1) / TPB);
    k_grain_sums<<<blocks, TPB, 0, h->stream>>>(h->d_gid, h->d_gkind, h->d_acc, h->N, sums);
    k_grain_final<<<(h->ngrains + 127) / 128, 128, 0, h->stream>>>(sums, h->ngrains, h->opt.fs_k, h->opt.fs_sigma_y, pc,
                                                                    w, fs);
    return cudaGetLastError();
}

}  // namespace gff
