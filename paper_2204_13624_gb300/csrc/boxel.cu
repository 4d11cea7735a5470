// boxel.cu -- rank-one laminate law of the composite boxels (paper Sec. 4), FP64.
//
// One thread per boxel:
//   F(+/-) = F_box +/- (1/c(+/-)) a (x) N                     (Eq. Fpm)
//   f(a)   = (P+ - P-) N                                      (Eq. tractionbalance)
//   Newton-Raphson on a (Algorithm 1) with the Hessian of Eq. (hessian),
//   selective back-projection of inadmissible iterates (Algorithm 2, Sec. 4.2),
//   P_box = c+ P+ + c- P-                                     (Eq. Peff:Seff)
//   A_box = c+ A+ + c- A- - dA D Delta^{-1} D^T dA            (Sec. 4.1; the
//   volume average c+ A+ + c- A- is used in the first term, as in the
//   cheat-sheet table -- the printed "c- A+" is read as a typo).
//
// For the Neo-Hookean law (Sec. 6.1) with G = F^{-1}, g = G^T N, m = mu - lam ln J:
//   N.A.N      = mu |N|^2 I + (lam + m) g (x) g
//   (A D)_(iJ),k = mu d_ik N_J + lam G_Ji g_k + m G_Jk g_i
// so the Hessian and the tangent correction need no 9x9 products.
#include <type_traits>

#include "combo_internal.cuh"
#include "../../include/combo.h"

namespace combo {

struct Phase {
    double F[9], G[9], g[3], P[9], lnJ, J;
};

__device__ __forceinline__ bool nh_phase(Phase& s, double mu, double lam, const double N[3])
{
    const double* F = s.F;
    const double c0 = F[4] * F[8] - F[5] * F[7];
    const double c1 = F[5] * F[6] - F[3] * F[8];
    const double c2 = F[3] * F[7] - F[4] * F[6];
    const double J = F[0] * c0 + F[1] * c1 + F[2] * c2;
    s.J = J;
    if (!(J > 0.0)) return false;
    const double iJ = 1.0 / J;
    s.G[0] = c0 * iJ;
    s.G[1] = (F[2] * F[7] - F[1] * F[8]) * iJ;
    s.G[2] = (F[1] * F[5] - F[2] * F[4]) * iJ;
    s.G[3] = c1 * iJ;
    s.G[4] = (F[0] * F[8] - F[2] * F[6]) * iJ;
    s.G[5] = (F[2] * F[3] - F[0] * F[5]) * iJ;
    s.G[6] = c2 * iJ;
    s.G[7] = (F[1] * F[6] - F[0] * F[7]) * iJ;
    s.G[8] = (F[0] * F[4] - F[1] * F[3]) * iJ;
    s.lnJ = log(J);
    const double k = lam * s.lnJ - mu;
#pragma unroll
    for (int i = 0; i < 3; i++) {
#pragma unroll
        for (int j = 0; j < 3; j++) s.P[3 * i + j] = mu * F[3 * i + j] + k * s.G[3 * j + i];
        s.g[i] = s.G[i] * N[0] + s.G[3 + i] * N[1] + s.G[6 + i] * N[2];
    }
    return true;
}

struct LamEval {
    Phase p, m;
    double f[3];
    double err, eps;
};

// (icp, icm = 1/c+, 1/c-: the jump enters as (a/c) (x) N)
__device__ __forceinline__ bool lam_eval(LamEval& e, const double Fb[9], const double N[3], double icp, double icm,
                                         const double a[3], const double mu[2], const double lam[2], double tol_rel,
                                         double tol_abs)
{
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const double ap = a[i] * icp, am = a[i] * icm;
#pragma unroll
        for (int j = 0; j < 3; j++) {
            e.p.F[3 * i + j] = Fb[3 * i + j] + ap * N[j];
            e.m.F[3 * i + j] = Fb[3 * i + j] - am * N[j];
        }
    }
    if (!nh_phase(e.p, mu[1], lam[1], N)) return false;
    if (!nh_phase(e.m, mu[0], lam[0], N)) return false;
    double tp = 0.0, tm = 0.0, ff = 0.0;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const double a1 = e.p.P[3 * i] * N[0] + e.p.P[3 * i + 1] * N[1] + e.p.P[3 * i + 2] * N[2];
        const double a2 = e.m.P[3 * i] * N[0] + e.m.P[3 * i + 1] * N[1] + e.m.P[3 * i + 2] * N[2];
        e.f[i] = a1 - a2;
        tp += a1 * a1;
        tm += a2 * a2;
        ff += e.f[i] * e.f[i];
    }
    e.err = sqrt(ff);
    e.eps = tol_rel * (sqrt(tp) + sqrt(tm)) + tol_abs * fmax(mu[0], mu[1]);
    return true;
}

// Delta = sum_phase (1/c) [mu I + (lam + mu - lam ln J) g g^T]   (|N| = 1; wp, wm = 1/c+, 1/c-)
__device__ __forceinline__ void hessian(const LamEval& e, double wp, double wm, const double mu[2],
                                        const double lam[2], double D[9])
{
    const double sp = (lam[1] + mu[1] - lam[1] * e.p.lnJ) * wp;
    const double sm = (lam[0] + mu[0] - lam[0] * e.m.lnJ) * wm;
    const double d = mu[1] * wp + mu[0] * wm;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int k = 0; k < 3; k++)
            D[3 * i + k] = (i == k ? d : 0.0) + sp * e.p.g[i] * e.p.g[k] + sm * e.m.g[i] * e.m.g[k];
}

__device__ __forceinline__ bool inv3(const double A[9], double B[9])
{
    const double c0 = A[4] * A[8] - A[5] * A[7];
    const double c1 = A[5] * A[6] - A[3] * A[8];
    const double c2 = A[3] * A[7] - A[4] * A[6];
    const double det = A[0] * c0 + A[1] * c1 + A[2] * c2;
    if (det == 0.0 || !isfinite(det)) return false;
    const double id = 1.0 / det;
    B[0] = c0 * id;
    B[1] = (A[2] * A[7] - A[1] * A[8]) * id;
    B[2] = (A[1] * A[5] - A[2] * A[4]) * id;
    B[3] = c1 * id;
    B[4] = (A[0] * A[8] - A[2] * A[6]) * id;
    B[5] = (A[2] * A[3] - A[0] * A[5]) * id;
    B[6] = c2 * id;
    B[7] = (A[1] * A[6] - A[0] * A[7]) * id;
    B[8] = (A[0] * A[4] - A[1] * A[3]) * id;
    return true;
}

// ---- double-float form of the laminate solve (refined precision form with
// double-float residuals): the jump a, the phase states F, F^{-1}, J, ln J
// and P and the traction residual f in df32 (ln J by df_log), the Hessian,
// its inverse, the Newton direction and the admissibility test of
// Algorithm 2 in FP32.  The iterations run on the FP32 pipe alone (the
// per-boxel constants are split once) and stop at the rounding level of the
// df32 residual; the FP64 residual then decides convergence.
struct PhaseD {
    df32 F[9], G[9], P[9], J, lnJ;
    float g[3];  // G^T N
};

// Per-boxel constants of the double-float iterations: the phase constants
// (0 matrix, 1 inclusion) split into df32, and the stopping test
// |f| <= tol_rel (|P+ N| + |P- N|) + eps_abs with the rounding level
// floor_scale (1 + |P+ N| + |P- N|) of f.
struct DfLam {
    df32 mu[2], lam[2];
    float tol_rel, eps_abs, floor_scale;
};

__device__ __forceinline__ DfLam df_lam(const double mu[2], const double lam[2], double tol_rel, double tol_abs)
{
    DfLam k;
#pragma unroll
    for (int i = 0; i < 2; i++) {
        k.mu[i] = df32(mu[i]);
        k.lam[i] = df32(lam[i]);
    }
    k.tol_rel = (float)tol_rel;
    k.eps_abs = (float)(tol_abs * fmax(mu[0], mu[1]));
    // P = mu F + k F^{-T} is formed from terms of size ~(mu + lam) |F|: 2^-44 of that
    k.floor_scale = (float)(0x1p-44 * (fmax(mu[0], mu[1]) + fmax(lam[0], lam[1])));
    return k;
}

__device__ __forceinline__ bool nh_phase_df(PhaseD& s, df32 mud, df32 lamd, const df32 N[3], double* gd = nullptr)
{
    const df32* F = s.F;
    const df32 c0 = F[4] * F[8] - F[5] * F[7];
    const df32 c1 = F[5] * F[6] - F[3] * F[8];
    const df32 c2 = F[3] * F[7] - F[4] * F[6];
    const df32 J = F[0] * c0 + F[1] * c1 + F[2] * c2;
    s.J = J;
    if (!(J.hi > 0.f)) return false;
    const df32 iJ = df32(1.f, 0.f) / J;
    s.G[0] = c0 * iJ;
    s.G[1] = (F[2] * F[7] - F[1] * F[8]) * iJ;
    s.G[2] = (F[1] * F[5] - F[2] * F[4]) * iJ;
    s.G[3] = c1 * iJ;
    s.G[4] = (F[0] * F[8] - F[2] * F[6]) * iJ;
    s.G[5] = (F[2] * F[3] - F[0] * F[5]) * iJ;
    s.G[6] = c2 * iJ;
    s.G[7] = (F[1] * F[6] - F[0] * F[7]) * iJ;
    s.G[8] = (F[0] * F[4] - F[1] * F[3]) * iJ;
    s.lnJ = df_log(J);
    const df32 k = lamd * s.lnJ - mud;
#pragma unroll
    for (int i = 0; i < 3; i++) {
#pragma unroll
        for (int j = 0; j < 3; j++) s.P[3 * i + j] = mud * F[3 * i + j] + k * s.G[3 * j + i];
        const df32 gi = s.G[i] * N[0] + s.G[3 + i] * N[1] + s.G[6 + i] * N[2];
        s.g[i] = (float)gi;
        if (gd) gd[i] = (double)gi;
    }
    return true;
}

struct LamEvalD {
    PhaseD p, m;
    float f[3];
    float err, eps;
    float tol;    // the laminate tolerance (eps before the rounding-level floor)
    float floor;  // rounding level of f in double-float: below it only FP64 can decide
};

__device__ __forceinline__ bool lam_eval(LamEvalD& e, const df32 Fb[9], const df32 N[3], df32 icp, df32 icm,
                                         const df32 a[3], const DfLam& k)
{
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const df32 t = a[i] * N[j];
            e.p.F[3 * i + j] = Fb[3 * i + j] + t * icp;
            e.m.F[3 * i + j] = Fb[3 * i + j] - t * icm;
        }
    if (!nh_phase_df(e.p, k.mu[1], k.lam[1], N)) return false;
    if (!nh_phase_df(e.m, k.mu[0], k.lam[0], N)) return false;
    float tp = 0.f, tm = 0.f, ff = 0.f;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const df32 a1 = e.p.P[3 * i] * N[0] + e.p.P[3 * i + 1] * N[1] + e.p.P[3 * i + 2] * N[2];
        const df32 a2 = e.m.P[3 * i] * N[0] + e.m.P[3 * i + 1] * N[1] + e.m.P[3 * i + 2] * N[2];
        const df32 fi = a1 - a2;
        e.f[i] = (float)fi;
        tp += a1.hi * a1.hi;
        tm += a2.hi * a2.hi;
        ff += fi.hi * fi.hi;
    }
    const float nt = sqrtf(tp) + sqrtf(tm);
    e.err = sqrtf(ff);
    e.eps = e.tol = k.tol_rel * nt + k.eps_abs;
    e.floor = k.floor_scale * (1.f + nt);
    return true;
}

// The laminate Hessian in FP32, scaled by 1/d (d = mu+/c+ + mu-/c-):
//   Delta / d = I + s+ g+ g+^T + s- g- g-^T,  s = K - L ln J,
//   K = (lam + mu) / (c d), L = lam / (c d)  (per phase; formed once per boxel)
struct HessF {
    float Kp, Lp, Km, Lm, id0;
};

__device__ __forceinline__ HessF hess_f(const double mu[2], const double lam[2], double wp, double wm)
{
    const double id = 1.0 / (mu[1] * wp + mu[0] * wm);
    HessF h;
    h.Kp = (float)((lam[1] + mu[1]) * wp * id);
    h.Lp = (float)(lam[1] * wp * id);
    h.Km = (float)((lam[0] + mu[0]) * wm * id);
    h.Lm = (float)(lam[0] * wm * id);
    h.id0 = (float)id;
    return h;
}

// Delta^{-1} = (Delta / d)^{-1} / d in FP32.  False when the rank-one parts
// outweigh the isotropic part by more than 1e4 (a phase close to collapse,
// J -> 0): an FP32 inverse would not give a Newton direction there, and the
// caller continues in FP64.
__device__ __forceinline__ bool hess_inv_f(const HessF& h, float lnJp, float lnJm, const float gp[3],
                                           const float gm[3], float Di[9])
{
    const float sp = h.Kp - h.Lp * lnJp;
    const float sm = h.Km - h.Lm * lnJm;
    const float gp2 = gp[0] * gp[0] + gp[1] * gp[1] + gp[2] * gp[2];
    const float gm2 = gm[0] * gm[0] + gm[1] * gm[1] + gm[2] * gm[2];
    if (!(fabsf(sp) * gp2 <= 1e4f && fabsf(sm) * gm2 <= 1e4f)) return false;
    float A[9];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int k = 0; k < 3; k++) A[3 * i + k] = (i == k ? 1.f : 0.f) + sp * gp[i] * gp[k] + sm * gm[i] * gm[k];
    const float c0 = A[4] * A[8] - A[5] * A[7];
    const float c1 = A[5] * A[6] - A[3] * A[8];
    const float c2 = A[3] * A[7] - A[4] * A[6];
    const float det = A[0] * c0 + A[1] * c1 + A[2] * c2;
    if (det == 0.f || !isfinite(det)) return false;
    const float id = h.id0 / det;
    Di[0] = c0 * id;
    Di[1] = (A[2] * A[7] - A[1] * A[8]) * id;
    Di[2] = (A[1] * A[5] - A[2] * A[4]) * id;
    Di[3] = c1 * id;
    Di[4] = (A[0] * A[8] - A[2] * A[6]) * id;
    Di[5] = (A[2] * A[3] - A[0] * A[5]) * id;
    Di[6] = c2 * id;
    Di[7] = (A[1] * A[6] - A[0] * A[7]) * id;
    Di[8] = (A[0] * A[4] - A[1] * A[3]) * id;
    return true;
}

// from a double-float laminate state (the Newton direction of its iterations)
__device__ __forceinline__ bool hessian_inv(const LamEvalD& e, const HessF& h, float Di[9])
{
    return hess_inv_f(h, (float)e.p.lnJ, (float)e.m.lnJ, e.p.g, e.m.g, Di);
}

// from an FP64 laminate state: the Delta^{-1} of an FP32 boxel tangent, and
// the direction of the certifying FP64 steps of the double-float form
__device__ __forceinline__ bool hessian_inv32(const LamEval& e, const HessF& h, float Di[9])
{
    const float gp[3] = {(float)e.p.g[0], (float)e.p.g[1], (float)e.p.g[2]};
    const float gm[3] = {(float)e.m.g[0], (float)e.m.g[1], (float)e.m.g[2]};
    return hess_inv_f(h, (float)e.p.lnJ, (float)e.m.lnJ, gp, gm, Di);
}

// One Neo-Hookean phase's tangent data in precision S:
//   A_iJkL     = mu d_ik d_JL + lam G_Ji G_Lk + m G_Jk G_Li,   m = mu - lam ln J
//   (A D)_(iJ),k = mu d_ik N_J + lam G_Ji g_k + m G_Jk g_i,     g = G^T N
template <typename S> struct TanPhase {
    S G[9], g[3], mu, lam, m;
    __device__ __forceinline__ void load(const Phase& s, double mu_, double lam_)
    {
#pragma unroll
        for (int q = 0; q < 9; q++) G[q] = (S)s.G[q];
#pragma unroll
        for (int q = 0; q < 3; q++) g[q] = (S)s.g[q];
        mu = (S)mu_;
        lam = (S)lam_;
        m = (S)(mu_ - lam_ * s.lnJ);
    }
    __device__ __forceinline__ void load(const PhaseD& s, double mu_, double lam_)
    {
#pragma unroll
        for (int q = 0; q < 9; q++) G[q] = (S)(double)s.G[q];
#pragma unroll
        for (int q = 0; q < 3; q++) g[q] = (S)s.g[q];
        mu = (S)mu_;
        lam = (S)lam_;
        m = (S)(mu_ - lam_ * (double)s.lnJ);
    }

    __device__ __forceinline__ S AD(const S N[3], int i, int Jx, int k) const
    {
        return (i == k ? mu * N[Jx] : (S)0) + lam * G[3 * Jx + i] * g[k] + m * G[3 * Jx + k] * g[i];
    }
    __device__ __forceinline__ S A(int i, int Jx, int k, int L) const
    {
        return ((i == k && Jx == L) ? mu : (S)0) + lam * G[3 * Jx + i] * G[3 * L + k] + m * G[3 * Jx + k] * G[3 * L + i];
    }
};

// Newton-Raphson on the jump a (Algorithm 1) with selective back-projection
// (Algorithm 2) from the current a, until e.err <= max(e.eps, floor); it counts
// the iterations of every call against max_iter.  Returns 0, or the failure
// reason: 2 a phase inadmissible, 3 singular Hessian, 4 iteration cap.
template <class LE, class EV, class INV>
__device__ __forceinline__ int nr_loop(LE& e, double a[3], const double m[3], double bcp, double bcm, double floor,
                                       int& it, int max_iter, double& nbp, const EV& evaluate, const INV& inverse)
{
    if (!evaluate(e)) return 2;
    while (e.err > fmax(e.eps, floor)) {
        if (it >= max_iter) return 4;
        double Di[9];
        if (!inverse(e, Di)) return 3;
        double a1[3];
#pragma unroll
        for (int i = 0; i < 3; i++) a1[i] = a[i] - (Di[3 * i] * e.f[0] + Di[3 * i + 1] * e.f[1] + Di[3 * i + 2] * e.f[2]);
        const double b1 = a1[0] * m[0] + a1[1] * m[1] + a1[2] * m[2];
        if (!(b1 > bcp && b1 < bcm)) {
            // Algorithm 2: keep M_perp a1, move the m_beta coordinate to the
            // midpoint between the admissible beta0 and the crossed bound
            const double b0 = a[0] * m[0] + a[1] * m[1] + a[2] * m[2];
            const double bc = (b1 <= bcp) ? bcp : bcm;
            const double bs = 0.5 * (b0 + bc);
#pragma unroll
            for (int i = 0; i < 3; i++) a1[i] = (a1[i] - b1 * m[i]) + bs * m[i];
            nbp += 1.0;
        }
        a[0] = a1[0];
        a[1] = a1[1];
        a[2] = a1[2];
        it++;
        if (!evaluate(e)) return 2;
    }
    return 0;
}

// The same iterations in the double-float form, on the FP32 pipe: the jump
// in df32, the direction Delta^{-1} f from the FP32 Hessian inverse, the
// admissibility test and the back-projection of Algorithm 2 on the FP32
// values of m_beta . a; until |f| <= max(eps, its rounding level).  Returns
// as nr_loop.
template <class EV>
__device__ __forceinline__ int nr_loop_df(LamEvalD& e, df32 a[3], const float m[3], float bcp, float bcm, int& it,
                                          int max_iter, double& nbp, const HessF& h, const EV& evaluate)
{
    if (!evaluate(e)) return 2;
    while (e.err > fmaxf(e.eps, e.floor)) {
        if (it >= max_iter) return 4;
        float Di[9];
        if (!hessian_inv(e, h, Di)) return 3;
        df32 a1[3];
#pragma unroll
        for (int i = 0; i < 3; i++)
            a1[i] = a[i] - df32(Di[3 * i] * e.f[0] + Di[3 * i + 1] * e.f[1] + Di[3 * i + 2] * e.f[2], 0.f);
        const float b1 = (float)a1[0] * m[0] + (float)a1[1] * m[1] + (float)a1[2] * m[2];
        if (!(b1 > bcp && b1 < bcm)) {
            const float b0 = (float)a[0] * m[0] + (float)a[1] * m[1] + (float)a[2] * m[2];
            const float bc = (b1 <= bcp) ? bcp : bcm;
            const float db = 0.5f * (b0 + bc) - b1;
#pragma unroll
            for (int i = 0; i < 3; i++) a1[i] = a1[i] + df32(db * m[i], 0.f);
            nbp += 1.0;
        }
#pragma unroll
        for (int i = 0; i < 3; i++) a[i] = a1[i];
        it++;
        if (!evaluate(e)) return 2;
    }
    return 0;
}

// The packed boxel tangent A_box = c+ A+ + c- A- - dA D Delta^{-1} D^T dA
// (Sec. 4.1) in precision Tc from a converged laminate state (FP64 or double-
// float phases ep, em) and Delta^{-1} (Di): the 45 entries of its upper
// triangle (major symmetry) go to out[sym_idx * stride + col].
template <typename Tc, typename PH>
__device__ __forceinline__ void boxel_tangent_store(const PH& ep, const PH& em, const double N[3], double cp,
                                                    double cm, const double mu[2], const double lam[2],
                                                    const double Di[9], Tc* out, int64_t stride, int64_t col)
{
    TanPhase<Tc> tp, tm;
    tp.load(ep, mu[1], lam[1]);
    tm.load(em, mu[0], lam[0]);
    Tc Nt[3] = {(Tc)N[0], (Tc)N[1], (Tc)N[2]};
    Tc Dt[9];
#pragma unroll
    for (int q = 0; q < 9; q++) Dt[q] = (Tc)Di[q];
    const Tc cpt = (Tc)cp, cmt = (Tc)cm;
    // B = dA D (9x3), W = B Delta^{-1}
    Tc B[27], W[27];
#pragma unroll
    for (int r = 0; r < 9; r++)
#pragma unroll
        for (int k = 0; k < 3; k++) B[3 * r + k] = tp.AD(Nt, r / 3, r % 3, k) - tm.AD(Nt, r / 3, r % 3, k);
#pragma unroll
    for (int r = 0; r < 9; r++)
#pragma unroll
        for (int k = 0; k < 3; k++)
            W[3 * r + k] = B[3 * r] * Dt[k] + B[3 * r + 1] * Dt[3 + k] + B[3 * r + 2] * Dt[6 + k];
#pragma unroll
    for (int r = 0; r < 9; r++)
#pragma unroll
        for (int s2 = r; s2 < 9; s2++) {
            const Tc avg = cpt * tp.A(r / 3, r % 3, s2 / 3, s2 % 3) + cmt * tm.A(r / 3, r % 3, s2 / 3, s2 % 3);
            const Tc corr = W[3 * r] * B[3 * s2] + W[3 * r + 1] * B[3 * s2 + 1] + W[3 * r + 2] * B[3 * s2 + 2];
            out[(int64_t)sym_idx(r, s2) * stride + col] = avg - corr;
        }
}

// DFM: the double-float form: the Newton iterations run on the double-float
// residual down to its rounding level, then the FP64 residual decides
// convergence (and takes the last step if needed), so the stopping test and
// the returned state are those of the FP64 form.
// (body of block vb of 128 boxels; a grouped launch over several grids
// calls it once per work item)
template <typename Tc, bool DFM> __device__ __forceinline__ void boxel_body(const BoxelArgs<Tc>& A, int vb)
{
    __shared__ double red[64];
    __shared__ int same_problem;
    const int64_t b = (int64_t)vb * blockDim.x + threadIdx.x;
    // the problem of this boxel (stacked problems: boxels in problem order)
    const int pb = (A.bprob && b < A.nb) ? A.bprob[b] : 0;
    Scalars* sc = A.sc + pb;
    double its = 0.0, nbp = 0.0, nev = 0.0;
    if (b < A.nb && !(A.guard == 2 && sc->outer_done)) {
        nev = 1.0;
        const int64_t v = A.bidx[b];
        double Fb[9], N[3], a[3];
#pragma unroll
        for (int c = 0; c < 9; c++) Fb[c] = A.F[c * A.V + v];
#pragma unroll
        for (int i = 0; i < 3; i++) {
            N[i] = A.bN[3 * b + i];
            a[i] = A.ba[3 * b + i];
        }
        const double cp = A.bc[b], cm = 1.0 - cp;
        const double* mp = A.matp ? A.matp + 4 * pb : nullptr;
        const double mu[2] = {mp ? mp[0] : A.mu[0], mp ? mp[1] : A.mu[1]};
        const double lam[2] = {mp ? mp[2] : A.lam[0], mp ? mp[3] : A.lam[1]};
        int status = 0, reason = 0;
        // m_beta = F^{-T} N / |F^{-T} N|, beta_c(+/-) = -/+ c(+/-) / |F^{-T} N|  (Sec. 4.2)
        double gbox[3];
        // 1/c+-, once (the iterations multiply by them)
        const double icp64 = 1.0 / cp, icm64 = 1.0 / cm;
        const HessF hf = hess_f(mu, lam, icp64, icm64);
        df32 Fd[9], Nd[3], icp, icm;
        DfLam dk;
        if constexpr (DFM) {
#pragma unroll
            for (int c = 0; c < 9; c++) Fd[c] = df32(Fb[c]);
#pragma unroll
            for (int i = 0; i < 3; i++) Nd[i] = df32(N[i]);
            icp = df32(icp64);
            icm = df32(icm64);
            dk = df_lam(mu, lam, A.tol_rel, A.tol_abs);
            PhaseD box;
#pragma unroll
            for (int c = 0; c < 9; c++) box.F[c] = Fd[c];
            if (!nh_phase_df(box, dk.mu[0], dk.lam[0], Nd, gbox)) status = finite9(Fb) ? COMBO_E_INADMISSIBLE : COMBO_E_NAN;
        } else {
            Phase box;
#pragma unroll
            for (int c = 0; c < 9; c++) box.F[c] = Fb[c];
            if (!nh_phase(box, mu[0], lam[0], N)) status = finite9(Fb) ? COMBO_E_INADMISSIBLE : COMBO_E_NAN;
#pragma unroll
            for (int i = 0; i < 3; i++) gbox[i] = box.g[i];
        }
        LamEval e;
        auto eval64 = [&](LamEval& x) {
            return lam_eval(x, Fb, N, icp64, icm64, a, mu, lam, A.tol_rel, A.tol_abs);
        };
        auto inv64 = [&](const LamEval& x, double Di[9]) {
            double Dl[9];
            hessian(x, icp64, icm64, mu, lam, Dl);
            return inv3(Dl, Di);
        };
        // the FP64 steps that follow double-float iterations take the FP32
        // inverse (their residual is already at the df32 rounding level)
        auto inv_cert = [&](const LamEval& x, double Di[9]) {
            float Df[9];
            if (!hessian_inv32(x, hf, Df)) return inv64(x, Di);
#pragma unroll
            for (int q = 0; q < 9; q++) Di[q] = Df[q];
            return true;
        };
        double Di[9];
        LamEvalD ed;           // (double-float form) the last double-float evaluation
        bool df_done = false;  // (double-float form) its state is the converged one
        if (!status) {
            const double ng = sqrt(gbox[0] * gbox[0] + gbox[1] * gbox[1] + gbox[2] * gbox[2]);
            const double m[3] = {gbox[0] / ng, gbox[1] / ng, gbox[2] / ng};
            const double bcp = -cp / ng, bcm = cm / ng;
            double beta = a[0] * m[0] + a[1] * m[1] + a[2] * m[2];
            if (!(beta > bcp && beta < bcm)) a[0] = a[1] = a[2] = 0.0;
            int it = 0, it_df = 0;
            if constexpr (DFM) {
                // double-float iterations from a copy of the start; if they
                // stop early (a phase near collapse, an ill-conditioned
                // Hessian), the FP64 iterations start over from a
                df32 ad[3] = {df32(a[0]), df32(a[1]), df32(a[2])};
                const float mf[3] = {(float)m[0], (float)m[1], (float)m[2]};
                const int rdf = nr_loop_df(ed, ad, mf, (float)bcp, (float)bcm, it_df, A.max_iter, nbp, hf,
                                           [&](LamEvalD& x) { return lam_eval(x, Fd, Nd, icp, icm, ad, dk); });
                if (rdf == 0) {
#pragma unroll
                    for (int i = 0; i < 3; i++) a[i] = (double)ad[i];
                    // the double-float residual lies below the tolerance by
                    // more than its own rounding level: the FP64 residual
                    // passes the same test, and the FP64 evaluation is skipped
                    float Df[9];
                    df_done = ed.err + ed.floor <= 0.99f * ed.tol && hessian_inv(ed, hf, Df);
                    if (df_done)
#pragma unroll
                        for (int q = 0; q < 9; q++) Di[q] = Df[q];
                }
            }
            if (!df_done) {
                if constexpr (DFM)
                    reason = nr_loop(e, a, m, bcp, bcm, 0.0, it, A.max_iter, nbp, eval64, inv_cert);
                else
                    reason = nr_loop(e, a, m, bcp, bcm, 0.0, it, A.max_iter, nbp, eval64, inv64);
                if (reason) status = COMBO_E_LAMINATE;
            }
            its = it + it_df;
        } else {
            reason = 1;
        }
        if (status) {
            raise_status(sc, status);
            if (atomicCAS(&sc->fail_boxel, 0, (int32_t)(b + 1)) == 0) {
                sc->fail_reason = reason;
#pragma unroll
                for (int c = 0; c < 9; c++) sc->fail_state[c] = Fb[c];
#pragma unroll
                for (int i = 0; i < 3; i++) {
                    sc->fail_state[9 + i] = N[i];
                    sc->fail_state[13 + i] = a[i];
                }
                sc->fail_state[12] = cp;
            }
        } else {
            // The boxel tangent only feeds the Krylov iterations: it is formed
            // in their precision Tc from the converged state (FP64, or the
            // accepted double-float state); A_box is major-symmetric (the
            // second derivative of the condensed energy): its upper triangle
            // is stored, column rank[b]
            const int64_t kb = A.rank ? (int64_t)A.rank[b] : b;
            auto tangent = [&](const auto& ep, const auto& em) {
                boxel_tangent_store<Tc>(ep, em, N, cp, cm, mu, lam, Di, A.bA, A.nb, kb);
            };
            if (df_done) {
#pragma unroll
                for (int c = 0; c < 9; c++) A.bP[9 * b + c] = cp * (double)ed.p.P[c] + cm * (double)ed.m.P[c];
            } else {
#pragma unroll
                for (int c = 0; c < 9; c++) A.bP[9 * b + c] = cp * e.p.P[c] + cm * e.m.P[c];
            }
#pragma unroll
            for (int i = 0; i < 3; i++) A.ba[3 * b + i] = a[i];
            if (A.bA) {
                // (an FP32 tangent takes Delta^{-1} in FP32, off the FP64 pipe)
                bool inv_ok = false;
                if (!df_done) {
                    if constexpr (sizeof(Tc) == 4) {
                        float Df[9];
                        inv_ok = hessian_inv32(e, hf, Df);
                        if (inv_ok)
#pragma unroll
                            for (int q = 0; q < 9; q++) Di[q] = Df[q];
                    }
                    if (!inv_ok) inv_ok = inv64(e, Di);
                }
                if (df_done) {
                    tangent(ed.p, ed.m);
                } else if (!inv_ok) {
                    raise_status(sc, COMBO_E_LAMINATE);
                } else {
                    tangent(e.p, e.m);
                }
            }
        }
    }
    // counters: one atomic per block when its boxels share a problem
    if (threadIdx.x == 0) {
        const int64_t first = (int64_t)vb * blockDim.x;
        const int64_t last = min(first + (int64_t)blockDim.x, A.nb) - 1;
        same_problem = (!A.bprob || A.bprob[first] == A.bprob[last]) ? 1 : 0;
    }
    __syncthreads();
    if (same_problem) {
        const double s1 = block_sum(its, red);
        const double s2 = block_sum(nbp, red + 32);
        __syncthreads();
        const double s3 = block_sum(nev, red);
        if (threadIdx.x == 0) {
            Scalars* s0 = A.sc + (A.bprob ? A.bprob[(int64_t)vb * blockDim.x] : 0);
            atomicAdd(&s0->nr_iters, (unsigned long long)s1);
            atomicAdd(&s0->n_backproj, (unsigned long long)s2);
            atomicAdd(&s0->n_lam, (unsigned long long)s3);
        }
    } else if (nev > 0.0) {
        atomicAdd(&sc->nr_iters, (unsigned long long)its);
        atomicAdd(&sc->n_backproj, (unsigned long long)nbp);
        atomicAdd(&sc->n_lam, (unsigned long long)nev);
    }
}

template <typename Tc, bool DFM> __global__ void __launch_bounds__(128) k_boxel(BoxelArgs<Tc> A)
{
    boxel_body<Tc, DFM>(A, blockIdx.x);
}

// Infinitesimal-strain composite boxel in closed form (cheat sheet of the
// appendix, right column), |N| = 1:
//   Delta = N . (C+/c+ + C-/c-) . N = (mu+/c+ + mu-/c-) I + ((lam+ + mu+)/c+ + (lam- + mu-)/c-) N N^T,
//   f = N . (C- - C+) : eps = (lam- - lam+) tr(eps) N + 2 (mu- - mu+) eps N,   a = Delta^{-1} f,
//   eps+- = eps +- sym(a (x) N) / c+-,  sigma_box = c+ sigma+ + c- sigma-,
//   C_box = (c+ C+ + c- C-) - dC (N (x) Delta^{-1} (x) N) dC  (packed, in Tc).
// The tangent reuses TanPhase with G = I, g = N, m = mu, which is C.
template <typename Tc> __device__ __forceinline__ void boxel_linear_body(const BoxelArgs<Tc>& A, int vb)
{
    __shared__ double red[32];
    __shared__ int same_problem;
    const int64_t b = (int64_t)vb * blockDim.x + threadIdx.x;
    const int pb = (A.bprob && b < A.nb) ? A.bprob[b] : 0;
    Scalars* sc = A.sc + pb;
    double nev = 0.0;
    if (b < A.nb && !(A.guard == 2 && sc->outer_done)) {
        nev = 1.0;
        const int64_t v = A.bidx[b];
        double e[9], N[3];
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++)
                e[3 * i + j] = 0.5 * (A.F[(3 * i + j) * A.V + v] + A.F[(3 * j + i) * A.V + v]) - (i == j ? 1.0 : 0.0);
#pragma unroll
        for (int i = 0; i < 3; i++) N[i] = A.bN[3 * b + i];
        const double cp = A.bc[b], cm = 1.0 - cp;
        const double* mp = A.matp ? A.matp + 4 * pb : nullptr;
        const double mu[2] = {mp ? mp[0] : A.mu[0], mp ? mp[1] : A.mu[1]};
        const double lam[2] = {mp ? mp[2] : A.lam[0], mp ? mp[3] : A.lam[1]};
        const double d0 = mu[1] / cp + mu[0] / cm;
        const double d1 = (lam[1] + mu[1]) / cp + (lam[0] + mu[0]) / cm;
        double Dl[9], Di[9];
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int k = 0; k < 3; k++) Dl[3 * i + k] = (i == k ? d0 : 0.0) + d1 * N[i] * N[k];
        const double tr = e[0] + e[4] + e[8];
        double f[3], a[3];
#pragma unroll
        for (int i = 0; i < 3; i++)
            f[i] = (lam[0] - lam[1]) * tr * N[i] +
                   2.0 * (mu[0] - mu[1]) * (e[3 * i] * N[0] + e[3 * i + 1] * N[1] + e[3 * i + 2] * N[2]);
        if (!inv3(Dl, Di)) {
            raise_status(sc, COMBO_E_LAMINATE);
        } else {
#pragma unroll
            for (int i = 0; i < 3; i++) a[i] = Di[3 * i] * f[0] + Di[3 * i + 1] * f[1] + Di[3 * i + 2] * f[2];
            double trp = tr, trm = tr;
            const double aN = a[0] * N[0] + a[1] * N[1] + a[2] * N[2];
            trp += aN / cp;
            trm -= aN / cm;
#pragma unroll
            for (int i = 0; i < 3; i++)
#pragma unroll
                for (int j = 0; j < 3; j++) {
                    const double s = 0.5 * (a[i] * N[j] + a[j] * N[i]);
                    const double ep = e[3 * i + j] + s / cp, em = e[3 * i + j] - s / cm;
                    const double sp = 2.0 * mu[1] * ep + (i == j ? lam[1] * trp : 0.0);
                    const double sm = 2.0 * mu[0] * em + (i == j ? lam[0] * trm : 0.0);
                    A.bP[9 * b + 3 * i + j] = cp * sp + cm * sm;
                }
#pragma unroll
            for (int i = 0; i < 3; i++) A.ba[3 * b + i] = a[i];
            if (A.bA) {
                TanPhase<Tc> tp, tm;
#pragma unroll
                for (int q = 0; q < 9; q++) tp.G[q] = tm.G[q] = (Tc)((q == 0 || q == 4 || q == 8) ? 1.0 : 0.0);
#pragma unroll
                for (int q = 0; q < 3; q++) tp.g[q] = tm.g[q] = (Tc)N[q];
                tp.mu = (Tc)mu[1], tp.lam = (Tc)lam[1], tp.m = (Tc)mu[1];
                tm.mu = (Tc)mu[0], tm.lam = (Tc)lam[0], tm.m = (Tc)mu[0];
                Tc Nt[3] = {(Tc)N[0], (Tc)N[1], (Tc)N[2]};
                Tc Dt[9];
#pragma unroll
                for (int q = 0; q < 9; q++) Dt[q] = (Tc)Di[q];
                const Tc cpt = (Tc)cp, cmt = (Tc)cm;
                Tc B[27], W[27];
#pragma unroll
                for (int r = 0; r < 9; r++)
#pragma unroll
                    for (int k = 0; k < 3; k++) B[3 * r + k] = tp.AD(Nt, r / 3, r % 3, k) - tm.AD(Nt, r / 3, r % 3, k);
#pragma unroll
                for (int r = 0; r < 9; r++)
#pragma unroll
                    for (int k = 0; k < 3; k++)
                        W[3 * r + k] = B[3 * r] * Dt[k] + B[3 * r + 1] * Dt[3 + k] + B[3 * r + 2] * Dt[6 + k];
                const int64_t kb = A.rank ? (int64_t)A.rank[b] : b;
#pragma unroll
                for (int r = 0; r < 9; r++)
#pragma unroll
                    for (int s2 = r; s2 < 9; s2++) {
                        const Tc avg = cpt * tp.A(r / 3, r % 3, s2 / 3, s2 % 3) + cmt * tm.A(r / 3, r % 3, s2 / 3, s2 % 3);
                        const Tc corr = W[3 * r] * B[3 * s2] + W[3 * r + 1] * B[3 * s2 + 1] + W[3 * r + 2] * B[3 * s2 + 2];
                        A.bA[(int64_t)sym_idx(r, s2) * A.nb + kb] = avg - corr;
                    }
            }
        }
    }
    if (threadIdx.x == 0) {
        const int64_t first = (int64_t)vb * blockDim.x;
        const int64_t last = min(first + (int64_t)blockDim.x, A.nb) - 1;
        same_problem = (!A.bprob || A.bprob[first] == A.bprob[last]) ? 1 : 0;
    }
    __syncthreads();
    if (same_problem) {
        const double s3 = block_sum(nev, red);
        if (threadIdx.x == 0)
            atomicAdd(&(A.sc + (A.bprob ? A.bprob[(int64_t)vb * blockDim.x] : 0))->n_lam, (unsigned long long)s3);
    } else if (nev > 0.0) {
        atomicAdd(&sc->n_lam, (unsigned long long)nev);
    }
}

template <typename Tc> __global__ void __launch_bounds__(128) k_boxel_linear(BoxelArgs<Tc> A)
{
    boxel_linear_body<Tc>(A, blockIdx.x);
}

template <typename Tc> void launch_boxel(const BoxelArgs<Tc>& a, cudaStream_t st)
{
    if (a.nb <= 0) return;
    if (a.linear) {
        k_boxel_linear<Tc><<<(int)((a.nb + 127) / 128), 128, 0, st>>>(a);
        return;
    }
    const int grid = (int)((a.nb + 127) / 128);
    if constexpr (std::is_same<Tc, float>::value) {
        if (a.dfloat) {
            k_boxel<Tc, true><<<grid, 128, 0, st>>>(a);
            return;
        }
    }
    k_boxel<Tc, false><<<grid, 128, 0, st>>>(a);
}

// grouped: items of 128 boxels of several grids' boxel lists
template <typename Tc, bool DFM, bool LIN>
__global__ void __launch_bounds__(128)
    k_group_boxel(const BoxelArgs<Tc>* __restrict__ args, const int* __restrict__ vstart, int nd)
{
    const int total = __ldg(vstart + nd);
    for (int v = blockIdx.x; v < total; v += gridDim.x) {
        const int d = group_of(vstart, nd, v);
        if constexpr (LIN)
            boxel_linear_body<Tc>(args[d], v - __ldg(vstart + d));
        else
            boxel_body<Tc, DFM>(args[d], v - __ldg(vstart + d));
        __syncthreads();  // the next item reuses the block's shared sums
    }
}

template <typename Tc> void launch_group_boxel(const GroupTab<BoxelArgs<Tc>>& t, bool dfloat, bool linear,
                                               cudaStream_t st)
{
    if (t.total <= 0) return;
    if (linear) {
        auto k = k_group_boxel<Tc, false, true>;
        k<<<group_grid((const void*)k, 128, 0, t.total), 128, 0, st>>>(t.args, t.vstart, t.nd);
        return;
    }
    if constexpr (std::is_same<Tc, float>::value) {
        if (dfloat) {
            auto k = k_group_boxel<Tc, true, false>;
            k<<<group_grid((const void*)k, 128, 0, t.total), 128, 0, st>>>(t.args, t.vstart, t.nd);
            return;
        }
    }
    auto k = k_group_boxel<Tc, false, false>;
    k<<<group_grid((const void*)k, 128, 0, t.total), 128, 0, st>>>(t.args, t.vstart, t.nd);
}
template void launch_group_boxel<float>(const GroupTab<BoxelArgs<float>>&, bool, bool, cudaStream_t);
template void launch_group_boxel<double>(const GroupTab<BoxelArgs<double>>&, bool, bool, cudaStream_t);

// Doubly-fine material grid (App. A): the laminate of every sub-cell l of
// every composite boxel, at F_sub(c, l) (the cell's diagonal, the staggered
// off-diagonals nearest the sub-cell), from the sub-cell's own warm start
// a [nb][8][3]; the boxel stress c+ P+ + c- P- goes to S[9 l + comp][v].
// One thread per (boxel, sub-cell), FP64 (the fixed point and nonlinear CG
// run in FP64 only).
template <bool DFM> __global__ void __launch_bounds__(128) k_boxel_dfmg(BoxelArgs<double> A)
{
    __shared__ double red[64];
    __shared__ int same_problem;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nt = 8 * A.nb;
    const int64_t b = t >> 3;
    const int l = (int)(t & 7);
    const int pb = (A.bprob && t < nt) ? A.bprob[b] : 0;
    Scalars* sc = A.sc + pb;
    double its = 0.0, nbp = 0.0, nev = 0.0;
    if (t < nt && !(A.guard == 2 && sc->outer_done)) {
        nev = 1.0;
        const int64_t v = A.bidx[b];
        const int64_t base = (int64_t)pb * A.Vp, lv = v - base;
        const int i = (int)(lv % A.n1), j = (int)((lv / A.n1) % A.n2), k = (int)(lv / ((int64_t)A.n1 * A.n2));
        double Fb[9], N[3], a[3];
        dfmg_fsub(A.F, A.V, base, A.n1, A.n2, A.n3, i, j, k, l, Fb);
#pragma unroll
        for (int q = 0; q < 3; q++) {
            N[q] = A.bN[3 * b + q];
            a[q] = A.ba[24 * b + 3 * l + q];
        }
        const double cp = A.bc[b], cm = 1.0 - cp;
        const double* mp = A.matp ? A.matp + 4 * pb : nullptr;
        const double mu[2] = {mp ? mp[0] : A.mu[0], mp ? mp[1] : A.mu[1]};
        const double lam[2] = {mp ? mp[2] : A.lam[0], mp ? mp[3] : A.lam[1]};
        int status = 0, reason = 0;
        double gbox[3];
        // 1/c+-, once (the iterations multiply by them)
        const double icp64 = 1.0 / cp, icm64 = 1.0 / cm;
        const HessF hf = hess_f(mu, lam, icp64, icm64);
        df32 Fd[9], Nd[3], icp, icm;
        DfLam dk;
        if constexpr (DFM) {
#pragma unroll
            for (int c = 0; c < 9; c++) Fd[c] = df32(Fb[c]);
#pragma unroll
            for (int q = 0; q < 3; q++) Nd[q] = df32(N[q]);
            icp = df32(icp64);
            icm = df32(icm64);
            dk = df_lam(mu, lam, A.tol_rel, A.tol_abs);
            PhaseD box;
#pragma unroll
            for (int c = 0; c < 9; c++) box.F[c] = Fd[c];
            if (!nh_phase_df(box, dk.mu[0], dk.lam[0], Nd, gbox)) status = finite9(Fb) ? COMBO_E_INADMISSIBLE : COMBO_E_NAN;
        } else {
            Phase box;
#pragma unroll
            for (int c = 0; c < 9; c++) box.F[c] = Fb[c];
            if (!nh_phase(box, mu[0], lam[0], N)) status = finite9(Fb) ? COMBO_E_INADMISSIBLE : COMBO_E_NAN;
#pragma unroll
            for (int q = 0; q < 3; q++) gbox[q] = box.g[q];
        }
        LamEval e;
        auto eval64 = [&](LamEval& x) {
            return lam_eval(x, Fb, N, icp64, icm64, a, mu, lam, A.tol_rel, A.tol_abs);
        };
        auto inv64 = [&](const LamEval& x, double Di[9]) {
            double Dl[9];
            hessian(x, icp64, icm64, mu, lam, Dl);
            return inv3(Dl, Di);
        };
        LamEvalD ed;
        bool df_done = false;  // the double-float iterations converged: their state is the result
        if (!status) {
            const double ng = sqrt(gbox[0] * gbox[0] + gbox[1] * gbox[1] + gbox[2] * gbox[2]);
            const double m[3] = {gbox[0] / ng, gbox[1] / ng, gbox[2] / ng};
            const double bcp = -cp / ng, bcm = cm / ng;
            const double beta = a[0] * m[0] + a[1] * m[1] + a[2] * m[2];
            if (!(beta > bcp && beta < bcm)) a[0] = a[1] = a[2] = 0.0;
            int it = 0, it_df = 0;
            if constexpr (DFM) {
                // the double-float residual form: Newton iterations on the
                // double-float residual down to its rounding level; FP64
                // iterations only where they stop early (a phase near
                // collapse, an ill-conditioned Hessian)
                df32 ad[3] = {df32(a[0]), df32(a[1]), df32(a[2])};
                const float mf[3] = {(float)m[0], (float)m[1], (float)m[2]};
                const int rdf = nr_loop_df(ed, ad, mf, (float)bcp, (float)bcm, it_df, A.max_iter, nbp, hf,
                                           [&](LamEvalD& x) { return lam_eval(x, Fd, Nd, icp, icm, ad, dk); });
                if (rdf == 0) {
#pragma unroll
                    for (int q = 0; q < 3; q++) a[q] = (double)ad[q];
                    df_done = true;
                }
            }
            if (!df_done) {
                reason = nr_loop(e, a, m, bcp, bcm, 0.0, it, A.max_iter, nbp, eval64, inv64);
                if (reason) status = COMBO_E_LAMINATE;
            }
            its = it + it_df;
        } else {
            reason = 1;
        }
        if (status) {
            raise_status(sc, status);
            if (atomicCAS(&sc->fail_boxel, 0, (int32_t)(b + 1)) == 0) {
                sc->fail_reason = reason;
#pragma unroll
                for (int c = 0; c < 9; c++) sc->fail_state[c] = Fb[c];
#pragma unroll
                for (int q = 0; q < 3; q++) {
                    sc->fail_state[9 + q] = N[q];
                    sc->fail_state[13 + q] = a[q];
                }
                sc->fail_state[12] = cp;
            }
        } else {
            if (A.dfloat) {  // S in (hi, lo) pairs: the double-float residual form
                float2* S2 = reinterpret_cast<float2*>(A.S);
                const df32 cpd(cp), cmd(cm);
#pragma unroll
                for (int c = 0; c < 9; c++) {
                    const df32 t = df_done ? cpd * ed.p.P[c] + cmd * ed.m.P[c] : df32(cp * e.p.P[c] + cm * e.m.P[c]);
                    S2[(int64_t)(9 * l + c) * A.V + v] = make_float2(t.hi, t.lo);
                }
            } else {
#pragma unroll
                for (int c = 0; c < 9; c++) A.S[(int64_t)(9 * l + c) * A.V + v] = cp * e.p.P[c] + cm * e.m.P[c];
            }
#pragma unroll
            for (int q = 0; q < 3; q++) A.ba[24 * b + 3 * l + q] = a[q];
            if (A.bAsub) {
                // the sub-cell's tangent for the doubly-fine Newton-CG, in
                // the Krylov precision, from the converged state
                double Di[9];
                float Df[9];
                bool ok;
                if (df_done && hessian_inv(ed, hf, Df)) {
                    ok = true;
#pragma unroll
                    for (int q = 0; q < 9; q++) Di[q] = Df[q];
                    if (A.sub_f32)
                        boxel_tangent_store<float>(ed.p, ed.m, N, cp, cm, mu, lam, Di, (float*)A.bAsub, 8 * A.nb, t);
                    else
                        boxel_tangent_store<double>(ed.p, ed.m, N, cp, cm, mu, lam, Di, (double*)A.bAsub, 8 * A.nb,
                                                    t);
                } else {
                    ok = (df_done ? eval64(e) : true) && inv64(e, Di);
                    if (ok) {
                        if (A.sub_f32)
                            boxel_tangent_store<float>(e.p, e.m, N, cp, cm, mu, lam, Di, (float*)A.bAsub, 8 * A.nb, t);
                        else
                            boxel_tangent_store<double>(e.p, e.m, N, cp, cm, mu, lam, Di, (double*)A.bAsub, 8 * A.nb,
                                                        t);
                    }
                }
                if (!ok) raise_status(sc, COMBO_E_LAMINATE);
            }
        }
    }
    if (threadIdx.x == 0) {
        const int64_t first = ((int64_t)blockIdx.x * blockDim.x) >> 3;
        const int64_t last = (min((int64_t)(blockIdx.x + 1) * blockDim.x, nt) - 1) >> 3;
        same_problem = (!A.bprob || A.bprob[first] == A.bprob[last]) ? 1 : 0;
    }
    __syncthreads();
    if (same_problem) {
        const double s1 = block_sum(its, red);
        const double s2 = block_sum(nbp, red + 32);
        __syncthreads();
        const double s3 = block_sum(nev, red);
        if (threadIdx.x == 0) {
            Scalars* s0 = A.sc + (A.bprob ? A.bprob[((int64_t)blockIdx.x * blockDim.x) >> 3] : 0);
            atomicAdd(&s0->nr_iters, (unsigned long long)s1);
            atomicAdd(&s0->n_backproj, (unsigned long long)s2);
            atomicAdd(&s0->n_lam, (unsigned long long)s3);
        }
    } else if (nev > 0.0) {
        atomicAdd(&sc->nr_iters, (unsigned long long)its);
        atomicAdd(&sc->n_backproj, (unsigned long long)nbp);
        atomicAdd(&sc->n_lam, (unsigned long long)nev);
    }
}

void launch_boxel_dfmg(const BoxelArgs<double>& a, cudaStream_t st)
{
    if (a.nb <= 0) return;
    const int grid = (int)((8 * a.nb + 127) / 128);
    if (a.dfloat)
        k_boxel_dfmg<true><<<grid, 128, 0, st>>>(a);
    else
        k_boxel_dfmg<false><<<grid, 128, 0, st>>>(a);
}

template void launch_boxel<double>(const BoxelArgs<double>&, cudaStream_t);
template void launch_boxel<float>(const BoxelArgs<float>&, cudaStream_t);

}  // namespace combo
