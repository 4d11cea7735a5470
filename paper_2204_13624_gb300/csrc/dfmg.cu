// Doubly-fine material grid of the staggered scheme (App. A, Eq.
// constitutive_law).  Every cell c is cut into 8 sub-cells l in {0,1}^3; the
// sub-cell carries F_sub(c, l): the diagonal of F at c and the off-diagonal
// pairs from the staggered positions nearest the sub-cell (dfmg_fsub).  The
// law evaluates the material of c at every F_sub(c, l) once -- 8 evaluations
// per cell -- and gathers
//   P_aa[xi] = 1/8 sum_l S(xi, l)_aa,
//   P_ab[xi] = 1/8 sum_l S(xi - l_a e_a - l_b e_b, l)_ab   (a != b),
// S(c, l) the stress of sub-cell l of cell c.  This is the gradient of the
// sub-cell energy 1/8 sum_c sum_l W_c(F_sub(c, l)), so the discrete problem
// keeps the variational structure of the staggered scheme.
//
//   k_dfmg_pure    pure cells: 8 Neo-Hookean stresses per cell -> S [72][V]
//   (boxel.cu)     composite boxels: 8 laminates per boxel -> S
//   k_dfmg_gather  S -> P [9][V], the operand of the residual's x-pass
//
// The work is FP64 arithmetic (per sub-cell a logarithm, a division and ~70
// FMAs) and 2 x 576 B of S traffic per cell; on this part FP64 issues at a
// small fraction of the FP32 rate, so both kernels are FP64-pipe bound.  The
// double-float residual form (k_dfmg_pure_df, k_dfmg_gather_df) keeps only
// the conversions on the FP64 pipe and stores S as (hi, lo) float pairs of
// the same size.
#include <cuda_runtime.h>

#include "../../include/combo.h"
#include "combo_internal.cuh"

namespace combo {

static int dfmg_grid(int64_t n)
{
    const int64_t g = (n + 255) / 256;
    return (int)(g < 1 ? 1 : (g > 152 * 16 ? 152 * 16 : g));
}

// Neo-Hookean P of F_sub in double-float: cofactors, J, 1/J, ln J (df_log)
// and P in df32.  False if J <= 0.
__device__ __forceinline__ bool nh_P_df(const df32 F[9], double mu, double lam, df32 P[9])
{
    const df32 c0 = F[4] * F[8] - F[5] * F[7];
    const df32 c1 = F[5] * F[6] - F[3] * F[8];
    const df32 c2 = F[3] * F[7] - F[4] * F[6];
    const df32 J = F[0] * c0 + F[1] * c1 + F[2] * c2;
    if (!(J.hi > 0.f)) return false;
    const df32 iJ = df32(1.f, 0.f) / J;
    df32 G[9];
    G[0] = c0 * iJ;
    G[1] = (F[2] * F[7] - F[1] * F[8]) * iJ;
    G[2] = (F[1] * F[5] - F[2] * F[4]) * iJ;
    G[3] = c1 * iJ;
    G[4] = (F[0] * F[8] - F[2] * F[6]) * iJ;
    G[5] = (F[2] * F[3] - F[0] * F[5]) * iJ;
    G[6] = c2 * iJ;
    G[7] = (F[1] * F[6] - F[0] * F[7]) * iJ;
    G[8] = (F[0] * F[4] - F[1] * F[3]) * iJ;
    const df32 mud = df32(mu);
    const df32 k = df32(lam) * df_log(J) - mud;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) P[3 * i + j] = mud * F[3 * i + j] + k * G[3 * j + i];
    return true;
}

// Double-float form of k_dfmg_pure: the 27 distinct entries a cell's
// sub-cells draw from F (the diagonal, each off-diagonal pair at its four
// staggered positions) are converted once; S receives (hi, lo) pairs.
__global__ void __launch_bounds__(256) k_dfmg_pure_df(DfmgArgs a)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t V = a.V;
    float2* __restrict__ S = reinterpret_cast<float2*>(a.S);
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += stride) {
        const int ph = a.phase[v];
        if (ph == 2) continue;  // composite boxel: k_boxel_dfmg
        const int pb = (int)(v / a.Vp);
        Scalars* sc = a.sc + pb;
        if (a.guard == 2 && sc->outer_done) continue;
        const int64_t base = (int64_t)pb * a.Vp, lv = v - base;
        const int i = (int)(lv % a.n1), j = (int)((lv / a.n1) % a.n2), k = (int)(lv / ((int64_t)a.n1 * a.n2));
        const int ip = (i + 1 == a.n1) ? 0 : i + 1, jp = (j + 1 == a.n2) ? 0 : j + 1, kp = (k + 1 == a.n3) ? 0 : k + 1;
        const double mu = a.matp ? a.matp[4 * pb + ph] : a.mu[ph];
        const double lam = a.matp ? a.matp[4 * pb + 2 + ph] : a.lam[ph];
        auto at = [&](int c, int x, int y, int z) {
            return df32(a.F[(int64_t)c * V + base + x + (int64_t)a.n1 * (y + (int64_t)a.n2 * z)]);
        };
        const df32 d0 = at(0, i, j, k), d4 = at(4, i, j, k), d8 = at(8, i, j, k);
        df32 o12[4][2], o13[4][2], o23[4][2];  // [la + 2 lb][first, second component of the pair]
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int x1 = (q & 1) ? ip : i, y1 = (q & 2) ? jp : j;  // (l1, l2) for the 12 pair
            o12[q][0] = at(1, x1, y1, k);
            o12[q][1] = at(3, x1, y1, k);
            const int z1 = (q & 2) ? kp : k;  // (l1, l3) for the 13 pair
            o13[q][0] = at(2, x1, j, z1);
            o13[q][1] = at(6, x1, j, z1);
            const int y2 = (q & 1) ? jp : j;  // (l2, l3) for the 23 pair
            o23[q][0] = at(5, i, y2, z1);
            o23[q][1] = at(7, i, y2, z1);
        }
        bool ok = true;
#pragma unroll
        for (int l = 0; l < 8; l++) {
            const int l1 = l & 1, l2 = (l >> 1) & 1, l3 = (l >> 2) & 1;
            const int q12 = l1 + 2 * l2, q13 = l1 + 2 * l3, q23 = l2 + 2 * l3;
            df32 f[9], P[9];
            f[0] = d0;
            f[4] = d4;
            f[8] = d8;
            f[1] = o12[q12][0];
            f[3] = o12[q12][1];
            f[2] = o13[q13][0];
            f[6] = o13[q13][1];
            f[5] = o23[q23][0];
            f[7] = o23[q23][1];
            if (!nh_P_df(f, mu, lam, P)) {
                ok = false;
#pragma unroll
                for (int c = 0; c < 9; c++) P[c] = df32(0.f, 0.f);
            }
#pragma unroll
            for (int c = 0; c < 9; c++) S[(int64_t)(9 * l + c) * V + v] = make_float2(P[c].hi, P[c].lo);
        }
        if (!ok) raise_status(sc, COMBO_E_INADMISSIBLE);
    }
}

// Double-float form of k_dfmg_gather: sums of (hi, lo) pairs in df32, P in FP64.
__global__ void __launch_bounds__(256) k_dfmg_gather_df(DfmgArgs a)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t V = a.V;
    const float2* __restrict__ S = reinterpret_cast<const float2*>(a.S);
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += stride) {
        const int pb = (int)(v / a.Vp);
        if (a.guard == 2 && a.sc[pb].outer_done) continue;
        const int64_t base = (int64_t)pb * a.Vp, lv = v - base;
        const int i = (int)(lv % a.n1), j = (int)((lv / a.n1) % a.n2), k = (int)(lv / ((int64_t)a.n1 * a.n2));
        const int im = (i == 0) ? a.n1 - 1 : i - 1;
        const int jm = (j == 0) ? a.n2 - 1 : j - 1;
        const int km = (k == 0) ? a.n3 - 1 : k - 1;
        df32 o[9];
#pragma unroll
        for (int c = 0; c < 9; c++) o[c] = df32(0.f, 0.f);
        auto ld = [&](int64_t idx) {
            const float2 t = S[idx];
            return df32(t.x, t.y);
        };
#pragma unroll 2
        for (int l = 0; l < 8; l++) {
            const int ii = (l & 1) ? im : i, jj = (l & 2) ? jm : j, kk = (l & 4) ? km : k;
            const int64_t c12 = base + ii + (int64_t)a.n1 * (jj + (int64_t)a.n2 * k);
            const int64_t c13 = base + ii + (int64_t)a.n1 * (j + (int64_t)a.n2 * kk);
            const int64_t c23 = base + i + (int64_t)a.n1 * (jj + (int64_t)a.n2 * kk);
            const int64_t r0 = (int64_t)9 * l * V;
            o[0] += ld(r0 + 0 * V + v);
            o[4] += ld(r0 + 4 * V + v);
            o[8] += ld(r0 + 8 * V + v);
            o[1] += ld(r0 + 1 * V + c12);
            o[3] += ld(r0 + 3 * V + c12);
            o[2] += ld(r0 + 2 * V + c13);
            o[6] += ld(r0 + 6 * V + c13);
            o[5] += ld(r0 + 5 * V + c23);
            o[7] += ld(r0 + 7 * V + c23);
        }
#pragma unroll
        for (int c = 0; c < 9; c++) a.P[(int64_t)c * V + v] = 0.125 * (double)o[c];
    }
}

__global__ void __launch_bounds__(256) k_dfmg_pure(DfmgArgs a)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t V = a.V;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += stride) {
        const int ph = a.phase[v];
        if (ph == 2) continue;  // composite boxel: k_boxel_dfmg
        const int pb = (int)(v / a.Vp);
        Scalars* sc = a.sc + pb;
        if (a.guard == 2 && sc->outer_done) continue;
        const int64_t base = (int64_t)pb * a.Vp, lv = v - base;
        const int i = (int)(lv % a.n1), j = (int)((lv / a.n1) % a.n2), k = (int)(lv / ((int64_t)a.n1 * a.n2));
        const double mu = a.matp ? a.matp[4 * pb + ph] : a.mu[ph];
        const double lam = a.matp ? a.matp[4 * pb + 2 + ph] : a.lam[ph];
        bool ok = true;
#pragma unroll 1
        for (int l = 0; l < 8; l++) {
            double f[9], P[9];
            dfmg_fsub(a.F, V, base, a.n1, a.n2, a.n3, i, j, k, l, f);
            if (!nh_P64(f, mu, lam, P)) {
                ok = false;
#pragma unroll
                for (int c = 0; c < 9; c++) P[c] = 0.0;
            }
#pragma unroll
            for (int c = 0; c < 9; c++) a.S[(int64_t)(9 * l + c) * V + v] = P[c];
        }
        if (!ok) raise_status(sc, COMBO_E_INADMISSIBLE);
    }
}

__global__ void __launch_bounds__(256) k_dfmg_gather(DfmgArgs a)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t V = a.V;
    const double* __restrict__ S = a.S;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += stride) {
        const int pb = (int)(v / a.Vp);
        if (a.guard == 2 && a.sc[pb].outer_done) continue;
        const int64_t base = (int64_t)pb * a.Vp, lv = v - base;
        const int i = (int)(lv % a.n1), j = (int)((lv / a.n1) % a.n2), k = (int)(lv / ((int64_t)a.n1 * a.n2));
        const int im = (i == 0) ? a.n1 - 1 : i - 1;
        const int jm = (j == 0) ? a.n2 - 1 : j - 1;
        const int km = (k == 0) ? a.n3 - 1 : k - 1;
        double o[9];
#pragma unroll
        for (int c = 0; c < 9; c++) o[c] = 0.0;
#pragma unroll
        for (int l = 0; l < 8; l++) {
            const int ii = (l & 1) ? im : i, jj = (l & 2) ? jm : j, kk = (l & 4) ? km : k;
            const int64_t c12 = base + ii + (int64_t)a.n1 * (jj + (int64_t)a.n2 * k);
            const int64_t c13 = base + ii + (int64_t)a.n1 * (j + (int64_t)a.n2 * kk);
            const int64_t c23 = base + i + (int64_t)a.n1 * (jj + (int64_t)a.n2 * kk);
            const double* Sl = S + (int64_t)9 * l * V;
            o[0] += Sl[0 * V + v];
            o[4] += Sl[4 * V + v];
            o[8] += Sl[8 * V + v];
            o[1] += Sl[1 * V + c12];
            o[3] += Sl[3 * V + c12];
            o[2] += Sl[2 * V + c13];
            o[6] += Sl[6 * V + c13];
            o[5] += Sl[5 * V + c23];
            o[7] += Sl[7 * V + c23];
        }
#pragma unroll
        for (int c = 0; c < 9; c++) a.P[(int64_t)c * V + v] = 0.125 * o[c];
    }
}

__global__ void k_dfmg_amean(const double* __restrict__ ba8, double* __restrict__ ba, int64_t nb)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * nb) return;
    const int64_t b = t / 3;
    const int q = (int)(t - 3 * b);
    double s = 0.0;
    for (int l = 0; l < 8; l++) s += ba8[24 * b + 3 * l + q];
    ba[t] = 0.125 * s;
}

void launch_dfmg_pure(const DfmgArgs& a, cudaStream_t st)
{
    if (a.dfloat)
        k_dfmg_pure_df<<<dfmg_grid(a.V), 256, 0, st>>>(a);
    else
        k_dfmg_pure<<<dfmg_grid(a.V), 256, 0, st>>>(a);
}

void launch_dfmg_gather(const DfmgArgs& a, cudaStream_t st)
{
    if (a.dfloat)
        k_dfmg_gather_df<<<dfmg_grid(a.V), 256, 0, st>>>(a);
    else
        k_dfmg_gather<<<dfmg_grid(a.V), 256, 0, st>>>(a);
}

void launch_dfmg_amean(const double* ba8, double* ba, int64_t nb, cudaStream_t st)
{
    if (nb <= 0) return;
    k_dfmg_amean<<<(int)((3 * nb + 255) / 256), 256, 0, st>>>(ba8, ba, nb);
}

// ---------------------------------------------------------------- Newton-CG
// The tangent of the doubly-fine law is the Hessian of the sub-cell energy:
// applied to a direction p it is the gather of A_sub(c, l) : p_sub(c, l),
// p_sub assembled from p like F_sub from F and A_sub the tangent of the
// material of c at F_sub(c, l) (symmetric).  One CG iteration runs
//   k_dfmg_cg_update  x += alpha_prev p, p = r + beta p          (elementwise)
//   k_dfmg_tangent    S_t(c, l) = A_sub(c, l) : p_sub(c, l)     [72][V]
//   k_dfmg_tgather    y = gather of S_t, (p, y) -> alpha         [9][V]
// then the x-pass transform of y and the unchanged y-, z- and x-inverse
// passes.  A pure sub-cell's tangent is formed from F_sub on the fly in the
// Krylov precision (G = F_sub^{-1}, m = mu - lam ln J: cheaper than storing
// it); a composite boxel's sub-cells read the packed tangents the laminate
// kernel stored at the last residual evaluation.

// Neo-Hookean tangent data of F in precision S: G = F^{-1}, m = mu - lam ln J
template <typename S> __device__ __forceinline__ void nh_tan_data(const S f[9], S mu, S lam, S G[9], S& m)
{
    const S c0 = f[4] * f[8] - f[5] * f[7];
    const S c1 = f[5] * f[6] - f[3] * f[8];
    const S c2 = f[3] * f[7] - f[4] * f[6];
    const S J = f[0] * c0 + f[1] * c1 + f[2] * c2;
    const S iJ = (S)1 / J;
    G[0] = c0 * iJ;
    G[1] = (f[2] * f[7] - f[1] * f[8]) * iJ;
    G[2] = (f[1] * f[5] - f[2] * f[4]) * iJ;
    G[3] = c1 * iJ;
    G[4] = (f[0] * f[8] - f[2] * f[6]) * iJ;
    G[5] = (f[2] * f[3] - f[0] * f[5]) * iJ;
    G[6] = c2 * iJ;
    G[7] = (f[1] * f[6] - f[0] * f[7]) * iJ;
    G[8] = (f[0] * f[4] - f[1] * f[3]) * iJ;
    m = mu - lam * log(J);
}

template <typename Tc> __global__ void __launch_bounds__(256) k_dfmg_cg_update(DfmgTanArgs<Tc> a)
{
    Scalars* sc = a.sc;
    if (sc->cg_done) return;
    const bool first = sc->cg_iter == 0;
    const Tc beta = first ? (Tc)0 : (Tc)sc->beta;
    const Tc apend = first ? (Tc)0 : (Tc)sc->alpha_pending;
    const int64_t V = a.V;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < 9; c++) {
            const Tc rv = a.r[c * V + v];
            Tc pn = rv;
            if (!first) {
                const Tc po = a.p[c * V + v];
                if (apend != (Tc)0) a.x[c * V + v] += apend * po;
                pn = rv + beta * po;
            }
            a.p[c * V + v] = pn;
        }
    }
}

template <typename Tc> __global__ void __launch_bounds__(256) k_dfmg_tangent(DfmgTanArgs<Tc> a)
{
    if (a.sc->cg_done) return;
    const int64_t V = a.V;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(v % a.n1), j = (int)((v / a.n1) % a.n2), k = (int)(v / ((int64_t)a.n1 * a.n2));
        const int ph = a.phase[v];
        const int64_t b = (ph == 2) ? (int64_t)a.vox2box[v] : -1;
        const Tc mu = (Tc)a.mu[ph == 1 ? 1 : 0], lam = (Tc)a.lam[ph == 1 ? 1 : 0];
#pragma unroll 1
        for (int l = 0; l < 8; l++) {
            double fd[9];
            double pd[9];
            dfmg_fsub(a.F, V, 0, a.n1, a.n2, a.n3, i, j, k, l, fd);
            dfmg_fsub_t(a.p, V, a.n1, a.n2, a.n3, i, j, k, l, pd);
            Tc ps[9], y[9];
#pragma unroll
            for (int c = 0; c < 9; c++) ps[c] = (Tc)pd[c];
            if (b < 0) {
                Tc f[9], G[9], m;
#pragma unroll
                for (int c = 0; c < 9; c++) f[c] = (Tc)fd[c];
                nh_tan_data<Tc>(f, mu, lam, G, m);
                nh_tangent<Tc>(G, m, mu, lam, ps, y);
            } else {
                const int64_t col = 8 * b + l, stride = 8 * a.nb;
#pragma unroll
                for (int r = 0; r < 9; r++) {
                    Tc yr = 0;
#pragma unroll
                    for (int c = 0; c < 9; c++) yr += a.bAsub[(int64_t)sym_idx(r, c) * stride + col] * ps[c];
                    y[r] = yr;
                }
            }
#pragma unroll
            for (int r = 0; r < 9; r++) a.St[(int64_t)(9 * l + r) * V + v] = y[r];
        }
    }
}

template <typename Tc> __global__ void __launch_bounds__(256) k_dfmg_tgather(DfmgTanArgs<Tc> a)
{
    __shared__ double red[256];
    __shared__ int flag;
    Scalars* sc = a.sc;
    if (sc->cg_done) return;
    const int64_t V = a.V;
    double acc = 0.0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(v % a.n1), j = (int)((v / a.n1) % a.n2), k = (int)(v / ((int64_t)a.n1 * a.n2));
        Tc o[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int l = 0; l < 8; l++) {
            const int l1 = l & 1, l2 = (l >> 1) & 1, l3 = (l >> 2) & 1;
            const int im = l1 ? (i == 0 ? a.n1 - 1 : i - 1) : i;
            const int jm = l2 ? (j == 0 ? a.n2 - 1 : j - 1) : j;
            const int km = l3 ? (k == 0 ? a.n3 - 1 : k - 1) : k;
            const int64_t c12 = im + (int64_t)a.n1 * (jm + (int64_t)a.n2 * k);
            const int64_t c13 = im + (int64_t)a.n1 * (j + (int64_t)a.n2 * km);
            const int64_t c23 = i + (int64_t)a.n1 * (jm + (int64_t)a.n2 * km);
            const Tc* S = a.St + (int64_t)(9 * l) * V;
            o[0] += S[0 * V + v];
            o[4] += S[4 * V + v];
            o[8] += S[8 * V + v];
            o[1] += S[1 * V + c12];
            o[3] += S[3 * V + c12];
            o[2] += S[2 * V + c13];
            o[6] += S[6 * V + c13];
            o[5] += S[5 * V + c23];
            o[7] += S[7 * V + c23];
        }
        Tc s = 0;
#pragma unroll
        for (int c = 0; c < 9; c++) {
            const Tc yc = (Tc)0.125 * o[c];
            a.y[c * V + v] = yc;
            s += a.p[c * V + v] * yc;
        }
        acc += (double)s;
    }
    const double tot_b = block_sum(acc, red);
    if (threadIdx.x == 0) a.partial[blockIdx.x] = tot_b;
    if (last_block(&sc->ticket[0], &flag, gridDim.x)) {
        const double tot = sum_partials_fixed(a.partial, gridDim.x, red);
        if (threadIdx.x == 0) cg_alpha(sc, tot);
    }
}

int dfmg_cg_blocks(int64_t V) { return dfmg_grid(V); }

template <typename Tc> void launch_dfmg_cg(const DfmgTanArgs<Tc>& a, int stage, cudaStream_t st)
{
    const int grid = dfmg_grid(a.V);
    if (stage == 0)
        k_dfmg_cg_update<Tc><<<grid, 256, 0, st>>>(a);
    else if (stage == 1)
        k_dfmg_tangent<Tc><<<grid, 256, 0, st>>>(a);
    else
        k_dfmg_tgather<Tc><<<grid, 256, 0, st>>>(a);
}
template void launch_dfmg_cg<float>(const DfmgTanArgs<float>&, int, cudaStream_t);
template void launch_dfmg_cg<double>(const DfmgTanArgs<double>&, int, cudaStream_t);

}  // namespace combo
