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
// The work is FP64 arithmetic (8 logarithms, divisions and ~70 FMAs per cell)
// and 2 x 576 B of S traffic per cell; on this part FP64 issues at a small
// fraction of the FP32 rate, so the pure-cell kernel is FP64-pipe bound.
#include <cuda_runtime.h>

#include "../../include/combo.h"
#include "combo_internal.cuh"

namespace combo {

static int dfmg_grid(int64_t n)
{
    const int64_t g = (n + 255) / 256;
    return (int)(g < 1 ? 1 : (g > 152 * 16 ? 152 * 16 : g));
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

void launch_dfmg_pure(const DfmgArgs& a, cudaStream_t st) { k_dfmg_pure<<<dfmg_grid(a.V), 256, 0, st>>>(a); }

void launch_dfmg_gather(const DfmgArgs& a, cudaStream_t st) { k_dfmg_gather<<<dfmg_grid(a.V), 256, 0, st>>>(a); }

void launch_dfmg_amean(const double* ba8, double* ba, int64_t nb, cudaStream_t st)
{
    if (nb <= 0) return;
    k_dfmg_amean<<<(int)((3 * nb + 255) / 256), 256, 0, st>>>(ba8, ba, nb);
}

}  // namespace combo
