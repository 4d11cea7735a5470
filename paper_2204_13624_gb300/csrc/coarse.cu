// coarse.cu -- coarse-graining of a binary fine image into composite boxels
// with the interface normal of Sec. 5: Laplacian interface weights (Sec. 5.1),
// the weighted least-squares plane through the interface voxels of each boxel
// (Sec. 5.2, the smallest eigenvector of the second moment M) and its sign
// from the barycentre normal (Eqs. normal:kabel, normal:flip).
//
// Exact integer moments.  For a binary image the three second differences of
// a fine voxel all carry the sign of -chi (or vanish), so the weight
// |S * chi| = sum_i r_i m_i, with m_i in {0, 1, 2} the number of its two
// neighbours along e_i that belong to the other phase.  With the offset of a
// fine voxel from its boxel's centre written x = q h / 2 (q = 2 i' + 1 - b an
// integer per axis),
//     sum w         = sum_i r_i T0_i,
//     sum w x_c     = h_c / 2       sum_i r_i T1_ic,
//     sum w x_c x_d = h_c h_d / 4   sum_i r_i T2_icd,
// where T are integer sums of m_i, m_i q_c and m_i q_c q_d over the boxel.
// The kernel gets them from XOR masks of neighbouring bit rows; M about the
// weighted barycentre is S2 - S1 S1^T / S0 in FP64 and its smallest
// eigenvector comes from cyclic Jacobi rotations.  The barycentre normal is
// -(h o Q) / |h o Q| with Q the integer sum of q over the inclusion voxels
// (the offsets of all voxels of a boxel sum to zero).
//
// Work layout.  One CTA per slab (J, K) of coarse voxels (all I along x): the
// b2 b3 fine rows of the slab are read once from HBM with 16-byte loads and
// packed to bit rows in shared memory (one bit per fine voxel).  Coarse
// voxels are counted with popcounts; only a slab that holds a composite boxel
// loads the one-voxel halo rows (periodic in y and z; x wraps inside a row)
// and accumulates the moments, a group of G lanes per boxel.  The boxels are
// written to a dense per-coarse-voxel scratch; a one-CTA scan of the per-slab
// counts and a scatter kernel compact them in increasing coarse index.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "combo.h"
#include "combo_internal.cuh"

namespace combo {
namespace {

constexpr int CG_THREADS = 256;
constexpr int SCAN_THREADS = 1024;
constexpr int SCATTER_THREADS = 256;
constexpr size_t CG_SMEM_MAX = 200 * 1024;

struct CgArgs {
    const uint8_t* chi;  // [n3][n2][n1]
    int n1, n2, n3;
    int b1, b2, b3;
    int nc1, nc2, nc3;
    int nw;      // words per shared-memory bit row: ceil(n1 / 32) + 1 (zero pad)
    int vec;     // 16-byte loads (n1 % 32 == 0 and chi 16-byte aligned)
    int G;       // lanes per composite boxel (power of two, <= 32)
    int method;  // COMBO_NORMAL_LAPLACE / COMBO_NORMAL_KABEL
    double h[3], r[3];
    uint8_t* phase;  // [nc]
    int* slab_cnt;   // [nc2 nc3] boxels per slab
    double* sN;      // [nc][3] dense scratch (boxels only)
    double* sc;      // [nc]
};

__device__ __forceinline__ int lrow(int jj, int kk, int b2) { return (kk + 1) * (b2 + 2) + (jj + 1); }

__device__ __forceinline__ int wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// bits [x, x + L) of a bit row, L in [0, 32]
__device__ __forceinline__ uint32_t ext(const uint32_t* row, int x, int L)
{
    if (L <= 0) return 0u;
    const int w = x >> 5, s = x & 31;
    const uint64_t v = (((uint64_t)row[w + 1] << 32) | row[w]) >> s;
    return (uint32_t)v & (L == 32 ? 0xFFFFFFFFu : ((1u << L) - 1u));
}

__device__ __forceinline__ uint32_t bit_at(const uint32_t* row, int x) { return (row[x >> 5] >> (x & 31)) & 1u; }

// sum of the positions of the set bits of m
__device__ __forceinline__ int pos_sum(uint32_t m)
{
    return __popc(m & 0xAAAAAAAAu) + (__popc(m & 0xCCCCCCCCu) << 1) + (__popc(m & 0xF0F0F0F0u) << 2) +
           (__popc(m & 0xFF00FF00u) << 3) + (__popc(m & 0xFFFF0000u) << 4);
}

// 16 fine voxels (bytes, nonzero = inclusion) -> 16 bits, voxel x0 + k at bit k
__device__ __forceinline__ uint32_t pack16(uint4 v)
{
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    uint32_t m = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        // byte flags at bits 0, 8, 16, 24; the product gathers them at bits 21..24
        const uint32_t f = __vcmpne4(w[k], 0u) & 0x01010101u;
        m |= ((f * 0x00204081u) >> 21 & 0xFu) << (4 * k);
    }
    return m;
}

// Map t in [0, nrows) to the slab-local row (jj, kk): the interior rows, or the
// halo rows (planes kk = -1 and kk = b3, then the y edges jj = -1, b2 of the
// interior planes).
template <bool HALO> __device__ __forceinline__ void row_of(int t, int b2, int& jj, int& kk)
{
    if (!HALO) {
        jj = t % b2;
        kk = t / b2;
        return;
    }
    const int pl = b2 + 2;
    if (t < pl) {
        kk = -1;
        jj = t - 1;
    } else if (t < 2 * pl) {
        kk = -2;  // placeholder, fixed by the caller (b3)
        jj = t - pl - 1;
    } else {
        const int u = t - 2 * pl;
        kk = u >> 1;
        jj = (u & 1) ? b2 : -1;
    }
}

template <bool HALO> __device__ void load_rows(const CgArgs& a, uint32_t* bits, int J, int K)
{
    const int nrows = HALO ? 2 * (a.b2 + 2) + 2 * a.b3 : a.b2 * a.b3;
    const int nwr = a.nw - 1;
    if (a.vec) {
        const int ipr = a.n1 >> 4;  // 16-byte items per row (even)
        const int total = nrows * ipr;
        constexpr int U = 4;
        for (int base = 0; base < total; base += U * CG_THREADS) {
            uint4 v[U];
            int lr[U], u[U];
#pragma unroll
            for (int k = 0; k < U; k++) {
                const int it = base + k * CG_THREADS + (int)threadIdx.x;
                v[k] = make_uint4(0u, 0u, 0u, 0u);
                lr[k] = -1;
                if (it < total) {
                    const int t = it / ipr;
                    u[k] = it - t * ipr;
                    int jj, kk;
                    row_of<HALO>(t, a.b2, jj, kk);
                    if (kk == -2) kk = a.b3;
                    const int y = wrap(J * a.b2 + jj, a.n2), z = wrap(K * a.b3 + kk, a.n3);
                    const uint4* src =
                        reinterpret_cast<const uint4*>(a.chi + ((size_t)z * a.n2 + y) * (size_t)a.n1) + u[k];
                    v[k] = __ldg(src);
                    lr[k] = lrow(jj, kk, a.b2);
                }
            }
#pragma unroll
            for (int k = 0; k < U; k++) {
                const uint32_t m = pack16(v[k]);
                const uint32_t o = __shfl_xor_sync(0xFFFFFFFFu, m, 1);
                // lanes 2m and 2m+1 hold the two halves of one 32-bit word
                if (lr[k] >= 0 && !(u[k] & 1)) bits[lr[k] * a.nw + (u[k] >> 1)] = m | (o << 16);
            }
        }
    } else {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const int total = nrows * nwr;
        for (int it = warp; it < total; it += CG_THREADS / 32) {
            const int t = it / nwr, wd = it - t * nwr;
            int jj, kk;
            row_of<HALO>(t, a.b2, jj, kk);
            if (kk == -2) kk = a.b3;
            const int y = wrap(J * a.b2 + jj, a.n2), z = wrap(K * a.b3 + kk, a.n3);
            const int x = 32 * wd + lane;
            const uint8_t c = x < a.n1 ? __ldg(a.chi + ((size_t)z * a.n2 + y) * (size_t)a.n1 + x) : (uint8_t)0;
            const uint32_t m = __ballot_sync(0xFFFFFFFFu, c != 0);
            if (lane == 0) bits[lrow(jj, kk, a.b2) * a.nw + wd] = m;
        }
    }
    for (int t = threadIdx.x; t < nrows; t += CG_THREADS) {
        int jj, kk;
        row_of<HALO>(t, a.b2, jj, kk);
        if (kk == -2) kk = a.b3;
        bits[lrow(jj, kk, a.b2) * a.nw + nwr] = 0u;
    }
}

// Smallest-eigenvalue eigenvector of the symmetric 3x3 matrix
// m = (xx, xy, xz, yy, yz, zz) by cyclic Jacobi rotations: each rotation in
// the (p, q) plane annihilates a_pq with tan(phi) the smaller root of
// t^2 + 2 theta t - 1 = 0, theta = (a_qq - a_pp) / (2 a_pq) (the stable form
// of the classical method, Golub & Van Loan, Matrix Computations, Sec. 8.5).
__device__ void sym3_min_eigvec(const double m[6], double v[3])
{
    double a[3][3] = {{m[0], m[1], m[2]}, {m[1], m[3], m[4]}, {m[2], m[4], m[5]}};
    double V[3][3] = {{1.0, 0.0, 0.0}, {0.0, 1.0, 0.0}, {0.0, 0.0, 1.0}};
    for (int sweep = 0; sweep < 32; sweep++) {
        bool rotated = false;
#pragma unroll
        for (int pq = 0; pq < 3; pq++) {
            const int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2, r = 3 - p - q;
            const double apq = a[p][q];
            if (fabs(apq) <= 0x1p-60 * (fabs(a[p][p]) + fabs(a[q][q])) || fabs(apq) < 1e-300) {
                a[p][q] = a[q][p] = 0.0;
                continue;
            }
            const double theta = (a[q][q] - a[p][p]) / (2.0 * apq);
            const double t = fabs(theta) > 1e150 ? 0.5 / theta
                                                 : (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
            a[p][p] -= t * apq;
            a[q][q] += t * apq;
            a[p][q] = a[q][p] = 0.0;
            const double arp = a[r][p], arq = a[r][q];
            a[r][p] = a[p][r] = c * arp - s * arq;
            a[r][q] = a[q][r] = s * arp + c * arq;
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const double vp = V[k][p], vq = V[k][q];
                V[k][p] = c * vp - s * vq;
                V[k][q] = s * vp + c * vq;
            }
            rotated = true;
        }
        if (!rotated) break;
    }
    // the column of the smallest diagonal entry (selected without a dynamic
    // index so the matrices stay in registers)
    const bool k1 = a[1][1] < a[0][0];
    const double d01 = k1 ? a[1][1] : a[0][0];
    const bool k2 = a[2][2] < d01;
#pragma unroll
    for (int i = 0; i < 3; i++) v[i] = k2 ? V[i][2] : (k1 ? V[i][1] : V[i][0]);
    const double nv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
#pragma unroll
    for (int i = 0; i < 3; i++) v[i] /= nv;
}

// acc: [0..2] Q (sum of q over the inclusion voxels), then per axis i the ten
// integer moments T0, T1x, T1y, T1z, T2xx, T2xy, T2xz, T2yy, T2yz, T2zz of m_i.
constexpr int NACC = 33;

__device__ __forceinline__ void boxel_result(const CgArgs& a, const int* acc, double* N)
{
    const bool has_nt = acc[0] != 0 || acc[1] != 0 || acc[2] != 0;
    double nt[3] = {0.0, 0.0, 0.0};
    if (has_nt) {
        const double d[3] = {-a.h[0] * acc[0], -a.h[1] * acc[1], -a.h[2] * acc[2]};
        const double nd = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
#pragma unroll
        for (int c = 0; c < 3; c++) nt[c] = d[c] / nd;
    }
    if (a.method == COMBO_NORMAL_KABEL && has_nt) {
        for (int c = 0; c < 3; c++) N[c] = nt[c];
        return;
    }
    double S0 = 0.0, S1[3] = {0.0, 0.0, 0.0}, S2[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const int* T = acc + 3 + 10 * i;
        const double ri = a.r[i];
        S0 += ri * T[0];
#pragma unroll
        for (int c = 0; c < 3; c++) S1[c] += ri * T[1 + c];
#pragma unroll
        for (int c = 0; c < 6; c++) S2[c] += ri * T[4 + c];
    }
    for (int c = 0; c < 3; c++) S1[c] *= 0.5 * a.h[c];
    const int ci[6] = {0, 0, 0, 1, 1, 2}, di[6] = {0, 1, 2, 1, 2, 2};
    double M[6];
#pragma unroll
    for (int c = 0; c < 6; c++) M[c] = S2[c] * (0.25 * a.h[ci[c]] * a.h[di[c]]) - S1[ci[c]] * S1[di[c]] / S0;
    sym3_min_eigvec(M, N);
    // Eq. normal:flip: keep N only where it agrees with the barycentre normal
    if (!(nt[0] * N[0] + nt[1] * N[1] + nt[2] * N[2] > 0.0))
        for (int c = 0; c < 3; c++) N[c] = -N[c];
}

__global__ void __launch_bounds__(CG_THREADS) k_cg_slab(CgArgs a)
{
    extern __shared__ __align__(16) uint32_t bits[];
    const int nrow_all = (a.b2 + 2) * (a.b3 + 2);
    int* cnt = reinterpret_cast<int*>(bits + (size_t)nrow_all * a.nw);
    int* mixed = cnt + a.nc1;
    __shared__ int nmixed;
    const int slab = blockIdx.x;
    const int J = slab % a.nc2, K = slab / a.nc2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NWARP = CG_THREADS / 32;
    if (threadIdx.x == 0) nmixed = 0;
    load_rows<false>(a, bits, J, K);
    __syncthreads();
    // inclusion voxels per coarse voxel
    const int rows = a.b2 * a.b3;
    for (int I = warp; I < a.nc1; I += NWARP) {
        int s = 0;
        for (int t = lane; t < rows; t += 32) {
            const uint32_t* row = bits + lrow(t % a.b2, t / a.b2, a.b2) * a.nw;
            for (int c0 = 0; c0 < a.b1; c0 += 32) s += __popc(ext(row, I * a.b1 + c0, min(32, a.b1 - c0)));
        }
        s = __reduce_add_sync(0xFFFFFFFFu, s);
        if (lane == 0) cnt[I] = s;
    }
    __syncthreads();
    const int nblock = a.b1 * a.b2 * a.b3;
    const size_t cbase = (size_t)slab * a.nc1;
    for (int I = threadIdx.x; I < a.nc1; I += CG_THREADS) {
        const int c = cnt[I];
        const uint8_t ph = c == 0 ? 0 : (c == nblock ? 1 : 2);
        a.phase[cbase + I] = ph;
        if (ph == 2) mixed[atomicAdd(&nmixed, 1)] = I;
    }
    __syncthreads();
    const int nm = nmixed;
    if (threadIdx.x == 0) a.slab_cnt[slab] = nm;
    if (nm == 0) return;
    load_rows<true>(a, bits, J, K);
    __syncthreads();

    const int G = a.G, gpw = 32 / G, g = lane / G, lg = lane & (G - 1);
    for (int mb = warp * gpw; mb < nm; mb += NWARP * gpw) {
        const int m = mb + g;
        const bool act = m < nm;
        const int I = act ? mixed[m] : 0;
        int acc[NACC];
#pragma unroll
        for (int k = 0; k < NACC; k++) acc[k] = 0;
        if (act) {
            for (int t = lg; t < rows; t += G) {
                const int jj = t % a.b2, kk = t / a.b2;
                const uint32_t* C = bits + lrow(jj, kk, a.b2) * a.nw;
                const uint32_t* YM = bits + lrow(jj - 1, kk, a.b2) * a.nw;
                const uint32_t* YP = bits + lrow(jj + 1, kk, a.b2) * a.nw;
                const uint32_t* ZM = bits + lrow(jj, kk - 1, a.b2) * a.nw;
                const uint32_t* ZP = bits + lrow(jj, kk + 1, a.b2) * a.nw;
                const int qy = 2 * jj + 1 - a.b2, qz = 2 * kk + 1 - a.b3;
                for (int c0 = 0; c0 < a.b1; c0 += 32) {
                    const int L = min(32, a.b1 - c0), x = I * a.b1 + c0;
                    const uint32_t W = ext(C, x, L);
                    const uint32_t Wm = x > 0 ? ext(C, x - 1, L) : ((ext(C, 0, L - 1) << 1) | bit_at(C, a.n1 - 1));
                    const uint32_t Wp =
                        x + L < a.n1 ? ext(C, x + 1, L) : (ext(C, x + 1, L - 1) | (bit_at(C, 0) << (L - 1)));
                    const uint32_t msk = L == 32 ? 0xFFFFFFFFu : ((1u << L) - 1u);
                    const int o = 2 * c0 + 1 - a.b1;  // q = 2 i + o for bit i
                    const int np = __popc(W);
                    acc[0] += 2 * pos_sum(W) + o * np;
                    acc[1] += qy * np;
                    acc[2] += qz * np;
                    const uint32_t e[6] = {(W ^ Wm) & msk, (W ^ Wp) & msk, W ^ ext(YM, x, L),
                                           W ^ ext(YP, x, L),  W ^ ext(ZM, x, L), W ^ ext(ZP, x, L)};
#pragma unroll
                    for (int i = 0; i < 3; i++) {
                        const int n = __popc(e[2 * i]) + __popc(e[2 * i + 1]);
                        if (n == 0) continue;
                        int s1 = 0, s2 = 0;
#pragma unroll
                        for (int h = 0; h < 2; h++) {
                            uint32_t mm = e[2 * i + h];
                            while (mm) {
                                const int q = 2 * (__ffs(mm) - 1) + o;
                                mm &= mm - 1u;
                                s1 += q;
                                s2 += q * q;
                            }
                        }
                        int* T = acc + 3 + 10 * i;
                        T[0] += n;
                        T[1] += s1;
                        T[2] += qy * n;
                        T[3] += qz * n;
                        T[4] += s2;
                        T[5] += qy * s1;
                        T[6] += qz * s1;
                        T[7] += qy * qy * n;
                        T[8] += qy * qz * n;
                        T[9] += qz * qz * n;
                    }
                }
            }
        }
        for (int off = G >> 1; off >= 1; off >>= 1)
#pragma unroll
            for (int k = 0; k < NACC; k++) acc[k] += __shfl_xor_sync(0xFFFFFFFFu, acc[k], off);
        if (act && lg == 0) {
            double N[3];
            boxel_result(a, acc, N);
            const size_t ci = cbase + I;
            a.sN[3 * ci + 0] = N[0];
            a.sN[3 * ci + 1] = N[1];
            a.sN[3 * ci + 2] = N[2];
            a.sc[ci] = (double)cnt[I] / (double)nblock;
        }
    }
}

// exclusive scan of the per-slab boxel counts (one CTA)
__global__ void __launch_bounds__(SCAN_THREADS) k_cg_scan(const int* cnt, int nslab, int64_t* off, int64_t* total)
{
    __shared__ int64_t wsum[SCAN_THREADS / 32];
    const int per = (nslab + SCAN_THREADS - 1) / SCAN_THREADS;
    const int s0 = threadIdx.x * per, s1 = min(nslab, s0 + per);
    int64_t mine = 0;
    for (int s = s0; s < s1; s++) mine += cnt[s];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t incl = mine;
    for (int d = 1; d < 32; d <<= 1) {
        const int64_t v = __shfl_up_sync(0xFFFFFFFFu, incl, d);
        if (lane >= d) incl += v;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int64_t w = wsum[lane];
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t v = __shfl_up_sync(0xFFFFFFFFu, w, d);
            if (lane >= d) w += v;
        }
        wsum[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    int64_t run = incl - mine + (warp > 0 ? wsum[warp - 1] : 0);
    for (int s = s0; s < s1; s++) {
        off[s] = run;
        run += cnt[s];
    }
    if (threadIdx.x == SCAN_THREADS - 1) *total = run;
}

// compact the boxels of one slab into the output lists (increasing index)
__global__ void __launch_bounds__(SCATTER_THREADS)
    k_cg_scatter(const uint8_t* phase, const int* cnt, const int64_t* off, const double* sN, const double* sc,
                 int nc1, int64_t cap, int64_t* idx_out, double* N_out, double* c_out)
{
    __shared__ int wtot[SCATTER_THREADS / 32];
    const int slab = blockIdx.x;
    if (cnt[slab] == 0) return;
    const size_t base = (size_t)slab * nc1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t run = off[slab];
    for (int I0 = 0; I0 < nc1; I0 += SCATTER_THREADS) {
        const int I = I0 + threadIdx.x;
        const bool f = I < nc1 && phase[base + I] == 2;
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, f);
        if (lane == 0) wtot[warp] = __popc(bal);
        __syncthreads();
        int before = 0, all = 0;
        for (int w = 0; w < SCATTER_THREADS / 32; w++) {
            before += w < warp ? wtot[w] : 0;
            all += wtot[w];
        }
        const int64_t pos = run + before + __popc(bal & ((1u << lane) - 1u));
        if (f && pos < cap) {
            const size_t ci = base + I;
            idx_out[pos] = (int64_t)ci;
            N_out[3 * pos + 0] = sN[3 * ci + 0];
            N_out[3 * pos + 1] = sN[3 * ci + 1];
            N_out[3 * pos + 2] = sN[3 * ci + 2];
            c_out[pos] = sc[ci];
        }
        run += all;
        __syncthreads();
    }
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace
}  // namespace combo

using namespace combo;

#define CGK(call)                                                                                            \
    do {                                                                                                     \
        cudaError_t e_ = (call);                                                                             \
        if (e_ != cudaSuccess) return set_error(COMBO_E_CUDA, (std::string(#call ": ") + cudaGetErrorString(e_)).c_str()); \
    } while (0)

extern "C" int combo_coarse_grain(combo_ctx* ctx, const int32_t n[3], const int32_t b[3], const double h[3],
                                  int32_t method, const uint8_t* chi, uint8_t* phase_out, int64_t cap,
                                  int64_t* idx_out, double* N_out, double* c_out, int64_t* n_boxels, int32_t mem)
{
    if (!ctx || !n || !b || !h || !chi || !phase_out || !n_boxels)
        return set_error(COMBO_E_INVALID_ARG, "combo_coarse_grain: null argument");
    if (cap < 0 || (cap > 0 && (!idx_out || !N_out || !c_out)))
        return set_error(COMBO_E_INVALID_ARG, "combo_coarse_grain: cap > 0 needs the boxel output arrays");
    if (method != COMBO_NORMAL_LAPLACE && method != COMBO_NORMAL_KABEL)
        return set_error(COMBO_E_INVALID_ARG, "combo_coarse_grain: unknown normal method");
    if (mem != COMBO_MEM_HOST && mem != COMBO_MEM_DEVICE)
        return set_error(COMBO_E_INVALID_ARG, "combo_coarse_grain: bad mem");
    for (int j = 0; j < 3; j++) {
        if (n[j] < 1 || b[j] < 1 || n[j] % b[j] != 0)
            return set_error(COMBO_E_INVALID_ARG, "combo_coarse_grain: b_j must divide n_j (both >= 1)");
        if (!(h[j] > 0.0) || !std::isfinite(h[j]))
            return set_error(COMBO_E_INVALID_ARG, "combo_coarse_grain: h_j must be finite and > 0");
    }
    const int64_t nblock = (int64_t)b[0] * b[1] * b[2];
    const int64_t bmax = std::max(b[0], std::max(b[1], b[2]));
    if (2 * nblock * bmax * bmax >= ((int64_t)1 << 31))
        return set_error(COMBO_E_INVALID_ARG, "combo_coarse_grain: boxel too large for the integer moments");
    CgArgs a{};
    a.n1 = n[0];
    a.n2 = n[1];
    a.n3 = n[2];
    a.b1 = b[0];
    a.b2 = b[1];
    a.b3 = b[2];
    a.nc1 = n[0] / b[0];
    a.nc2 = n[1] / b[1];
    a.nc3 = n[2] / b[2];
    a.nw = (a.n1 + 31) / 32 + 1;
    a.method = method;
    for (int j = 0; j < 3; j++) a.h[j] = h[j];
    a.r[0] = h[1] * h[2] / h[0];  // r_i = h_j h_k / h_i
    a.r[1] = h[0] * h[2] / h[1];
    a.r[2] = h[0] * h[1] / h[2];
    const int rows = a.b2 * a.b3;
    int G = 1;
    while (G < 32 && 4 * G < rows) G <<= 1;  // about four rows per lane
    a.G = G;
    const size_t smem = (size_t)(a.b2 + 2) * (a.b3 + 2) * a.nw * 4 + (size_t)8 * a.nc1;
    if (smem > CG_SMEM_MAX)
        return set_error(COMBO_E_INVALID_ARG, "combo_coarse_grain: slab rows exceed the shared-memory limit");
    const size_t V = (size_t)n[0] * n[1] * n[2];
    const size_t nc = (size_t)a.nc1 * a.nc2 * a.nc3;
    const int nslab = a.nc2 * a.nc3;
    const bool dev = mem == COMBO_MEM_DEVICE;
    CGK(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;

    // scratch: [chi copy] [phase] slab_cnt slab_off total sN sc [idx N c]
    size_t o_chi = 0, sz = 0;
    if (!dev) sz += align256(V);
    const size_t o_phase = sz;
    if (!dev) sz += align256(nc);
    const size_t o_cnt = sz;
    sz += align256(4 * (size_t)nslab);
    const size_t o_off = sz;
    sz += align256(8 * (size_t)nslab);
    const size_t o_tot = sz;
    sz += 256;
    const size_t o_sN = sz;
    sz += align256(24 * nc);
    const size_t o_sc = sz;
    sz += align256(8 * nc);
    const int64_t ncap = std::min<int64_t>(cap, (int64_t)nc);
    const size_t o_out = sz;
    if (!dev) sz += align256(40 * (size_t)std::max<int64_t>(ncap, 1));
    if (ctx->scratch_bytes < sz) {
        CGK(cudaStreamSynchronize(st));
        if (ctx->scratch) cudaFree(ctx->scratch);
        ctx->scratch = nullptr;
        ctx->scratch_bytes = 0;
        if (cudaMalloc(&ctx->scratch, sz) != cudaSuccess) {
            cudaGetLastError();
            ctx->scratch = nullptr;
            return set_error(COMBO_E_OOM, "combo_coarse_grain: scratch allocation failed");
        }
        ctx->scratch_bytes = sz;
    }
    char* S = static_cast<char*>(ctx->scratch);
    if (!dev) {
        CGK(cudaMemcpyAsync(S + o_chi, chi, V, cudaMemcpyHostToDevice, st));
        a.chi = reinterpret_cast<const uint8_t*>(S + o_chi);
        a.phase = reinterpret_cast<uint8_t*>(S + o_phase);
    } else {
        a.chi = chi;
        a.phase = phase_out;
    }
    a.vec = (a.n1 % 32 == 0) && ((reinterpret_cast<uintptr_t>(a.chi) & 15) == 0);
    a.slab_cnt = reinterpret_cast<int*>(S + o_cnt);
    int64_t* d_off = reinterpret_cast<int64_t*>(S + o_off);
    int64_t* d_tot = reinterpret_cast<int64_t*>(S + o_tot);
    a.sN = reinterpret_cast<double*>(S + o_sN);
    a.sc = reinterpret_cast<double*>(S + o_sc);
    int64_t* oi = idx_out;
    double* oN = N_out;
    double* oc = c_out;
    if (!dev) {
        oi = reinterpret_cast<int64_t*>(S + o_out);
        oN = reinterpret_cast<double*>(S + o_out + 8 * (size_t)std::max<int64_t>(ncap, 1));
        oc = reinterpret_cast<double*>(S + o_out + 32 * (size_t)std::max<int64_t>(ncap, 1));
    }
    CGK(cudaFuncSetAttribute(k_cg_slab, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CG_SMEM_MAX));
    k_cg_slab<<<nslab, CG_THREADS, smem, st>>>(a);
    CGK(cudaGetLastError());
    k_cg_scan<<<1, SCAN_THREADS, 0, st>>>(a.slab_cnt, nslab, d_off, d_tot);
    CGK(cudaGetLastError());
    k_cg_scatter<<<nslab, SCATTER_THREADS, 0, st>>>(a.phase, a.slab_cnt, d_off, a.sN, a.sc, a.nc1, ncap, oi, oN,
                                                    oc);
    CGK(cudaGetLastError());
    int64_t total = 0;
    CGK(cudaMemcpyAsync(&total, d_tot, 8, cudaMemcpyDeviceToHost, st));
    CGK(cudaStreamSynchronize(st));
    *n_boxels = total;
    if (!dev) {
        const int64_t k = std::min<int64_t>(total, ncap);
        CGK(cudaMemcpyAsync(phase_out, a.phase, nc, cudaMemcpyDeviceToHost, st));
        if (k > 0) {
            CGK(cudaMemcpyAsync(idx_out, oi, 8 * k, cudaMemcpyDeviceToHost, st));
            CGK(cudaMemcpyAsync(N_out, oN, 24 * k, cudaMemcpyDeviceToHost, st));
            CGK(cudaMemcpyAsync(c_out, oc, 8 * k, cudaMemcpyDeviceToHost, st));
        }
        CGK(cudaStreamSynchronize(st));
    }
    return COMBO_OK;
}
