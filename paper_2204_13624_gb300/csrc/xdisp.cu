// xdisp.cu -- the x side of the displacement form of the rotated Green
// operator in the FP32 CG.
//
// The rotated symbol k_J = i P kr_J (P = e^{i (theta_1 + theta_2 + theta_3) / 2},
// kr_J = (2 / h_J) sin(theta_J / 2) prod_{m != J} cos(theta_m / 2), the cosine
// zero at a Nyquist index) is the Fourier symbol of the HEX8R gradient: the
// difference of a nodal field along the edges of a voxel parallel to axis J,
// averaged over the voxel's 4 such edges (Sec. 3, the rotated scheme).  So
// G X = k (k^H X) / |k|^2 is, row by row, that gradient of the nodal field
// u_i = IFFT(k^H X_i / |k|^2).  The z-pass leaves the three spectra of u_i,
// the y-inverse transforms only those, and here
//   * k_xinv_disp turns each x-line of them into real u_i (packed half-length
//     inverse, as the CG x-inverse), three line transforms per output line
//     instead of nine;
//   * k_disp_grad_cg forms F_iJ from the 8 corners of every voxel and applies
//     the CG update r -= alpha F with the fused (r, r) reduction and, in the
//     problem's last block, beta and the stopping test.
#include <algorithm>

#include "async_copy.cuh"
#include "combo_internal.cuh"
#include "fft_fast.cuh"
#include "../../include/combo.h"

namespace combo {

namespace {

int num_sms_disp()
{
    static int nsm = 0;
    if (nsm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) nsm = 152;
    }
    return nsm;
}

// lines per group of the x-inverse: three components x LB lines, about 12 KB
// of spectrum per stage
template <int M> __host__ __device__ constexpr int disp_lb() { return M == 64 ? 8 : (M == 128 ? 8 : 4); }
template <int M> __host__ __device__ constexpr int xdisp_threads() { return (3 * disp_lb<M>() * FastPlan<M>::TPL + 31) / 32 * 32; }

}  // namespace

// y rows of one work item of the gradient pass (a sliding window along y)
constexpr int kDispSY = 4;

bool disp_x_ok(const GridDims& g)
{
    const int M = g.M;
    if (!(M == 64 || M == 128 || M == 256) || 2 * M != g.n1 || g.n2 % kDispSY != 0) return false;
    const int lb = (M == 256) ? disp_lb<256>() : disp_lb<128>();
    return (g.n2 * g.n3p) % lb == 0;
}

// ------------------------------------------------------------- x-inverse to u
// Stage layout: spectrum rows [3][LB][lsx] (components 0, 3, 6 of the
// spectrum); each line is transformed in place in its stage row (the first
// stage's loads finish before its stores), and the last stage writes the
// real pairs 2e, 2e + 1 of u_c straight to global memory.
template <int M>
__global__ void __launch_bounds__(xdisp_threads<M>()) k_xinv_disp(DispArgs a)
{
    int pb, pj, gp;  // problem of this block, index among its gp blocks
    prob_block(a.g, blockIdx.x, gridDim.x, pb, pj, gp);
    const Scalars* scp = a.sc + pb;
    if (scp->cg_done) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int LB = disp_lb<M>();
    constexpr int n1 = 2 * M;
    constexpr int lsx = (M + 2) / 2 * 2;  // M + 1 rounded up to even: 16-byte rows
    constexpr int TPL = FastPlan<M>::TPL;
    constexpr int NL = 3 * LB;
    constexpr size_t SB = (size_t)NL * lsx * 8;
    const GridDims g = a.g;
    float2* stage[2] = {reinterpret_cast<float2*>(smem_raw), reinterpret_cast<float2*>(smem_raw + SB)};
    float2* w2 = reinterpret_cast<float2*>(smem_raw + 2 * SB);  // exp(-2 pi i k / n1), k < M
    float2* tws = w2 + M;                                       // exp(-2 pi i t / M)
    uint64_t* bar = reinterpret_cast<uint64_t*>(tws + M);

    const int nlp = g.n2 * g.n3p;  // x-lines of one problem
    const int ngroups = nlp / LB;  // disp_x_ok guarantees nlp % LB == 0
    const int gbase = pb * ngroups;
    constexpr uint32_t tx_bytes = (uint32_t)SB;

    auto issue = [&](int grp, int s) {
        mbar_arrive_expect_tx(&bar[s], tx_bytes);
        for (int l = 0; l < LB; l++) {
            const int64_t L = (int64_t)grp * LB + l;
            for (int c = 0; c < 3; c++)
                bulk_g2s(stage[s] + ((size_t)c * LB + l) * lsx, a.spec + 3 * c * g.Vs + L * g.nhp, lsx * 8, &bar[s]);
        }
    };

    for (int k = threadIdx.x; k < M; k += blockDim.x) {
        w2[k] = a.tw2[k];
        tws[k] = a.tw[k];
    }
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_proxy_async();
    }
    __syncthreads();
    if (threadIdx.x == 0 && pj < ngroups) issue(gbase + pj, 0);

    const int q = threadIdx.x / TPL, tau = threadIdx.x - (threadIdx.x / TPL) * TPL;
    const bool act = q < NL;
    const int c = act ? q / LB : 0, l = act ? q - (q / LB) * LB : 0;
    int it = 0;
    bool timed_out = false;
    for (int lgrp = pj; lgrp < ngroups; lgrp += gp, it++) {
        const int grp = gbase + lgrp;
        const int s = it & 1;
        if (threadIdx.x == 0 && lgrp + gp < ngroups) issue(grp + gp, s ^ 1);
        const bool ok = mbar_wait_bounded(&bar[s], (uint32_t)((it >> 1) & 1), wait_cap_of(a.wait_cap));
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            break;
        }
        float2* X = stage[s] + (size_t)(act ? q : 0) * lsx;
        float* ug = a.u + (int64_t)c * a.ustride + ((int64_t)grp * LB + l) * n1;
        // Z[k] = Ze + i Zo,  Ze = (X[k] + conj X[M-k]) / 2,  Zo = (X[k] - conj X[M-k]) W^{-k} / 2
        auto lg = [&](int k) -> float2 {
            if (!act) return float2{0.f, 0.f};
            const float2 A = X[k];
            const float2 Bc = c_conj(X[M - k]);
            const float2 Ze = c_scale(c_add(A, Bc), 0.5f);
            const float2 Zo = c_mul(c_scale(c_sub(A, Bc), 0.5f), c_conj(w2[k]));
            return float2{Ze.x - Zo.y, Ze.y + Zo.x};
        };
        auto lx = [&](int e) -> float2 { return act ? X[e] : float2{0.f, 0.f}; };
        auto sx = [&](int e, float2 v) {
            if (act) X[e] = v;
        };
        // output e of the packed inverse holds the reals 2e, 2e + 1
        auto sg = [&](int e, float2 v) {
            if (act) *reinterpret_cast<float2*>(ug + 2 * e) = v;
        };
        fft_fast<float, M, true, true, false>(lg, sg, lx, sx, tau, tws);
        fence_proxy_async();  // this thread's stage writes, before a bulk copy refills the stage
        __syncthreads();      // stage s is refilled two groups on
    }
    if (timed_out && threadIdx.x == 0) {
        raise_status(const_cast<Scalars*>(scp), COMBO_E_TIMEOUT);
        // copies possibly in flight: the group waited on and, if it was
        // issued, the prefetch of the next one
        const int s = it & 1;
        mbar_wait_bounded(&bar[s], (uint32_t)((it >> 1) & 1));
        if (pj + (it + 1) * gp < ngroups) mbar_wait_bounded(&bar[s ^ 1], (uint32_t)(((it + 1) >> 1) & 1));
    }
}

// ------------------------------------------------------------- gradient + CG update
// Block of 256 threads = 256 / M line groups of M threads; thread tx of a
// group owns the voxels x0 = 2 tx and x0 + 1 of its line and holds, per
// field, the nodal values at x0, x0 + 1 and x0 + 2 (the third from the next
// lane, or from memory on the warp's last lane; x wraps).  A work item is
// kDispSY consecutive y rows at one z: the rows (y, z) and (y, z + 1) slide
// along y, so each step loads the two rows at y + 1 (y, z wrap within the
// problem).  For the voxel at x with corners c_abc = u(x + a, y + b, z + c):
//   F_i0 = c_0 (sum of c_1bc - sum of c_0bc)   (the 4 edges along x)
//   F_i1 = c_1 (sum of c_a1c - sum of c_a0c)
//   F_i2 = c_2 (sum of c_ab1 - sum of c_ab0)
template <int M>
__global__ void __launch_bounds__(256, 2) k_disp_grad_cg(DispArgs a)
{
    int pb, pj, gp;
    prob_block(a.g, blockIdx.x, gridDim.x, pb, pj, gp);
    Scalars* scp = a.sc + pb;
    if (scp->cg_done) return;
    __shared__ double red[256];  // block_sum and sum_partials_fixed (one per thread)
    __shared__ int flag[4];
    constexpr int n1 = 2 * M, LPB = 256 / M;
    static_assert(M % 32 == 0, "a warp lies within one line group");
    const GridDims g = a.g;
    const int lgi = threadIdx.x / M, tx = threadIdx.x - lgi * M;
    const int x0 = 2 * tx;
    const bool last_lane = (threadIdx.x & 31) == 31;
    const int nseg = g.n2 / kDispSY;
    const int items = g.n3p * nseg;
    const float alpha = (float)scp->alpha;
    const float cx0 = a.cJ[0], cx1 = a.cJ[1], cx2 = a.cJ[2];
    const float* __restrict__ u = a.u;
    float* __restrict__ r = a.r;
    const int64_t V = g.V, us = a.ustride;

    // nodal values at x0, x0 + 1, x0 + 2 of one row
    auto row3 = [&](const float* row, float (&v)[3]) {
        const float2 p = __ldg(reinterpret_cast<const float2*>(row + x0));
        float nx = __shfl_down_sync(0xffffffffu, p.x, 1);
        if (last_lane) nx = __ldg(row + ((x0 + 2) & (n1 - 1)));
        v[0] = p.x;
        v[1] = p.y;
        v[2] = nx;
    };

    double acc = 0.0;
    for (int item = pj * LPB + lgi; item < items; item += gp * LPB) {
        const int zl = item / nseg, y0 = (item - zl * nseg) * kDispSY;
        const int64_t zo = (int64_t)(pb * g.n3p + zl) * g.n2;                       // row offset of z
        const int64_t z1 = (int64_t)(pb * g.n3p + (zl + 1 == g.n3p ? 0 : zl + 1)) * g.n2;  // and of z + 1
        float A[3][3], B[3][3];  // rows (y, z), (y, z + 1) of the three fields
#pragma unroll
        for (int i = 0; i < 3; i++) {
            row3(u + i * us + (zo + y0) * n1, A[i]);
            row3(u + i * us + (z1 + y0) * n1, B[i]);
        }
        float accp = 0.f;
        for (int yy = 0; yy < kDispSY; yy++) {
            const int y = y0 + yy, yn = (y + 1 == g.n2) ? 0 : y + 1;
            const int64_t o = (zo + y) * n1 + x0;  // this thread's voxels in a component of r
            float2 rv[9];
#pragma unroll
            for (int c = 0; c < 9; c++) rv[c] = *reinterpret_cast<const float2*>(r + c * V + o);
            float C[3][3], D[3][3];  // rows (y + 1, z), (y + 1, z + 1)
#pragma unroll
            for (int i = 0; i < 3; i++) {
                row3(u + i * us + (zo + yn) * n1, C[i]);
                row3(u + i * us + (z1 + yn) * n1, D[i]);
            }
#pragma unroll
            for (int i = 0; i < 3; i++) {
                float s0[3], s1[3], t0[3], t1[3];
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    s0[k] = A[i][k] + B[i][k];  // y side: (y, z) + (y, z + 1)
                    s1[k] = C[i][k] + D[i][k];  //         (y + 1, z) + (y + 1, z + 1)
                    t0[k] = A[i][k] + C[i][k];  // z side: (y, z) + (y + 1, z)
                    t1[k] = B[i][k] + D[i][k];  //         (y, z + 1) + (y + 1, z + 1)
                }
                float F[3][2];
#pragma unroll
                for (int p = 0; p < 2; p++) {
                    F[0][p] = cx0 * ((s0[p + 1] + s1[p + 1]) - (s0[p] + s1[p]));
                    F[1][p] = cx1 * ((s1[p] + s1[p + 1]) - (s0[p] + s0[p + 1]));
                    F[2][p] = cx2 * ((t1[p] + t1[p + 1]) - (t0[p] + t0[p + 1]));
                }
#pragma unroll
                for (int J = 0; J < 3; J++) {
                    float2& q = rv[3 * i + J];
                    q.x -= alpha * F[J][0];
                    q.y -= alpha * F[J][1];
                    accp += q.x * q.x + q.y * q.y;
                }
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    A[i][k] = C[i][k];
                    B[i][k] = D[i][k];
                }
            }
#pragma unroll
            for (int c = 0; c < 9; c++) *reinterpret_cast<float2*>(r + c * V + o) = rv[c];
        }
        acc += (double)accp;
    }
    if (a.partial) {
        const double sacc = block_sum(acc, red);
        if (threadIdx.x == 0) a.partial[blockIdx.x] = sacc;
        if (a.fuse && last_block(&scp->ticket[1], flag, gp)) {
            const double tot = sum_partials_fixed(a.partial + (size_t)pb * gp, gp, red);
            if (threadIdx.x == 0) cg_beta(scp, tot, a.cg_tol, a.cg_max, a.cg_fixed);
        }
    }
}

// ------------------------------------------------------------- fused x-inverse + gradient
// The two kernels above in one pass, without the round trip of the nodal
// fields through global memory.  A block takes an even share of the problem's
// (column, plane) pairs in column-major order, a column being TY voxel lines
// y0 .. y0 + TY - 1: runs of planes, each marched along z.  For each node
// plane it turns the TY + 1 node lines y0 .. y0 + TY of the three fields into
// real lines (packed half-length inverse in place in the stage, output into
// a ring of two node planes in shared memory), then forms the gradient of the
// voxel plane between that node plane and the previous one with the CG
// update.  The spectrum rows of the next node plane are copied into the stage
// (bulk copies, mbarrier, bounded wait) while the gradient is formed.  The
// node line y0 + TY and the node plane after a run's last are formed twice
// (by this run and by the neighbour's).
template <int M> __host__ __device__ constexpr int fused_ty() { return M == 256 ? 4 : 8; }
template <int M, int TY> __host__ __device__ constexpr size_t fused_smem()
{
    // stage [3 (TY + 1)][lsx] complex; node planes [2][3][TY + 1][n1] floats;
    // w2 [M], twiddles [M]; reduction [256] doubles; flag; barrier
    return (size_t)3 * (TY + 1) * ((M + 2) / 2 * 2) * 8 + (size_t)2 * 3 * (TY + 1) * 2 * M * 4 + (size_t)2 * M * 8 +
           256 * 8 + 16 + 16;
}

template <int M, int TY>
__global__ void __launch_bounds__(256, 2) k_xinv_grad(DispArgs a)
{
    int pb, pj, gp;
    prob_block(a.g, blockIdx.x, gridDim.x, pb, pj, gp);
    Scalars* scp = a.sc + pb;
    if (scp->cg_done) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int n1 = 2 * M;
    constexpr int lsx = (M + 2) / 2 * 2;
    constexpr int TPL = FastPlan<M>::TPL;
    constexpr int NL = 3 * (TY + 1);  // node lines per node plane
    constexpr int NBAR = (NL * TPL + 31) / 32 * 32;
    constexpr int LPB = 256 / M;      // voxel lines of the gradient at a time
    static_assert(NBAR <= 256 && M % 32 == 0, "block shape");
    constexpr size_t SB = (size_t)NL * lsx * 8;
    const GridDims g = a.g;
    float2* stage = reinterpret_cast<float2*>(smem_raw);
    float* up = reinterpret_cast<float*>(smem_raw + SB);  // [2][3][TY + 1][n1]
    float2* w2 = reinterpret_cast<float2*>(up + 2 * NL * n1);
    float2* tws = w2 + M;
    double* red = reinterpret_cast<double*>(tws + M);
    int* flag = reinterpret_cast<int*>(red + 256);
    uint64_t* bar = reinterpret_cast<uint64_t*>(flag + 4);
    const int tid = threadIdx.x;
    for (int k = tid; k < M; k += blockDim.x) {
        w2[k] = a.tw2[k];
        tws[k] = a.tw[k];
    }
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        fence_proxy_async();
    }
    __syncthreads();

    const int ncol = g.n2 / TY;
    const int64_t total = (int64_t)ncol * g.n3p;
    const int64_t lin_b = total * pj / gp, lin_e = total * (pj + 1) / gp;
    const float alpha = (float)scp->alpha;
    const float cx0 = a.cJ[0], cx1 = a.cJ[1], cx2 = a.cJ[2];
    float* __restrict__ r = a.r;
    const int64_t V = g.V;
    // spectrum rows of node plane zn (local index, wraps) of the column at y0
    auto issue = [&](int y0, int zn) {
        const int zl = zn >= g.n3p ? zn - g.n3p : zn;
        mbar_arrive_expect_tx(&bar[0], (uint32_t)SB);
        for (int c = 0; c < 3; c++)
            for (int ly = 0; ly <= TY; ly++) {
                const int y = (y0 + ly >= g.n2) ? y0 + ly - g.n2 : y0 + ly;
                const int64_t L = (int64_t)(pb * g.n3p + zl) * g.n2 + y;
                bulk_g2s(stage + (size_t)(c * (TY + 1) + ly) * lsx, a.spec + 3 * c * g.Vs + L * g.nhp, lsx * 8,
                         &bar[0]);
            }
    };
    // FFT roles: line q of the node plane, tau of its TPL threads
    const int q = tid / TPL, tau = tid - (tid / TPL) * TPL;
    const bool act = q < NL;
    // gradient roles: x pair tx of voxel lines lg, lg + LPB, ...
    const int lg = tid / M, tx = tid - (tid / M) * M, x0 = 2 * tx;
    const int x2 = (x0 + 2) & (n1 - 1);

    double acc = 0.0;
    uint32_t phase = 0;
    bool timed_out = false;
    for (int64_t lin = lin_b; lin < lin_e && !timed_out;) {
        const int col = (int)(lin / g.n3p), z0 = (int)(lin - (int64_t)col * g.n3p);
        const int z1 = (int)min((int64_t)g.n3p, z0 + (lin_e - lin));
        lin += z1 - z0;
        const int y0 = col * TY;
        float accp = 0.f;
        if (tid == 0) issue(y0, z0);
        for (int zn = z0; zn <= z1; zn++) {
            const int sl = (zn - z0) & 1;  // ring slot of this node plane
            const bool ok = mbar_wait_bounded(&bar[0], phase, wait_cap_of(a.wait_cap));
            phase ^= 1u;
            if (__syncthreads_or(!ok)) {
                timed_out = true;
                break;
            }
            // node plane zn: packed inverse in place in the stage, real pairs
            // into the ring
            if (tid < NBAR) {
                float2* X = stage + (size_t)(act ? q : 0) * lsx;
                float* ug = up + ((size_t)sl * NL + (act ? q : 0)) * n1;
                auto lgz = [&](int k) -> float2 {
                    if (!act) return float2{0.f, 0.f};
                    const float2 A = X[k];
                    const float2 Bc = c_conj(X[M - k]);
                    const float2 Ze = c_scale(c_add(A, Bc), 0.5f);
                    const float2 Zo = c_mul(c_scale(c_sub(A, Bc), 0.5f), c_conj(w2[k]));
                    return float2{Ze.x - Zo.y, Ze.y + Zo.x};
                };
                auto lx = [&](int e) -> float2 { return act ? X[e] : float2{0.f, 0.f}; };
                auto sx = [&](int e, float2 v) {
                    if (act) X[e] = v;
                };
                auto sg = [&](int e, float2 v) {
                    if (act) *reinterpret_cast<float2*>(ug + 2 * e) = v;
                };
                fft_fast<float, M, true, true, false, NBAR>(lgz, sg, lx, sx, act ? tau : 0, tws);
            }
            fence_proxy_async();  // the stage's generic writes, before the next bulk copy
            __syncthreads();
            if (tid == 0 && zn < z1) issue(y0, zn + 1);
            if (zn == z0) continue;
            // voxel plane zn - 1 between ring slots sl ^ 1 (z) and sl (z + 1)
            const int zv = zn - 1;
            const int64_t zrow = (int64_t)(pb * g.n3p + zv) * g.n2;
            const float* P0 = up + (size_t)(sl ^ 1) * NL * n1;
            const float* P1 = up + (size_t)sl * NL * n1;
            for (int ly = lg; ly < TY; ly += LPB) {
                const int64_t o = (zrow + y0 + ly) * n1 + x0;
                float2 rv[9];
#pragma unroll
                for (int c = 0; c < 9; c++) rv[c] = *reinterpret_cast<const float2*>(r + c * V + o);
#pragma unroll
                for (int i = 0; i < 3; i++) {
                    const int ra = (i * (TY + 1) + ly) * n1, rb = ra + n1;  // node lines y, y + 1
                    float A3[3], B3[3], C3[3], D3[3];  // (y, z), (y, z + 1), (y + 1, z), (y + 1, z + 1)
                    A3[0] = P0[ra + x0], A3[1] = P0[ra + x0 + 1], A3[2] = P0[ra + x2];
                    B3[0] = P1[ra + x0], B3[1] = P1[ra + x0 + 1], B3[2] = P1[ra + x2];
                    C3[0] = P0[rb + x0], C3[1] = P0[rb + x0 + 1], C3[2] = P0[rb + x2];
                    D3[0] = P1[rb + x0], D3[1] = P1[rb + x0 + 1], D3[2] = P1[rb + x2];
                    float s0[3], s1[3], t0[3], t1[3];
#pragma unroll
                    for (int k = 0; k < 3; k++) {
                        s0[k] = A3[k] + B3[k];
                        s1[k] = C3[k] + D3[k];
                        t0[k] = A3[k] + C3[k];
                        t1[k] = B3[k] + D3[k];
                    }
                    float F[3][2];
#pragma unroll
                    for (int p = 0; p < 2; p++) {
                        F[0][p] = cx0 * ((s0[p + 1] + s1[p + 1]) - (s0[p] + s1[p]));
                        F[1][p] = cx1 * ((s1[p] + s1[p + 1]) - (s0[p] + s0[p + 1]));
                        F[2][p] = cx2 * ((t1[p] + t1[p + 1]) - (t0[p] + t0[p + 1]));
                    }
#pragma unroll
                    for (int J = 0; J < 3; J++) {
                        float2& qv = rv[3 * i + J];
                        qv.x -= alpha * F[J][0];
                        qv.y -= alpha * F[J][1];
                        accp += qv.x * qv.x + qv.y * qv.y;
                    }
                }
#pragma unroll
                for (int c = 0; c < 9; c++) *reinterpret_cast<float2*>(r + c * V + o) = rv[c];
            }
            // (the ring slot read here is rewritten two node planes on, after
            // the barrier that follows the next transform)
        }
        acc += (double)accp;
    }
    if (timed_out) {
        if (tid == 0) {
            raise_status(scp, COMBO_E_TIMEOUT);
            mbar_wait_bounded(&bar[0], phase ^ 1u);  // the copy waited on, if it is still in flight
        }
        return;
    }
    if (a.partial) {
        const double sacc = block_sum(acc, red);
        if (tid == 0) a.partial[blockIdx.x] = sacc;
        if (a.fuse && last_block(&scp->ticket[1], flag, gp)) {
            const double tot = sum_partials_fixed(a.partial + (size_t)pb * gp, gp, red);
            if (tid == 0) cg_beta(scp, tot, a.cg_tol, a.cg_max, a.cg_fixed);
        }
    }
}

// ------------------------------------------------------------- launchers
template <int M> static void xinv_disp_launch(const DispArgs& a, cudaStream_t st)
{
    constexpr int LB = disp_lb<M>();
    constexpr int lsx = (M + 2) / 2 * 2;
    constexpr int threads = xdisp_threads<M>();
    constexpr size_t sm = 2 * (size_t)3 * LB * lsx * 8 + (size_t)2 * M * 8 + 16;
    static int per_sm = 0;
    if (per_sm == 0) {
        cudaFuncSetAttribute(k_xinv_disp<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_xinv_disp<M>, threads, sm) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
    }
    const int grid = a.g.nprob * xpass_gp(a.g, LB, per_sm * num_sms_disp());
    k_xinv_disp<M><<<grid, threads, sm, st>>>(a);
}

void launch_xinv_disp(const DispArgs& a, cudaStream_t st)
{
    switch (a.g.M) {
        case 64: xinv_disp_launch<64>(a, st); break;
        case 128: xinv_disp_launch<128>(a, st); break;
        default: xinv_disp_launch<256>(a, st); break;
    }
}

int disp_grad_partials_max() { return 4 * num_sms_disp(); }

template <int M> static void disp_grad_launch(const DispArgs& a, cudaStream_t st)
{
    constexpr int LPB = 256 / M;
    static int per_sm = 0;
    if (per_sm == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_disp_grad_cg<M>, 256, 0) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        per_sm = std::min(per_sm, 4);
    }
    const int items = a.g.n3p * (a.g.n2 / kDispSY);
    const int cap = std::max(1, per_sm * num_sms_disp() / a.g.nprob);
    const int gp = std::max(1, std::min((items + LPB - 1) / LPB, cap));
    k_disp_grad_cg<M><<<a.g.nprob * gp, 256, 0, st>>>(a);
}

void launch_disp_grad_cg(const DispArgs& a, cudaStream_t st)
{
    switch (a.g.M) {
        case 64: disp_grad_launch<64>(a, st); break;
        case 128: disp_grad_launch<128>(a, st); break;
        default: disp_grad_launch<256>(a, st); break;
    }
}

template <int M, int TY> static void xinv_grad_launch(const DispArgs& a, cudaStream_t st)
{
    constexpr size_t sm = fused_smem<M, TY>();
    static int per_sm = 0;
    if (per_sm == 0) {
        cudaFuncSetAttribute(k_xinv_grad<M, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_xinv_grad<M, TY>, 256, sm) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        per_sm = std::min(per_sm, 4);
    }
    const int64_t total = (int64_t)(a.g.n2 / TY) * a.g.n3p;
    const int gp = (int)std::max<int64_t>(1, std::min<int64_t>(total, std::max(1, per_sm * num_sms_disp() / a.g.nprob)));
    k_xinv_grad<M, TY><<<a.g.nprob * gp, 256, sm, st>>>(a);
}

bool xinv_grad_ok(const GridDims& g)
{
    return disp_x_ok(g) && g.n2 % (g.M == 256 ? 4 : 8) == 0;
}

void launch_xinv_grad(const DispArgs& a, cudaStream_t st)
{
    switch (a.g.M) {
        case 64: xinv_grad_launch<64, fused_ty<64>()>(a, st); break;
        case 128: xinv_grad_launch<128, fused_ty<128>()>(a, st); break;
        default: xinv_grad_launch<256, fused_ty<256>()>(a, st); break;
    }
}

}  // namespace combo
