// xpass_stream.cu -- the FP32 CG x-inverse with streamed inputs.
//
// Same arithmetic as the CG x-inverse of xpass.cu (r -= alpha G[A:p] with the
// fused beta reduction), restructured so that memory and arithmetic overlap inside a block: a
// persistent block walks its groups of x-lines, and while it transforms
// group i the input rows of group i+1 arrive in the other of two shared-
// memory stage buffers through bulk asynchronous copies (cp.async.bulk,
// completion counted on an mbarrier).  Outputs are written with ordinary
// coalesced stores.  Waits are bounded: a block that exhausts the cap
// raises COMBO_E_TIMEOUT, waits (bounded) for its own copies and returns.
#include <algorithm>

#include "async_copy.cuh"
#include "combo_internal.cuh"
#include "fft_fast.cuh"
#include "../../include/combo.h"

namespace combo {

namespace {

template <typename K> void allow_smem_stream(K kernel, bool& done)
{
    if (!done) {
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        done = true;
    }
}

int num_sms()
{
    static int nsm = 0;
    if (nsm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) nsm = 152;
    }
    return nsm;
}

}  // namespace

// ------------------------------------------------------------- CG x-inverse
// Thread q * TPL + tau transforms line q = c * LB + l of the group with the
// TPL threads of its compile-time plan; the block has just enough warps.
template <int M, int LB> __host__ __device__ constexpr int xinv_threads()
{
    return (9 * LB * FastPlan<M>::TPL + 31) / 32 * 32;
}

// stage layout: spectrum rows [9][LB][lsx] complex, then r rows [9][LB][n1].
// Per group: the first FFT stage reads the spectrum rows and forms the packed
// half-length input (Hermitian combine) on the fly; the last stage hands each
// output pair straight to the CG update r -= alpha G[A:p] and (r, r).
template <int M, int LB>
__global__ void __launch_bounds__(xinv_threads<M, LB>()) k_xinv_stream(XinvArgs<float, float> a)
{
    int pb, pj, gp;  // problem of this block, index among its gp blocks
    prob_block(a.g, blockIdx.x, gridDim.x, pb, pj, gp);
    Scalars* scp = a.sc + pb;
    if (scp->cg_done) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int n1 = 2 * M;
    constexpr int lsx = (M + 2) / 2 * 2;  // M + 1 rounded up to even: 16-byte rows
    constexpr int TPL = FastPlan<M>::TPL;
    constexpr int NL = 9 * LB;
    constexpr size_t SPEC = (size_t)NL * lsx * 8;
    constexpr size_t SB = SPEC + (size_t)NL * n1 * 4;
    const GridDims g = a.g;
    unsigned char* stage[2] = {smem_raw, smem_raw + SB};
    float2* xb = reinterpret_cast<float2*>(smem_raw + 2 * SB);  // exchange rows [NL][lsx]
    float2* w2 = xb + (size_t)NL * lsx;                          // exp(-2 pi i k / n1), k < M
    float2* tws = w2 + M;                                        // exp(-2 pi i t / M)
    double* red = reinterpret_cast<double*>(tws + M);
    int* flag = reinterpret_cast<int*>(red + 256);
    uint64_t* bar = reinterpret_cast<uint64_t*>(flag + 4);

    const int nlp = g.n2 * g.n3p;  // x-lines of one problem
    const int ngroups = nlp / LB;  // the launcher guarantees nlp % LB == 0
    const int gbase = pb * ngroups;
    const int64_t V = g.V;
    const float alpha = (float)scp->alpha;
    constexpr uint32_t tx_bytes = (uint32_t)SB;

    auto issue = [&](int grp, int s) {
        float2* sp = reinterpret_cast<float2*>(stage[s]);
        float* rr = reinterpret_cast<float*>(stage[s] + SPEC);
        mbar_arrive_expect_tx(&bar[s], tx_bytes);
        for (int l = 0; l < LB; l++) {
            const int L = grp * LB + l;
            for (int c = 0; c < 9; c++) {
                bulk_g2s(sp + ((size_t)c * LB + l) * lsx, a.spec + c * g.Vs + (int64_t)L * g.nhp, lsx * 8, &bar[s]);
                bulk_g2s(rr + ((size_t)c * LB + l) * n1, a.r + c * V + (int64_t)L * n1, n1 * 4, &bar[s]);
            }
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
    float2* xq = xb + (size_t)(act ? q : 0) * lsx;
    double acc = 0.0;
    int it = 0;
    bool timed_out = false;
    for (int lgrp = pj; lgrp < ngroups; lgrp += gp, it++) {
        const int grp = gbase + lgrp;
        const int s = it & 1;
        if (threadIdx.x == 0 && lgrp + gp < ngroups) {
            fence_proxy_async();
            issue(grp + gp, s ^ 1);
        }
        const bool ok = mbar_wait_bounded(&bar[s], (uint32_t)((it >> 1) & 1), wait_cap_of(a.wait_cap));
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            break;
        }
        const float2* X = reinterpret_cast<const float2*>(stage[s]) + (size_t)(act ? q : 0) * lsx;
        const float* rr = reinterpret_cast<const float*>(stage[s] + SPEC) + (size_t)(act ? q : 0) * n1;
        float* rg = a.r + (int64_t)c * V + (int64_t)(grp * LB + l) * n1;
        float accp = 0.f;
        // Z[k] = Ze + i Zo,  Ze = (X[k] + conj X[M-k]) / 2,  Zo = (X[k] - conj X[M-k]) W^{-k} / 2
        auto lg = [&](int k) -> float2 {
            if (!act) return float2{0.f, 0.f};
            const float2 A = X[k];
            const float2 Bc = c_conj(X[M - k]);
            const float2 Ze = c_scale(c_add(A, Bc), 0.5f);
            const float2 Zo = c_mul(c_scale(c_sub(A, Bc), 0.5f), c_conj(w2[k]));
            return float2{Ze.x - Zo.y, Ze.y + Zo.x};
        };
        auto lx = [&](int e) -> float2 { return act ? xq[e] : float2{0.f, 0.f}; };
        auto sx = [&](int e, float2 v) {
            if (act) xq[e] = v;
        };
        // output e of the packed inverse holds the reals 2e, 2e + 1
        auto sg = [&](int e, float2 v) {
            if (!act) return;
            const float2 r0 = *reinterpret_cast<const float2*>(rr + 2 * e);
            const float2 rn = float2{r0.x - alpha * v.x, r0.y - alpha * v.y};
            *reinterpret_cast<float2*>(rg + 2 * e) = rn;
            accp += rn.x * rn.x + rn.y * rn.y;
        };
        fft_fast<float, M, true, false, false>(lg, sg, lx, sx, tau, tws);
        acc += (double)accp;
        __syncthreads();  // stage s and the exchange rows are reused
    }
    if (timed_out) {
        if (threadIdx.x == 0) {
            raise_status(scp, COMBO_E_TIMEOUT);
            // copies possibly in flight: the group waited on and, if it was
            // issued, the prefetch of the next one (the block's shared memory
            // must outlive them)
            const int s = it & 1;
            mbar_wait_bounded(&bar[s], (uint32_t)((it >> 1) & 1));
            if (pj + (it + 1) * gp < ngroups) mbar_wait_bounded(&bar[s ^ 1], (uint32_t)(((it + 1) >> 1) & 1));
        }
        return;
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

// ------------------------------------------------------------- launchers
static int stream_lines(const GridDims& g) { return (g.n1 <= 128 && (g.n2 * g.n3p) % 2 == 0) ? 2 : 1; }

bool stream_xpass_ok(const GridDims& g)
{
    const int M = g.M;
    return (M == 64 || M == 128 || M == 256) && (g.n1 % 16) == 0 && (g.n2 * g.n3p) % stream_lines(g) == 0;
}

template <int M, int LB> static void xinv_stream_launch(const XinvArgs<float, float>& a, cudaStream_t st)
{
    constexpr int lsx = (M + 2) / 2 * 2;
    constexpr int threads = xinv_threads<M, LB>();
    constexpr size_t sb = (size_t)9 * LB * lsx * 8 + (size_t)9 * LB * 2 * M * 4;
    constexpr size_t sm = 2 * sb + (size_t)9 * LB * lsx * 8 + (size_t)2 * M * 8 + 256 * 8 + 16 + 16;
    static int per_sm = 0;
    if (per_sm == 0) {
        cudaFuncSetAttribute(k_xinv_stream<M, LB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_xinv_stream<M, LB>, threads, sm) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
    }
    const int grid = a.g.nprob * xpass_gp(a.g, LB, per_sm * num_sms());
    k_xinv_stream<M, LB><<<grid, threads, sm, st>>>(a);
}

// lines per group: candidate 0 (default) and candidate 1 (autotuner)
void launch_xinv_stream(const XinvArgs<float, float>& a, cudaStream_t st)
{
    const bool even = (a.g.n2 * a.g.n3p) % 2 == 0;
    switch (a.g.M) {
        case 64:
            if (stream_lines(a.g) == 2 && a.cfg != 1)
                xinv_stream_launch<64, 2>(a, st);
            else
                xinv_stream_launch<64, 1>(a, st);
            break;
        case 128:
            if (a.cfg == 1 && even)
                xinv_stream_launch<128, 2>(a, st);
            else
                xinv_stream_launch<128, 1>(a, st);
            break;
        default: xinv_stream_launch<256, 1>(a, st); break;
    }
}

}  // namespace combo
