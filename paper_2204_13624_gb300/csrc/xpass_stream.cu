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
// stage layout: spectrum rows [9][LB][lsx] complex, then r rows [9][LB][n1]
template <int M>
__global__ void __launch_bounds__(256) k_xinv_stream(XinvArgs<float, float> a, int LB)
{
    if (a.sc->cg_done) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int n1 = 2 * M;
    constexpr int lsx = (M + 2) / 2 * 2;  // M + 1 rounded up to even: 16-byte rows
    const GridDims g = a.g;
    const size_t spec_bytes = (size_t)9 * LB * lsx * 8;
    const size_t sb = spec_bytes + (size_t)9 * LB * n1 * 4;
    unsigned char* stage[2] = {smem_raw, smem_raw + sb};
    float2* buf1 = reinterpret_cast<float2*>(smem_raw + 2 * sb);
    float2* buf2 = buf1 + (size_t)9 * LB * lsx;
    double* red = reinterpret_cast<double*>(buf2 + (size_t)9 * LB * lsx);
    int* flag = reinterpret_cast<int*>(red + 256);
    uint64_t* bar = reinterpret_cast<uint64_t*>(flag + 4);

    const int nlines = g.n2 * g.n3;
    const int ngroups = nlines / LB;
    const int64_t V = g.V;
    const float alpha = (float)a.sc->alpha;
    const uint32_t tx_bytes = (uint32_t)(9 * LB * lsx * 8 + 9 * LB * n1 * 4);

    auto issue = [&](int grp, int s) {
        float2* sp = reinterpret_cast<float2*>(stage[s]);
        float* rr = reinterpret_cast<float*>(stage[s] + spec_bytes);
        mbar_arrive_expect_tx(&bar[s], tx_bytes);
        for (int l = 0; l < LB; l++) {
            const int L = grp * LB + l;
            for (int c = 0; c < 9; c++) {
                bulk_g2s(sp + ((size_t)c * LB + l) * lsx, a.spec + c * g.Vs + (int64_t)L * g.nhp, lsx * 8, &bar[s]);
                bulk_g2s(rr + ((size_t)c * LB + l) * n1, a.r + c * V + (int64_t)L * n1, n1 * 4, &bar[s]);
            }
        }
    };

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_proxy_async();
    }
    __syncthreads();
    if (threadIdx.x == 0 && (int)blockIdx.x < ngroups) issue(blockIdx.x, 0);

    double acc = 0.0;
    int it = 0;
    bool timed_out = false;
    const int nl = 9 * LB;
    for (int grp = blockIdx.x; grp < ngroups; grp += gridDim.x, it++) {
        const int s = it & 1;
        const int nxt = grp + gridDim.x;
        if (threadIdx.x == 0 && nxt < ngroups) {
            fence_proxy_async();
            issue(nxt, s ^ 1);
        }
        const bool ok = mbar_wait_bounded(&bar[s], (uint32_t)((it >> 1) & 1));
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            break;
        }
        const float2* X = reinterpret_cast<const float2*>(stage[s]);
        const float* rr = reinterpret_cast<const float*>(stage[s] + spec_bytes);
        // Z[k] = Ze + i Zo,  Ze = (X[k] + conj X[M-k]) / 2,  Zo = (X[k] - conj X[M-k]) W^{-k} / 2
        for (int e = threadIdx.x; e < nl * M; e += blockDim.x) {
            const int q = e / M, k = e - q * M;
            const float2 A = X[(size_t)q * lsx + k];
            const float2 Bc = c_conj(X[(size_t)q * lsx + (M - k)]);
            const float2 Ze = c_scale(c_add(A, Bc), 0.5f);
            const float2 Zo = c_mul(c_scale(c_sub(A, Bc), 0.5f), c_conj(a.tw2[k]));
            buf1[(size_t)q * lsx + k] = float2{Ze.x - Zo.y, Ze.y + Zo.x};
        }
        __syncthreads();
        float2* Zr = fft_lines_fast<float, M, true>(buf1, buf2, nl, lsx, a.tw);
        const float* gq = reinterpret_cast<const float*>(Zr);
        const int L0 = grp * LB;
        float accp = 0.f;
        for (int e = threadIdx.x; e < LB * n1; e += blockDim.x) {
            const int l = e / n1, x = e - l * n1;
            const int64_t v = (int64_t)(L0 + l) * n1 + x;
#pragma unroll
            for (int c = 0; c < 9; c++) {
                const float rn = rr[((size_t)c * LB + l) * n1 + x] - alpha * gq[(size_t)2 * (c * LB + l) * lsx + x];
                a.r[c * V + v] = rn;
                accp += rn * rn;
            }
        }
        acc += (double)accp;
        __syncthreads();
    }
    if (timed_out) {
        if (threadIdx.x == 0) {
            raise_status(a.sc, COMBO_E_TIMEOUT);
            mbar_wait_bounded(&bar[it & 1 ^ 1], (uint32_t)(((it + 1) >> 1) & 1));
        }
        return;
    }
    if (a.partial) {
        const double sacc = block_sum(acc, red);
        if (threadIdx.x == 0) a.partial[blockIdx.x] = sacc;
        if (a.fuse && last_block(&a.sc->ticket[1], flag)) {
            const double tot = sum_partials_fixed(a.partial, gridDim.x, red);
            if (threadIdx.x == 0) cg_beta(a.sc, tot, a.cg_tol, a.cg_max, a.cg_fixed);
        }
    }
}

// ------------------------------------------------------------- launchers
static int stream_lines(const GridDims& g) { return (g.n1 <= 128 && (g.n2 * g.n3) % 2 == 0) ? 2 : 1; }

bool stream_xpass_ok(const GridDims& g)
{
    const int M = g.M;
    return (M == 64 || M == 128 || M == 256) && (g.n1 % 16) == 0 && (g.n2 * g.n3) % stream_lines(g) == 0;
}

template <int M> static void xinv_stream_launch(const XinvArgs<float, float>& a, cudaStream_t st)
{
    const int LB = stream_lines(a.g);
    constexpr int lsx = (M + 2) / 2 * 2;
    const size_t sb = (size_t)9 * LB * lsx * 8 + (size_t)9 * LB * 2 * M * 4;
    const size_t sm = 2 * sb + (size_t)2 * 9 * LB * lsx * 8 + 256 * 8 + 16 + 16;
    const int per_sm = sm > 72 * 1024 ? 2 : 3;
    const int groups = a.g.n2 * a.g.n3 / LB;
    const int grid = groups < per_sm * num_sms() ? groups : per_sm * num_sms();
    static bool attr = false;
    allow_smem_stream(k_xinv_stream<M>, attr);
    k_xinv_stream<M><<<grid, 256, sm, st>>>(a, LB);
}

void launch_xinv_stream(const XinvArgs<float, float>& a, cudaStream_t st)
{
    switch (a.g.M) {
        case 64: xinv_stream_launch<64>(a, st); break;
        case 128: xinv_stream_launch<128>(a, st); break;
        default: xinv_stream_launch<256>(a, st); break;
    }
}

}  // namespace combo
