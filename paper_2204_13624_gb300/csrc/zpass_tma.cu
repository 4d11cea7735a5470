// zpass_tma.cu -- FP32 z-pass (forward z FFT, Green operator, inverse z FFT)
// and y-passes with tensor-memory-accelerator (TMA) tile movement.
//
// Same arithmetic as k_zpass_fast of yzpass.cu for the Krylov operator (no
// norm accumulation).  A persistent block walks tiles of the half spectrum;
// a tile is the three components of one tensor row i, all N z-planes, one y
// and TX consecutive x frequencies: a 4-D box {TX, 1, N, 3} of the tensor
// [9][n3][n2][nhp] of complex FP32 (8-byte elements).  One TMA load brings a
// whole tile into shared memory (completion counted on an mbarrier) while the
// previous tile is transformed in the other buffer; the result leaves by one
// TMA store, so no thread waits on global memory.  The column stride of the
// z direction (n2 * nhp complex) makes this pass the one with the least
// contiguous rows; the copy engine issues them without occupying warps.
//
// Waits on the mbarrier are bounded: a block that exhausts the cap raises
// COMBO_E_TIMEOUT, waits (bounded) for its own copies in flight and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "async_copy.cuh"
#include "combo_internal.cuh"
#include "fft_fast.cuh"
#include "../../include/combo.h"

namespace combo {

namespace {

// x-frequency widths of a z-pass tile: two candidates per size (the
// autotuner picks one per grid; candidate 0 is the default)
template <int N, int C> __host__ __device__ constexpr int tma_tx()
{
    return (N > 128 ? 8 : 16) >> C;
}
__host__ __device__ constexpr int tma_tx_rt(int n, int c) { return (n > 128 ? 8 : 16) >> c; }
// x-frequency widths of a y-pass tile
template <int C> __host__ __device__ constexpr int tma_tyx() { return 16 >> C; }

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

}  // namespace

bool zpass_tma_size(int n3) { return n3 == 64 || n3 == 128 || n3 == 256 || n3 == 512 || fast3_size(n3); }

// Encode a tiled map of the complex FP32 spectrum [9][n3][n2][nhp]; an axis
// of 512 (the tile's long axis: z for the z-pass, y for the y-pass) is split
// into 256 x 2 (5-D map), since a box dimension holds at most 256 elements;
// the box then covers the whole axis as 256 x 2 with the shared-memory
// layout of the 4-D box.
static bool encode_spec_map(void* map, const GridDims& g, const void* spec, const cuuint32_t box4[4], int split_axis)
{
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t d4[4] = {(cuuint64_t)g.nhp, (cuuint64_t)g.n2, (cuuint64_t)g.n3, 9};
    const cuuint64_t s4[4] = {8, (cuuint64_t)g.nhp * 8, (cuuint64_t)g.n2 * g.nhp * 8,
                              (cuuint64_t)g.n3 * g.n2 * g.nhp * 8};
    cuuint64_t dim[5], stride[4];
    cuuint32_t box[5], estr[5] = {1, 1, 1, 1, 1};
    int nd = 0;
    for (int a = 0; a < 4; a++) {
        if (a == split_axis) {
            if (d4[a] % 256 != 0 || box4[a] != 512) return false;
            dim[nd] = 256;
            box[nd] = 256;
            if (nd > 0) stride[nd - 1] = s4[a];
            nd++;
            dim[nd] = d4[a] / 256;
            box[nd] = 2;
            stride[nd - 1] = s4[a] * 256;
            nd++;
        } else {
            dim[nd] = d4[a];
            box[nd] = box4[a];
            if (nd > 0) stride[nd - 1] = s4[a];
            nd++;
        }
    }
    const CUresult r = fn(reinterpret_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_UINT64, nd,
                          const_cast<void*>(spec), dim, stride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Tensor map of a complex FP32 half spectrum [9][n3][n2][nhp] for the z-pass
// tile box {TX, 1, n3, 3}.  False (map unusable) for other sizes or when the
// driver entry point is missing.
bool zpass_tma_encode(void* map, const GridDims& g, const void* spec, int cand)
{
    if (!zpass_tma_size(g.n3p) || !spec) return false;
    const int tx = tma_tx_rt(g.n3p, cand);
    if ((g.nhp * 8) % 16 != 0 || (reinterpret_cast<uintptr_t>(spec) & 15) != 0) return false;
    const cuuint32_t box[4] = {(cuuint32_t)tx, 1, (cuuint32_t)g.n3p, 3};
    return encode_spec_map(map, g, spec, box, g.n3p > 256 ? 2 : -1);
}

// Tensor map of the same spectrum with a one-component tile box {TX, 1, n3,
// 1}: the store of the displacement form's z-pass (one spectrum per row).
bool zpass_tma_encode_u(void* map, const GridDims& g, const void* spec, int cand)
{
    if (!zpass_tma_size(g.n3p) || !spec) return false;
    const int tx = tma_tx_rt(g.n3p, cand);
    if ((g.nhp * 8) % 16 != 0 || (reinterpret_cast<uintptr_t>(spec) & 15) != 0) return false;
    const cuuint32_t box[4] = {(cuuint32_t)tx, 1, (cuuint32_t)g.n3p, 1};
    return encode_spec_map(map, g, spec, box, g.n3p > 256 ? 2 : -1);
}

// DISP: the displacement form of the rotated operator.  The rotated symbol is
// k_J = i P kr_J with P = e^{i (theta_1 + theta_2 + theta_3) / 2} and the real
// kr of the symbol tables, so G X_i = k (k^H X_i) / |k|^2 is the HEX8R
// gradient (the 8-node trilinear element's average gradient, an edge
// difference averaged over the 4 parallel edges of the voxel) of the nodal
// field u_i = IFFT(-i conj(P) (kr . X_i) / |kr|^2).  The tile's row then
// leaves as that one spectrum, into component 3 i: the inverse z transform
// runs on one component instead of three, by the first component group of
// threads on named barrier 1 while the others wait at the block barrier.
template <int N, int TX, bool DISP>
__global__ void __launch_bounds__(3 * TX * FastPlan<N>::TPL)
    k_zpass_tma(const __grid_constant__ CUtensorMap tm, const __grid_constant__ CUtensorMap tmu, ZArgs<float> a)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    constexpr int TPL = FastPlan<N>::TPL;
    constexpr int GS = TX * TPL;  // threads per component group
    constexpr int TILE = 3 * N * TX;
    constexpr uint32_t TILE_BYTES = TILE * 8;
    typedef cx<float> C;
    C* tiles = reinterpret_cast<C*>(smem_raw);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + 2 * TILE_BYTES);
    C* tws = reinterpret_cast<C*>(bar + 2);  // twiddles exp(-2 pi i t / N) in shared memory
    const GridDims g = a.g;
    for (int i = threadIdx.x; i < N; i += blockDim.x) tws[i] = a.tw[i];
    const int c = threadIdx.x / GS;
    const int r = threadIdx.x - c * GS;
    const int line = r % TX, tau = r / TX;
    const int nxt = (g.nh + TX - 1) / TX;
    const int tpp = nxt * g.n2 * 3;  // tiles per problem
    const int ntiles = tpp * g.nprob;
    // a tile of a finished problem is skipped (guard 1: CG done, 2: outer done)
    auto done_of = [&](const Scalars* q) { return (a.guard == 1 && q->cg_done) || (a.guard == 2 && q->outer_done); };
    const bool done0 = done_of(a.sc);
    auto active = [&](int t) { return g.nprob == 1 ? !done0 : !done_of(a.sc + t / tpp); };
    auto next_tile = [&](int t) {
        while (t < ntiles && !active(t)) t += gridDim.x;
        return t;
    };

    // tile t = ((b * 3 + row) * n2 + y) * nxt + xt: consecutive blocks take
    // neighbouring x tiles of the same rows of DRAM
    auto issue = [&](int t, int s) {
        const int xt = t % nxt, rest = t / nxt;
        const int y = rest % g.n2, rb = rest / g.n2;
        const int b = rb / 3, row = rb - 3 * b;
        mbar_arrive_expect_tx(&bar[s], TILE_BYTES);
        if constexpr (N > 256)
            tma_load_5d(tiles + s * TILE, &tm, xt * TX, y, 0, b * (N / 256), 3 * row, &bar[s]);
        else
            tma_load_4d(tiles + s * TILE, &tm, xt * TX, y, b * N, 3 * row, &bar[s]);
    };

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_proxy_async();
    }
    __syncthreads();
    const int t0 = next_tile(blockIdx.x);
    if (threadIdx.x == 0 && t0 < ntiles) issue(t0, 0);

    int it = 0, tn = ntiles;
    bool timed_out = false;
    for (int t = t0; t < ntiles; t = tn, it++) {
        const int s = it & 1;
        tn = next_tile(t + gridDim.x);
        if (threadIdx.x == 0 && tn < ntiles) {
            bulk_wait_read_all();  // the store of the previous tile has left buffer s ^ 1
            issue(tn, s ^ 1);
        }
        const bool ok = mbar_wait_bounded(&bar[s], (uint32_t)((it >> 1) & 1), wait_cap_of(a.wait_cap));
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            break;
        }
        const int xt = t % nxt, rest = t / nxt;
        const int y = rest % g.n2, rb = rest / g.n2;
        const int pb = rb / 3, row = rb - 3 * pb;
        const int x0 = xt * TX;
        C* park = tiles + s * TILE;
        C* pc = park + c * N * TX + line;
        auto lp = [&](int e) { return pc[e * TX]; };
        auto sp = [&](int e, C v) { pc[e * TX] = v; };

        // forward along z, in place in the tile
        fft_fast<float, N, false, true, true>(lp, sp, lp, sp, tau, tws);
        __syncthreads();

        // projection: row i of G X at every (xi3, column) = k (k . X_i) / |k|^2
        const float ay = a.sa[1][y], by = a.sb[1][y];
        for (int f = threadIdx.x; f < N * TX; f += blockDim.x) {
            const int z = f / TX, ln = f - z * TX;
            const int xi1 = x0 + ln;
            C* p = park + f;
            if (xi1 >= g.nh) {
                p[0] = p[N * TX] = p[2 * N * TX] = C{0.f, 0.f};
                continue;
            }
            C X0 = p[0], X1 = p[N * TX], X2 = p[2 * N * TX];
            C u0, u1, u2;
            if (a.ph[0]) {
                u0 = stag_u(row, 0, a.ph[0][xi1]);
                u1 = stag_u(row, 1, a.ph[1][y]);
                u2 = stag_u(row, 2, a.ph[2][z]);
                X0 = c_mul(X0, u0);
                X1 = c_mul(X1, u1);
                X2 = c_mul(X2, u2);
            }
            const float ax = a.sa[0][xi1], bx = a.sb[0][xi1];
            const float az = a.sa[2][z], bz = a.sb[2][z];
            const float k0 = ax * by * bz, k1 = ay * bx * bz, k2 = az * bx * by;
            const float kk = k0 * k0 + k1 * k1 + k2 * k2;
            if constexpr (DISP) {
                C o{0.f, 0.f};
                if (kk > 0.f) {
                    const float ik = a.scale / kk;
                    const float sr = (k0 * X0.x + k1 * X1.x + k2 * X2.x) * ik;
                    const float si = (k0 * X0.y + k1 * X1.y + k2 * X2.y) * ik;
                    const C P = c_mul(c_mul(a.rph[0][xi1], a.rph[1][y]), a.rph[2][z]);
                    // -i conj(P) (sr + i si)
                    o = C{P.x * si - P.y * sr, -(P.x * sr + P.y * si)};
                }
                p[0] = o;
                continue;
            }
            C o0{0.f, 0.f}, o1{0.f, 0.f}, o2{0.f, 0.f};
            if (kk > 0.f) {
                const float ik = 1.f / kk;
                const float sr = (k0 * X0.x + k1 * X1.x + k2 * X2.x) * ik;
                const float si = (k0 * X0.y + k1 * X1.y + k2 * X2.y) * ik;
                o0 = C{k0 * sr, k0 * si};
                o1 = C{k1 * sr, k1 * si};
                o2 = C{k2 * sr, k2 * si};
                if (a.ph[0]) {
                    o0 = c_mul(o0, c_conj(u0));
                    o1 = c_mul(o1, c_conj(u1));
                    o2 = c_mul(o2, c_conj(u2));
                }
            }
            p[0] = c_scale(o0, a.scale);
            p[N * TX] = c_scale(o1, a.scale);
            p[2 * N * TX] = c_scale(o2, a.scale);
        }
        __syncthreads();

        // inverse along z, in place; then the whole tile leaves by one store
        if constexpr (DISP) {
            // component 0 only, by the warps of the first group (threads of
            // its last warp beyond GS transform lines of component 1, which
            // is not stored)
            constexpr int GSW = (GS + 31) / 32 * 32;
            if (threadIdx.x < GSW) fft_fast<float, N, true, true, true, GSW>(lp, sp, lp, sp, tau, tws);
        } else {
            fft_fast<float, N, true, true, true>(lp, sp, lp, sp, tau, tws);
        }
        fence_proxy_async();  // this thread's tile writes, before the copy engine reads them
        __syncthreads();
        if (threadIdx.x == 0) {
            const CUtensorMap* ts = DISP ? &tmu : &tm;
            if constexpr (N > 256)
                tma_store_5d(ts, x0, y, 0, pb * (N / 256), 3 * row, park);
            else
                tma_store_4d(ts, x0, y, pb * N, 3 * row, park);
            bulk_commit();
        }
    }
    if (threadIdx.x == 0) {
        if (timed_out) {
            raise_status(a.sc, COMBO_E_TIMEOUT);
            // loads possibly in flight: this iteration's and the prefetch
            const int s = it & 1;
            mbar_wait_bounded(&bar[s], (uint32_t)((it >> 1) & 1));
            if (tn < ntiles) mbar_wait_bounded(&bar[s ^ 1], (uint32_t)(((it + 1) >> 1) & 1));
        }
        bulk_wait_all();  // the stores are complete before the block's shared memory goes away
    }
}

// ------------------------------------------------------------- y-pass
// Tile: one component, one z plane, all n2 y rows, TX consecutive x
// frequencies: box {TX, n2, 1, 1}; the transform runs in place in the tile.
bool ypass_tma_encode(void* map, const GridDims& g, const void* spec, int cand)
{
    const int TYX = 16 >> cand;
    if (!zpass_tma_size(g.n2) || !spec) return false;
    if ((g.nhp * 8) % 16 != 0 || (reinterpret_cast<uintptr_t>(spec) & 15) != 0) return false;
    const cuuint32_t box[4] = {(cuuint32_t)TYX, (cuuint32_t)g.n2, 1, 1};
    return encode_spec_map(map, g, spec, box, g.n2 > 256 ? 1 : -1);
}

template <int N, int TX, bool INV>
__global__ void __launch_bounds__(TX * FastPlan<N>::TPL)
    k_ypass_tma(const __grid_constant__ CUtensorMap tm, YArgs<float> a)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    constexpr int TILE = N * TX;
    constexpr uint32_t TILE_BYTES = TILE * 8;
    typedef cx<float> C;
    C* tiles = reinterpret_cast<C*>(smem_raw);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + 2 * TILE_BYTES);
    C* tws = reinterpret_cast<C*>(bar + 2);  // twiddles in shared memory
    const GridDims g = a.g;
    for (int i = threadIdx.x; i < N; i += blockDim.x) tws[i] = a.tw[i];
    const int line = threadIdx.x % TX, tau = threadIdx.x / TX;
    const int nxt = (g.nh + TX - 1) / TX;
    const int cs = a.disp ? 3 : 1;  // component stride: the displacement form's y-inverse takes 0, 3, 6
    const int ntiles = nxt * g.n3 * (9 / cs);
    // a tile of a finished problem (the problem of its z plane) is skipped
    auto done_of = [&](const Scalars* q) { return (a.guard == 1 && q->cg_done) || (a.guard == 2 && q->outer_done); };
    const bool done0 = done_of(a.sc);
    auto active = [&](int t) { return g.nprob == 1 ? !done0 : !done_of(a.sc + ((t / nxt) % g.n3) / g.n3p); };
    auto next_tile = [&](int t) {
        while (t < ntiles && !active(t)) t += gridDim.x;
        return t;
    };

    // tile t = (c * n3 + z) * nxt + xt
    auto issue = [&](int t, int s) {
        const int xt = t % nxt, rest = t / nxt;
        const int z = rest % g.n3, c = (rest / g.n3) * cs;
        mbar_arrive_expect_tx(&bar[s], TILE_BYTES);
        if constexpr (N > 256)
            tma_load_5d(tiles + s * TILE, &tm, xt * TX, 0, 0, z, c, &bar[s]);
        else
            tma_load_4d(tiles + s * TILE, &tm, xt * TX, 0, z, c, &bar[s]);
    };

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_proxy_async();
    }
    __syncthreads();
    const int t0 = next_tile(blockIdx.x);
    if (threadIdx.x == 0 && t0 < ntiles) issue(t0, 0);

    int it = 0, tn = ntiles;
    bool timed_out = false;
    for (int t = t0; t < ntiles; t = tn, it++) {
        const int s = it & 1;
        tn = next_tile(t + gridDim.x);
        if (threadIdx.x == 0 && tn < ntiles) {
            bulk_wait_read_all();  // the store of the previous tile has left buffer s ^ 1
            issue(tn, s ^ 1);
        }
        const bool ok = mbar_wait_bounded(&bar[s], (uint32_t)((it >> 1) & 1), wait_cap_of(a.wait_cap));
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            break;
        }
        const int xt = t % nxt, rest = t / nxt;
        const int z = rest % g.n3, c = (rest / g.n3) * cs;
        C* park = tiles + s * TILE;
        C* pc = park + line;
        auto lp = [&](int e) { return pc[e * TX]; };
        auto sp = [&](int e, C v) { pc[e * TX] = v; };
        fft_fast<float, N, INV, true, true>(lp, sp, lp, sp, tau, tws);
        fence_proxy_async();  // this thread's tile writes, before the copy engine reads them
        __syncthreads();
        if (threadIdx.x == 0) {
            if constexpr (N > 256)
                tma_store_5d(&tm, xt * TX, 0, 0, z, c, park);
            else
                tma_store_4d(&tm, xt * TX, 0, z, c, park);
            bulk_commit();
        }
    }
    if (threadIdx.x == 0) {
        if (timed_out) {
            raise_status(const_cast<Scalars*>(a.sc), COMBO_E_TIMEOUT);
            const int s = it & 1;
            mbar_wait_bounded(&bar[s], (uint32_t)((it >> 1) & 1));
            if (tn < ntiles) mbar_wait_bounded(&bar[s ^ 1], (uint32_t)(((it + 1) >> 1) & 1));
        }
        bulk_wait_all();
    }
}

template <int N, int TX, bool INV>
static void ypass_tma_launch(const YArgs<float>& a, const void* map, cudaStream_t st)
{
    constexpr int threads = TX * FastPlan<N>::TPL;
    const size_t sm = (size_t)2 * N * TX * 8 + 16 + (size_t)N * 8;
    static int grid_per_sm = 0;
    static int nsm = 0;
    if (grid_per_sm == 0) {
        cudaFuncSetAttribute(k_ypass_tma<N, TX, INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) nsm = 152;
        int per = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_ypass_tma<N, TX, INV>, threads, sm) != cudaSuccess ||
            per < 1)
            per = 1;
        grid_per_sm = per;
    }
    const int ntiles = ((a.g.nh + TX - 1) / TX) * a.g.n3 * (a.disp ? 3 : 9);
    const int grid = std::min(ntiles, grid_per_sm * nsm);
    k_ypass_tma<N, TX, INV><<<grid, threads, sm, st>>>(*reinterpret_cast<const CUtensorMap*>(map), a);
}

template <int N, bool INV> static void ypass_tma_pick(const YArgs<float>& a, const void* map, cudaStream_t st)
{
    if (a.cfg == 1)
        ypass_tma_launch<N, tma_tyx<1>(), INV>(a, map, st);
    else
        ypass_tma_launch<N, tma_tyx<0>(), INV>(a, map, st);
}

template <bool INV> void launch_ypass_tma(const YArgs<float>& a, const void* map, cudaStream_t st)
{
    switch (a.g.n2) {
        case 48: ypass_tma_pick<48, INV>(a, map, st); break;
        case 64: ypass_tma_pick<64, INV>(a, map, st); break;
        case 72: ypass_tma_pick<72, INV>(a, map, st); break;
        case 96: ypass_tma_pick<96, INV>(a, map, st); break;
        case 108: ypass_tma_pick<108, INV>(a, map, st); break;
        case 128: ypass_tma_pick<128, INV>(a, map, st); break;
        case 144: ypass_tma_pick<144, INV>(a, map, st); break;
        case 192: ypass_tma_pick<192, INV>(a, map, st); break;
        case 216: ypass_tma_pick<216, INV>(a, map, st); break;
        case 256: ypass_tma_pick<256, INV>(a, map, st); break;
        default: ypass_tma_pick<512, INV>(a, map, st); break;
    }
}
template void launch_ypass_tma<false>(const YArgs<float>&, const void*, cudaStream_t);
template void launch_ypass_tma<true>(const YArgs<float>&, const void*, cudaStream_t);

// ------------------------------------------------------------- z-pass launch
template <int N, int TX, bool DISP>
static void zpass_tma_launch(const ZArgs<float>& a, const void* map, cudaStream_t st)
{
    constexpr int threads = 3 * TX * FastPlan<N>::TPL;
    const size_t sm = (size_t)2 * 3 * N * TX * 8 + 16 + (size_t)N * 8;
    static int grid_per_sm = 0;
    static int nsm = 0;
    if (grid_per_sm == 0) {
        cudaFuncSetAttribute(k_zpass_tma<N, TX, DISP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) nsm = 152;
        int per = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_zpass_tma<N, TX, DISP>, threads, sm) !=
                cudaSuccess ||
            per < 1)
            per = 1;
        grid_per_sm = per;
    }
    const int ntiles = ((a.g.nh + TX - 1) / TX) * a.g.n2 * 3 * a.g.nprob;
    const int grid = std::min(ntiles, grid_per_sm * nsm);
    const CUtensorMap& tm = *reinterpret_cast<const CUtensorMap*>(map);
    const CUtensorMap& tmu = DISP ? *reinterpret_cast<const CUtensorMap*>(a.tmap_u) : tm;
    k_zpass_tma<N, TX, DISP><<<grid, threads, sm, st>>>(tm, tmu, a);
}

template <int N> static void zpass_tma_pick(const ZArgs<float>& a, const void* map, cudaStream_t st)
{
    const bool disp = a.disp && a.tmap_u;
    if (a.cfg == 1) {
        if (disp)
            zpass_tma_launch<N, tma_tx<N, 1>(), true>(a, map, st);
        else
            zpass_tma_launch<N, tma_tx<N, 1>(), false>(a, map, st);
    } else {
        if (disp)
            zpass_tma_launch<N, tma_tx<N, 0>(), true>(a, map, st);
        else
            zpass_tma_launch<N, tma_tx<N, 0>(), false>(a, map, st);
    }
}

void launch_zpass_tma(const ZArgs<float>& a, const void* map, cudaStream_t st)
{
    switch (a.g.n3p) {
        case 48: zpass_tma_pick<48>(a, map, st); break;
        case 64: zpass_tma_pick<64>(a, map, st); break;
        case 72: zpass_tma_pick<72>(a, map, st); break;
        case 96: zpass_tma_pick<96>(a, map, st); break;
        case 108: zpass_tma_pick<108>(a, map, st); break;
        case 128: zpass_tma_pick<128>(a, map, st); break;
        case 144: zpass_tma_pick<144>(a, map, st); break;
        case 192: zpass_tma_pick<192>(a, map, st); break;
        case 216: zpass_tma_pick<216>(a, map, st); break;
        case 256: zpass_tma_pick<256>(a, map, st); break;
        default: zpass_tma_pick<512>(a, map, st); break;
    }
}

// ------------------------------------------------------------- scalar z-pass
// The nodal form's z-pass: a tile is one of the components 0, 3, 6 (the
// nodal forces f_i), all N z-planes, one y and TX x-frequencies (box {TX, 1,
// N, 1}); forward z FFT, multiplication by scale / |kr|^2 (zero where |kr| is
// zero), inverse z FFT, in place, then one TMA store.
// tile width: candidate 0 (default) or 1 (half as wide; autotuner)
__host__ __device__ constexpr int tma_txs(int n, int c = 0) { return (n > 256 ? 8 : 16) >> c; }

bool zpass_scalar_encode(void* map, const GridDims& g, const void* spec, int cand)
{
    if (!zpass_tma_size(g.n3p) || !spec) return false;
    if ((g.nhp * 8) % 16 != 0 || (reinterpret_cast<uintptr_t>(spec) & 15) != 0) return false;
    const cuuint32_t box[4] = {(cuuint32_t)tma_txs(g.n3p, cand), 1, (cuuint32_t)g.n3p, 1};
    return encode_spec_map(map, g, spec, box, g.n3p > 256 ? 2 : -1);
}

template <int N, int TX>
__global__ void __launch_bounds__(TX * FastPlan<N>::TPL)
    k_zpass_scalar(const __grid_constant__ CUtensorMap tm, ZArgs<float> a)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    constexpr int TILE = N * TX;
    constexpr uint32_t TILE_BYTES = TILE * 8;
    typedef cx<float> C;
    C* tiles = reinterpret_cast<C*>(smem_raw);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + 2 * TILE_BYTES);
    C* tws = reinterpret_cast<C*>(bar + 2);
    const GridDims g = a.g;
    for (int i = threadIdx.x; i < N; i += blockDim.x) tws[i] = a.tw[i];
    const int line = threadIdx.x % TX, tau = threadIdx.x / TX;
    const int nxt = (g.nh + TX - 1) / TX;
    const int tpp = nxt * g.n2 * 3;  // tiles per problem
    const int ntiles = tpp * g.nprob;
    auto done_of = [&](const Scalars* q) { return (a.guard == 1 && q->cg_done) || (a.guard == 2 && q->outer_done); };
    const bool done0 = done_of(a.sc);
    auto active = [&](int t) { return g.nprob == 1 ? !done0 : !done_of(a.sc + t / tpp); };
    auto next_tile = [&](int t) {
        while (t < ntiles && !active(t)) t += gridDim.x;
        return t;
    };
    // tile t = ((b * 3 + row) * n2 + y) * nxt + xt
    auto issue = [&](int t, int s) {
        const int xt = t % nxt, rest = t / nxt;
        const int y = rest % g.n2, rb = rest / g.n2;
        const int b = rb / 3, row = rb - 3 * b;
        mbar_arrive_expect_tx(&bar[s], TILE_BYTES);
        if constexpr (N > 256)
            tma_load_5d(tiles + s * TILE, &tm, xt * TX, y, 0, b * (N / 256), 3 * row, &bar[s]);
        else
            tma_load_4d(tiles + s * TILE, &tm, xt * TX, y, b * N, 3 * row, &bar[s]);
    };
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_proxy_async();
    }
    __syncthreads();
    const int t0 = next_tile(blockIdx.x);
    if (threadIdx.x == 0 && t0 < ntiles) issue(t0, 0);

    int it = 0, tn = ntiles;
    bool timed_out = false;
    for (int t = t0; t < ntiles; t = tn, it++) {
        const int s = it & 1;
        tn = next_tile(t + gridDim.x);
        if (threadIdx.x == 0 && tn < ntiles) {
            bulk_wait_read_all();  // the store of the previous tile has left buffer s ^ 1
            issue(tn, s ^ 1);
        }
        const bool ok = mbar_wait_bounded(&bar[s], (uint32_t)((it >> 1) & 1), wait_cap_of(a.wait_cap));
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            break;
        }
        const int xt = t % nxt, rest = t / nxt;
        const int y = rest % g.n2, rb = rest / g.n2;
        const int pb = rb / 3, row = rb - 3 * pb;
        const int x0 = xt * TX;
        C* park = tiles + s * TILE;
        C* pc = park + line;
        auto lp = [&](int e) { return pc[e * TX]; };
        auto sp = [&](int e, C v) { pc[e * TX] = v; };
        fft_fast<float, N, false, true, true>(lp, sp, lp, sp, tau, tws);
        __syncthreads();
        const float ay = a.sa[1][y], by = a.sb[1][y];
        for (int f = threadIdx.x; f < N * TX; f += blockDim.x) {
            const int z = f / TX, ln = f - z * TX;
            const int xi1 = x0 + ln;
            float w = 0.f;
            if (xi1 < g.nh) {
                const float ax = a.sa[0][xi1], bx = a.sb[0][xi1];
                const float az = a.sa[2][z], bz = a.sb[2][z];
                const float k0 = ax * by * bz, k1 = ay * bx * bz, k2 = az * bx * by;
                const float kk = k0 * k0 + k1 * k1 + k2 * k2;
                if (kk > 0.f) w = a.scale / kk;
            }
            park[f] = c_scale(park[f], w);
        }
        __syncthreads();
        fft_fast<float, N, true, true, true>(lp, sp, lp, sp, tau, tws);
        fence_proxy_async();
        __syncthreads();
        if (threadIdx.x == 0) {
            if constexpr (N > 256)
                tma_store_5d(&tm, x0, y, 0, pb * (N / 256), 3 * row, park);
            else
                tma_store_4d(&tm, x0, y, pb * N, 3 * row, park);
            bulk_commit();
        }
    }
    if (threadIdx.x == 0) {
        if (timed_out) {
            raise_status(a.sc, COMBO_E_TIMEOUT);
            const int s = it & 1;
            mbar_wait_bounded(&bar[s], (uint32_t)((it >> 1) & 1));
            if (tn < ntiles) mbar_wait_bounded(&bar[s ^ 1], (uint32_t)(((it + 1) >> 1) & 1));
        }
        bulk_wait_all();
    }
}

template <int N, int C> static void zpass_scalar_launch(const ZArgs<float>& a, cudaStream_t st)
{
    constexpr int TX = tma_txs(N, C);
    constexpr int threads = TX * FastPlan<N>::TPL;
    const size_t sm = (size_t)2 * N * TX * 8 + 16 + (size_t)N * 8;
    static int grid_per_sm = 0;
    static int nsm = 0;
    if (grid_per_sm == 0) {
        cudaFuncSetAttribute(k_zpass_scalar<N, TX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) nsm = 152;
        int per = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_zpass_scalar<N, TX>, threads, sm) != cudaSuccess ||
            per < 1)
            per = 1;
        grid_per_sm = per;
    }
    const int ntiles = ((a.g.nh + TX - 1) / TX) * a.g.n2 * 3 * a.g.nprob;
    const int grid = std::min(ntiles, grid_per_sm * nsm);
    k_zpass_scalar<N, TX><<<grid, threads, sm, st>>>(*reinterpret_cast<const CUtensorMap*>(a.tmap_u), a);
}

template <int C> static void zpass_scalar_pick(const ZArgs<float>& a, cudaStream_t st)
{
    switch (a.g.n3p) {
        case 48: zpass_scalar_launch<48, C>(a, st); break;
        case 64: zpass_scalar_launch<64, C>(a, st); break;
        case 72: zpass_scalar_launch<72, C>(a, st); break;
        case 96: zpass_scalar_launch<96, C>(a, st); break;
        case 108: zpass_scalar_launch<108, C>(a, st); break;
        case 128: zpass_scalar_launch<128, C>(a, st); break;
        case 144: zpass_scalar_launch<144, C>(a, st); break;
        case 192: zpass_scalar_launch<192, C>(a, st); break;
        case 216: zpass_scalar_launch<216, C>(a, st); break;
        case 256: zpass_scalar_launch<256, C>(a, st); break;
        default: zpass_scalar_launch<512, C>(a, st); break;
    }
}

// (a.tmap_u: the map encoded for the candidate a.cfg selects)
void launch_zpass_scalar(const ZArgs<float>& a, cudaStream_t st)
{
    if (a.cfg == 1)
        zpass_scalar_pick<1>(a, st);
    else
        zpass_scalar_pick<0>(a, st);
}

}  // namespace combo
