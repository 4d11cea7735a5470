// yzpass.cu -- y and z passes of one operator application.
//
//   y-pass : complex FFT along y of one component tile, in place.
//   z-pass : complex FFT along z of one tensor row (3 components), the
//            Green-operator projection of Sec. 3 (Eq. Gamma0) per frequency,
//            partial sums of |G X|^2 (Parseval), and the inverse FFT along z.
//
// The half spectrum is [9][n3][n2][nhp] complex.  Power-of-two line lengths
// use the compile-time plans of fft_fast.cuh (global -> registers -> one
// shared-memory exchange -> global); other lengths use the runtime
// mixed-radix Stockham of combo_internal.cuh.
#include "combo_internal.cuh"
#include "fft_fast.cuh"
#include "../../include/combo.h"

namespace combo {

template <typename K> static void allow_smem(K kernel, bool& done)
{
    if (!done) {
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        done = true;
    }
}

// ------------------------------------------------------------- y pass (generic)
// The pass bodies take the block index explicitly (VBlock): a launch of its
// own passes blockIdx, a grouped launch the work item of one grid.
template <typename T, bool INV>
__device__ __forceinline__ void ypass_body(const YArgs<T>& a, const VBlock& bi, unsigned char* smem_raw)
{
    const Scalars* sc = a.sc + bi.y / a.g.n3p;  // this z plane's problem
    if (a.guard == 1 && sc->cg_done) return;
    if (a.guard == 2 && sc->outer_done) return;
    const GridDims g = a.g;
    const int TX = a.tx;
    const int n2 = g.n2;
    cx<T>* buf0 = reinterpret_cast<cx<T>*>(smem_raw);
    cx<T>* buf1 = buf0 + (size_t)n2 * TX;
    const int x0 = bi.x * TX;
    const int z = bi.y;
    cx<T>* base = a.spec + bi.z * g.Vs + (int64_t)z * n2 * g.nhp + x0;
    for (int e = threadIdx.x; e < n2 * TX; e += blockDim.x) {
        const int y = e / TX, t = e - y * TX;
        buf0[e] = (x0 + t < g.nh) ? base[(int64_t)y * g.nhp + t] : cx<T>{(T)0, (T)0};
    }
    __syncthreads();
    cx<T>* res = fft_lines<T, INV>(buf0, buf1, a.plan, TX, 1, TX, a.tw);
    for (int e = threadIdx.x; e < n2 * TX; e += blockDim.x) {
        const int y = e / TX, t = e - y * TX;
        if (x0 + t < g.nh) base[(int64_t)y * g.nhp + t] = res[e];
    }
}

template <typename T, bool INV>
__global__ void __launch_bounds__(256) k_ypass(YArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ypass_body<T, INV>(a, VBlock::of_launch(), smem_raw);
}

// ------------------------------------------------------------- y pass (power of two)
// Block: TX columns x TPL threads; column fastest in the thread index so that
// every global access of a warp covers TX consecutive complex values.
template <typename T, int N, int TX, bool INV>
__device__ __forceinline__ void ypass_fast_body(const YArgs<T>& a, const VBlock& bi, unsigned char* smem_raw)
{
    const Scalars* sc = a.sc + bi.y / a.g.n3p;  // this z plane's problem
    if (a.guard == 1 && sc->cg_done) return;
    if (a.guard == 2 && sc->outer_done) return;
    cx<T>* ex = reinterpret_cast<cx<T>*>(smem_raw);
    const GridDims g = a.g;
    const int line = threadIdx.x % TX, tau = threadIdx.x / TX;
    const int x0 = bi.x * TX;
    const bool valid = x0 + line < g.nh;
    cx<T>* base = a.spec + bi.z * g.Vs + (int64_t)bi.y * N * g.nhp + x0 + line;
    const int64_t st = g.nhp;
    if constexpr (std::is_same<T, df32>::value && INV) {
        if (a.inv32) {
            float2* ex32 = reinterpret_cast<float2*>(smem_raw);
            fft_fast<float, N, true>(
                [&](int e) {
                    if (!valid) return float2{0.f, 0.f};
                    const cx<df32> v = base[e * st];
                    return float2{v.x.hi + v.x.lo, v.y.hi + v.y.lo};
                },
                [&](int e, float2 v) {
                    if (valid) base[e * st] = cx<df32>{df32(v.x, 0.f), df32(v.y, 0.f)};
                },
                [&](int e) { return ex32[e * TX + line]; }, [&](int e, float2 v) { ex32[e * TX + line] = v; }, tau,
                a.tw32);
            return;
        }
    }
    fft_fast<T, N, INV>([&](int e) { return valid ? base[e * st] : cx<T>{(T)0, (T)0}; },
                        [&](int e, cx<T> v) {
                            if (valid) base[e * st] = v;
                        },
                        [&](int e) { return ex[e * TX + line]; }, [&](int e, cx<T> v) { ex[e * TX + line] = v; }, tau,
                        a.tw);
}

template <typename T, int N, int TX, bool INV>
__global__ void __launch_bounds__(TX * FastPlan<N>::TPL) k_ypass_fast(YArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ypass_fast_body<T, N, TX, INV>(a, VBlock::of_launch(), smem_raw);
}

// ------------------------------------------------------------- z pass + Gamma (generic)
template <typename T>
__device__ __forceinline__ void zpass_body(const ZArgs<T>& a, const VBlock& bi, unsigned char* smem_raw)
{
    const int pb = bi.z / 3;  // problem; gz = 3 nprob
    Scalars* sc = a.sc + pb;
    if (a.guard == 1 && sc->cg_done) return;
    if (a.guard == 2 && sc->outer_done) return;
    const GridDims g = a.g;
    const int TX = a.tx;
    const int n3 = g.n3p;
    const int W = 3 * TX;  // elements per z row of the tile
    cx<T>* buf0 = reinterpret_cast<cx<T>*>(smem_raw);
    cx<T>* buf1 = buf0 + (size_t)n3 * W;
    double* red = reinterpret_cast<double*>(buf1 + (size_t)n3 * W);
    const int x0 = bi.x * TX;
    const int y = bi.y;
    const int row = bi.z - 3 * pb;  // tensor row i: components 3i, 3i+1, 3i+2
    const int64_t zstride = (int64_t)g.n2 * g.nhp;
    cx<T>* base = a.spec + (int64_t)(3 * row) * g.Vs + (int64_t)pb * g.n3p * zstride + (int64_t)y * g.nhp + x0;

    for (int e = threadIdx.x; e < n3 * W; e += blockDim.x) {
        const int z = e / W, r = e - z * W;
        const int c = r / TX, t = r - c * TX;
        buf0[e] = (x0 + t < g.nh) ? base[c * g.Vs + z * zstride + t] : cx<T>{(T)0, (T)0};
    }
    __syncthreads();
    cx<T>* X = fft_lines<T, false>(buf0, buf1, a.plan, W, 1, W, a.tw);

    double acc = 0.0;
    const T ay = a.sa[1][y], by = a.sb[1][y];
    for (int e = threadIdx.x; e < n3 * TX; e += blockDim.x) {
        const int z = e / TX, t = e - z * TX;
        const int xi1 = x0 + t;
        cx<T>* p = X + (size_t)z * W + t;
        if (xi1 >= g.nh) {
            p[0] = p[TX] = p[2 * TX] = cx<T>{(T)0, (T)0};
            continue;
        }
        const T ax = a.sa[0][xi1], bx = a.sb[0][xi1];
        const T az = a.sa[2][z], bz = a.sb[2][z];
        const T k0 = ax * by * bz, k1 = ay * bx * bz, k2 = az * bx * by;
        const T kk = k0 * k0 + k1 * k1 + k2 * k2;
        cx<T> X0 = p[0], X1 = p[TX], X2 = p[2 * TX];
        if (a.want_norm && xi1 == 0 && y == 0 && z == 0) {
            sc->dc[3 * row + 0] = (double)X0.x;
            sc->dc[3 * row + 1] = (double)X1.x;
            sc->dc[3 * row + 2] = (double)X2.x;
        }
        cx<T> u0, u1, u2;
        if (a.ph[0]) {
            u0 = stag_u(row, 0, a.ph[0][xi1]);
            u1 = stag_u(row, 1, a.ph[1][y]);
            u2 = stag_u(row, 2, a.ph[2][z]);
            X0 = c_mul(X0, u0);
            X1 = c_mul(X1, u1);
            X2 = c_mul(X2, u2);
        }
        cx<T> o0{(T)0, (T)0}, o1{(T)0, (T)0}, o2{(T)0, (T)0};
        if (kk > (T)0) {
            // row i of G X: k (k . X_i) / |k|^2
            const T ik = (T)1 / kk;
            const T sr = (k0 * X0.x + k1 * X1.x + k2 * X2.x) * ik;
            const T si = (k0 * X0.y + k1 * X1.y + k2 * X2.y) * ik;
            o0 = cx<T>{k0 * sr, k0 * si};
            o1 = cx<T>{k1 * sr, k1 * si};
            o2 = cx<T>{k2 * sr, k2 * si};
            if (a.ph[0]) {
                o0 = c_mul(o0, c_conj(u0));
                o1 = c_mul(o1, c_conj(u1));
                o2 = c_mul(o2, c_conj(u2));
            }
            if (a.want_norm) {
                const double wgt = (xi1 == 0 || xi1 == g.M) ? 1.0 : 2.0;
                acc += wgt * sq3(o0, o1, o2);
            }
        }
        p[0] = c_scale(o0, a.scale);
        p[TX] = c_scale(o1, a.scale);
        p[2 * TX] = c_scale(o2, a.scale);
    }
    __syncthreads();
    cx<T>* other = (X == buf0) ? buf1 : buf0;
    cx<T>* res = fft_lines<T, true>(X, other, a.plan, W, 1, W, a.tw);
    for (int e = threadIdx.x; e < n3 * W; e += blockDim.x) {
        const int z = e / W, r = e - z * W;
        const int c = r / TX, t = r - c * TX;
        if (x0 + t < g.nh) base[c * g.Vs + z * zstride + t] = res[e];
    }
    if (a.want_norm && a.partial) {
        const double s = block_sum(acc, red);
        if (threadIdx.x == 0) a.partial[bi.linear()] = s;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_zpass(ZArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    zpass_body<T>(a, VBlock::of_launch(), smem_raw);
}

// ------------------------------------------------------------- z pass + Gamma (power of two)
// Block: 3 groups (one per component of tensor row i) x TX columns x TPL
// threads; the three components are transformed concurrently.  The tile
// [3][N][TX] is both the exchange buffer and the place where the forward
// transform ends; after a barrier every frequency's three components are in
// shared memory, the projection runs in place, and each group's inverse
// transform starts from the positions its own last forward stage wrote.
template <typename T, int N, int TX>
__device__ __forceinline__ void zpass_fast_body(const ZArgs<T>& a, const VBlock& bi, unsigned char* smem_raw)
{
    const int pb = bi.z / 3;  // problem; gz = 3 nprob
    Scalars* sc = a.sc + pb;
    if (a.guard == 1 && sc->cg_done) return;
    if (a.guard == 2 && sc->outer_done) return;
    constexpr int TPL = FastPlan<N>::TPL;
    constexpr int GS = TX * TPL;  // threads per component group
    cx<T>* park = reinterpret_cast<cx<T>*>(smem_raw);  // [3][N][TX]
    double* red = reinterpret_cast<double*>(park + 3 * N * TX);
    const GridDims g = a.g;
    const int c = threadIdx.x / GS;
    const int r = threadIdx.x - c * GS;
    const int line = r % TX, tau = r / TX;
    const int x0 = bi.x * TX;
    const bool valid = x0 + line < g.nh;
    const int y = bi.y;
    const int row = bi.z - 3 * pb;
    const int64_t zst = (int64_t)g.n2 * g.nhp;
    cx<T>* bc = a.spec + (int64_t)(3 * row + c) * g.Vs + (int64_t)pb * N * zst + (int64_t)y * g.nhp + x0 + line;
    cx<T>* pc = park + c * N * TX + line;
    auto lp = [&](int e) { return pc[e * TX]; };
    auto sp = [&](int e, cx<T> v) { pc[e * TX] = v; };

    // forward along z, ending in the tile (in place: barrier inside the last stage)
    fft_fast<T, N, false, false, true>([&](int e) { return valid ? bc[e * zst] : cx<T>{(T)0, (T)0}; }, sp, lp, sp,
                                       tau, a.tw);
    __syncthreads();

    // projection: row i of G X at every (xi3, column) = k (k . X_i) / |k|^2
    double acc = 0.0;
    const T ay = a.sa[1][y], by = a.sb[1][y];
    for (int f = threadIdx.x; f < N * TX; f += blockDim.x) {
        const int z = f / TX, ln = f - z * TX;
        const int xi1 = x0 + ln;
        cx<T>* p = park + f;
        if (xi1 >= g.nh) {
            p[0] = p[N * TX] = p[2 * N * TX] = cx<T>{(T)0, (T)0};
            continue;
        }
        cx<T> X0 = p[0], X1 = p[N * TX], X2 = p[2 * N * TX];
        const T ax = a.sa[0][xi1], bx = a.sb[0][xi1];
        const T az = a.sa[2][z], bz = a.sb[2][z];
        const T k0 = ax * by * bz, k1 = ay * bx * bz, k2 = az * bx * by;
        const T kk = k0 * k0 + k1 * k1 + k2 * k2;
        if (a.want_norm && xi1 == 0 && y == 0 && z == 0) {
            sc->dc[3 * row + 0] = (double)X0.x;
            sc->dc[3 * row + 1] = (double)X1.x;
            sc->dc[3 * row + 2] = (double)X2.x;
        }
        cx<T> u0, u1, u2;
        if (a.ph[0]) {
            u0 = stag_u(row, 0, a.ph[0][xi1]);
            u1 = stag_u(row, 1, a.ph[1][y]);
            u2 = stag_u(row, 2, a.ph[2][z]);
            X0 = c_mul(X0, u0);
            X1 = c_mul(X1, u1);
            X2 = c_mul(X2, u2);
        }
        cx<T> o0{(T)0, (T)0}, o1{(T)0, (T)0}, o2{(T)0, (T)0};
        if (kk > (T)0) {
            const T ik = (T)1 / kk;
            const T sr = (k0 * X0.x + k1 * X1.x + k2 * X2.x) * ik;
            const T si = (k0 * X0.y + k1 * X1.y + k2 * X2.y) * ik;
            o0 = cx<T>{k0 * sr, k0 * si};
            o1 = cx<T>{k1 * sr, k1 * si};
            o2 = cx<T>{k2 * sr, k2 * si};
            if (a.ph[0]) {
                o0 = c_mul(o0, c_conj(u0));
                o1 = c_mul(o1, c_conj(u1));
                o2 = c_mul(o2, c_conj(u2));
            }
            if (a.want_norm) {
                const double wgt = (xi1 == 0 || xi1 == g.M) ? 1.0 : 2.0;
                acc += wgt * sq3(o0, o1, o2);
            }
        }
        p[0] = c_scale(o0, a.scale);
        p[N * TX] = c_scale(o1, a.scale);
        p[2 * N * TX] = c_scale(o2, a.scale);
    }
    __syncthreads();

    // inverse along z from the tile (in place: barrier inside the first stage)
    bool inv_done = false;
    if constexpr (std::is_same<T, df32>::value) {
        if (a.inv32) {
            // in FP32 on the rounded values: the first stage converts from the
            // double-float tile, the later ones use an FP32 view of it (the
            // barrier inside the first stage orders every load before it)
            float2* pc32 = reinterpret_cast<float2*>(park) + c * N * TX + line;
            fft_fast<float, N, true, true, false>(
                [&](int e) {
                    const cx<df32> v = pc[e * TX];
                    return float2{v.x.hi + v.x.lo, v.y.hi + v.y.lo};
                },
                [&](int e, float2 v) {
                    if (valid) bc[e * zst] = cx<df32>{df32(v.x, 0.f), df32(v.y, 0.f)};
                },
                [&](int e) { return pc32[e * TX]; }, [&](int e, float2 v) { pc32[e * TX] = v; }, tau, a.tw32);
            inv_done = true;
        }
    }
    if (!inv_done)
        fft_fast<T, N, true, true, false>(lp,
                                          [&](int e, cx<T> v) {
                                              if (valid) bc[e * zst] = v;
                                          },
                                          lp, sp, tau, a.tw);
    if (a.want_norm && a.partial) {
        const double s = block_sum(acc, red);
        if (threadIdx.x == 0) a.partial[bi.linear()] = s;
    }
}

template <typename T, int N, int TX>
__global__ void __launch_bounds__(3 * TX * FastPlan<N>::TPL) k_zpass_fast(ZArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    zpass_fast_body<T, N, TX>(a, VBlock::of_launch(), smem_raw);
}

// ------------------------------------------------------------- launch configuration
template <typename T> int ytx_fast(int n) { return sizeof(T) == 4 ? 16 : 8; }
// z-pass columns per block: 3 * N * TX complex values of shared memory (48 KB
// at N >= 256)
template <typename T> constexpr int ztx_const(int n)
{
    return sizeof(T) == 4 ? (n == 512 ? 4 : (n == 256 ? 8 : 16)) : (n == 512 ? 4 : (n == 256 ? 4 : 8));
}
template <typename T> int ztx_fast(int n) { return ztx_const<T>(n); }

// z-pass blocks per problem of a launch that is not TMA-tiled (a launch
// that accumulates norm partials writes one per block): the power-of-two
// kernels fix their tile width by the line length, the generic one takes tx
int zpass_blocks(const GridDims& g, int tx, size_t cxbytes)
{
    const int t = fast_size(g.n3p) ? (cxbytes == 8 ? ztx_const<float>(g.n3p) : ztx_const<double>(g.n3p)) : tx;
    return ((g.nh + t - 1) / t) * g.n2 * 3;
}

int zpass_tx(int n, size_t cxbytes)
{
    if (fast_size(n)) return cxbytes == 8 ? ztx_fast<float>(n) : ztx_fast<double>(n);
    int tx = 16;
    while (tx > 1 && 2 * (size_t)3 * n * tx * cxbytes > 96 * 1024) tx /= 2;
    return tx;
}

int ypass_tx(int n, size_t cxbytes)
{
    if (fast_size(n)) return cxbytes == 8 ? ytx_fast<float>(n) : ytx_fast<double>(n);
    int tx = 16;
    while (tx > 1 && 2 * (size_t)n * tx * cxbytes > 64 * 1024) tx /= 2;
    return tx;
}


template <typename T, int N, bool INV> static void ypass_fast_launch(const YArgs<T>& a, cudaStream_t st)
{
    constexpr int TX = sizeof(T) == 4 ? 16 : 8;
    dim3 grid((a.g.nh + TX - 1) / TX, a.g.n3, 9);
    const size_t sm = (size_t)N * TX * sizeof(cx<T>);
    static bool attr = false;
    allow_smem(k_ypass_fast<T, N, TX, INV>, attr);
    k_ypass_fast<T, N, TX, INV><<<grid, TX * FastPlan<N>::TPL, sm, st>>>(a);
}

template <typename T, bool INV> void launch_ypass(const YArgs<T>& a, cudaStream_t st)
{
    if constexpr (sizeof(T) == 4) {
        if (a.tmap && zpass_tma_size(a.g.n2)) {
            launch_ypass_tma<INV>(a, a.tmap, st);
            return;
        }
    }
    switch (a.g.n2) {
        case 64: ypass_fast_launch<T, 64, INV>(a, st); return;
        case 128: ypass_fast_launch<T, 128, INV>(a, st); return;
        case 256: ypass_fast_launch<T, 256, INV>(a, st); return;
        case 512: ypass_fast_launch<T, 512, INV>(a, st); return;
        default: break;
    }
    dim3 grid((a.g.nh + a.tx - 1) / a.tx, a.g.n3, 9);
    const size_t sm = 2 * (size_t)a.g.n2 * a.tx * sizeof(cx<T>);
    static bool attr = false;
    allow_smem(k_ypass<T, INV>, attr);
    k_ypass<T, INV><<<grid, 256, sm, st>>>(a);
}

template <typename T, int N> static void zpass_fast_launch(const ZArgs<T>& a, cudaStream_t st)
{
    constexpr int TX = ztx_const<T>(N);
    dim3 grid((a.g.nh + TX - 1) / TX, a.g.n2, 3 * a.g.nprob);
    static_assert(sizeof(cx<T>) != 8 || TX == ztx_const<float>(N), "zpass_blocks tile width");
    const size_t sm = (size_t)3 * N * TX * sizeof(cx<T>) + 64 * sizeof(double);
    static bool attr = false;
    allow_smem(k_zpass_fast<T, N, TX>, attr);
    k_zpass_fast<T, N, TX><<<grid, 3 * TX * FastPlan<N>::TPL, sm, st>>>(a);
}

template <typename T> void launch_zpass(const ZArgs<T>& a, cudaStream_t st)
{
    if constexpr (sizeof(T) == 4) {
        if (a.tmap && !a.want_norm && zpass_tma_size(a.g.n3p)) {
            launch_zpass_tma(a, a.tmap, st);
            return;
        }
    }
    switch (a.g.n3p) {
        case 64: zpass_fast_launch<T, 64>(a, st); return;
        case 128: zpass_fast_launch<T, 128>(a, st); return;
        case 256: zpass_fast_launch<T, 256>(a, st); return;
        case 512: zpass_fast_launch<T, 512>(a, st); return;
        default: break;
    }
    dim3 grid((a.g.nh + a.tx - 1) / a.tx, a.g.n2, 3 * a.g.nprob);
    const size_t sm = 2 * (size_t)a.g.n3p * 3 * a.tx * sizeof(cx<T>) + 64 * sizeof(double);
    static bool attr = false;
    allow_smem(k_zpass<T>, attr);
    k_zpass<T><<<grid, 256, sm, st>>>(a);
}

// ------------------------------------------------------------- grouped launches
// Block size of the grouped y-pass: the power-of-two body's TX x TPL for
// lengths 64 and 128 (every other length runs the generic body, which takes
// any block size); z-pass: 3 TX TPL for lengths 64, 128 and 256.
template <typename T> constexpr int group_y_threads() { return (sizeof(T) == 4 ? 16 : 8) * FastPlan<64>::TPL; }
template <typename T> constexpr int group_z_threads() { return 3 * ztx_const<T>(64) * FastPlan<64>::TPL; }
template <typename T> constexpr bool group_y_fast(int n) { return n == 64 || n == 128; }
template <typename T> constexpr bool group_z_fast(int n)
{
    return (n == 64 || n == 128 || n == 256) && 3 * ztx_const<T>(n) * (n == 256 ? 16 : 8) == group_z_threads<T>();
}

void ypass_group_shape(const GridDims& g, int tx, size_t cxbytes, int& gx, int& gy, int& gz, size_t& smem)
{
    const bool fast = (g.n2 == 64 || g.n2 == 128);
    const int t = fast ? (cxbytes == 8 ? 16 : 8) : tx;
    gx = (g.nh + t - 1) / t;
    gy = g.n3;
    gz = 9;
    smem = fast ? (size_t)g.n2 * t * cxbytes : 2 * (size_t)g.n2 * t * cxbytes;
}

void zpass_group_shape(const GridDims& g, int tx, size_t cxbytes, int& gx, int& gy, int& gz, size_t& smem)
{
    const int n = g.n3p;
    const bool fast = cxbytes == 8 ? group_z_fast<float>(n) : group_z_fast<double>(n);
    const int t = fast ? (cxbytes == 8 ? ztx_const<float>(n) : ztx_const<double>(n)) : tx;
    gx = (g.nh + t - 1) / t;
    gy = g.n2;
    gz = 3 * g.nprob;
    smem = fast ? (size_t)3 * n * t * cxbytes + 64 * sizeof(double)
                : 2 * (size_t)n * 3 * t * cxbytes + 64 * sizeof(double);
}

template <typename T, bool INV>
__global__ void __launch_bounds__(group_y_threads<T>())
    k_group_ypass(const YArgs<T>* __restrict__ args, const int* __restrict__ vstart, const int* __restrict__ dims,
                  int nd)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int TX = sizeof(T) == 4 ? 16 : 8;
    const int total = __ldg(vstart + nd);
    for (int v = blockIdx.x; v < total; v += gridDim.x) {
        const int d = group_of(vstart, nd, v);
        const YArgs<T>& a = args[d];
        const VBlock bi = VBlock::of_item(v - __ldg(vstart + d), __ldg(dims + 2 * d), __ldg(dims + 2 * d + 1), 9);
        switch (a.g.n2) {
            case 64: ypass_fast_body<T, 64, TX, INV>(a, bi, smem_raw); break;
            case 128: ypass_fast_body<T, 128, TX, INV>(a, bi, smem_raw); break;
            default: ypass_body<T, INV>(a, bi, smem_raw); break;
        }
        __syncthreads();
    }
}

template <typename T>
__global__ void __launch_bounds__(group_z_threads<T>())
    k_group_zpass(const ZArgs<T>* __restrict__ args, const int* __restrict__ vstart, const int* __restrict__ dims,
                  int nd)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int total = __ldg(vstart + nd);
    for (int v = blockIdx.x; v < total; v += gridDim.x) {
        const int d = group_of(vstart, nd, v);
        const ZArgs<T>& a = args[d];
        const VBlock bi = VBlock::of_item(v - __ldg(vstart + d), __ldg(dims + 2 * d), __ldg(dims + 2 * d + 1),
                                          3 * a.g.nprob);
        const int n = a.g.n3p;
        if (n == 64 && group_z_fast<T>(64))
            zpass_fast_body<T, 64, ztx_const<T>(64)>(a, bi, smem_raw);
        else if (n == 128 && group_z_fast<T>(128))
            zpass_fast_body<T, 128, ztx_const<T>(128)>(a, bi, smem_raw);
        else if (n == 256 && group_z_fast<T>(256))
            zpass_fast_body<T, 256, ztx_const<T>(256)>(a, bi, smem_raw);
        else
            zpass_body<T>(a, bi, smem_raw);
        __syncthreads();
    }
}

template <typename T, bool INV> void launch_group_ypass(const GroupTab<YArgs<T>>& t, cudaStream_t st)
{
    if (t.total <= 0) return;
    auto k = k_group_ypass<T, INV>;
    constexpr int th = group_y_threads<T>();
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t.smem);
    k<<<group_grid((const void*)k, th, t.smem, t.total), th, t.smem, st>>>(t.args, t.vstart, t.dims, t.nd);
}

template <typename T> void launch_group_zpass(const GroupTab<ZArgs<T>>& t, cudaStream_t st)
{
    if (t.total <= 0) return;
    auto k = k_group_zpass<T>;
    constexpr int th = group_z_threads<T>();
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t.smem);
    k<<<group_grid((const void*)k, th, t.smem, t.total), th, t.smem, st>>>(t.args, t.vstart, t.dims, t.nd);
}

template void launch_group_ypass<float, false>(const GroupTab<YArgs<float>>&, cudaStream_t);
template void launch_group_ypass<float, true>(const GroupTab<YArgs<float>>&, cudaStream_t);
template void launch_group_ypass<double, false>(const GroupTab<YArgs<double>>&, cudaStream_t);
template void launch_group_ypass<double, true>(const GroupTab<YArgs<double>>&, cudaStream_t);
template void launch_group_ypass<df32, false>(const GroupTab<YArgs<df32>>&, cudaStream_t);
template void launch_group_ypass<df32, true>(const GroupTab<YArgs<df32>>&, cudaStream_t);
template void launch_group_zpass<float>(const GroupTab<ZArgs<float>>&, cudaStream_t);
template void launch_group_zpass<double>(const GroupTab<ZArgs<double>>&, cudaStream_t);
template void launch_group_zpass<df32>(const GroupTab<ZArgs<df32>>&, cudaStream_t);

template void launch_ypass<double, false>(const YArgs<double>&, cudaStream_t);
template void launch_ypass<double, true>(const YArgs<double>&, cudaStream_t);
template void launch_ypass<float, false>(const YArgs<float>&, cudaStream_t);
template void launch_ypass<float, true>(const YArgs<float>&, cudaStream_t);
template void launch_zpass<double>(const ZArgs<double>&, cudaStream_t);
template void launch_zpass<float>(const ZArgs<float>&, cudaStream_t);
template void launch_ypass<df32, false>(const YArgs<df32>&, cudaStream_t);
template void launch_ypass<df32, true>(const YArgs<df32>&, cudaStream_t);
template void launch_zpass<df32>(const ZArgs<df32>&, cudaStream_t);

}  // namespace combo
