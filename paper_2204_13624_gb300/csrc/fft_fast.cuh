// fft_fast.cuh -- compile-time power-of-two FFT plans for the hot sizes.
//
// A line of N complex values is transformed by TPL threads with a
// self-sorting Stockham decomposition whose radices are template constants:
// powers of two (N = 64: 8x8, 128: 16x8, 256: 16x16, 512: 8x8x8), where every
// index is a shift or a mask, and 2^a 3^b lengths of the grids between them
// (48: 12x4, 72: 12x6, 96: 4x4x6, 108: 6x6x3, 144: 12x12, 192: 4x4x12,
// 216: 6x6x6, and the half lengths 24 .. 108 of the x transforms), whose
// register DFTs of sizes 3, 6, 12 split by radices 2 and 3 with the
// constants cos(2 pi m / 144).  Each stage keeps its R values in registers and runs
// a register DFT of size R; consecutive stages exchange through shared
// memory.  The first stage may read global memory directly and the last one
// may write it directly.  The last forward stage leaves thread tau holding
// the frequencies j + t (N / R_last), j = tau + TPL u, which are exactly the
// inputs of the first stage of the inverse plan (radices reversed), so a
// pointwise operation between the two needs no exchange.
#pragma once
#include <type_traits>

#include "combo_internal.cuh"

namespace combo {

// cos(2 pi m / 32) for integer m (mathematical constants, folded at compile time)
__host__ __device__ __forceinline__ constexpr double kcos32(int m)
{
    m &= 31;
    constexpr double C[9] = {1.0,
                             0.9807852804032304491262,
                             0.9238795325112867561282,
                             0.8314696123025452370788,
                             0.7071067811865475244008,
                             0.5555702330196022247428,
                             0.3826834323650897717285,
                             0.1950903220161282678483,
                             0.0};
    return m <= 8 ? C[m] : (m <= 16 ? -C[16 - m] : (m <= 24 ? -C[m - 16] : C[32 - m]));
}
__host__ __device__ __forceinline__ constexpr double ksin32(int m) { return kcos32(m - 8); }

// cos(2 pi m / 144) for integer m (mathematical constants): the twiddles of
// register DFTs whose size divides 144
__host__ __device__ __forceinline__ constexpr double kcos144(int m)
{
    m %= 144;
    if (m < 0) m += 144;
    constexpr double C[37] = {
                             1.000000000000000000000,
                             0.9990482215818577624037,
                             0.9961946980917455322950,
                             0.9914448613738104111446,
                             0.9848077530122080593667,
                             0.9762960071199333659709,
                             0.9659258262890682867497,
                             0.9537169507482269211438,
                             0.9396926207859083840541,
                             0.9238795325112867561282,
                             0.9063077870366499632426,
                             0.8870108331782217010546,
                             0.8660254037844386467637,
                             0.8433914458128857012729,
                             0.8191520442889917896845,
                             0.7933533402912351645798,
                             0.7660444431189780352024,
                             0.7372773368101240413843,
                             0.7071067811865475244008,
                             0.6755902076156602443483,
                             0.6427876096865393263226,
                             0.6087614290087206394161,
                             0.5735764363510460961080,
                             0.5372996083468238318408,
                             0.5000000000000000000000,
                             0.4617486132350339305629,
                             0.4226182617406994361870,
                             0.3826834323650897717285,
                             0.3420201433256687330441,
                             0.3007057995042731216225,
                             0.2588190451025207623489,
                             0.2164396139381028797596,
                             0.1736481776669303488517,
                             0.1305261922200515915484,
                             0.08715574274765817355806,
                             0.04361938736533599978175,
                             0.0};
    return m <= 36 ? C[m] : (m <= 72 ? -C[72 - m] : (m <= 108 ? -C[m - 72] : C[144 - m]));
}
__host__ __device__ __forceinline__ constexpr double ksin144(int m) { return kcos144(m - 36); }

__host__ __device__ constexpr bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// v * exp(-/+ 2 pi i m / 144) (forward / inverse)
template <bool INV, typename V> __device__ __forceinline__ V tw144(V o, int m)
{
    typedef decltype(o.x) S;
    const S cr = (S)kcos144(m), si = (S)ksin144(m);
    return INV ? V{o.x * cr - o.y * si, o.x * si + o.y * cr} : V{o.x * cr + o.y * si, o.y * cr - o.x * si};
}

// DFT of size R in registers, natural order in and out: decimation in time by
// radix 2 (powers of two: constants cos(2 pi m / 32); even sizes with a factor
// 3: cos(2 pi m / 144)) or by radix 3 (odd sizes).
template <int R, bool INV> struct RegDFT {
    template <typename V> static __device__ __forceinline__ void run(V* v)
    {
        if constexpr (is_pow2(R)) {
            run_pow2(v);
        } else if constexpr (R == 3) {
            dft3<INV>(v);
        } else if constexpr (R % 2 == 0) {
            static_assert(144 % R == 0, "register DFT size must divide 144");
            V e[R / 2], o[R / 2];
#pragma unroll
            for (int k = 0; k < R / 2; k++) {
                e[k] = v[2 * k];
                o[k] = v[2 * k + 1];
            }
            RegDFT<R / 2, INV>::run(e);
            RegDFT<R / 2, INV>::run(o);
#pragma unroll
            for (int k = 0; k < R / 2; k++) {
                const V t = (k == 0) ? o[0] : (4 * k == R ? c_rot<INV>(o[k]) : tw144<INV>(o[k], k * (144 / R)));
                v[k] = c_add(e[k], t);
                v[k + R / 2] = c_sub(e[k], t);
            }
        } else {
            static_assert(R % 3 == 0 && 144 % R == 0, "odd register DFT sizes: 3, 9");
            constexpr int Q = R / 3;
            V x0[Q], x1[Q], x2[Q];
#pragma unroll
            for (int k = 0; k < Q; k++) {
                x0[k] = v[3 * k];
                x1[k] = v[3 * k + 1];
                x2[k] = v[3 * k + 2];
            }
            RegDFT<Q, INV>::run(x0);
            RegDFT<Q, INV>::run(x1);
            RegDFT<Q, INV>::run(x2);
#pragma unroll
            for (int k = 0; k < Q; k++) {
                V y[3] = {x0[k], k == 0 ? x1[0] : tw144<INV>(x1[k], k * (144 / R)),
                          k == 0 ? x2[0] : tw144<INV>(x2[k], 2 * k * (144 / R))};
                dft3<INV>(y);
                v[k] = y[0];
                v[k + Q] = y[1];
                v[k + 2 * Q] = y[2];
            }
        }
    }
    template <typename V> static __device__ __forceinline__ void run_pow2(V* v)
    {
        typedef decltype(v[0].x) S;
        V e[R / 2], o[R / 2];
#pragma unroll
        for (int k = 0; k < R / 2; k++) {
            e[k] = v[2 * k];
            o[k] = v[2 * k + 1];
        }
        RegDFT<R / 2, INV>::run(e);
        RegDFT<R / 2, INV>::run(o);
#pragma unroll
        for (int k = 0; k < R / 2; k++) {
            V t;
            if (k == 0) {
                t = o[0];
            } else if (4 * k == R) {
                t = c_rot<INV>(o[k]);
            } else {
                const S cr = (S)kcos32(k * (32 / R)), si = (S)ksin32(k * (32 / R));
                // forward: o * (cos - i sin); inverse: o * (cos + i sin)
                t = INV ? V{o[k].x * cr - o[k].y * si, o[k].x * si + o[k].y * cr}
                        : V{o[k].x * cr + o[k].y * si, o[k].y * cr - o[k].x * si};
            }
            v[k] = c_add(e[k], t);
            v[k + R / 2] = c_sub(e[k], t);
        }
    }
};
template <bool INV> struct RegDFT<1, INV> {
    template <typename V> static __device__ __forceinline__ void run(V*) {}
    template <typename V> static __device__ __forceinline__ void run_pow2(V*) {}
};

template <int N> struct FastPlan;
template <> struct FastPlan<32> {
    static constexpr int NST = 2, R0 = 8, R1 = 4, R2 = 1, TPL = 4;
};
template <> struct FastPlan<64> {
    static constexpr int NST = 2, R0 = 8, R1 = 8, R2 = 1, TPL = 8;
};
template <> struct FastPlan<128> {
    static constexpr int NST = 2, R0 = 16, R1 = 8, R2 = 1, TPL = 8;
};
template <> struct FastPlan<256> {
    static constexpr int NST = 2, R0 = 16, R1 = 16, R2 = 1, TPL = 16;
};
template <> struct FastPlan<512> {
    static constexpr int NST = 3, R0 = 8, R1 = 8, R2 = 8, TPL = 32;  // two butterflies per thread and stage
};
// 2^a 3^b lengths: every stage's butterfly count N / R is a multiple of TPL
template <> struct FastPlan<24> {
    static constexpr int NST = 2, R0 = 6, R1 = 4, R2 = 1, TPL = 2;
};
template <> struct FastPlan<36> {
    static constexpr int NST = 2, R0 = 6, R1 = 6, R2 = 1, TPL = 6;
};
template <> struct FastPlan<48> {
    static constexpr int NST = 2, R0 = 12, R1 = 4, R2 = 1, TPL = 4;
};
template <> struct FastPlan<54> {
    static constexpr int NST = 3, R0 = 3, R1 = 3, R2 = 6, TPL = 9;
};
template <> struct FastPlan<72> {
    static constexpr int NST = 2, R0 = 12, R1 = 6, R2 = 1, TPL = 6;
};
template <> struct FastPlan<96> {
    static constexpr int NST = 3, R0 = 4, R1 = 4, R2 = 6, TPL = 8;
};
template <> struct FastPlan<108> {
    static constexpr int NST = 3, R0 = 6, R1 = 6, R2 = 3, TPL = 18;
};
template <> struct FastPlan<144> {
    static constexpr int NST = 2, R0 = 12, R1 = 12, R2 = 1, TPL = 12;
};
template <> struct FastPlan<192> {
    static constexpr int NST = 3, R0 = 4, R1 = 4, R2 = 12, TPL = 16;
};
template <> struct FastPlan<216> {
    static constexpr int NST = 3, R0 = 6, R1 = 6, R2 = 6, TPL = 36;
};

__host__ __device__ constexpr bool fast_size(int n) { return n == 64 || n == 128 || n == 256 || n == 512; }
__host__ __device__ constexpr bool fast_size_x(int m) { return m == 32 || m == 64 || m == 128 || m == 256; }
// 2^a 3^b lengths with compile-time plans on the FP32 Krylov passes (the
// TMA-tiled y- and z-passes, the x-forward tangent pass and the x-inverse)
__host__ __device__ constexpr bool fast3_size(int n)
{
    return n == 48 || n == 72 || n == 96 || n == 108 || n == 144 || n == 192 || n == 216;
}
__host__ __device__ constexpr bool fast3_size_x(int m)
{
    return m == 24 || m == 36 || m == 48 || m == 54 || m == 72 || m == 96 || m == 108;
}

// Radix of stage s of the forward (INV = false) or inverse (reversed) plan.
template <class P, bool INV, int S> struct StageRP {
    static constexpr int FWD = (S == 0) ? P::R0 : ((S == 1) ? P::R1 : P::R2);
    static constexpr int RS = INV ? ((P::NST - 1 - S == 0) ? P::R0 : ((P::NST - 1 - S == 1) ? P::R1 : P::R2)) : FWD;
};
template <int N, bool INV, int S> struct StageR : StageRP<FastPlan<N>, INV, S> {};

// Plans for 8-byte words (FP64, double-float): at N = 128 and 256 the radix-16
// register DFTs of those words are long enough that the z-pass stalled on
// instruction fetch; radix 8 / 4 stages with the same threads per line
struct FastPlanW128 {
    static constexpr int NST = 3, R0 = 8, R1 = 4, R2 = 4, TPL = 8;
};
struct FastPlanW256 {
    static constexpr int NST = 3, R0 = 8, R1 = 8, R2 = 4, TPL = 16;
};
template <int N> struct WidePlan {
    using type = FastPlan<N>;
};
template <> struct WidePlan<128> {
    using type = FastPlanW128;
};
template <> struct WidePlan<256> {
    using type = FastPlanW256;
};
template <typename T, int N>
using PlanOf = typename std::conditional<(sizeof(T) >= 8), typename WidePlan<N>::type, FastPlan<N>>::type;

// Load phase of one stage (radix R, NS = product of the earlier radices):
// inputs j + t (N/R) of butterflies j = tau + TPL u, twiddled and transformed.
template <typename T, int N, int R, int NS, int TPL, bool INV, class LD>
__device__ __forceinline__ void stage_load(cx<T> (&v)[(N / R) / TPL][R], const LD& ld, int tau,
                                           const cx<T>* __restrict__ tw)
{
    constexpr int B = N / R;
    constexpr int U = B / TPL;
    static_assert(B % TPL == 0, "every stage gives each thread whole butterflies");
#pragma unroll
    for (int u = 0; u < U; u++) {
        const int j = tau + TPL * u;
#pragma unroll
        for (int t = 0; t < R; t++) v[u][t] = ld(j + t * B);
    }
#pragma unroll
    for (int u = 0; u < U; u++) {
        const int j = tau + TPL * u;
        if (NS > 1) {
            const int k = (int)((unsigned)j % (unsigned)NS);
#pragma unroll
            for (int t = 1; t < R; t++) {
                cx<T> w = tw[t * k * (N / (NS * R))];
                if (INV) w.y = -w.y;
                v[u][t] = c_mul(v[u][t], w);
            }
        }
        RegDFT<R, INV>::run(v[u]);
    }
}

// Store phase: outputs (j / NS) NS R + (j mod NS) + t NS.
template <typename T, int N, int R, int NS, int TPL, class ST>
__device__ __forceinline__ void stage_store(cx<T> (&v)[(N / R) / TPL][R], const ST& st, int tau)
{
    constexpr int B = N / R;
    constexpr int U = B / TPL;
#pragma unroll
    for (int u = 0; u < U; u++) {
        const int j = tau + TPL * u;
        const int d = (int)((unsigned)j / (unsigned)NS) * NS * R + (int)((unsigned)j % (unsigned)NS);
#pragma unroll
        for (int t = 0; t < R; t++) st(d + t * NS, v[u][t]);
    }
}

// Whole transform of one line by the TPL threads tau = 0..TPL-1 of a group.
// lg / sg: first-stage input and last-stage output accessors; lx / sx: the
// exchange buffer of this line.  SYNC_FIRST / SYNC_LAST put a block barrier
// between the loads and the stores of the first / last stage, for when lg or
// sg alias the exchange buffer.  Every thread of the block must call it with
// the same plan (it holds __syncthreads); the caller synchronises before
// reusing the exchange buffer.  NBAR > 0: the calling threads are only the
// first NBAR of the block (a multiple of 32), which synchronise on named
// barrier 1 instead; the rest of the block must not use that barrier meanwhile.
template <int NBAR> __device__ __forceinline__ void fft_sync()
{
    if constexpr (NBAR == 0)
        __syncthreads();
    else
        asm volatile("bar.sync 1, %0;" ::"n"(NBAR) : "memory");
}

template <typename T, int N, bool INV, bool SYNC_FIRST = false, bool SYNC_LAST = false, int NBAR = 0, class LG,
          class SG, class LX, class SX>
__device__ __forceinline__ void fft_fast(const LG& lg, const SG& sg, const LX& lx, const SX& sx, int tau,
                                         const cx<T>* __restrict__ tw)
{
    using P = PlanOf<T, N>;
    constexpr int TPL = P::TPL;
    constexpr int RA = StageRP<P, INV, 0>::RS;
    if constexpr (P::NST == 2) {
        constexpr int RB = StageRP<P, INV, 1>::RS;
        {
            cx<T> v[(N / RA) / TPL][RA];
            stage_load<T, N, RA, 1, TPL, INV>(v, lg, tau, tw);
            if constexpr (SYNC_FIRST) fft_sync<NBAR>();
            stage_store<T, N, RA, 1, TPL>(v, sx, tau);
        }
        fft_sync<NBAR>();
        {
            cx<T> v[(N / RB) / TPL][RB];
            stage_load<T, N, RB, RA, TPL, INV>(v, lx, tau, tw);
            if constexpr (SYNC_LAST) fft_sync<NBAR>();
            stage_store<T, N, RB, RA, TPL>(v, sg, tau);
        }
    } else {
        constexpr int RB = StageRP<P, INV, 1>::RS;
        constexpr int RC = StageRP<P, INV, 2>::RS;
        {
            cx<T> v[(N / RA) / TPL][RA];
            stage_load<T, N, RA, 1, TPL, INV>(v, lg, tau, tw);
            if constexpr (SYNC_FIRST) fft_sync<NBAR>();
            stage_store<T, N, RA, 1, TPL>(v, sx, tau);
        }
        fft_sync<NBAR>();
        {
            cx<T> v[(N / RB) / TPL][RB];
            stage_load<T, N, RB, RA, TPL, INV>(v, lx, tau, tw);
            fft_sync<NBAR>();
            stage_store<T, N, RB, RA, TPL>(v, sx, tau);
        }
        fft_sync<NBAR>();
        {
            cx<T> v[(N / RC) / TPL][RC];
            stage_load<T, N, RC, RA * RB, TPL, INV>(v, lx, tau, tw);
            if constexpr (SYNC_LAST) fft_sync<NBAR>();
            stage_store<T, N, RC, RA * RB, TPL>(v, sg, tau);
        }
    }
}

// Positions held by thread tau after the last forward stage (= inputs of the
// first inverse stage): j + t (N / R_last), j = tau + TPL u.
template <int N> struct LastStage {
    using P = FastPlan<N>;
    static constexpr int R = (P::NST == 2) ? P::R1 : P::R2;
    static constexpr int B = N / R;
    static constexpr int U = B / P::TPL;
};

// Many lines held in shared memory (line q at buf + q*ls, unit stride), ping-
// pong between b0 and b1; every block thread takes (line, tau) pairs.
// Returns the buffer that holds the result; ends with __syncthreads().
template <typename T, int N, bool INV>
__device__ cx<T>* fft_lines_fast(cx<T>* b0, cx<T>* b1, int nl, int ls, const cx<T>* __restrict__ tw)
{
    using P = PlanOf<T, N>;
    constexpr int TPL = P::TPL;
    const int tid = threadIdx.x, nthr = blockDim.x;
    cx<T>* src = b0;
    cx<T>* dst = b1;
    auto one = [&](auto stage_tag) {
        constexpr int S = decltype(stage_tag)::value;
        constexpr int R = StageRP<P, INV, S>::RS;
        constexpr int NS = (S == 0) ? 1 : ((S == 1) ? StageRP<P, INV, 0>::RS : StageRP<P, INV, 0>::RS * StageRP<P, INV, 1>::RS);
        for (int p = tid; p < nl * TPL; p += nthr) {
            const int q = p % nl, tau = p / nl;
            const cx<T>* s = src + (size_t)q * ls;
            cx<T>* d = dst + (size_t)q * ls;
            cx<T> v[(N / R) / TPL][R];
            stage_load<T, N, R, NS, TPL, INV>(v, [&](int e) { return s[e]; }, tau, tw);
            stage_store<T, N, R, NS, TPL>(v, [&](int e, cx<T> x) { d[e] = x; }, tau);
        }
        __syncthreads();
        cx<T>* t = src;
        src = dst;
        dst = t;
    };
    one(std::integral_constant<int, 0>{});
    one(std::integral_constant<int, 1>{});
    if constexpr (P::NST == 3) one(std::integral_constant<int, 2>{});
    return src;
}

}  // namespace combo
