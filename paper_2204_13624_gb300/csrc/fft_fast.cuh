// fft_fast.cuh -- compile-time power-of-two FFT plans for the hot sizes.
//
// A line of N complex values is transformed by TPL = N / max(R) threads with
// a self-sorting Stockham decomposition whose radices are template
// constants (N = 64: 8x8, 128: 16x8, 256: 16x16, 512: 8x8x8), so every index
// is a shift or a mask.  Each stage keeps its R values in registers and runs
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

// DFT of size R in registers, natural order in and out (radix-2 decimation in time).
template <int R, bool INV> struct RegDFT {
    template <typename V> static __device__ __forceinline__ void run(V* v)
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
    static constexpr int NST = 3, R0 = 8, R1 = 8, R2 = 8, TPL = 64;
};

__host__ __device__ constexpr bool fast_size(int n) { return n == 64 || n == 128 || n == 256 || n == 512; }
__host__ __device__ constexpr bool fast_size_x(int m) { return m == 32 || m == 64 || m == 128 || m == 256; }

// Radix of stage s of the forward (INV = false) or inverse (reversed) plan.
template <int N, bool INV, int S> struct StageR {
    using P = FastPlan<N>;
    static constexpr int FWD = (S == 0) ? P::R0 : ((S == 1) ? P::R1 : P::R2);
    static constexpr int RS = INV ? ((P::NST - 1 - S == 0) ? P::R0 : ((P::NST - 1 - S == 1) ? P::R1 : P::R2)) : FWD;
};

// Load phase of one stage (radix R, NS = product of the earlier radices):
// inputs j + t (N/R) of butterflies j = tau + TPL u, twiddled and transformed.
template <typename T, int N, int R, int NS, int TPL, bool INV, class LD>
__device__ __forceinline__ void stage_load(cx<T> (&v)[(N / R) / TPL][R], const LD& ld, int tau,
                                           const cx<T>* __restrict__ tw)
{
    constexpr int B = N / R;
    constexpr int U = B / TPL;
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
            const int k = j & (NS - 1);
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
        const int d = (j / NS) * NS * R + (j & (NS - 1));
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
// reusing the exchange buffer.
template <typename T, int N, bool INV, bool SYNC_FIRST = false, bool SYNC_LAST = false, class LG, class SG, class LX,
          class SX>
__device__ __forceinline__ void fft_fast(const LG& lg, const SG& sg, const LX& lx, const SX& sx, int tau,
                                         const cx<T>* __restrict__ tw)
{
    using P = FastPlan<N>;
    constexpr int TPL = P::TPL;
    constexpr int RA = StageR<N, INV, 0>::RS;
    if constexpr (P::NST == 2) {
        constexpr int RB = StageR<N, INV, 1>::RS;
        {
            cx<T> v[(N / RA) / TPL][RA];
            stage_load<T, N, RA, 1, TPL, INV>(v, lg, tau, tw);
            if constexpr (SYNC_FIRST) __syncthreads();
            stage_store<T, N, RA, 1, TPL>(v, sx, tau);
        }
        __syncthreads();
        {
            cx<T> v[(N / RB) / TPL][RB];
            stage_load<T, N, RB, RA, TPL, INV>(v, lx, tau, tw);
            if constexpr (SYNC_LAST) __syncthreads();
            stage_store<T, N, RB, RA, TPL>(v, sg, tau);
        }
    } else {
        constexpr int RB = StageR<N, INV, 1>::RS;
        constexpr int RC = StageR<N, INV, 2>::RS;
        {
            cx<T> v[(N / RA) / TPL][RA];
            stage_load<T, N, RA, 1, TPL, INV>(v, lg, tau, tw);
            if constexpr (SYNC_FIRST) __syncthreads();
            stage_store<T, N, RA, 1, TPL>(v, sx, tau);
        }
        __syncthreads();
        {
            cx<T> v[(N / RB) / TPL][RB];
            stage_load<T, N, RB, RA, TPL, INV>(v, lx, tau, tw);
            __syncthreads();
            stage_store<T, N, RB, RA, TPL>(v, sx, tau);
        }
        __syncthreads();
        {
            cx<T> v[(N / RC) / TPL][RC];
            stage_load<T, N, RC, RA * RB, TPL, INV>(v, lx, tau, tw);
            if constexpr (SYNC_LAST) __syncthreads();
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
    using P = FastPlan<N>;
    constexpr int TPL = P::TPL;
    const int tid = threadIdx.x, nthr = blockDim.x;
    cx<T>* src = b0;
    cx<T>* dst = b1;
    auto one = [&](auto stage_tag) {
        constexpr int S = decltype(stage_tag)::value;
        constexpr int R = StageR<N, INV, S>::RS;
        constexpr int NS = (S == 0) ? 1 : ((S == 1) ? StageR<N, INV, 0>::RS : StageR<N, INV, 0>::RS * StageR<N, INV, 1>::RS);
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
