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
// The kernel gets them from XOR masks of neighbouring bit rows and byte tables
// of bit-position sums (branch-free, so a warp never waits on its densest
// lane); M about the
// weighted barycentre is S2 - S1 S1^T / S0 in FP64 and its smallest
// eigenvector comes from cyclic Jacobi rotations.  The barycentre normal is
// -(h o Q) / |h o Q| with Q the integer sum of q over the inclusion voxels
// (the offsets of all voxels of a boxel sum to zero).
//
// Work layout.  A streaming pass packs the image to one bit per fine voxel
// (16-byte loads, the image read from HBM once).  Then one CTA per slab (J, K)
// of coarse voxels (all I along x) copies the bit rows of the slab and its
// one-voxel halo (periodic in y and z; x wraps inside a row) to shared
// memory.  Coarse voxels are counted with popcounts, and each composite boxel's integer sums are
// accumulated by a group of G lanes and written to a dense per-coarse-voxel
// scratch.  A one-CTA scan of the per-slab counts and a scatter kernel list
// the boxels in increasing coarse index; a last kernel finishes one boxel per
// thread (eigenvector, sign, c+), so the scarce FP64 pipe runs full warps.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>

#include "combo.h"
#include "combo_internal.cuh"

namespace combo {
namespace {

constexpr int CG_THREADS = 256;
constexpr int SCAN_THREADS = 1024;
constexpr int SCATTER_THREADS = 256;
constexpr size_t CG_SMEM_MAX = 200 * 1024;
constexpr int FIN_THREADS = 256;
// Per-boxel integer sums: [0..2] Q (sum of q over the inclusion voxels), then
// per axis i the ten moments T0, T1x, T1y, T1z, T2xx, T2xy, T2xz, T2yy, T2yz,
// T2zz of m_i, then the inclusion-voxel count; NSUM pads the record to 16 bytes.
constexpr int NACC = 33;
constexpr int NSUM = 36;

struct CgArgs {
    const uint32_t* bitimg;  // [n3][n2][nw] bit rows of the image (padded rows)
    const uint32_t* glut;    // byte tables of bit-position sums
    int n1, n2, n3;
    int b1, b2, b3;
    int nc1, nc2, nc3;
    int nwr;     // words per fine row: ceil(n1 / 32)
    int nw;      // words per padded bit row: nwr + 3 rounded up to a multiple of 4
    int G;       // lanes per composite boxel (power of two, <= 32): G = Gq b2 + Gr
    int Gq, Gr;
    int R;       // lanes per coarse voxel in the count (power of two, <= 32): R = Rq b2 + Rr
    int Rq, Rr;
    int NGq, NGr;  // column count: row groups NG = NGq b2 + NGr
    float inv_b2, inv_per, inv_nw4, inv_nwr;  // reciprocals for the divisions in the loops
    int method;  // COMBO_NORMAL_LAPLACE / COMBO_NORMAL_KABEL
    int iso;     // h1 == h2 == h3: the moments combine exactly in int64
    int nblock_pow2;  // b1 b2 b3 a power of two: c+ = count * inv_nblock exactly
    double inv_nblock;
    double h[3], r[3];
    uint8_t* phase;  // [nc]
    int* slab_cnt;   // [nc2 nc3] boxels per slab
    int* sums;       // [nc][NSUM] dense scratch: the integer sums of each boxel
};

__device__ __forceinline__ int lrow(int jj, int kk, int b2) { return (kk + 1) * (b2 + 2) + (jj + 1); }

__device__ __forceinline__ int wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

__device__ __forceinline__ uint32_t bit_at(const uint32_t* row, int x) { return (row[x >> 5] >> (x & 31)) & 1u; }

// 16 fine voxels (bytes, nonzero = inclusion) -> 16 bits, voxel x0 + k at bit k
__device__ __forceinline__ uint32_t pack16(uint4 v)
{
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    uint32_t m = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        // bit 7 of each byte: the byte is nonzero (adding 0x7F to its low
        // seven bits carries into bit 7 unless they are all zero)
        const uint32_t t = (((w[k] & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | w[k]) & 0x80808080u;
        // the product moves bits 7, 15, 23, 31 to bits 28..31 without carries
        m |= ((t * 0x00204081u) >> 28) << (4 * k);
    }
    return m;
}

// q = v / d for 0 <= v < 2^22, d >= 1, inv = 1.0f / d: the float quotient is
// within one of the exact one, so one correction either way makes it exact.
__device__ __forceinline__ int fdiv(int v, int d, float inv)
{
    int q = __float2int_rz((float)v * inv);
    const int r = v - q * d;
    return q + (r >= d) - (r < 0);
}

// Byte tables of bit-position sums.  lut[k][v] packs, for the set bits j of
// the byte v taken as positions i = 8 k + j of a 32-bit mask, the count (bits
// 0-6), sum i (bits 7-16) and sum i^2 (bits 17-31).  The fields of two
// masks' sums still fit (count <= 64, sum i <= 992, sum i^2 <= 20832), so the
// packed words of two masks add with one integer add.
constexpr int LUT_N = 4 * 256;

__device__ void build_lut(uint32_t* lut)
{
    for (int e = threadIdx.x; e < LUT_N; e += blockDim.x) {
        const uint32_t k = e >> 8, v = e & 255;
        // positions j of the set bits from the bit planes of j (0..7)
        const uint32_t p0 = v & 0xAAu, p1 = v & 0xCCu, p2 = v & 0xF0u;
        const uint32_t n = __popc(v);
        const uint32_t sj = __popc(p0) + 2 * __popc(p1) + 4 * __popc(p2);
        const uint32_t sjj = __popc(p0) + 4 * __popc(p1) + 16 * __popc(p2) + 4 * __popc(p0 & p1) +
                             8 * __popc(p0 & p2) + 16 * __popc(p1 & p2);
        // i = 8 k + j
        const uint32_t si = 8 * k * n + sj, sii = 64 * k * k * n + 16 * k * sj + sjj;
        lut[e] = n | (si << 7) | (sii << 17);
    }
}

// Pass 1: the binary image packed to bit rows of nw words (nw a multiple of
// four, >= nwr + 3, nwr = ceil(n1 / 32)): word 1 + w of row (y, z) holds bit
// j = voxel (32 w + j, y, z), zero past n1; where n1 % 32 == 0, word 0 and
// word nwr + 1 repeat the row's last and first words (the periodic x
// neighbours of its two ends); the other words are zero.  Block 0 also
// writes the byte tables.
constexpr int PACK_THREADS = 256;

__device__ __forceinline__ void put_word(uint32_t* dst, int w, int nwr, int nw, uint32_t m, bool wrapx)
{
    dst[1 + w] = m;
    if (w == nwr - 1) dst[0] = wrapx ? m : 0u;
    if (w == 0) {
        dst[nwr + 1] = wrapx ? m : 0u;
        for (int p = nwr + 2; p < nw; p++) dst[p] = 0u;
    }
}

// n1 % 32 == 0, chi 16-byte aligned: a lane per word (two 16-byte loads),
// 32 / nwr rows a warp step where a row has fewer than 32 words
__global__ void __launch_bounds__(PACK_THREADS) k_cg_pack_vec(const uint8_t* chi, int n1, int nwr, int nw,
                                                              int64_t nrows, uint32_t* bitimg, uint32_t* lut)
{
    if (blockIdx.x == 0) build_lut(lut);
    const int lane = threadIdx.x & 31;
    const int rpw = nwr <= 32 ? 32 / nwr : 1;
    const int rs = nwr <= 32 ? lane / nwr : 0, w0 = nwr <= 32 ? lane - rs * nwr : lane;
    const bool on = rs < rpw;
    const int64_t nwarps = (int64_t)gridDim.x * (PACK_THREADS / 32);
    const int64_t step = nwarps * rpw;
    // four rows a lane per step: eight 16-byte loads in flight
    constexpr int RU = 4;
    for (int64_t r0 = ((int64_t)blockIdx.x * (PACK_THREADS / 32) + (threadIdx.x >> 5)) * rpw; r0 < nrows;
         r0 += RU * step) {
        for (int w = w0; w < nwr; w += 32) {
            uint4 v[2 * RU];
#pragma unroll
            for (int k = 0; k < RU; k++) {
                const int64_t row = r0 + k * step + rs;
                v[2 * k] = make_uint4(0u, 0u, 0u, 0u);
                v[2 * k + 1] = v[2 * k];
                if (on && row < nrows) {
                    const uint4* src = reinterpret_cast<const uint4*>(chi + row * n1 + 32 * w);
                    v[2 * k] = __ldcs(src);
                    v[2 * k + 1] = __ldcs(src + 1);
                }
            }
#pragma unroll
            for (int k = 0; k < RU; k++) {
                const int64_t row = r0 + k * step + rs;
                if (on && row < nrows)
                    put_word(bitimg + row * nw, w, nwr, nw, pack16(v[2 * k]) | (pack16(v[2 * k + 1]) << 16), true);
            }
        }
    }
}

// any n1 and alignment: a warp per row, one byte a lane
__global__ void __launch_bounds__(PACK_THREADS) k_cg_pack_bytes(const uint8_t* chi, int n1, int nwr, int nw,
                                                                int64_t nrows, uint32_t* bitimg, uint32_t* lut)
{
    if (blockIdx.x == 0) build_lut(lut);
    const int lane = threadIdx.x & 31;
    const bool wrapx = (n1 & 31) == 0;
    const int64_t nwarps = (int64_t)gridDim.x * (PACK_THREADS / 32);
    for (int64_t row = (int64_t)blockIdx.x * (PACK_THREADS / 32) + (threadIdx.x >> 5); row < nrows; row += nwarps) {
        for (int w = 0; w < nwr; w++) {
            const int x = 32 * w + lane;
            const uint8_t c = x < n1 ? __ldcs(chi + row * n1 + x) : (uint8_t)0;
            const uint32_t m = __ballot_sync(0xFFFFFFFFu, c != 0);
            if (lane == 0) put_word(bitimg + row * nw, w, nwr, nw, m, wrapx);
        }
    }
}

// Pass 2 input: the slab's (b2 + 2)(b3 + 2) bit rows -- its own b2 b3 rows and
// the one-voxel halo around them, periodic in y and z -- copied from the bit
// image with 16-byte loads (row layout as in the bit image).  Slab-local row t
// holds (jj, kk) = (t mod (b2 + 2), t div (b2 + 2)) - 1.  Also copies the byte
// tables.
__device__ void load_rows(const CgArgs& a, uint32_t* bits, uint32_t* lut, int J, int K)
{
    if (threadIdx.x < LUT_N / 4)
        reinterpret_cast<uint4*>(lut)[threadIdx.x] = __ldg(reinterpret_cast<const uint4*>(a.glut) + threadIdx.x);
    const int pl = a.b2 + 2, nw4 = a.nw >> 2;
    const int per = pl * nw4;  // 16-byte words per plane of rows
    const int total = (a.b3 + 2) * per;
    const uint4* src = reinterpret_cast<const uint4*>(a.bitimg);
    uint4* dst = reinterpret_cast<uint4*>(bits);
    constexpr int U = 4;
    for (int base = 0; base < total; base += U * CG_THREADS) {
        uint4 v[U];
        int d[U];
#pragma unroll
        for (int k = 0; k < U; k++) {
            const int it = base + k * CG_THREADS + (int)threadIdx.x;
            d[k] = -1;
            if (it < total) {
                const int pk = fdiv(it, per, a.inv_per), u = it - pk * per;
                const int jr = fdiv(u, nw4, a.inv_nw4), q = u - jr * nw4;
                const int y = wrap(J * a.b2 + jr - 1, a.n2), z = wrap(K * a.b3 + pk - 1, a.n3);
                v[k] = __ldg(src + ((size_t)z * a.n2 + y) * nw4 + q);
                d[k] = it;
            }
        }
#pragma unroll
        for (int k = 0; k < U; k++)
            if (d[k] >= 0) dst[d[k]] = v[k];
    }
}

// The part of a fine row that one boxel covers: bits [x, x + L) of the
// slab's bit row, x = I b1 + x0, L <= 32.
struct Span {
    int w, s, L;    // word, shift and width
    uint32_t msk;   // L low bits
    int o;          // offset q = 2 i + o of bit i (q = 2 i' + 1 - b1)
    int nbytes;     // bytes of the L-bit masks (table lookups)
    bool one;       // s + L <= 32: the span lies in one word
    bool left_in;   // x > 0: bit x - 1 is in the row (else it wraps to n1 - 1)
    bool right_in;  // x + L < n1: bit x + L is in the row (else it wraps to 0)
};

__device__ __forceinline__ Span make_span(const CgArgs& a, int I, int x0)
{
    Span c;
    const int x = I * a.b1 + x0;
    c.L = min(32, a.b1 - x0);
    c.w = x >> 5;
    c.s = x & 31;
    c.msk = c.L == 32 ? 0xFFFFFFFFu : ((1u << c.L) - 1u);
    c.o = 2 * x0 + 1 - a.b1;
    c.nbytes = (c.L + 7) >> 3;
    c.one = c.s + c.L <= 32;
    c.left_in = x > 0;
    c.right_in = x + c.L < a.n1;
    return c;
}

__device__ __forceinline__ uint32_t take(const uint32_t* row, const Span& c)
{
    if (c.one) return (row[c.w] >> c.s) & c.msk;
    return (uint32_t)((((uint64_t)row[c.w + 1] << 32) | row[c.w]) >> c.s) & c.msk;
}

template <int NB> __device__ __forceinline__ uint32_t look(const uint32_t* lut, uint32_t m)
{
    uint32_t v = lut[m & 255u];
    if (NB > 1) v += lut[256 + (m >> 8 & 255u)];
    if (NB > 2) v += lut[512 + (m >> 16 & 255u)];
    if (NB > 3) v += lut[768 + (m >> 24)];
    return v;
}

// Smallest-eigenvalue eigenvector of a symmetric positive semidefinite 3x3
// matrix K = (xx, xy, xz, yy, yz, zz).
//
// A start vector comes from cyclic Jacobi rotations in FP32 on K / tr K: each
// rotation in the (p, q) plane annihilates a_pq, tan(phi) being the smaller
// root of t^2 + 2 theta t - 1 = 0 with theta = (a_qq - a_pp) / (2 a_pq) (the
// classical method in its stable form, Golub & Van Loan, Matrix
// Computations, Sec. 8.5).  It is refined in FP64 by Rayleigh-quotient
// iteration written with the adjugate: for sigma the Rayleigh quotient of v,
// adj(K - sigma I) = sum_i prod_{j != i} (lambda_j - sigma) u_i u_i^T, so
// adj(K - sigma I) v keeps v's component along the sought eigenvector u_0
// and damps the others by (lambda_0 - sigma) / (lambda_i - sigma) -- cubic
// convergence, one step from an FP32 start except where the two smallest
// eigenvalues are close (then two).  FP64 is the scarce pipe on this GPU,
// so the FP64 part is a few dozen operations.
__device__ void min_eigvec(const double K[6], const float Kf[6], double N[3])
{
    // Kf: K rounded to FP32 (any positive multiple), scaled to unit trace
    const float trf = Kf[0] + Kf[3] + Kf[5];
    const float sc = trf > 0.f ? 1.f / trf : 1.f;
    float a[3][3] = {{Kf[0] * sc, Kf[1] * sc, Kf[2] * sc},
                     {Kf[1] * sc, Kf[3] * sc, Kf[4] * sc},
                     {Kf[2] * sc, Kf[4] * sc, Kf[5] * sc}};
    float V[3][3] = {{1.f, 0.f, 0.f}, {0.f, 1.f, 0.f}, {0.f, 0.f, 1.f}};
    for (int sweep = 0; sweep < 8; sweep++) {
        bool rotated = false;
#pragma unroll
        for (int pq = 0; pq < 3; pq++) {
            const int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2, r = 3 - p - q;
            const float apq = a[p][q];
            if (fabsf(apq) <= 1e-9f * (fabsf(a[p][p]) + fabsf(a[q][q])) || fabsf(apq) < 1e-30f) {
                a[p][q] = a[q][p] = 0.f;
                continue;
            }
            const float theta = (a[q][q] - a[p][p]) / (2.f * apq);
            const float t = fabsf(theta) > 1e9f ? 0.5f / theta
                                                : copysignf(1.f, theta) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
            const float c = rsqrtf(t * t + 1.f), s = t * c;
            a[p][p] -= t * apq;
            a[q][q] += t * apq;
            a[p][q] = a[q][p] = 0.f;
            const float arp = a[r][p], arq = a[r][q];
            a[r][p] = a[p][r] = c * arp - s * arq;
            a[r][q] = a[q][r] = s * arp + c * arq;
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const float vp = V[k][p], vq = V[k][q];
                V[k][p] = c * vp - s * vq;
                V[k][q] = s * vp + c * vq;
            }
            rotated = true;
        }
        if (!rotated) break;
    }
    // smallest and middle diagonal entries (no dynamic index: registers only)
    const float d0 = a[0][0], d1 = a[1][1], d2 = a[2][2];
    const int k = (d0 <= d1 && d0 <= d2) ? 0 : (d1 <= d2 ? 1 : 2);
    const float lo = k == 0 ? d0 : (k == 1 ? d1 : d2);
    const float mid = k == 0 ? fminf(d1, d2) : (k == 1 ? fminf(d0, d2) : fminf(d0, d1));
    // the FP32 start: a unit vector to FP32 rounding
    double v[3];
#pragma unroll
    for (int i = 0; i < 3; i++) v[i] = (double)(k == 0 ? V[i][0] : (k == 1 ? V[i][1] : V[i][2]));
    double nv;
    const int steps = (mid - lo) < 1e-3f ? 2 : 1;
    for (int it = 0; it < steps; it++) {
        const double kv0 = K[0] * v[0] + K[1] * v[1] + K[2] * v[2];
        const double kv1 = K[1] * v[0] + K[3] * v[1] + K[4] * v[2];
        const double kv2 = K[2] * v[0] + K[4] * v[1] + K[5] * v[2];
        // Rayleigh quotient v^T K v / v^T v, with 1 / (1 + d) ~ 1 - d for the
        // FP32-sized d = v^T v - 1 (second-order error ~ 1e-15)
        const double vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        const double sg = (v[0] * kv0 + v[1] * kv1 + v[2] * kv2) * (2.0 - vv);
        const double A00 = K[0] - sg, A11 = K[3] - sg, A22 = K[5] - sg, A01 = K[1], A02 = K[2], A12 = K[4];
        const double C00 = A11 * A22 - A12 * A12, C11 = A00 * A22 - A02 * A02, C22 = A00 * A11 - A01 * A01;
        const double C01 = A02 * A12 - A01 * A22, C02 = A01 * A12 - A02 * A11, C12 = A01 * A02 - A00 * A12;
        const double y0 = C00 * v[0] + C01 * v[1] + C02 * v[2];
        const double y1 = C01 * v[0] + C11 * v[1] + C12 * v[2];
        const double y2 = C02 * v[0] + C12 * v[1] + C22 * v[2];
        const double ny = y0 * y0 + y1 * y1 + y2 * y2;
        if (!(ny > 0.0) || !isfinite(ny)) {  // v already spans a multiple eigenvalue
            nv = rsqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            v[0] *= nv;
            v[1] *= nv;
            v[2] *= nv;
            break;
        }
        nv = rsqrt(ny);
        v[0] = y0 * nv;
        v[1] = y1 * nv;
        v[2] = y2 * nv;
    }
    N[0] = v[0];
    N[1] = v[1];
    N[2] = v[2];
}


__device__ void boxel_finish(const CgArgs& a, const int* acc, double* N)
{
    const int Qx = acc[0], Qy = acc[1], Qz = acc[2];
    // the barycentre normal's direction, unnormalised: -(h o Q)
    const double d0 = -a.h[0] * Qx, d1 = -a.h[1] * Qy, d2 = -a.h[2] * Qz;
    const bool has_nt = (Qx | Qy | Qz) != 0;
    if (a.method == COMBO_NORMAL_KABEL && has_nt) {
        const double s = rsqrt(d0 * d0 + d1 * d1 + d2 * d2);
        N[0] = d0 * s;
        N[1] = d1 * s;
        N[2] = d2 * s;
        return;
    }
    // K = 4 S0 M = (h_c h_d) (S0 U2_cd - U1_c U1_d), U = sum_i r_i T_i, a
    // positive multiple of M with the same eigenvectors
    double K[6];
    float Kf[6];
    const int ci[6] = {0, 0, 0, 1, 1, 2}, di[6] = {0, 1, 2, 1, 2, 2};
    if (a.iso) {
        // equal r_i and h_c: K is h^4 r^2 (T0 T2 - T1 T1^T), exact in int64
        int64_t T0 = 0, T1[3] = {0, 0, 0}, T2[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int i = 0; i < 3; i++) {
            const int* T = acc + 3 + 10 * i;
            T0 += T[0];
#pragma unroll
            for (int c = 0; c < 3; c++) T1[c] += T[1 + c];
#pragma unroll
            for (int c = 0; c < 6; c++) T2[c] += T[4 + c];
        }
#pragma unroll
        for (int c = 0; c < 6; c++) {
            const int64_t D = T0 * T2[c] - T1[ci[c]] * T1[di[c]];
            K[c] = (double)D;
            Kf[c] = (float)D;
        }
    } else {
        double S0 = 0.0, U1[3] = {0.0, 0.0, 0.0}, U2[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int i = 0; i < 3; i++) {
            const int* T = acc + 3 + 10 * i;
            const double ri = a.r[i];
            S0 += ri * T[0];
#pragma unroll
            for (int c = 0; c < 3; c++) U1[c] += ri * T[1 + c];
#pragma unroll
            for (int c = 0; c < 6; c++) U2[c] += ri * T[4 + c];
        }
#pragma unroll
        for (int c = 0; c < 6; c++) {
            K[c] = (a.h[ci[c]] * a.h[di[c]]) * (S0 * U2[c] - U1[ci[c]] * U1[di[c]]);
            Kf[c] = (float)K[c];
        }
    }
    min_eigvec(K, Kf, N);
    // Eq. normal:flip: keep N only where it agrees with the barycentre normal
    if (!(d0 * N[0] + d1 * N[1] + d2 * N[2] > 0.0)) {
        N[0] = -N[0];
        N[1] = -N[1];
        N[2] = -N[2];
    }
}

// Accumulate the integer moments of one boxel row span into acc, given its
// bits W, its x neighbours Wm (bits x - 1 ..) and Wp (bits x + 1 ..), and the
// same span of the four y / z neighbour rows; q = 2 i + o for bit i.
template <int NB>
__device__ __forceinline__ void span_moments(const uint32_t* lut, uint32_t W, uint32_t Wm, uint32_t Wp,
                                             uint32_t Ym, uint32_t Yp, uint32_t Zm, uint32_t Zp, int o, int qy,
                                             int qz, int* acc)
{
    const uint32_t vw = look<NB>(lut, W);
    const int np = vw & 127, sw = vw >> 7 & 1023;
    acc[0] += 2 * sw + o * np;
    acc[1] += qy * np;
    acc[2] += qz * np;
    const uint32_t e[6] = {W ^ Wm, W ^ Wp, W ^ Ym, W ^ Yp, W ^ Zm, W ^ Zp};
    const int qyy = qy * qy, qyz = qy * qz, qzz = qz * qz;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        // m_i over the span: its two neighbours' XOR masks
        const uint32_t v = look<NB>(lut, e[2 * i]) + look<NB>(lut, e[2 * i + 1]);
        const int n = v & 127, si = v >> 7 & 1023, sii = v >> 17;
        const int s1 = 2 * si + o * n;                       // sum of q
        const int s2 = 4 * sii + 4 * o * si + o * o * n;     // sum of q^2
        int* T = acc + 3 + 10 * i;
        T[0] += n;
        T[1] += s1;
        T[2] += qy * n;
        T[3] += qz * n;
        T[4] += s2;
        T[5] += qy * s1;
        T[6] += qz * s1;
        T[7] += qyy * n;
        T[8] += qyz * n;
        T[9] += qzz * n;
    }
}

// General spans (any n1, any b1): bits [x, x + L) of the row whose global
// word w is C[w]; the row's ends wrap explicitly.
__device__ __forceinline__ void row_moments(const CgArgs& a, const uint32_t* lut, const Span& c, const uint32_t* C,
                                            int rstride, int qy, int qz, int* acc)
{
    const uint64_t win = ((uint64_t)C[c.w + 1] << 32) | C[c.w];
    const uint32_t W = (uint32_t)(win >> c.s) & c.msk;
    const uint32_t Wp = c.right_in ? ((uint32_t)(win >> (c.s + 1)) & c.msk)
                                   : ((W >> 1) | ((C[0] & 1u) << (c.L - 1)));
    uint32_t Wm;
    if (c.s > 0)
        Wm = (uint32_t)(win >> (c.s - 1)) & c.msk;
    else
        Wm = ((W << 1) | (c.left_in ? (C[c.w - 1] >> 31) : bit_at(C, a.n1 - 1))) & c.msk;
    span_moments<4>(lut, W, Wm, Wp, take(C - a.nw, c), take(C + a.nw, c), take(C - rstride, c),
                    take(C + rstride, c), c.o, qy, qz, acc);
}

// Fast spans: n1 % 32 == 0 and b1 <= 32, so x = I b1 and every neighbour bit
// lies in the three padded words around the span (the wrap words included).
struct FastSpan {
    int w;         // padded index of the word before the span's first word
    int s, o;
    uint32_t msk;
};

__device__ __forceinline__ FastSpan make_fast_span(const CgArgs& a, int I)
{
    FastSpan c;
    const int x = I * a.b1;
    c.w = x >> 5;
    c.s = x & 31;
    c.o = 1 - a.b1;
    c.msk = a.b1 == 32 ? 0xFFFFFFFFu : ((1u << a.b1) - 1u);
    return c;
}

template <bool ONE> __device__ __forceinline__ uint32_t take_fast(const uint32_t* R, const FastSpan& c)
{
    if (ONE) return (R[c.w + 1] >> c.s) & c.msk;
    return __funnelshift_r(R[c.w + 1], R[c.w + 2], c.s) & c.msk;
}

// The fast path's lanes keep one y row offset qy (the group size is a
// multiple of b2), so a lane sums only what varies with its rows: per axis
// i, n, sum q, sum q^2, sum qz n, sum qz q, sum qz^2 n (f[6 i ..]), then
// sum q over the inclusion bits, their count and sum qz count (f[18 ..]).
constexpr int NFAST = 21;

template <int NB, bool ONE>
__device__ __forceinline__ void row_moments_fast(const uint32_t* lut, const FastSpan& c, const uint32_t* R, int nw,
                                                 int rstride, int qz, int* f)
{
    const uint32_t lo = R[c.w], mid = R[c.w + 1], hi = R[c.w + 2];
    const uint32_t W = (ONE ? (mid >> c.s) : __funnelshift_r(mid, hi, c.s)) & c.msk;
    const uint32_t Wm = (c.s == 0 ? __funnelshift_r(lo, mid, 31) : __funnelshift_r(mid, hi, c.s - 1)) & c.msk;
    const uint32_t Wp = (c.s == 31 ? hi : __funnelshift_r(mid, hi, c.s + 1)) & c.msk;
    const uint32_t e[6] = {W ^ Wm, W ^ Wp, W ^ take_fast<ONE>(R - nw, c), W ^ take_fast<ONE>(R + nw, c),
                           W ^ take_fast<ONE>(R - rstride, c), W ^ take_fast<ONE>(R + rstride, c)};
    const int o = c.o, qzz = qz * qz;
    const uint32_t vw = look<NB>(lut, W);
    const int np = vw & 127, sw = vw >> 7 & 1023;
    f[18] += 2 * sw + o * np;
    f[19] += np;
    f[20] += qz * np;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const uint32_t v = look<NB>(lut, e[2 * i]) + look<NB>(lut, e[2 * i + 1]);
        const int n = v & 127, si = v >> 7 & 1023, sii = v >> 17;
        const int s1 = 2 * si + o * n;                    // sum of q
        const int s2 = 4 * sii + 4 * o * si + o * o * n;  // sum of q^2
        int* F = f + 6 * i;
        F[0] += n;
        F[1] += s1;
        F[2] += s2;
        F[3] += qz * n;
        F[4] += qz * s1;
        F[5] += qzz * n;
    }
}

// the lane's sums with its qy folded in, in the layout of the per-boxel record
__device__ __forceinline__ void expand_fast(const int* f, int qy, int* acc)
{
    acc[0] = f[18];
    acc[1] = qy * f[19];
    acc[2] = f[20];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const int* F = f + 6 * i;
        int* T = acc + 3 + 10 * i;
        T[0] = F[0];
        T[1] = F[1];
        T[2] = qy * F[0];
        T[3] = F[3];
        T[4] = F[2];
        T[5] = qy * F[1];
        T[6] = F[4];
        T[7] = qy * qy * F[0];
        T[8] = qy * F[3];
        T[9] = F[5];
    }
}

template <int NB, bool ONE, bool FAST>
__global__ void __launch_bounds__(CG_THREADS, 4) k_cg_slab(CgArgs a)
{
    extern __shared__ __align__(16) uint32_t bits[];
    const int pl = a.b2 + 2;  // bit rows per slab plane
    int* cnt = reinterpret_cast<int*>(bits + (size_t)pl * (a.b3 + 2) * a.nw);
    int* mixed = cnt + a.nc1;
    __shared__ int nmixed;
    __shared__ __align__(16) uint32_t lut[LUT_N];
    const int slab = blockIdx.x;
    const int J = slab % a.nc2, K = slab / a.nc2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NWARP = CG_THREADS / 32;
    const int rows = a.b2 * a.b3;
    if (threadIdx.x == 0) nmixed = 0;
    // column counts (b1 = 8, 16, 32 on the fast path) accumulate with atomics
    const bool colcount = FAST && ONE && a.b1 >= 8;
    if (colcount)
        for (int I = threadIdx.x; I < a.nc1; I += CG_THREADS) cnt[I] = 0;
    load_rows(a, bits, lut, J, K);
    __syncthreads();

    // inclusion voxels per coarse voxel
    if (colcount) {
        // a thread per (word column w, row group g): byte-wise popcounts of the
        // words, summed over every NG-th row in packed bytes (flushed before a
        // byte can overflow), then added to the word's 32 / b1 coarse voxels
        const int NG = a.NGq * a.b2 + a.NGr;
        for (int it = threadIdx.x; it < a.nwr * NG; it += CG_THREADS) {
            const int g = fdiv(it, a.nwr, a.inv_nwr), w = it - g * a.nwr;
            int kk = fdiv(g, a.b2, a.inv_b2), jj = g - kk * a.b2;
            uint32_t packed = 0;
            int c0 = 0, c1 = 0, c2 = 0, c3 = 0, nrow = 0;
            for (int r = g; r < rows; r += NG) {
                uint32_t x = bits[lrow(jj, kk, a.b2) * a.nw + 1 + w];
                x = x - ((x >> 1) & 0x55555555u);
                x = (x & 0x33333333u) + ((x >> 2) & 0x33333333u);
                packed += (x + (x >> 4)) & 0x0F0F0F0Fu;
                if (++nrow == 31) {
                    c0 += packed & 255u;
                    c1 += packed >> 8 & 255u;
                    c2 += packed >> 16 & 255u;
                    c3 += packed >> 24;
                    packed = 0;
                    nrow = 0;
                }
                jj += a.NGr;
                kk += a.NGq;
                if (jj >= a.b2) {
                    jj -= a.b2;
                    kk++;
                }
            }
            c0 += packed & 255u;
            c1 += packed >> 8 & 255u;
            c2 += packed >> 16 & 255u;
            c3 += packed >> 24;
            if (a.b1 == 8) {
                if (c0) atomicAdd(&cnt[4 * w], c0);
                if (c1) atomicAdd(&cnt[4 * w + 1], c1);
                if (c2) atomicAdd(&cnt[4 * w + 2], c2);
                if (c3) atomicAdd(&cnt[4 * w + 3], c3);
            } else if (a.b1 == 16) {
                if (c0 + c1) atomicAdd(&cnt[2 * w], c0 + c1);
                if (c2 + c3) atomicAdd(&cnt[2 * w + 1], c2 + c3);
            } else if (c0 + c1 + c2 + c3) {
                atomicAdd(&cnt[w], c0 + c1 + c2 + c3);
            }
        }
    } else {
        // R consecutive lanes per coarse voxel, each summing the popcounts of
        // every R-th fine row
        const int R = a.R;
        const int per = CG_THREADS / R;
        for (int I0 = 0; I0 < a.nc1; I0 += per) {
            const int I = I0 + (int)threadIdx.x / R, rg = threadIdx.x & (R - 1);
            int s = 0;
            if (I < a.nc1) {
                int kk = fdiv(rg, a.b2, a.inv_b2), jj = rg - kk * a.b2;
                const FastSpan fc = make_fast_span(a, I);
                const Span c = make_span(a, I, 0);
                for (int t = rg; t < rows; t += R) {
                    const uint32_t* row = bits + lrow(jj, kk, a.b2) * a.nw;
                    if (FAST)
                        s += __popc(take_fast<ONE>(row, fc));
                    else
                        for (int x0 = 0; x0 < a.b1; x0 += 32)
                            s += __popc(take(row + 1, x0 == 0 ? c : make_span(a, I, x0)));
                    jj += a.Rr;
                    kk += a.Rq;
                    if (jj >= a.b2) {
                        jj -= a.b2;
                        kk++;
                    }
                }
            }
            for (int off = R >> 1; off >= 1; off >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, off);
            if (I < a.nc1 && rg == 0) cnt[I] = s;
        }
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

    // integer moments: G lanes per boxel, every G-th fine row a lane
    const int G = a.G, gpw = 32 / G, g = lane / G, lg = lane & (G - 1);
    const int rstride = pl * a.nw;  // one plane of bit rows
    const int kk0 = fdiv(lg, a.b2, a.inv_b2), jj0 = lg - kk0 * a.b2;
    for (int mb = warp * gpw; mb < nm; mb += NWARP * gpw) {
        const int m = mb + g;
        const bool act = m < nm;
        const int I = act ? mixed[m] : 0;
        int acc[NACC];
        if (FAST) {
            // rows t = lg + G k: jj = jj0 for all of them (G % b2 == 0)
            int f[NFAST];
#pragma unroll
            for (int k = 0; k < NFAST; k++) f[k] = 0;
            if (act) {
                const FastSpan c = make_fast_span(a, I);
                const uint32_t* R = bits + lrow(jj0, kk0, a.b2) * a.nw;
                const int rstep = a.Gq * pl * a.nw;
                for (int kk = kk0; kk < a.b3; kk += a.Gq, R += rstep)
                    row_moments_fast<NB, ONE>(lut, c, R, a.nw, rstride, 2 * kk + 1 - a.b3, f);
            }
            expand_fast(f, 2 * jj0 + 1 - a.b2, acc);
        } else {
#pragma unroll
            for (int k = 0; k < NACC; k++) acc[k] = 0;
            if (act) {
                int jj = jj0, kk = kk0;
                for (int t = lg; t < rows; t += G) {
                    const uint32_t* C = bits + lrow(jj, kk, a.b2) * a.nw + 1;
                    for (int x0 = 0; x0 < a.b1; x0 += 32)
                        row_moments(a, lut, make_span(a, I, x0), C, rstride, 2 * jj + 1 - a.b2, 2 * kk + 1 - a.b3,
                                    acc);
                    jj += a.Gr;
                    kk += a.Gq;
                    if (jj >= a.b2) {
                        jj -= a.b2;
                        kk++;
                    }
                }
            }
        }
        for (int off = G >> 1; off >= 1; off >>= 1)
#pragma unroll
            for (int k = 0; k < NACC; k++) acc[k] += __shfl_xor_sync(0xFFFFFFFFu, acc[k], off);
        if (act && lg == 0) {
            int4* dst = reinterpret_cast<int4*>(a.sums + (cbase + I) * NSUM);
#pragma unroll
            for (int k = 0; k < 8; k++) dst[k] = make_int4(acc[4 * k], acc[4 * k + 1], acc[4 * k + 2], acc[4 * k + 3]);
            dst[8] = make_int4(acc[32], cnt[I], 0, 0);
        }
    }
}

using SlabKernel = void (*)(CgArgs);

SlabKernel pick_slab_kernel(int n1, int b1, bool fast)
{
    if (!fast) return k_cg_slab<4, false, false>;
    const bool one = 32 % b1 == 0;
    if (b1 <= 8) return one ? k_cg_slab<1, true, true> : k_cg_slab<1, false, true>;
    if (b1 <= 16) return one ? k_cg_slab<2, true, true> : k_cg_slab<2, false, true>;
    return one ? k_cg_slab<4, true, true> : k_cg_slab<4, false, true>;
}

// the normals and c+ of the listed boxels, one boxel per thread
__global__ void __launch_bounds__(FIN_THREADS) k_cg_finish(CgArgs a, const int64_t* total, int64_t cap,
                                                           const int64_t* idx_out, double* N_out, double* c_out)
{
    const int64_t nb = min(*total, cap);
    const int nblock = a.b1 * a.b2 * a.b3;
    for (int64_t pos = blockIdx.x * (int64_t)FIN_THREADS + threadIdx.x; pos < nb;
         pos += (int64_t)gridDim.x * FIN_THREADS) {
        const int4* src = reinterpret_cast<const int4*>(a.sums + idx_out[pos] * NSUM);
        int acc[NACC + 3];
#pragma unroll
        for (int k = 0; k < 9; k++) {
            const int4 v = src[k];
            acc[4 * k] = v.x;
            acc[4 * k + 1] = v.y;
            acc[4 * k + 2] = v.z;
            acc[4 * k + 3] = v.w;
        }
        double N[3];
        boxel_finish(a, acc, N);
        N_out[3 * pos + 0] = N[0];
        N_out[3 * pos + 1] = N[1];
        N_out[3 * pos + 2] = N[2];
        const int npl = acc[NACC];
        c_out[pos] = a.nblock_pow2 ? npl * a.inv_nblock : (double)npl / (double)nblock;
    }
}

// exclusive scan of the per-slab boxel counts (one CTA, coalesced chunks)
__global__ void __launch_bounds__(SCAN_THREADS) k_cg_scan(const int* cnt, int nslab, int64_t* off, int64_t* total)
{
    __shared__ int64_t wsum[SCAN_THREADS / 32];
    __shared__ int64_t carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nslab; base += SCAN_THREADS) {
        const int s = base + threadIdx.x;
        const int64_t v = s < nslab ? cnt[s] : 0;
        int64_t incl = v;
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t t = __shfl_up_sync(0xFFFFFFFFu, incl, d);
            if (lane >= d) incl += t;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int64_t w = wsum[lane];
            for (int d = 1; d < 32; d <<= 1) {
                const int64_t t = __shfl_up_sync(0xFFFFFFFFu, w, d);
                if (lane >= d) w += t;
            }
            wsum[lane] = w;  // inclusive over warps
        }
        __syncthreads();
        const int64_t excl = carry + incl - v + (warp > 0 ? wsum[warp - 1] : 0);
        if (s < nslab) off[s] = excl;
        __syncthreads();  // every thread has read carry
        if (threadIdx.x == SCAN_THREADS - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

// the coarse indices of each slab's boxels into the output list (increasing):
// a warp per slab
__global__ void __launch_bounds__(SCATTER_THREADS)
    k_cg_scatter(const uint8_t* phase, const int* cnt, const int64_t* off, int nc1, int nslab, int64_t cap,
                 int64_t* idx_out)
{
    const int lane = threadIdx.x & 31;
    const int slab = blockIdx.x * (SCATTER_THREADS / 32) + (threadIdx.x >> 5);
    if (slab >= nslab || cnt[slab] == 0) return;
    const size_t base = (size_t)slab * nc1;
    int64_t run = off[slab];
    for (int I0 = 0; I0 < nc1; I0 += 32) {
        const int I = I0 + lane;
        const bool f = I < nc1 && phase[base + I] == 2;
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, f);
        const int64_t pos = run + __popc(bal & ((1u << lane) - 1u));
        if (f && pos < cap) idx_out[pos] = (int64_t)(base + I);
        run += __popc(bal);
    }
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// event timing of the launches (combo_coarse_grain_profile)
std::mutex g_prof_mu;
bool g_prof_on = false;
int g_prof_dev = -1;
cudaEvent_t g_prof_ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
bool g_prof_have = false;
double g_prof_ms[5] = {0.0, 0.0, 0.0, 0.0, 0.0};

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
    a.nwr = (a.n1 + 31) / 32;
    a.nw = (a.nwr + 3 + 3) & ~3;
    a.method = method;
    for (int j = 0; j < 3; j++) a.h[j] = h[j];
    a.r[0] = h[1] * h[2] / h[0];  // r_i = h_j h_k / h_i
    a.r[1] = h[0] * h[2] / h[1];
    a.r[2] = h[0] * h[1] / h[2];
    const int rows = a.b2 * a.b3;
    // lanes per boxel: about eight fine rows a lane (fewer reduction levels);
    // the fast path (n1 % 32 == 0, b1 <= 32, b2 a power of two <= 32) takes a
    // multiple of b2 so that each lane keeps one y row offset
    int G = 1;
    while (G < 32 && 16 * G <= rows) G <<= 1;
    const bool b2pow2 = (a.b2 & (a.b2 - 1)) == 0 && a.b2 <= 32;
    const bool fast = a.n1 % 32 == 0 && a.b1 <= 32 && b2pow2;
    if (fast) G = std::max(G, a.b2);
    a.G = G;
    a.Gq = G / a.b2;
    a.Gr = G % a.b2;
    // lanes per coarse voxel in the count
    int R = 1;
    while (R < 32 && 2 * R * a.nc1 <= CG_THREADS && 2 * R <= rows) R <<= 1;
    a.R = R;
    a.Rq = R / a.b2;
    a.Rr = R % a.b2;
    a.inv_b2 = 1.0f / (float)a.b2;
    a.inv_per = 1.0f / (float)((a.b2 + 2) * (a.nw / 4));
    a.inv_nw4 = 1.0f / (float)(a.nw / 4);
    a.inv_nwr = 1.0f / (float)a.nwr;
    {
        const int NG = std::max(1, CG_THREADS / a.nwr);
        a.NGq = NG / a.b2;
        a.NGr = NG % a.b2;
    }
    a.iso = h[0] == h[1] && h[1] == h[2];
    a.nblock_pow2 = (nblock & (nblock - 1)) == 0;
    a.inv_nblock = 1.0 / (double)nblock;
    const size_t smem = (size_t)(a.b2 + 2) * (a.b3 + 2) * a.nw * 4 + (size_t)8 * a.nc1;
    if (smem > CG_SMEM_MAX)
        return set_error(COMBO_E_INVALID_ARG, "combo_coarse_grain: slab rows exceed the shared-memory limit");
    const size_t V = (size_t)n[0] * n[1] * n[2];
    const size_t nc = (size_t)a.nc1 * a.nc2 * a.nc3;
    const int nslab = a.nc2 * a.nc3;
    const bool dev = mem == COMBO_MEM_DEVICE;
    CGK(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;

    // scratch: [chi copy] [phase] slab_cnt slab_off total sums [idx N c]
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
    const size_t o_sums = sz;
    sz += align256(4 * NSUM * nc);
    const size_t o_bits = sz;
    sz += align256(4 * (size_t)a.nw * (size_t)n[1] * n[2]);
    const size_t o_lut = sz;
    sz += align256(4 * LUT_N);
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
    const uint8_t* d_chi = chi;
    if (!dev) {
        CGK(cudaMemcpyAsync(S + o_chi, chi, V, cudaMemcpyHostToDevice, st));
        d_chi = reinterpret_cast<const uint8_t*>(S + o_chi);
        a.phase = reinterpret_cast<uint8_t*>(S + o_phase);
    } else {
        a.phase = phase_out;
    }
    uint32_t* d_bits = reinterpret_cast<uint32_t*>(S + o_bits);
    uint32_t* d_lut = reinterpret_cast<uint32_t*>(S + o_lut);
    a.bitimg = d_bits;
    a.glut = d_lut;
    const bool vec = (a.n1 % 32 == 0) && ((reinterpret_cast<uintptr_t>(d_chi) & 15) == 0);
    a.slab_cnt = reinterpret_cast<int*>(S + o_cnt);
    int64_t* d_off = reinterpret_cast<int64_t*>(S + o_off);
    int64_t* d_tot = reinterpret_cast<int64_t*>(S + o_tot);
    a.sums = reinterpret_cast<int*>(S + o_sums);
    int64_t* oi = idx_out;
    double* oN = N_out;
    double* oc = c_out;
    if (!dev) {
        oi = reinterpret_cast<int64_t*>(S + o_out);
        oN = reinterpret_cast<double*>(S + o_out + 8 * (size_t)std::max<int64_t>(ncap, 1));
        oc = reinterpret_cast<double*>(S + o_out + 32 * (size_t)std::max<int64_t>(ncap, 1));
    }
    const SlabKernel slab_kernel = pick_slab_kernel(a.n1, a.b1, fast);
    CGK(cudaFuncSetAttribute(slab_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CG_SMEM_MAX));
    std::unique_lock<std::mutex> plock(g_prof_mu);
    const bool prof = g_prof_on;
    if (prof && g_prof_dev != ctx->device) {
        for (auto& e : g_prof_ev)
            if (e) cudaEventDestroy(e), e = nullptr;
        for (auto& e : g_prof_ev) CGK(cudaEventCreate(&e));
        g_prof_dev = ctx->device;
    }
    if (!prof) plock.unlock();
    if (prof) CGK(cudaEventRecord(g_prof_ev[0], st));
    {
        const int64_t nrows = (int64_t)n[1] * n[2];
        const int rpw = a.nwr <= 32 ? 32 / a.nwr : 1;
        const int64_t warps = vec ? (nrows + rpw - 1) / rpw : nrows;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((warps + 7) / 8, 152 * 16));
        if (vec)
            k_cg_pack_vec<<<grid, PACK_THREADS, 0, st>>>(d_chi, a.n1, a.nwr, a.nw, nrows, d_bits, d_lut);
        else
            k_cg_pack_bytes<<<grid, PACK_THREADS, 0, st>>>(d_chi, a.n1, a.nwr, a.nw, nrows, d_bits, d_lut);
        CGK(cudaGetLastError());
    }
    if (prof) CGK(cudaEventRecord(g_prof_ev[1], st));
    slab_kernel<<<nslab, CG_THREADS, smem, st>>>(a);
    CGK(cudaGetLastError());
    if (prof) CGK(cudaEventRecord(g_prof_ev[2], st));
    k_cg_scan<<<1, SCAN_THREADS, 0, st>>>(a.slab_cnt, nslab, d_off, d_tot);
    CGK(cudaGetLastError());
    if (prof) CGK(cudaEventRecord(g_prof_ev[3], st));
    k_cg_scatter<<<(nslab + SCATTER_THREADS / 32 - 1) / (SCATTER_THREADS / 32), SCATTER_THREADS, 0, st>>>(
        a.phase, a.slab_cnt, d_off, a.nc1, nslab, ncap, oi);
    CGK(cudaGetLastError());
    if (prof) CGK(cudaEventRecord(g_prof_ev[4], st));
    if (ncap > 0) {
        const int fin_grid = (int)std::min<int64_t>((ncap + FIN_THREADS - 1) / FIN_THREADS, 152 * 8);
        k_cg_finish<<<fin_grid, FIN_THREADS, 0, st>>>(a, d_tot, ncap, oi, oN, oc);
        CGK(cudaGetLastError());
    }
    if (prof) CGK(cudaEventRecord(g_prof_ev[5], st));
    int64_t total = 0;
    CGK(cudaMemcpyAsync(&total, d_tot, 8, cudaMemcpyDeviceToHost, st));
    CGK(cudaStreamSynchronize(st));
    if (prof) {
        float t = 0.f;
        for (int k = 0; k < 5; k++) {
            CGK(cudaEventElapsedTime(&t, g_prof_ev[k], g_prof_ev[k + 1]));
            g_prof_ms[k] = t;
        }
        g_prof_have = true;
        plock.unlock();
    }
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

extern "C" int combo_coarse_grain_profile(int32_t enable)
{
    std::lock_guard<std::mutex> l(g_prof_mu);
    g_prof_on = enable != 0;
    return COMBO_OK;
}

extern "C" int combo_coarse_grain_profile_read(double ms[5])
{
    std::lock_guard<std::mutex> l(g_prof_mu);
    if (!ms || !g_prof_have) return set_error(COMBO_E_INVALID_ARG, "combo_coarse_grain_profile_read: nothing recorded");
    for (int k = 0; k < 5; k++) ms[k] = g_prof_ms[k];
    return COMBO_OK;
}
