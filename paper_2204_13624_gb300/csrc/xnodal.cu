// xnodal.cu -- the tangent pass of the nodal form of the rotated Green
// operator in the FP32 CG.
//
// With D the HEX8R gradient (nodal field -> voxel tensor: edge differences
// along J averaged over the voxel's 4 such edges, over h_J), the rotated
// operator is G = D (D^T D)^+ D^T: D's Fourier symbol is the rotated k
// (Sec. 3, the rotated scheme), so D^T D is the scalar |k|^2.  In the CG,
// G [A : p] is then D of the nodal field that solves D^T D u_i = f_i, where
// f_i = D^T (A : p)_i are the nodal forces of the direction's stress.  This
// pass assembles f in real space -- three nodal fields instead of the nine
// components of A : p -- and transforms them along x:
//
//   f_i(n) = sum over the 8 voxels v = n - b (b in {0,1}^3) of
//            sum_J c_J s(b_J) (A : p)_iJ(v),   s(1) = +1, s(0) = -1, c_J = 1/(4 h_J)
//
// A block takes runs of planes of columns, a column being TY node lines
// y0 .. y0 + TY - 1 -- equal chunks of planes per column, or an even share of
// the problem's (column, plane) pairs -- and marches each run along z; for
// each voxel plane it sweeps the voxel
// lines y0 - 1 .. y0 + TY - 1 (the first one, and the plane below its first,
// are halo: their A : p is formed but neither p, x nor pAp is written).  Per
// voxel line: (1) the voxels' direction update p = r + beta p_old, the
// deferred x += alpha_prev p_old and A : p -- at pure voxels from the tangent
// cache, at boxels from the packed boxel tangent (its column from the voxel's
// vrank entry) -- scaled by c_J into a shared line buffer; (2) (one barrier
// later) each thread combines its node's two
// x-neighbours (e = A(x-1) - A(x), f = B(x-1) + B(x), q = C(x-1) + C(x), with
// A, B, C the c_J-scaled columns J = 0, 1, 2 of row i), then the two voxel
// lines along y (P = e' + e + f' - f, Q = q' + q), and the two voxel planes
// along z: f_i = T + P - Q with T = P + Q of the plane below, kept per node.
// The nodal lines of a plane are then transformed along x (packed half-length
// FFT + Hermitian split) into components 0, 3, 6 of the spectrum.
#include <algorithm>

#include "combo_internal.cuh"
#include "fft_fast.cuh"
#include "../../include/combo.h"

namespace combo {

namespace {

int num_sms_nodal()
{
    static int nsm = 0;
    if (nsm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) nsm = 152;
    }
    return nsm;
}

// threads per block: one voxel of a line per thread
template <int M> __host__ __device__ constexpr int nodal_threads() { return 2 * M; }
// blocks per SM: two of 256 (or 128) threads (registers capped at 128); one of
// 512 at n1 = 512
template <int M, int C> __host__ __device__ constexpr int nodal_minb() { return M == 256 ? 1 : 2; }
// threads that transform the 3 TY nodal lines of a plane (named barrier 1)
template <int M, int TY> __host__ __device__ constexpr int nodal_fft_threads()
{
    return (3 * TY * FastPlan<M>::TPL + 31) / 32 * 32;
}
template <int M, int TY> __host__ __device__ constexpr size_t nodal_smem()
{
    // line buffers [2][9][n1], T [3][TY][n1] floats; nodal lines [3 TY][M + 1]
    // complex; twiddles [M]; reduction [max(256, threads)] doubles; flag
    return (size_t)2 * 9 * 2 * M * 4 + (size_t)3 * TY * 2 * M * 4 + (size_t)3 * TY * (M + 1) * 8 + (size_t)M * 8 +
           (size_t)(2 * M > 256 ? 2 * M : 256) * 8 + 16;
}

}  // namespace

bool nodal_ok(const GridDims& g)
{
    const int M = g.M;
    if (!(M == 64 || M == 128 || M == 256) || 2 * M != g.n1) return false;
    return g.n2 % 4 == 0;
}

int nodal_partials_max() { return 3 * num_sms_nodal(); }  // per_sm is capped at 3

template <int M, int TY, int C>
__global__ void __launch_bounds__(nodal_threads<M>(), (nodal_minb<M, C>())) k_xfwd_nodal(NodalArgs a)
{
    constexpr int n1 = 2 * M;
    constexpr int NT = nodal_threads<M>();
    constexpr int VPT = n1 / NT;  // voxels per thread and line
    constexpr int TPL = FastPlan<M>::TPL;
    constexpr int NLF = 3 * TY;   // nodal lines per plane
    constexpr int NBAR = nodal_fft_threads<M, TY>();
    constexpr int lsw = M + 1;    // complex stride of the nodal lines
    static_assert(NBAR <= NT, "the nodal lines of a plane are transformed in one round");
    int pb, pj, gp;
    prob_block(a.g, blockIdx.x, gridDim.x, pb, pj, gp);
    Scalars* sc = a.sc + pb;
    if (sc->cg_done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* lbuf = reinterpret_cast<float*>(smem_raw);      // [2][9][n1]
    float* tp = lbuf + 2 * 9 * n1;                          // [3][TY][n1]
    float2* W = reinterpret_cast<float2*>(tp + 3 * TY * n1);  // [NLF][lsw]
    float2* tws = W + (size_t)NLF * lsw;  // exp(-2 pi i t / M)
    double* red = reinterpret_cast<double*>(tws + M);
    int* flag = reinterpret_cast<int*>(red + (NT > 256 ? NT : 256));
    for (int i = threadIdx.x; i < M; i += blockDim.x) tws[i] = a.tw[i];

    const GridDims g = a.g;
    const int64_t V = g.V;
    const int tid = threadIdx.x;
    const int ncol = g.n2 / TY;
    // the problem's (column, plane) pairs, column-major, split evenly over its
    // gp blocks; a block's share is one or more runs of planes of a column
    const int64_t total = (int64_t)ncol * g.n3p;
    const int64_t lin_b = total * pj / gp, lin_e = total * (pj + 1) / gp;
    const bool first = sc->cg_iter == 0;
    const float beta = first ? 0.f : (float)sc->beta;
    const float apend = first ? 0.f : (float)sc->alpha_pending;
    const int kpar = sc->cg_iter & 1;
    const float* __restrict__ pin = a.p[kpar ^ 1];  // p of the previous iteration
    float* __restrict__ pout = a.p[kpar];
    const float* __restrict__ rg = a.r;
    float* __restrict__ xg = a.x;
    const float* __restrict__ tg = a.tc;
    const float c0 = a.cJ[0], c1 = a.cJ[1], c2 = a.cJ[2];
    float mu[2], lam[2];
    for (int i = 0; i < 2; i++) {
        mu[i] = (float)(a.matp ? a.matp[4 * pb + i] : a.mu[i]);
        lam[i] = (float)(a.matp ? a.matp[4 * pb + 2 + i] : a.lam[i]);
    }
    __syncthreads();

    double acc = 0.0;
    int s = 0;  // voxel lines swept (line buffer parity)
    // this block's runs: its even share (nch == 0), or, with nch chunks of
    // planes per column, items (chunk, column) in chunk-major order, so that
    // neighbouring columns march through the same planes at the same time and
    // a halo line is read while its owner's copy is still in L2
    const int nitems = a.nch > 0 ? ncol * a.nch : 0;
    int64_t lin = lin_b;
    int item = pj;
    for (;;) {
        int col, z0, z1;
        if (a.nch > 0) {
            if (item >= nitems) break;
            col = item % ncol;
            const int ch = item / ncol;
            z0 = (int)((int64_t)ch * g.n3p / a.nch);
            z1 = (int)((int64_t)(ch + 1) * g.n3p / a.nch);
            item += gp;
            if (z1 <= z0) continue;
        } else {
            if (lin >= lin_e) break;
            col = (int)(lin / g.n3p);
            z0 = (int)(lin - (int64_t)col * g.n3p);
            z1 = (int)min((int64_t)g.n3p, z0 + (lin_e - lin));
            lin += z1 - z0;
        }
        const int y0 = col * TY;
        float accp = 0.f;
        int vrc[VPT];  // vrank of this thread's voxels on the current voxel line
        {
            const int64_t L0 = (int64_t)(pb * g.n3p + (z0 == 0 ? g.n3p - 1 : z0 - 1)) * g.n2 + (y0 == 0 ? g.n2 - 1 : y0 - 1);
#pragma unroll
            for (int v = 0; v < VPT; v++) vrc[v] = a.vrank[L0 * n1 + tid + v * NT];
        }
        for (int zv = z0 - 1; zv < z1; zv++) {
            const bool zown = zv >= z0;
            const int zl = zv < 0 ? zv + g.n3p : zv;
            const int64_t zrow = (int64_t)(pb * g.n3p + zl) * g.n2;  // first line of the plane
            float pe[VPT][3], pf[VPT][3], pq[VPT][3];  // e, f, q of the previous voxel line
            for (int yy = -1; yy < TY; yy++, s++) {
                const int yl = (y0 + yy < 0) ? y0 + yy + g.n2 : y0 + yy;
                const bool own = zown && yy >= 0;
                const int64_t L = zrow + yl;
                float* LB = lbuf + (s & 1) * 9 * n1;
                int64_t Lnext = -1;  // the next voxel line of this run
                {
                    int yn = yy + 1, zn = zv;
                    if (yn >= TY) {
                        yn = -1;
                        zn++;
                    }
                    if (zn < z1) {
                        const int zln = zn < 0 ? zn + g.n3p : zn;
                        const int yln = (y0 + yn < 0) ? y0 + yn + g.n2 : y0 + yn;
                        Lnext = (int64_t)(pb * g.n3p + zln) * g.n2 + yln;
                    }
                }
                {
                    // the operand rows and boxel tangents of the voxel line pfd
                    // steps ahead (within this run) into L2: each step waits on
                    // its loads, so they should find L2 rather than DRAM
                    int ya = yy + a.pfd, za = zv;  // (pfd <= TY + 1: one wrap)
                    if (ya >= TY) {
                        ya -= TY + 1;
                        za++;
                    }
                    if (a.pfd > 0 && za < z1) {
                        const int zla = za < 0 ? za + g.n3p : za;
                        const int yla = (y0 + ya < 0) ? y0 + ya + g.n2 : y0 + ya;
                        const int64_t La = (int64_t)(pb * g.n3p + zla) * g.n2 + yla;
                        const bool owna = za >= z0 && ya >= 0;
                        constexpr int CH = n1 * 4 / 128;  // 128-byte chunks per row
                        const int nrow = 20 + (first ? 0 : 9) + ((owna && apend != 0.f) ? 9 : 0);
                        for (int e = tid; e < nrow * CH; e += NT) {
                            const int row = e / CH, qq = e - row * CH;
                            const float* base = row == 0 ? reinterpret_cast<const float*>(a.vrank)
                                                : row < 10 ? rg + (int64_t)(row - 1) * V
                                                : row < 20 ? tg + (int64_t)(row - 10) * V
                                                : (!first && row < 29) ? pin + (int64_t)(row - 20) * V
                                                : xg + (int64_t)(row - (first ? 20 : 29)) * V;
                            asm volatile("prefetch.global.L2 [%0];" ::"l"(base + La * n1 + qq * 32));
                        }
                        const int b0 = a.lofs[La], b1 = a.lofs[La + 1];
                        if (b1 > b0) {
                            const int nch = (b1 - b0 + 31) / 32 + 1;  // 128-byte chunks a row segment may touch
                            for (int e = tid; e < 45 * nch; e += NT) {
                                const int j = e / nch, q = e - j * nch;
                                const float* pa = a.bA + (int64_t)j * a.nb + b0 + 32 * q;
                                if (pa < a.bA + (int64_t)j * a.nb + b1)
                                    asm volatile("prefetch.global.L2 [%0];" ::"l"(pa));
                            }
                        }
                    }
                }
                // (1) voxels of the line: A : p at pure voxels from the tangent
                // cache, at boxels from their packed tangent (column vrank)
#pragma unroll
                for (int v = 0; v < VPT; v++) {
                    const int xx = tid + v * NT;
                    const int64_t vox = L * n1 + xx;
                    // this line's vrank was loaded one line ahead, so every
                    // operand load -- the boxel tangent's too, and the tangent
                    // cache, unused at boxels -- is issued before the first
                    // use: one memory latency per line; the stores follow
                    const int vr = vrc[v];
                    const bool xup = own && !first && apend != 0.f;
                    float p[9], po[9], xo[9], t[10], Ak[45];
#pragma unroll
                    for (int c = 0; c < 9; c++) p[c] = rg[c * V + vox];
#pragma unroll
                    for (int c = 0; c < 10; c++) t[c] = tg[c * V + vox];
                    if (!first) {
#pragma unroll
                        for (int c = 0; c < 9; c++) po[c] = pin[c * V + vox];
                    }
                    if (xup) {
#pragma unroll
                        for (int c = 0; c < 9; c++) xo[c] = xg[c * V + vox];
                    }
                    if (vr >= 0) {
#pragma unroll
                        for (int j = 0; j < 45; j++) Ak[j] = a.bA[(int64_t)j * a.nb + vr];
                    }
                    vrc[v] = Lnext >= 0 ? a.vrank[Lnext * n1 + xx] : 0;
                    if (!first) {
#pragma unroll
                        for (int c = 0; c < 9; c++) p[c] += beta * po[c];
                    }
                    float y[9];
                    if (vr >= 0) {
#pragma unroll
                        for (int r = 0; r < 9; r++) {
                            float yr = 0.f;
#pragma unroll
                            for (int c = 0; c < 9; c++) yr += Ak[sym_idx(r, c)] * p[c];
                            y[r] = yr;
                        }
                    } else {
                        const int ph = -1 - vr;
                        nh_tangent<float>(t, t[9], mu[ph], lam[ph], p, y);
                    }
                    if (own) {
                        float sp = 0.f;
#pragma unroll
                        for (int c = 0; c < 9; c++) sp += p[c] * y[c];
                        accp += sp;
#pragma unroll
                        for (int c = 0; c < 9; c++) pout[c * V + vox] = p[c];
                    }
                    if (xup) {
#pragma unroll
                        for (int c = 0; c < 9; c++) xg[c * V + vox] = xo[c] + apend * po[c];
                    }
#pragma unroll
                    for (int i = 0; i < 3; i++) {
                        LB[(3 * i) * n1 + xx] = c0 * y[3 * i];
                        LB[(3 * i + 1) * n1 + xx] = c1 * y[3 * i + 1];
                        LB[(3 * i + 2) * n1 + xx] = c2 * y[3 * i + 2];
                    }
                }
                __syncthreads();
                // (2) x-neighbours, then the y and z accumulation of the nodes
#pragma unroll
                for (int v = 0; v < VPT; v++) {
                    const int xx = tid + v * NT;
                    const int xm = xx == 0 ? n1 - 1 : xx - 1;
#pragma unroll
                    for (int i = 0; i < 3; i++) {
                        const float e = LB[(3 * i) * n1 + xm] - LB[(3 * i) * n1 + xx];
                        const float f = LB[(3 * i + 1) * n1 + xm] + LB[(3 * i + 1) * n1 + xx];
                        const float q = LB[(3 * i + 2) * n1 + xm] + LB[(3 * i + 2) * n1 + xx];
                        if (yy >= 0) {
                            const float P = (pe[v][i] + e) + (pf[v][i] - f);
                            const float Q = pq[v][i] + q;
                            float* T = tp + (i * TY + yy) * n1 + xx;
                            if (zown) reinterpret_cast<float*>(W + (size_t)(i * TY + yy) * lsw)[xx] = (*T + P) - Q;
                            *T = P + Q;
                        }
                        pe[v][i] = e;
                        pf[v][i] = f;
                        pq[v][i] = q;
                    }
                }
            }
            if (!zown) continue;
            __syncthreads();  // the plane's nodal lines are complete
            // packed half-length FFT of the NLF real nodal lines, in place
            if (tid < NBAR) {
                const int q = tid / TPL, tau = tid - (tid / TPL) * TPL;
                const bool act = q < NLF;
                float2* Z = W + (size_t)(act ? q : 0) * lsw;
                auto lz = [&](int e) -> float2 { return act ? Z[e] : float2{0.f, 0.f}; };
                auto sz = [&](int e, float2 v) {
                    if (act) Z[e] = v;
                };
                fft_fast<float, M, false, true, true, NBAR>(lz, sz, lz, sz, act ? tau : 0, tws);
            }
            __syncthreads();
            // Hermitian split: X[k] = Ze + W^k Zo, k = 0 .. M, into components 0, 3, 6
            constexpr int half = M / 2;
            for (int e = tid; e < NLF * (half + 1); e += NT) {
                const int q = e / (half + 1), k = e - q * (half + 1);
                const int i = q / TY, yy = q - i * TY;
                const float2* z = W + (size_t)q * lsw;
                float2* o = a.spec + (int64_t)(3 * i) * g.Vs + (zrow + y0 + yy) * g.nhp;
                if (k == 0) {
                    const float2 z0v = z[0];
                    o[0] = float2{z0v.x + z0v.y, 0.f};
                    o[M] = float2{z0v.x - z0v.y, 0.f};
                    continue;
                }
                const int k2 = M - k;
                const float2 A = z[k], B = z[k2];
                {
                    const float2 Bc = c_conj(B);
                    const float2 Ze = c_scale(c_add(A, Bc), 0.5f);
                    const float2 D = c_sub(A, Bc);
                    const float2 Zo = float2{0.5f * D.y, -0.5f * D.x};
                    o[k] = c_add(Ze, c_mul(a.tw2[k], Zo));
                }
                if (k2 != k) {
                    const float2 Ac = c_conj(A);
                    const float2 Ze = c_scale(c_add(B, Ac), 0.5f);
                    const float2 D = c_sub(B, Ac);
                    const float2 Zo = float2{0.5f * D.y, -0.5f * D.x};
                    o[k2] = c_add(Ze, c_mul(a.tw2[k2], Zo));
                }
            }
            __syncthreads();  // the nodal lines are rewritten by the next plane
        }
        acc += (double)accp;
    }
    if (a.partial) {
        const double sacc = block_sum(acc, red);
        if (tid == 0) a.partial[blockIdx.x] = sacc;
        if (a.fuse && last_block(&sc->ticket[0], flag, gp)) {
            const double tot = sum_partials_fixed(a.partial + (size_t)pb * gp, gp, red);
            if (tid == 0) cg_alpha(sc, tot);
        }
    }
}

// ------------------------------------------------------------- launcher
template <int M, int TY, int C> static void xfwd_nodal_launch(NodalArgs a, cudaStream_t st)
{
    constexpr int threads = nodal_threads<M>();
    constexpr size_t sm = nodal_smem<M, TY>();
    static int per_sm = 0;
    if (per_sm == 0) {
        cudaFuncSetAttribute(k_xfwd_nodal<M, TY, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_xfwd_nodal<M, TY, C>, threads, sm) !=
                cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        per_sm = std::min(per_sm, 3);
    }
    const GridDims& g = a.g;
    const int slots = per_sm * num_sms_nodal();
    // one resident block per share (each run of planes re-forms the voxel
    // plane below it as halo)
    const int ncol = g.n2 / TY;
    const int64_t total = (int64_t)ncol * g.n3p;
    const int cap = std::max(1, slots / g.nprob);  // blocks per problem (partials: nodal_partials_max)
    // the L2 prefetch runs one voxel line ahead (measured at 256^3: 0.894 ms
    // per launch, against 0.936 two lines ahead, 1.133 four, 0.950 none)
    a.pfd = 1;
    int gp;
    if (a.cfg == 1 && ncol <= cap) {
        // equal chunks of planes per column, one item per block
        a.nch = std::max(1, std::min(g.n3p, cap / ncol));
        gp = ncol * a.nch;
    } else {
        a.nch = 0;  // even shares, one block per resident slot
        gp = (int)std::max<int64_t>(1, std::min<int64_t>(total, cap));
    }
    k_xfwd_nodal<M, TY, C><<<g.nprob * gp, threads, sm, st>>>(a);
}

template <int C> static void xfwd_nodal_pick(const NodalArgs& a, cudaStream_t st)
{
    switch (a.g.M) {
        case 64: xfwd_nodal_launch<64, 4, C>(a, st); break;
        case 128:
            if (a.g.n2 % 8 == 0)
                xfwd_nodal_launch<128, 8, C>(a, st);
            else
                xfwd_nodal_launch<128, 4, C>(a, st);
            break;
        default:
            if (a.g.n2 % 8 == 0)
                xfwd_nodal_launch<256, 8, C>(a, st);
            else
                xfwd_nodal_launch<256, 4, C>(a, st);
            break;
    }
}

// candidate 0: an even share of the (column, plane) pairs per block; 1: equal
// chunks of planes per column (neighbouring columns in step)
void launch_xfwd_nodal(NodalArgs a, cudaStream_t st) { xfwd_nodal_pick<1>(a, st); }

}  // namespace combo
