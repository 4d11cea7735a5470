// xpass.cu -- x-axis passes of one operator application.
//
//   x-forward : per-voxel constitutive law (paper Sec. 6.1; boxel stresses
//               come from the laminate kernel) or tangent application, then
//               a real-to-complex FFT along x (packed half-length complex
//               transform + Hermitian split), written to the half spectrum.
//   x-inverse : complex-to-real FFT along x and the solver update fused in
//               (fixed point F -= G[P]/mu0, or the CG updates x += a p,
//               r -= a q with (r, r)).
//
// Real fields are [9][n3][n2][n1] (x fastest).  A block strides over groups
// of LB x-lines; each thread issues all of a voxel's loads before any
// arithmetic, so the DRAM round trips overlap.  Dot products are summed in
// FP32 within a thread's share of a group and in FP64 across groups: FP64
// arithmetic runs at a small fraction of the FP32 rate on this GPU.
#include <algorithm>
#include <type_traits>

#include "combo_internal.cuh"
#include "fft_fast.cuh"
#include "../../include/combo.h"

namespace combo {

// ping-pong line buffers, reduction scratch and flag, twiddle table
size_t xpass_smem(const GridDims& g, int lines, size_t cxbytes)
{
    return 2 * (size_t)9 * lines * (g.M + 1) * cxbytes + 256 * sizeof(double) + 16 + (size_t)g.M * cxbytes;
}

int xpass_lines(const GridDims& g, size_t cxbytes)
{
    // keep the two ping-pong buffers under ~48 KB while covering >= 512 voxels
    int lines = 1;
    while (lines * g.n1 < 512 && xpass_smem(g, lines * 2, cxbytes) <= 48 * 1024 &&
           (g.n2 * g.n3p) % (lines * 2) == 0)
        lines *= 2;
    return lines;
}

// x-pass grid: a few resident blocks per SM stride over the line groups, so
// that the fused reductions see few partials and few tickets.
static int grid_cap(const GridDims&)
{
    static int nsm = 0;
    if (nsm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) nsm = 152;
    }
    return 4 * nsm;
}

int xpass_partials_max(const GridDims& g) { return 2 * grid_cap(g) + g.nprob; }

// blocks per problem: the problem's line groups, at most cap / nprob
int xpass_gp(const GridDims& g, int lines, int cap)
{
    const int groups = (g.n2 * g.n3p + lines - 1) / lines;
    return std::max(1, std::min(groups, cap / g.nprob));
}

int xpass_grid(const GridDims& g, int lines) { return g.nprob * xpass_gp(g, lines, grid_cap(g)); }

template <typename K> static void allow_smem(K kernel, bool& done)
{
    if (!done) {
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        done = true;
    }
}

// x-pass FFT of the nl lines held in shared memory: compile-time plan when MF > 0
template <typename T, int MF, bool INV>
__device__ __forceinline__ cx<T>* xpass_fft(cx<T>* b0, cx<T>* b1, const Plan& plan, int nl, int ls, const cx<T>* tw)
{
    if constexpr (MF > 0)
        return fft_lines_fast<T, MF, INV>(b0, b1, nl, ls, tw);
    else
        return fft_lines<T, INV>(b0, b1, plan, nl, ls, 1, tw);
}

template <typename S> struct Pair;
template <> struct Pair<float> { typedef float2 type; };
template <> struct Pair<double> { typedef double2 type; };
template <typename S> using pair_t = typename Pair<S>::type;

template <typename S> __device__ __forceinline__ pair_t<S> ld2(const S* __restrict__ p)
{
    return *reinterpret_cast<const pair_t<S>*>(p);
}
template <typename S> __device__ __forceinline__ void st2(S* __restrict__ p, S a, S b)
{
    *reinterpret_cast<pair_t<S>*>(p) = pair_t<S>{a, b};
}

// Neo-Hookean stress (Sec. 6.1) in FP64: P = mu F + (lam ln J - mu) F^{-T};
// G = F^{-1} and m = mu - lam ln J for the tangent cache.  False if J <= 0.
__device__ __forceinline__ bool nh_stress(const double F[9], double mu, double lam, double P[9], double G[9], double& m)
{
    const double c0 = F[4] * F[8] - F[5] * F[7];
    const double c1 = F[5] * F[6] - F[3] * F[8];
    const double c2 = F[3] * F[7] - F[4] * F[6];
    const double J = F[0] * c0 + F[1] * c1 + F[2] * c2;
    if (!(J > 0.0)) return false;
    const double iJ = 1.0 / J;
    G[0] = c0 * iJ;
    G[1] = (F[2] * F[7] - F[1] * F[8]) * iJ;
    G[2] = (F[1] * F[5] - F[2] * F[4]) * iJ;
    G[3] = c1 * iJ;
    G[4] = (F[0] * F[8] - F[2] * F[6]) * iJ;
    G[5] = (F[2] * F[3] - F[0] * F[5]) * iJ;
    G[6] = c2 * iJ;
    G[7] = (F[1] * F[6] - F[0] * F[7]) * iJ;
    G[8] = (F[0] * F[4] - F[1] * F[3]) * iJ;
    const double lnJ = log(J);
    const double k = lam * lnJ - mu;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) P[3 * i + j] = mu * F[3 * i + j] + k * G[3 * j + i];
    m = mu - lam * lnJ;
    return true;
}

// The same stress with the cofactors, J, F^{-1}, ln J (df_log) and P in
// double-float; G and m, the tangent cache of the FP32 Krylov iterations, are
// rounded to FP32.  False if J <= 0.
__device__ __forceinline__ bool nh_stress_df(const double Fd[9], df32 mud, df32 lamd, df32 P[9], float G[9],
                                             float& m)
{
    df32 F[9];
#pragma unroll
    for (int c = 0; c < 9; c++) F[c] = df32(Fd[c]);
    const df32 c0 = F[4] * F[8] - F[5] * F[7];
    const df32 c1 = F[5] * F[6] - F[3] * F[8];
    const df32 c2 = F[3] * F[7] - F[4] * F[6];
    const df32 J = F[0] * c0 + F[1] * c1 + F[2] * c2;
    if (!(J.hi > 0.f)) return false;
    const df32 iJ = df32(1.f, 0.f) / J;
    df32 Gi[9];
    Gi[0] = c0 * iJ;
    Gi[1] = (F[2] * F[7] - F[1] * F[8]) * iJ;
    Gi[2] = (F[1] * F[5] - F[2] * F[4]) * iJ;
    Gi[3] = c1 * iJ;
    Gi[4] = (F[0] * F[8] - F[2] * F[6]) * iJ;
    Gi[5] = (F[2] * F[3] - F[0] * F[5]) * iJ;
    Gi[6] = c2 * iJ;
    Gi[7] = (F[1] * F[6] - F[0] * F[7]) * iJ;
    Gi[8] = (F[0] * F[4] - F[1] * F[3]) * iJ;
    const df32 lnJ = df_log(J);
    const df32 k = lamd * lnJ - mud;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) P[3 * i + j] = mud * F[3 * i + j] + k * Gi[3 * j + i];
#pragma unroll
    for (int c = 0; c < 9; c++) G[c] = (float)Gi[c];
    m = -(float)k;
    return true;
}

// ------------------------------------------------------------- x forward
// TAN: the Krylov tangent pass (a.mode == XF_TANGENT, no external X), whose
// FP32 instance is register-capped for three resident blocks per SM
// The pass body of one block: vb of vg blocks (a launch of its own: the
// block index and grid size; a grouped launch: a work item of one grid).
template <typename T, typename Tc, int MF, bool TAN>
__device__ __forceinline__ void xfwd_body(const XfwdArgs<T, Tc>& a, int guard, int vb, int vg,
                                          unsigned char* smem_raw)
{
    const GridDims g = a.g;
    int pb, pj, gp;  // problem of this block, index among its gp blocks
    prob_block(g, vb, vg, pb, pj, gp);
    Scalars* sc = a.sc + pb;
    if (guard == 1 && sc->cg_done) return;
    if (guard == 2 && sc->outer_done) return;
    const int LB = a.lines_per_block;
    const int ls = g.M + 1;
    cx<T>* buf0 = reinterpret_cast<cx<T>*>(smem_raw);
    cx<T>* buf1 = buf0 + (size_t)9 * LB * ls;
    double* red = reinterpret_cast<double*>(buf1 + (size_t)9 * LB * ls);
    int* flag = reinterpret_cast<int*>(red + 256);
    cx<T>* tws = reinterpret_cast<cx<T>*>(flag + 4);  // twiddles exp(-2 pi i t / M)
    for (int i = threadIdx.x; i < g.M; i += blockDim.x) tws[i] = a.tw[i];
    T* rb = reinterpret_cast<T*>(buf0);
    const int nlp = g.n2 * g.n3p;  // x-lines of one problem
    const int Lbase = pb * nlp, Lend = Lbase + nlp;
    const int ngroups = (nlp + LB - 1) / LB;
    const int64_t V = g.V;
    double acc = 0.0;
    double mu[2], lam[2];
    df32 mu_df[2], lam_df[2];  // their double-float splits (once per block, off the per-voxel FP64 pipe)
    for (int i = 0; i < 2; i++) {
        mu[i] = a.matp ? a.matp[4 * pb + i] : a.mu[i];
        lam[i] = a.matp ? a.matp[4 * pb + 2 + i] : a.lam[i];
        mu_df[i] = df32(mu[i]);
        lam_df[i] = df32(lam[i]);
    }

    const bool first = (a.mode == XF_TANGENT) ? (sc->cg_iter == 0) : false;
    const Tc beta = (a.mode == XF_TANGENT && !first) ? (Tc)sc->beta : (Tc)0;
    const Tc apend = (a.mode == XF_TANGENT && !first) ? (Tc)sc->alpha_pending : (Tc)0;
    const uint8_t* __restrict__ phase = a.phase;

    // grid-stride over the problem's groups of LB x-lines
    for (int grp = pj; grp < ngroups; grp += gp) {
        const int L0 = Lbase + grp * LB;
        // dot products: FP32 within a thread's share of a group, FP64 across
        // groups (FP64 arithmetic runs at a small fraction of the FP32 rate)
        Tc accp = 0;
        for (int e = threadIdx.x; e < LB * g.n1; e += blockDim.x) {
            const int l = e / g.n1, x = e - l * g.n1;
            const int L = L0 + l;
            if (L >= Lend) continue;
            const int64_t v = (int64_t)L * g.n1 + x;
            T o[9];
            if constexpr (!TAN) {
              if (a.X) {
#pragma unroll
                for (int c = 0; c < 9; c++) o[c] = (T)a.X[c * V + v];
              } else if (a.Xc) {
#pragma unroll
                for (int c = 0; c < 9; c++) o[c] = (T)a.Xc[c * V + v];
              } else {  // XF_RESID
                const int ph = phase[v];
                double F[9];
#pragma unroll
                for (int c = 0; c < 9; c++) F[c] = a.F[c * V + v];
                if (ph == 2) {
                    const int b = a.vox2box[v];
#pragma unroll
                    for (int c = 0; c < 9; c++) o[c] = (T)a.bP[(int64_t)b * 9 + c];
                    if (a.tc) {
#pragma unroll
                        for (int c = 0; c < 10; c++) a.tc[c * V + v] = (Tc)0;
                    }
                } else if (a.linear) {
                    // infinitesimal strain: sigma = C : sym(F - I); the tangent
                    // cache holds G = I, m = mu, for which the Neo-Hookean
                    // tangent formula is exactly C
                    double S[9];
                    lin_sigma(F, mu[ph], lam[ph], S);
#pragma unroll
                    for (int c = 0; c < 9; c++) o[c] = (T)S[c];
                    if (a.tc) {
#pragma unroll
                        for (int c = 0; c < 9; c++) a.tc[c * V + v] = (Tc)((c == 0 || c == 4 || c == 8) ? 1.0 : 0.0);
                        a.tc[9 * V + v] = (Tc)mu[ph];
                    }
                } else if constexpr (std::is_same<T, df32>::value) {
                    float G[9], m;
                    if (!nh_stress_df(F, mu_df[ph], lam_df[ph], o, G, m)) {
                        raise_status(sc, finite9(F) ? COMBO_E_INADMISSIBLE : COMBO_E_NAN);
#pragma unroll
                        for (int c = 0; c < 9; c++) {
                            o[c] = df32(0.f, 0.f);
                            G[c] = 0.f;
                        }
                        m = 0.f;
                    }
                    if (a.tc) {
#pragma unroll
                        for (int c = 0; c < 9; c++) a.tc[c * V + v] = (Tc)G[c];
                        a.tc[9 * V + v] = (Tc)m;
                    }
                } else {
                    double P[9], G[9], m;
                    if (!nh_stress(F, mu[ph], lam[ph], P, G, m)) {
                        raise_status(sc, finite9(F) ? COMBO_E_INADMISSIBLE : COMBO_E_NAN);
#pragma unroll
                        for (int c = 0; c < 9; c++) P[c] = G[c] = 0.0;
                        m = 0.0;
                    }
#pragma unroll
                    for (int c = 0; c < 9; c++) o[c] = (T)P[c];
                    if (a.tc) {
#pragma unroll
                        for (int c = 0; c < 9; c++) a.tc[c * V + v] = (Tc)G[c];
                        a.tc[9 * V + v] = (Tc)m;
                    }
                }
              }
            } else {  // XF_TANGENT: x += alpha_prev p, p = r + beta p, y = A : p
                // every load is issued before the first store and before the
                // phase branch, so that one memory latency covers all of them
                const Tc* __restrict__ rg = a.r;
                Tc* __restrict__ pg = a.p;
                Tc* __restrict__ xg = a.x;
                const Tc* __restrict__ tg = a.tc;
                const int ph = phase[v];
                Tc p[9], po[9], xo[9], t[10];
#pragma unroll
                for (int c = 0; c < 9; c++) p[c] = rg[c * V + v];
#pragma unroll
                for (int c = 0; c < 10; c++) t[c] = tg[c * V + v];
                if (!first) {
#pragma unroll
                    for (int c = 0; c < 9; c++) po[c] = pg[c * V + v];
                    if (apend != (Tc)0) {
#pragma unroll
                        for (int c = 0; c < 9; c++) xo[c] = xg[c * V + v];
#pragma unroll
                        for (int c = 0; c < 9; c++) xg[c * V + v] = xo[c] + apend * po[c];
                    }
#pragma unroll
                    for (int c = 0; c < 9; c++) p[c] += beta * po[c];
                }
#pragma unroll
                for (int c = 0; c < 9; c++) pg[c * V + v] = p[c];
                if (ph == 2) {
                    // boxel: p parks in the transform buffer; the boxel phase
                    // below replaces it by A_box : p
#pragma unroll
                    for (int c = 0; c < 9; c++) o[c] = (T)p[c];
                } else {
                    Tc y[9];
                    nh_tangent<Tc>(t, t[9], (Tc)mu[ph], (Tc)lam[ph], p, y);
                    Tc s = 0;
#pragma unroll
                    for (int c = 0; c < 9; c++) {
                        s += p[c] * y[c];
                        o[c] = (T)y[c];
                    }
                    accp += s;
                }
            }
#pragma unroll
            for (int c = 0; c < 9; c++) rb[(size_t)2 * (c * LB + l) * ls + x] = o[c];
        }
        if constexpr (TAN) {
            // boxels of the group, in voxel order: consecutive threads read
            // consecutive columns of the packed tangents (coalesced, no divergence)
            __syncthreads();
            const int k0 = a.lofs[L0], k1 = a.lofs[min(L0 + LB, Lend)];
            for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
                const int64_t v = a.bvox[k];
                const int l = (int)(v / g.n1) - L0, x = (int)(v % g.n1);
                Tc Ak[45], p[9];
#pragma unroll
                for (int j = 0; j < 45; j++) Ak[j] = a.bA[(int64_t)j * a.nb + k];
#pragma unroll
                for (int c = 0; c < 9; c++) p[c] = (Tc)rb[(size_t)2 * (c * LB + l) * ls + x];
                Tc s = 0;
#pragma unroll
                for (int r = 0; r < 9; r++) {
                    Tc yr = 0;
#pragma unroll
                    for (int c = 0; c < 9; c++) yr += Ak[sym_idx(r, c)] * p[c];
                    s += p[r] * yr;
                    rb[(size_t)2 * (r * LB + l) * ls + x] = (T)yr;
                }
                accp += s;
            }
        }
        acc += (double)accp;
        __syncthreads();

        if constexpr (TAN) {
            // the next group's operand rows (r, p, x, tangent cache) are
            // prefetched into L2 while this group is transformed, so that its
            // voxel phase finds them there
            const int gn = grp + gp;
            if (gn < ngroups) {
                const int L0n = Lbase + gn * LB;
                const int nlines = min(LB, Lend - L0n);
                const int chunks = (g.n1 * (int)sizeof(Tc) + 127) / 128;  // 128-B lines per x-line
                const int ncomp = 19 + (first ? 0 : 9) + (apend != (Tc)0 ? 9 : 0);
                const int total = ncomp * nlines * chunks;
                for (int e = threadIdx.x; e < total; e += blockDim.x) {
                    const int q = e % chunks, rest = e / chunks;
                    const int l = rest % nlines, c = rest / nlines;
                    const Tc* base;
                    if (c < 9)
                        base = a.r + (int64_t)c * V;
                    else if (c < 19)
                        base = a.tc + (int64_t)(c - 9) * V;
                    else if (!first && c < 28)
                        base = a.p + (int64_t)(c - 19) * V;
                    else
                        base = a.x + (int64_t)(c - (first ? 19 : 28)) * V;
                    const char* ptr = reinterpret_cast<const char*>(base + (int64_t)(L0n + l) * g.n1) + 128 * q;
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(ptr));
                }
            }
        }

        const int nl = 9 * LB;
        cx<T>* Z = xpass_fft<T, MF, false>(buf0, buf1, a.plan, nl, ls, tws);

        // Hermitian split of the packed transform: X[k] = Ze + W^k Zo, k = 0..M
        const int M = g.M;
        const int half = M / 2;
        for (int e = threadIdx.x; e < nl * (half + 1); e += blockDim.x) {
            const int q = e / (half + 1), k = e - q * (half + 1);  // k fastest: coalesced stores
            const int c = q / LB, l = q - c * LB;
            const int L = L0 + l;
            if (L >= Lend) continue;
            const cx<T>* z = Z + (size_t)q * ls;
            cx<T>* o = a.spec + c * g.Vs + (int64_t)L * g.nhp;
            if (k == 0) {
                const cx<T> z0 = z[0];
                o[0] = cx<T>{z0.x + z0.y, (T)0};
                o[M] = cx<T>{z0.x - z0.y, (T)0};
                continue;
            }
            const int k2 = M - k;
            const cx<T> A = z[k], B = z[k2];
            {
                const cx<T> Bc = c_conj(B);
                const cx<T> Ze = c_scale(c_add(A, Bc), (T)0.5);
                const cx<T> D = c_sub(A, Bc);
                const cx<T> Zo = cx<T>{(T)0.5 * D.y, (T)-0.5 * D.x};
                o[k] = c_add(Ze, c_mul(a.tw2[k], Zo));
            }
            if (k2 != k) {
                const cx<T> Ac = c_conj(A);
                const cx<T> Ze = c_scale(c_add(B, Ac), (T)0.5);
                const cx<T> D = c_sub(B, Ac);
                const cx<T> Zo = cx<T>{(T)0.5 * D.y, (T)-0.5 * D.x};
                o[k2] = c_add(Ze, c_mul(a.tw2[k2], Zo));
            }
        }
        __syncthreads();  // the next group reuses the shared buffers
    }
    if (TAN && a.partial) {
        const double s = block_sum(acc, red);
        if (threadIdx.x == 0) a.partial[vb] = s;
        if (a.fuse && last_block(&sc->ticket[0], flag, gp)) {
            const double tot = sum_partials_fixed(a.partial + (size_t)pb * gp, gp, red);
            if (threadIdx.x == 0) cg_alpha(sc, tot);
        }
    }
}

// blocks per SM the x-forward is register-capped for: FP32 tangent pass 4,
// FP64 / double-float constitutive pass 2, else 1
template <typename T, bool TAN> constexpr int xfwd_minb()
{
    return (TAN && sizeof(T) == 4) ? 4 : ((!TAN && sizeof(T) == 8) ? 2 : 1);
}

template <typename T, typename Tc, int MF, bool TAN>
__global__ void __launch_bounds__(256, (xfwd_minb<T, TAN>())) k_xfwd(XfwdArgs<T, Tc> a, int guard)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    xfwd_body<T, Tc, MF, TAN>(a, guard, blockIdx.x, gridDim.x, smem_raw);
}

// ------------------------------------------------------------- x inverse
template <typename T, typename Tc, int MF>
__device__ __forceinline__ void xinv_body(const XinvArgs<T, Tc>& a, int guard, int vb, int vg,
                                          unsigned char* smem_raw)
{
    const GridDims g = a.g;
    int pb, pj, gp;  // problem of this block, index among its gp blocks
    prob_block(g, vb, vg, pb, pj, gp);
    Scalars* sc = a.sc + pb;
    if (guard == 1 && sc->cg_done) return;
    if (guard == 2 && sc->outer_done) return;
    const int LB = a.lines_per_block;
    const int ls = g.M + 1;
    const int M = g.M;
    cx<T>* buf0 = reinterpret_cast<cx<T>*>(smem_raw);
    cx<T>* buf1 = buf0 + (size_t)9 * LB * ls;
    double* red = reinterpret_cast<double*>(buf1 + (size_t)9 * LB * ls);
    int* flag = reinterpret_cast<int*>(red + 256);
    cx<T>* tws = reinterpret_cast<cx<T>*>(flag + 4);  // twiddles exp(-2 pi i t / M)
    for (int i = threadIdx.x; i < g.M; i += blockDim.x) tws[i] = a.tw[i];
    const int nlp = g.n2 * g.n3p;  // x-lines of one problem
    const int Lbase = pb * nlp, Lend = Lbase + nlp;
    const int ngroups = (nlp + LB - 1) / LB;
    const int nl = 9 * LB;
    const int64_t V = g.V;
    double acc = 0.0;
    const bool skip_update = (a.mode == XI_FIXEDPOINT || a.mode == XI_NCG) && sc->outer_done;
    const double ncg_beta = (a.mode == XI_NCG) ? sc->beta : 0.0;
    const Tc alpha = (a.mode == XI_CG) ? (Tc)sc->alpha : (Tc)0;

    // grid-stride over the problem's groups of LB x-lines
    for (int grp = pj; grp < ngroups; grp += gp) {
        const int L0 = Lbase + grp * LB;
        for (int e = threadIdx.x; e < nl * (M + 1); e += blockDim.x) {
            const int q = e / (M + 1), k = e - q * (M + 1);
            const int c = q / LB, l = q - c * LB;
            const int L = L0 + l;
            buf0[(size_t)q * ls + k] =
                (L < Lend) ? a.spec[c * g.Vs + (int64_t)L * g.nhp + k] : cx<T>{(T)0, (T)0};
        }
        __syncthreads();
        // Z[k] = Ze + i Zo,  Ze = (X[k] + conj X[M-k]) / 2,  Zo = (X[k] - conj X[M-k]) W^{-k} / 2
        for (int e = threadIdx.x; e < nl * M; e += blockDim.x) {
            const int q = e / M, k = e - q * M;
            const cx<T> A = buf0[(size_t)q * ls + k];
            const cx<T> Bc = c_conj(buf0[(size_t)q * ls + (M - k)]);
            const cx<T> Ze = c_scale(c_add(A, Bc), (T)0.5);
            const cx<T> Zo = c_mul(c_scale(c_sub(A, Bc), (T)0.5), c_conj(a.tw2[k]));
            buf1[(size_t)q * ls + k] = cx<T>{Ze.x - Zo.y, Ze.y + Zo.x};
        }
        __syncthreads();
        cx<T>* Zr = xpass_fft<T, MF, true>(buf1, buf0, a.plan, nl, ls, tws);
        const T* rb = reinterpret_cast<const T*>(Zr);
        Tc accp = 0;  // FP32 within the group, FP64 across groups

        for (int e = threadIdx.x; e < LB * g.n1; e += blockDim.x) {
            const int l = e / g.n1, x = e - l * g.n1;
            const int L = L0 + l;
            if (L >= Lend) continue;
            const int64_t v = (int64_t)L * g.n1 + x;
            if (a.mode == XI_CG) {
                // r -= alpha q; the matching x += alpha p is done by the next
                // tangent x-pass (or the F update when CG stops)
                Tc rv[9];
#pragma unroll
                for (int c = 0; c < 9; c++) rv[c] = a.r[c * V + v];
#pragma unroll
                for (int c = 0; c < 9; c++) {
                    const Tc gv = (Tc)rb[(size_t)2 * (c * LB + l) * ls + x];
                    const Tc rn = rv[c] - alpha * gv;
                    a.r[c * V + v] = rn;
                    accp += rn * rn;
                }
            } else if (a.mode == XI_FIXEDPOINT) {
                if (skip_update) continue;
                double* __restrict__ Fg = a.F;
                double Fo[9];
#pragma unroll
                for (int c = 0; c < 9; c++) Fo[c] = Fg[c * V + v];
#pragma unroll
                for (int c = 0; c < 9; c++) Fg[c * V + v] = Fo[c] - (double)rb[(size_t)2 * (c * LB + l) * ls + x] * a.inv_mu0;
            } else if (a.mode == XI_NCG) {
                // d = -G[P]/mu0 + beta d, F += d (Fletcher-Reeves, basic-scheme step)
                if (skip_update) continue;
                double* __restrict__ Fg = a.F;
                double* __restrict__ dg = a.d;
                double Fo[9], dn[9];
#pragma unroll
                for (int c = 0; c < 9; c++) {
                    Fo[c] = Fg[c * V + v];
                    dn[c] = dg[c * V + v];
                }
#pragma unroll
                for (int c = 0; c < 9; c++) {
                    const double d = -(double)rb[(size_t)2 * (c * LB + l) * ls + x] * a.inv_mu0 + ncg_beta * dn[c];
                    dg[c * V + v] = d;
                    Fg[c * V + v] = Fo[c] + d;
                }
            } else if (a.mode == XI_RHS) {
#pragma unroll
                for (int c = 0; c < 9; c++) {
                    const Tc rn = (Tc)(-rb[(size_t)2 * (c * LB + l) * ls + x]);
                    a.r[c * V + v] = rn;
                    a.x[c * V + v] = (Tc)0;
                    accp += rn * rn;
                }
            } else {
#pragma unroll
                for (int c = 0; c < 9; c++) a.Y[c * V + v] = (double)rb[(size_t)2 * (c * LB + l) * ls + x];
            }
        }
        acc += (double)accp;
        __syncthreads();  // the next group reuses the shared buffers
    }
    if ((a.mode == XI_RHS || a.mode == XI_CG) && a.partial) {
        const double s = block_sum(acc, red);
        if (threadIdx.x == 0) a.partial[vb] = s;
        if (a.mode == XI_CG && a.fuse && last_block(&sc->ticket[1], flag, gp)) {
            const double tot = sum_partials_fixed(a.partial + (size_t)pb * gp, gp, red);
            if (threadIdx.x == 0) cg_beta(sc, tot, a.cg_tol, a.cg_max, a.cg_fixed);
        }
    }
}

template <typename T, typename Tc, int MF>
__global__ void __launch_bounds__(256) k_xinv(XinvArgs<T, Tc> a, int guard)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    xinv_body<T, Tc, MF>(a, guard, blockIdx.x, gridDim.x, smem_raw);
}

// ------------------------------------------------------------- launchers
template <typename T, typename Tc, int MF> static void xfwd_launch(const XfwdArgs<T, Tc>& a, int guard, cudaStream_t st)
{
    const int grid = xpass_grid(a.g, a.lines_per_block);
    const size_t sm = xpass_smem(a.g, a.lines_per_block, sizeof(cx<T>));
    if constexpr (std::is_same<T, Tc>::value) {  // the tangent pass runs in the Krylov precision
        if (a.mode == XF_TANGENT && !a.X) {
            static bool attr = false;
            allow_smem(k_xfwd<T, Tc, MF, true>, attr);
            if constexpr (sizeof(T) == 4 && MF > 0) {
                // FP32: small blocks of 128 threads whose FFT phase keeps most
                // of them busy (9 lines x TPL threads per x-line), as many
                // resident per SM as registers allow, one wave
                // candidate 1 (autotuner): the engine's group of lines in 256 threads
                constexpr int TPL = FastPlan<MF>::TPL;
                int lb = a.lines_per_block;
                if (a.cfg != 1)
                    while (lb > 1 && 9 * lb * TPL > 128) lb >>= 1;
                const int threads = (a.cfg != 1 && 9 * lb * TPL <= 128) ? 128 : 256;
                XfwdArgs<T, Tc> b = a;
                b.lines_per_block = lb;
                const size_t smb = xpass_smem(a.g, lb, sizeof(cx<T>));
                static int per_sm_c[2] = {0, 0};
                int& per_sm = per_sm_c[threads == 256 ? 1 : 0];
                if (per_sm == 0 &&
                    (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_xfwd<T, Tc, MF, true>, threads, smb) !=
                         cudaSuccess ||
                     per_sm < 1))
                    per_sm = 1;
                const int tgrid = a.g.nprob * xpass_gp(a.g, lb, per_sm * (grid_cap(a.g) / 4));
                k_xfwd<T, Tc, MF, true><<<tgrid, threads, smb, st>>>(b, guard);
            } else {
                k_xfwd<T, Tc, MF, true><<<grid, 256, sm, st>>>(a, guard);
            }
            return;
        }
    }
    {
        static bool attr = false;
        allow_smem(k_xfwd<T, Tc, MF, false>, attr);
        k_xfwd<T, Tc, MF, false><<<grid, 256, sm, st>>>(a, guard);
    }
}

template <typename T, typename Tc> void launch_xfwd(const XfwdArgs<T, Tc>& a, int guard, cudaStream_t st)
{
    if constexpr (std::is_same<T, float>::value && std::is_same<Tc, float>::value) {
        // 2^a 3^b half lengths: compile-time plans in the FP32 passes
        switch (a.g.M) {
            case 24: xfwd_launch<T, Tc, 24>(a, guard, st); return;
            case 36: xfwd_launch<T, Tc, 36>(a, guard, st); return;
            case 48: xfwd_launch<T, Tc, 48>(a, guard, st); return;
            case 54: xfwd_launch<T, Tc, 54>(a, guard, st); return;
            case 72: xfwd_launch<T, Tc, 72>(a, guard, st); return;
            case 96: xfwd_launch<T, Tc, 96>(a, guard, st); return;
            case 108: xfwd_launch<T, Tc, 108>(a, guard, st); return;
            default: break;
        }
    }
    switch (a.g.M) {
        case 32: xfwd_launch<T, Tc, 32>(a, guard, st); break;
        case 64: xfwd_launch<T, Tc, 64>(a, guard, st); break;
        case 128: xfwd_launch<T, Tc, 128>(a, guard, st); break;
        case 256: xfwd_launch<T, Tc, 256>(a, guard, st); break;
        default: xfwd_launch<T, Tc, 0>(a, guard, st); break;
    }
}

template <typename T, typename Tc, int MF> static void xinv_launch(const XinvArgs<T, Tc>& a, int guard, cudaStream_t st)
{
    const int grid = xpass_grid(a.g, a.lines_per_block);
    const size_t sm = xpass_smem(a.g, a.lines_per_block, sizeof(cx<T>));
    static bool attr = false;
    allow_smem(k_xinv<T, Tc, MF>, attr);
    k_xinv<T, Tc, MF><<<grid, 256, sm, st>>>(a, guard);
}

// ------------------------------------------------------------- Newton right-hand side, FP32
// The c2r of the double-float residual spectrum in the Newton right-hand-side
// mode: r = -G[P] and x = 0 are FP32 words (the Krylov precision), so the
// inverse transform runs in FP32 arithmetic on the double-float spectrum
// rounded to FP32 (the residual norm that decides convergence is summed in
// double-float by the z-pass).  Same groups, grid and partial sums as the
// double-float x-inverse it replaces.
template <int M>
__global__ void __launch_bounds__(256) k_xinv_rhs32(XinvArgs<df32, float> a, const float2* __restrict__ tw32,
                                                    const float2* __restrict__ tw2_32, int guard)
{
    const GridDims g = a.g;
    int pb, pj, gp;
    prob_block(g, blockIdx.x, gridDim.x, pb, pj, gp);
    Scalars* sc = a.sc + pb;
    if (guard == 1 && sc->cg_done) return;
    if (guard == 2 && sc->outer_done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int LB = a.lines_per_block;
    constexpr int ls = M + 1;
    float2* buf0 = reinterpret_cast<float2*>(smem_raw);
    float2* buf1 = buf0 + (size_t)9 * LB * ls;
    double* red = reinterpret_cast<double*>(buf1 + (size_t)9 * LB * ls);
    int* flag = reinterpret_cast<int*>(red + 256);
    float2* tws = reinterpret_cast<float2*>(flag + 4);
    for (int i = threadIdx.x; i < M; i += blockDim.x) tws[i] = tw32[i];
    const int nlp = g.n2 * g.n3p;
    const int Lbase = pb * nlp, Lend = Lbase + nlp;
    const int ngroups = (nlp + LB - 1) / LB;
    const int nl = 9 * LB;
    const int64_t V = g.V;
    double acc = 0.0;
    for (int grp = pj; grp < ngroups; grp += gp) {
        const int L0 = Lbase + grp * LB;
        // Z[k] = Ze + i Zo,  Ze = (X[k] + conj X[M-k]) / 2,  Zo = (X[k] - conj X[M-k]) W^{-k} / 2,
        // from the spectrum rounded to FP32
        for (int e = threadIdx.x; e < nl * M; e += blockDim.x) {
            const int q = e / M, k = e - q * M;
            const int c = q / LB, l = q - c * LB;
            const int L = L0 + l;
            float2 z{0.f, 0.f};
            if (L < Lend) {
                const cx<df32>* row = a.spec + c * g.Vs + (int64_t)L * g.nhp;
                const cx<df32> xa = row[k], xb = row[M - k];
                const float2 A{xa.x.hi + xa.x.lo, xa.y.hi + xa.y.lo};
                const float2 Bc{xb.x.hi + xb.x.lo, -(xb.y.hi + xb.y.lo)};
                const float2 Ze = c_scale(c_add(A, Bc), 0.5f);
                const float2 Zo = c_mul(c_scale(c_sub(A, Bc), 0.5f), c_conj(tw2_32[k]));
                z = float2{Ze.x - Zo.y, Ze.y + Zo.x};
            }
            buf1[(size_t)q * ls + k] = z;
        }
        __syncthreads();
        const float2* Zr = fft_lines_fast<float, M, true>(buf1, buf0, nl, ls, tws);
        const float* rb = reinterpret_cast<const float*>(Zr);
        float accp = 0.f;
        for (int e = threadIdx.x; e < LB * g.n1; e += blockDim.x) {
            const int l = e / g.n1, x = e - l * g.n1;
            const int L = L0 + l;
            if (L >= Lend) continue;
            const int64_t v = (int64_t)L * g.n1 + x;
#pragma unroll
            for (int c = 0; c < 9; c++) {
                const float rn = -rb[(size_t)2 * (c * LB + l) * ls + x];
                a.r[c * V + v] = rn;
                a.x[c * V + v] = 0.f;
                accp += rn * rn;
            }
        }
        acc += (double)accp;
        __syncthreads();  // the next group reuses the shared buffers
    }
    if (a.partial) {
        const double s2 = block_sum(acc, red);
        if (threadIdx.x == 0) a.partial[blockIdx.x] = s2;
    }
}

template <int M> static void xinv_rhs32_launch(const XinvArgs<df32, float>& a, const cx<float>* tw32,
                                               const cx<float>* tw2_32, int guard, cudaStream_t st)
{
    const int grid = xpass_grid(a.g, a.lines_per_block);
    const size_t sm = xpass_smem(a.g, a.lines_per_block, sizeof(cx<float>));
    static bool attr = false;
    allow_smem(k_xinv_rhs32<M>, attr);
    k_xinv_rhs32<M><<<grid, 256, sm, st>>>(a, tw32, tw2_32, guard);
}

bool xinv_rhs32_ok(const GridDims& g) { return fast_size_x(g.M) || fast3_size_x(g.M); }

void launch_xinv_rhs32(const XinvArgs<df32, float>& a, const cx<float>* tw32, const cx<float>* tw2_32, int guard,
                       cudaStream_t st)
{
    switch (a.g.M) {
        case 24: xinv_rhs32_launch<24>(a, tw32, tw2_32, guard, st); break;
        case 32: xinv_rhs32_launch<32>(a, tw32, tw2_32, guard, st); break;
        case 36: xinv_rhs32_launch<36>(a, tw32, tw2_32, guard, st); break;
        case 48: xinv_rhs32_launch<48>(a, tw32, tw2_32, guard, st); break;
        case 54: xinv_rhs32_launch<54>(a, tw32, tw2_32, guard, st); break;
        case 64: xinv_rhs32_launch<64>(a, tw32, tw2_32, guard, st); break;
        case 72: xinv_rhs32_launch<72>(a, tw32, tw2_32, guard, st); break;
        case 96: xinv_rhs32_launch<96>(a, tw32, tw2_32, guard, st); break;
        case 108: xinv_rhs32_launch<108>(a, tw32, tw2_32, guard, st); break;
        case 128: xinv_rhs32_launch<128>(a, tw32, tw2_32, guard, st); break;
        default: xinv_rhs32_launch<256>(a, tw32, tw2_32, guard, st); break;
    }
}

template <typename T, typename Tc> void launch_xinv(const XinvArgs<T, Tc>& a, int guard, cudaStream_t st)
{
    if constexpr (std::is_same<T, float>::value && std::is_same<Tc, float>::value) {
        if (a.mode == XI_CG && guard == 1 && stream_xpass_ok(a.g)) {
            launch_xinv_stream(a, st);
            return;
        }
    }
    if constexpr (std::is_same<T, float>::value && std::is_same<Tc, float>::value) {
        switch (a.g.M) {
            case 24: xinv_launch<T, Tc, 24>(a, guard, st); return;
            case 36: xinv_launch<T, Tc, 36>(a, guard, st); return;
            case 48: xinv_launch<T, Tc, 48>(a, guard, st); return;
            case 54: xinv_launch<T, Tc, 54>(a, guard, st); return;
            case 72: xinv_launch<T, Tc, 72>(a, guard, st); return;
            case 96: xinv_launch<T, Tc, 96>(a, guard, st); return;
            case 108: xinv_launch<T, Tc, 108>(a, guard, st); return;
            default: break;
        }
    }
    switch (a.g.M) {
        case 32: xinv_launch<T, Tc, 32>(a, guard, st); break;
        case 64: xinv_launch<T, Tc, 64>(a, guard, st); break;
        case 128: xinv_launch<T, Tc, 128>(a, guard, st); break;
        case 256: xinv_launch<T, Tc, 256>(a, guard, st); break;
        default: xinv_launch<T, Tc, 0>(a, guard, st); break;
    }
}

// ------------------------------------------------------------- grouped launches
int group_grid(const void* kernel, int threads, size_t smem, int items)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const int nsm = grid_cap(GridDims{}) / 4;
    return std::max(1, std::min(items, per_sm * nsm));
}

// x-forward over the items of several grids; each runs the body of its own
// grid's transform length (compile-time plan where there is one)
template <typename T, typename Tc, bool TAN>
__global__ void __launch_bounds__(256, (TAN && sizeof(T) == 4) ? 4 : 1)
    k_group_xfwd(const XfwdArgs<T, Tc>* __restrict__ args, const int* __restrict__ vstart, int nd, int guard)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int total = __ldg(vstart + nd);
    for (int v = blockIdx.x; v < total; v += gridDim.x) {
        const int d = group_of(vstart, nd, v);
        const XfwdArgs<T, Tc>& a = args[d];
        const int vb = v - __ldg(vstart + d), vg = __ldg(vstart + d + 1) - __ldg(vstart + d);
        switch (a.g.M) {
            case 32: xfwd_body<T, Tc, 32, TAN>(a, guard, vb, vg, smem_raw); break;
            case 64: xfwd_body<T, Tc, 64, TAN>(a, guard, vb, vg, smem_raw); break;
            case 128: xfwd_body<T, Tc, 128, TAN>(a, guard, vb, vg, smem_raw); break;
            default: xfwd_body<T, Tc, 0, TAN>(a, guard, vb, vg, smem_raw); break;
        }
        __syncthreads();  // the next item reuses the shared buffers
    }
}

template <typename T, typename Tc>
__global__ void __launch_bounds__(256)
    k_group_xinv(const XinvArgs<T, Tc>* __restrict__ args, const int* __restrict__ vstart, int nd, int guard)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int total = __ldg(vstart + nd);
    for (int v = blockIdx.x; v < total; v += gridDim.x) {
        const int d = group_of(vstart, nd, v);
        const XinvArgs<T, Tc>& a = args[d];
        const int vb = v - __ldg(vstart + d), vg = __ldg(vstart + d + 1) - __ldg(vstart + d);
        switch (a.g.M) {
            case 32: xinv_body<T, Tc, 32>(a, guard, vb, vg, smem_raw); break;
            case 64: xinv_body<T, Tc, 64>(a, guard, vb, vg, smem_raw); break;
            case 128: xinv_body<T, Tc, 128>(a, guard, vb, vg, smem_raw); break;
            default: xinv_body<T, Tc, 0>(a, guard, vb, vg, smem_raw); break;
        }
        __syncthreads();
    }
}

template <typename T, typename Tc>
void launch_group_xfwd(const GroupTab<XfwdArgs<T, Tc>>& t, bool tangent, int guard, cudaStream_t st)
{
    if (t.total <= 0) return;
    if (tangent) {
        if constexpr (std::is_same<T, Tc>::value) {
            auto k = k_group_xfwd<T, Tc, true>;
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t.smem);
            k<<<group_grid((const void*)k, 256, t.smem, t.total), 256, t.smem, st>>>(t.args, t.vstart, t.nd, guard);
        }
        return;
    }
    auto k = k_group_xfwd<T, Tc, false>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t.smem);
    k<<<group_grid((const void*)k, 256, t.smem, t.total), 256, t.smem, st>>>(t.args, t.vstart, t.nd, guard);
}

template <typename T, typename Tc>
void launch_group_xinv(const GroupTab<XinvArgs<T, Tc>>& t, int guard, cudaStream_t st)
{
    if (t.total <= 0) return;
    auto k = k_group_xinv<T, Tc>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t.smem);
    k<<<group_grid((const void*)k, 256, t.smem, t.total), 256, t.smem, st>>>(t.args, t.vstart, t.nd, guard);
}

template void launch_group_xfwd<float, float>(const GroupTab<XfwdArgs<float, float>>&, bool, int, cudaStream_t);
template void launch_group_xfwd<double, double>(const GroupTab<XfwdArgs<double, double>>&, bool, int, cudaStream_t);
template void launch_group_xfwd<double, float>(const GroupTab<XfwdArgs<double, float>>&, bool, int, cudaStream_t);
template void launch_group_xfwd<df32, float>(const GroupTab<XfwdArgs<df32, float>>&, bool, int, cudaStream_t);
template void launch_group_xinv<float, float>(const GroupTab<XinvArgs<float, float>>&, int, cudaStream_t);
template void launch_group_xinv<double, double>(const GroupTab<XinvArgs<double, double>>&, int, cudaStream_t);
template void launch_group_xinv<double, float>(const GroupTab<XinvArgs<double, float>>&, int, cudaStream_t);
template void launch_group_xinv<df32, float>(const GroupTab<XinvArgs<df32, float>>&, int, cudaStream_t);

template void launch_xfwd<double, double>(const XfwdArgs<double, double>&, int, cudaStream_t);
template void launch_xfwd<double, float>(const XfwdArgs<double, float>&, int, cudaStream_t);
template void launch_xfwd<float, float>(const XfwdArgs<float, float>&, int, cudaStream_t);
template void launch_xinv<double, double>(const XinvArgs<double, double>&, int, cudaStream_t);
template void launch_xinv<double, float>(const XinvArgs<double, float>&, int, cudaStream_t);
template void launch_xinv<float, float>(const XinvArgs<float, float>&, int, cudaStream_t);
template void launch_xfwd<df32, float>(const XfwdArgs<df32, float>&, int, cudaStream_t);
template void launch_xinv<df32, float>(const XinvArgs<df32, float>&, int, cudaStream_t);

}  // namespace combo
