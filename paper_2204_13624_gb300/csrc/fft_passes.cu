// fft_passes.cu -- the three FFT passes of one operator application.
//
//   x-forward : per-voxel constitutive law (paper Sec. 6.1; boxel stresses
//               come from the laminate kernel) or tangent application, then
//               a real-to-complex FFT along x (packed half-length complex
//               transform + Hermitian split), written to the half spectrum.
//   y-pass    : complex FFT along y of one component tile, in place.
//   z-pass    : complex FFT along z of one tensor row (3 components), the
//               Green-operator projection of Sec. 3 (Eq. Gamma0) per frequency,
//               partial sums of |G X|^2, and the inverse FFT along z.
//   x-inverse : complex-to-real FFT along x and the solver update fused in.
//
// Data layout: real fields [9][n3][n2][n1] (x fastest); the half spectrum is
// [9][n3][n2][nhp] complex, nhp >= n1/2 + 1.  Every pass reads and writes
// each element once.  Power-of-two line lengths use the compile-time plans
// of fft_fast.cuh (y/z passes go global -> registers -> one shared-memory
// exchange -> global); other lengths use the runtime mixed-radix Stockham of
// combo_internal.cuh.
#include "combo_internal.cuh"
#include "fft_fast.cuh"
#include "../../include/combo.h"

namespace combo {

size_t xpass_smem(const GridDims& g, int lines, size_t cxbytes)
{
    return 2 * (size_t)9 * lines * (g.M + 1) * cxbytes + 256 * sizeof(double) + 16;
}

int xpass_lines(const GridDims& g, size_t cxbytes)
{
    // keep the two ping-pong buffers under ~48 KB while covering >= 512 voxels
    int lines = 1;
    while (lines * g.n1 < 512 && xpass_smem(g, lines * 2, cxbytes) <= 48 * 1024 &&
           (g.n2 * g.n3) % (lines * 2) == 0)
        lines *= 2;
    return lines;
}

// x-pass grid: a few resident blocks per SM stride over the line groups, so
// that the fused reductions see few partials and few tickets.
int xpass_grid(const GridDims& g, int lines)
{
    static int nsm = 0;
    if (nsm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) nsm = 152;
    }
    const int groups = (g.n2 * g.n3 + lines - 1) / lines;
    return groups < 4 * nsm ? groups : 4 * nsm;
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

// ------------------------------------------------------------- x forward
template <typename T, typename Tc, int MF>
__global__ void __launch_bounds__(256) k_xfwd(XfwdArgs<T, Tc> a, int guard)
{
    if (guard == 1 && a.sc->cg_done) return;
    if (guard == 2 && a.sc->outer_done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const GridDims g = a.g;
    const int LB = a.lines_per_block;
    const int ls = g.M + 1;
    cx<T>* buf0 = reinterpret_cast<cx<T>*>(smem_raw);
    cx<T>* buf1 = buf0 + (size_t)9 * LB * ls;
    double* red = reinterpret_cast<double*>(buf1 + (size_t)9 * LB * ls);
    int* flag = reinterpret_cast<int*>(red + 256);
    T* rb = reinterpret_cast<T*>(buf0);
    const int nlines = g.n2 * g.n3;
    const int ngroups = (nlines + LB - 1) / LB;
    const int64_t V = g.V;
    double acc = 0.0;

    const bool first = (a.mode == XF_TANGENT) ? (a.sc->cg_iter == 0) : false;
    const double beta = (a.mode == XF_TANGENT && !first) ? a.sc->beta : 0.0;

    // grid-stride over groups of LB x-lines (a few blocks per SM)
    for (int grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    const int L0 = grp * LB;
    for (int e = threadIdx.x; e < LB * g.n1; e += blockDim.x) {
        const int l = e / g.n1, x = e - l * g.n1;
        const int L = L0 + l;
        if (L >= nlines) continue;
        const int64_t v = (int64_t)L * g.n1 + x;
        T out[9];
        if (a.X) {
#pragma unroll
            for (int c = 0; c < 9; c++) out[c] = (T)a.X[c * V + v];
        } else if (a.mode == XF_RESID) {
            const int ph = a.phase[v];
            if (ph == 2) {
                const int b = a.vox2box[v];
#pragma unroll
                for (int c = 0; c < 9; c++) out[c] = (T)a.bP[(int64_t)b * 9 + c];
            } else {
                double F[9];
#pragma unroll
                for (int c = 0; c < 9; c++) F[c] = a.F[c * V + v];
                const double mu = a.mu[ph], lam = a.lam[ph];
                const double c0 = F[4] * F[8] - F[5] * F[7];
                const double c1 = F[5] * F[6] - F[3] * F[8];
                const double c2 = F[3] * F[7] - F[4] * F[6];
                const double J = F[0] * c0 + F[1] * c1 + F[2] * c2;
                if (!(J > 0.0)) {
                    raise_status(a.sc, COMBO_E_INADMISSIBLE);
#pragma unroll
                    for (int c = 0; c < 9; c++) out[c] = (T)0;
                } else {
                    const double iJ = 1.0 / J;
                    // G = F^{-1} (row-major); P = mu F + (lam ln J - mu) G^T
                    double G[9];
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
                        for (int j = 0; j < 3; j++) out[3 * i + j] = (T)(mu * F[3 * i + j] + k * G[3 * j + i]);
                    if (a.tc) {
#pragma unroll
                        for (int c = 0; c < 9; c++) a.tc[c * V + v] = (Tc)G[c];
                        a.tc[9 * V + v] = (Tc)(mu - lam * lnJ);
                    }
                }
            }
        } else {  // XF_TANGENT: p = r + beta p, y = A : p
            Tc p[9];
#pragma unroll
            for (int c = 0; c < 9; c++) {
                Tc rv = a.r[c * V + v];
                p[c] = first ? rv : (Tc)(rv + (Tc)beta * a.p[c * V + v]);
                a.p[c * V + v] = p[c];
            }
            const int ph = a.phase[v];
            Tc y[9];
            if (ph == 2) {
                const int64_t b = a.vox2box[v];
#pragma unroll
                for (int r = 0; r < 9; r++) {
                    Tc s = 0;
#pragma unroll
                    for (int c = 0; c < 9; c++) s += a.bA[(int64_t)(r * 9 + c) * a.nb + b] * p[c];
                    y[r] = s;
                }
            } else {
                Tc G[9];
#pragma unroll
                for (int c = 0; c < 9; c++) G[c] = a.tc[c * V + v];
                const Tc m = a.tc[9 * V + v];
                const Tc mu = (Tc)a.mu[ph], lam = (Tc)a.lam[ph];
                Tc Gp[9], GpG[9];
#pragma unroll
                for (int i = 0; i < 3; i++)
#pragma unroll
                    for (int j = 0; j < 3; j++)
                        Gp[3 * i + j] = G[3 * i] * p[j] + G[3 * i + 1] * p[3 + j] + G[3 * i + 2] * p[6 + j];
                const Tc tr = Gp[0] + Gp[4] + Gp[8];
#pragma unroll
                for (int i = 0; i < 3; i++)
#pragma unroll
                    for (int j = 0; j < 3; j++)
                        GpG[3 * i + j] = Gp[3 * i] * G[j] + Gp[3 * i + 1] * G[3 + j] + Gp[3 * i + 2] * G[6 + j];
                // y_iJ = mu p_iJ + lam tr(G p) G_Ji + m (G p G)_Ji
#pragma unroll
                for (int i = 0; i < 3; i++)
#pragma unroll
                    for (int j = 0; j < 3; j++)
                        y[3 * i + j] = mu * p[3 * i + j] + lam * tr * G[3 * j + i] + m * GpG[3 * j + i];
            }
            double s = 0.0;
#pragma unroll
            for (int c = 0; c < 9; c++) {
                s += (double)p[c] * (double)y[c];
                out[c] = (T)y[c];
            }
            acc += s;
        }
#pragma unroll
        for (int c = 0; c < 9; c++) rb[(size_t)2 * (c * LB + l) * ls + x] = out[c];
    }
    __syncthreads();

    const int nl = 9 * LB;
    cx<T>* Z = xpass_fft<T, MF, false>(buf0, buf1, a.plan, nl, ls, a.tw);

    // Hermitian split of the packed transform: X[k] = Ze + W^k Zo, k = 0..M
    const int M = g.M;
    const int half = M / 2;
    for (int e = threadIdx.x; e < nl * (half + 1); e += blockDim.x) {
        const int q = e / (half + 1), k = e - q * (half + 1);  // k fastest: coalesced stores
        const int c = q / LB, l = q - c * LB;
        const int L = L0 + l;
        if (L >= nlines) continue;
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
    if (a.mode == XF_TANGENT && a.partial) {
        const double s = block_sum(acc, red);
        if (threadIdx.x == 0) a.partial[blockIdx.x] = s;
        if (a.fuse && last_block(&a.sc->ticket[0], flag)) {
            const double tot = sum_partials_fixed(a.partial, gridDim.x, red);
            if (threadIdx.x == 0) cg_alpha(a.sc, tot);
        }
    }
}

// ------------------------------------------------------------- x inverse
template <typename T, typename Tc, int MF>
__global__ void __launch_bounds__(256) k_xinv(XinvArgs<T, Tc> a, int guard)
{
    if (guard == 1 && a.sc->cg_done) return;
    if (guard == 2 && a.sc->outer_done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const GridDims g = a.g;
    const int LB = a.lines_per_block;
    const int ls = g.M + 1;
    const int M = g.M;
    cx<T>* buf0 = reinterpret_cast<cx<T>*>(smem_raw);
    cx<T>* buf1 = buf0 + (size_t)9 * LB * ls;
    double* red = reinterpret_cast<double*>(buf1 + (size_t)9 * LB * ls);
    int* flag = reinterpret_cast<int*>(red + 256);
    const int nlines = g.n2 * g.n3;
    const int ngroups = (nlines + LB - 1) / LB;
    const int nl = 9 * LB;
    const int64_t V = g.V;
    double acc = 0.0;
    const bool skip_update = (a.mode == XI_FIXEDPOINT) && a.sc->outer_done;
    const double alpha = (a.mode == XI_CG) ? a.sc->alpha : 0.0;

    // grid-stride over groups of LB x-lines (a few blocks per SM)
    for (int grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    const int L0 = grp * LB;
    for (int e = threadIdx.x; e < nl * (M + 1); e += blockDim.x) {
        const int q = e / (M + 1), k = e - q * (M + 1);
        const int c = q / LB, l = q - c * LB;
        const int L = L0 + l;
        buf0[(size_t)q * ls + k] = (L < nlines) ? a.spec[c * g.Vs + (int64_t)L * g.nhp + k] : cx<T>{(T)0, (T)0};
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
    cx<T>* Zr = xpass_fft<T, MF, true>(buf1, buf0, a.plan, nl, ls, a.tw);
    const T* rb = reinterpret_cast<const T*>(Zr);

    for (int e = threadIdx.x; e < LB * g.n1; e += blockDim.x) {
        const int l = e / g.n1, x = e - l * g.n1;
        const int L = L0 + l;
        if (L >= nlines) continue;
        const int64_t v = (int64_t)L * g.n1 + x;
#pragma unroll
        for (int c = 0; c < 9; c++) {
            const T gv = rb[(size_t)2 * (c * LB + l) * ls + x];
            const int64_t w = c * V + v;
            if (a.mode == XI_FIXEDPOINT) {
                if (!skip_update) a.F[w] -= (double)gv * a.inv_mu0;
            } else if (a.mode == XI_RHS) {
                const Tc rv = (Tc)(-gv);
                a.r[w] = rv;
                a.x[w] = (Tc)0;
                acc += (double)rv * (double)rv;
            } else if (a.mode == XI_CG) {
                const Tc rv = a.r[w] - (Tc)alpha * (Tc)gv;
                a.x[w] += (Tc)alpha * a.p[w];
                a.r[w] = rv;
                acc += (double)rv * (double)rv;
            } else {
                a.Y[w] = (double)gv;
            }
        }
    }
    __syncthreads();  // the next group reuses the shared buffers
    }
    if ((a.mode == XI_RHS || a.mode == XI_CG) && a.partial) {
        const double s = block_sum(acc, red);
        if (threadIdx.x == 0) a.partial[blockIdx.x] = s;
        if (a.mode == XI_CG && a.fuse && last_block(&a.sc->ticket[1], flag)) {
            const double tot = sum_partials_fixed(a.partial, gridDim.x, red);
            if (threadIdx.x == 0) cg_beta(a.sc, tot, a.cg_tol, a.cg_max, a.cg_fixed);
        }
    }
}

// ------------------------------------------------------------- y pass (generic)
template <typename T, bool INV>
__global__ void __launch_bounds__(256) k_ypass(YArgs<T> a)
{
    if (a.guard == 1 && a.sc->cg_done) return;
    if (a.guard == 2 && a.sc->outer_done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const GridDims g = a.g;
    const int TX = a.tx;
    const int n2 = g.n2;
    cx<T>* buf0 = reinterpret_cast<cx<T>*>(smem_raw);
    cx<T>* buf1 = buf0 + (size_t)n2 * TX;
    const int x0 = blockIdx.x * TX;
    const int z = blockIdx.y;
    cx<T>* base = a.spec + blockIdx.z * g.Vs + (int64_t)z * n2 * g.nhp + x0;
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

// ------------------------------------------------------------- y pass (power of two)
// Block: TX columns x TPL threads; column fastest in the thread index so that
// every global access of a warp covers TX consecutive complex values.
template <typename T, int N, int TX, bool INV>
__global__ void __launch_bounds__(TX * FastPlan<N>::TPL) k_ypass_fast(YArgs<T> a)
{
    if (a.guard == 1 && a.sc->cg_done) return;
    if (a.guard == 2 && a.sc->outer_done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T>* ex = reinterpret_cast<cx<T>*>(smem_raw);
    const GridDims g = a.g;
    const int line = threadIdx.x % TX, tau = threadIdx.x / TX;
    const int x0 = blockIdx.x * TX;
    const bool valid = x0 + line < g.nh;
    cx<T>* base = a.spec + blockIdx.z * g.Vs + (int64_t)blockIdx.y * N * g.nhp + x0 + line;
    const int64_t st = g.nhp;
    fft_fast<T, N, INV>([&](int e) { return valid ? base[e * st] : cx<T>{(T)0, (T)0}; },
                        [&](int e, cx<T> v) {
                            if (valid) base[e * st] = v;
                        },
                        [&](int e) { return ex[e * TX + line]; }, [&](int e, cx<T> v) { ex[e * TX + line] = v; }, tau,
                        a.tw);
}

// ------------------------------------------------------------- z pass + Gamma (generic)
template <typename T>
__global__ void __launch_bounds__(256) k_zpass(ZArgs<T> a)
{
    if (a.guard == 1 && a.sc->cg_done) return;
    if (a.guard == 2 && a.sc->outer_done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const GridDims g = a.g;
    const int TX = a.tx;
    const int n3 = g.n3;
    const int W = 3 * TX;  // elements per z row of the tile
    cx<T>* buf0 = reinterpret_cast<cx<T>*>(smem_raw);
    cx<T>* buf1 = buf0 + (size_t)n3 * W;
    double* red = reinterpret_cast<double*>(buf1 + (size_t)n3 * W);
    const int x0 = blockIdx.x * TX;
    const int y = blockIdx.y;
    const int row = blockIdx.z;  // tensor row i: components 3i, 3i+1, 3i+2
    const int64_t zstride = (int64_t)g.n2 * g.nhp;
    cx<T>* base = a.spec + (int64_t)(3 * row) * g.Vs + (int64_t)y * g.nhp + x0;

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
        const cx<T> X0 = p[0], X1 = p[TX], X2 = p[2 * TX];
        if (a.want_norm && xi1 == 0 && y == 0 && z == 0) {
            a.sc->dc[3 * row + 0] = (double)X0.x;
            a.sc->dc[3 * row + 1] = (double)X1.x;
            a.sc->dc[3 * row + 2] = (double)X2.x;
        }
        cx<T> o0{(T)0, (T)0}, o1{(T)0, (T)0}, o2{(T)0, (T)0};
        if (kk > (T)0) {
            // row i of G X: k (k . X_i) / |k|^2
            const T sr = (k0 * X0.x + k1 * X1.x + k2 * X2.x) / kk;
            const T si = (k0 * X0.y + k1 * X1.y + k2 * X2.y) / kk;
            o0 = cx<T>{k0 * sr, k0 * si};
            o1 = cx<T>{k1 * sr, k1 * si};
            o2 = cx<T>{k2 * sr, k2 * si};
            if (a.want_norm) {
                const double wgt = (xi1 == 0 || xi1 == g.M) ? 1.0 : 2.0;
                acc += wgt * ((double)o0.x * o0.x + (double)o0.y * o0.y + (double)o1.x * o1.x + (double)o1.y * o1.y +
                              (double)o2.x * o2.x + (double)o2.y * o2.y);
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
        if (threadIdx.x == 0) a.partial[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)] = s;
    }
}

// ------------------------------------------------------------- z pass + Gamma (power of two)
// Block: 3 groups (one per component of tensor row i) x TX columns x TPL
// threads; the three components are transformed concurrently.  The tile
// [3][N][TX] is both the exchange buffer and the place where the forward
// transform ends; after a barrier every frequency's three components are in
// shared memory, the projection runs in place, and each group's inverse
// transform starts from the positions its own last forward stage wrote.
template <typename T, int N, int TX>
__global__ void __launch_bounds__(3 * TX * FastPlan<N>::TPL) k_zpass_fast(ZArgs<T> a)
{
    if (a.guard == 1 && a.sc->cg_done) return;
    if (a.guard == 2 && a.sc->outer_done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int TPL = FastPlan<N>::TPL;
    constexpr int GS = TX * TPL;  // threads per component group
    cx<T>* park = reinterpret_cast<cx<T>*>(smem_raw);  // [3][N][TX]
    double* red = reinterpret_cast<double*>(park + 3 * N * TX);
    const GridDims g = a.g;
    const int c = threadIdx.x / GS;
    const int r = threadIdx.x - c * GS;
    const int line = r % TX, tau = r / TX;
    const int x0 = blockIdx.x * TX;
    const bool valid = x0 + line < g.nh;
    const int y = blockIdx.y;
    const int row = blockIdx.z;
    const int64_t zst = (int64_t)g.n2 * g.nhp;
    cx<T>* bc = a.spec + (int64_t)(3 * row + c) * g.Vs + (int64_t)y * g.nhp + x0 + line;
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
        const cx<T> X0 = p[0], X1 = p[N * TX], X2 = p[2 * N * TX];
        const T ax = a.sa[0][xi1], bx = a.sb[0][xi1];
        const T az = a.sa[2][z], bz = a.sb[2][z];
        const T k0 = ax * by * bz, k1 = ay * bx * bz, k2 = az * bx * by;
        const T kk = k0 * k0 + k1 * k1 + k2 * k2;
        if (a.want_norm && xi1 == 0 && y == 0 && z == 0) {
            a.sc->dc[3 * row + 0] = (double)X0.x;
            a.sc->dc[3 * row + 1] = (double)X1.x;
            a.sc->dc[3 * row + 2] = (double)X2.x;
        }
        cx<T> o0{(T)0, (T)0}, o1{(T)0, (T)0}, o2{(T)0, (T)0};
        if (kk > (T)0) {
            const T sr = (k0 * X0.x + k1 * X1.x + k2 * X2.x) / kk;
            const T si = (k0 * X0.y + k1 * X1.y + k2 * X2.y) / kk;
            o0 = cx<T>{k0 * sr, k0 * si};
            o1 = cx<T>{k1 * sr, k1 * si};
            o2 = cx<T>{k2 * sr, k2 * si};
            if (a.want_norm) {
                const double wgt = (xi1 == 0 || xi1 == g.M) ? 1.0 : 2.0;
                acc += wgt * ((double)o0.x * o0.x + (double)o0.y * o0.y + (double)o1.x * o1.x + (double)o1.y * o1.y +
                              (double)o2.x * o2.x + (double)o2.y * o2.y);
            }
        }
        p[0] = c_scale(o0, a.scale);
        p[N * TX] = c_scale(o1, a.scale);
        p[2 * N * TX] = c_scale(o2, a.scale);
    }
    __syncthreads();

    // inverse along z from the tile (in place: barrier inside the first stage)
    fft_fast<T, N, true, true, false>(lp,
                                      [&](int e, cx<T> v) {
                                          if (valid) bc[e * zst] = v;
                                      },
                                      lp, sp, tau, a.tw);
    if (a.want_norm && a.partial) {
        const double s = block_sum(acc, red);
        if (threadIdx.x == 0) a.partial[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)] = s;
    }
}

// ------------------------------------------------------------- launch configuration
template <typename T> int ytx_fast(int n) { return sizeof(T) == 4 ? 16 : 8; }
// z-pass columns per block: 3 * N * TX complex values of shared memory (48 KB
// at N >= 256)
template <typename T> constexpr int ztx_const(int n)
{
    return sizeof(T) == 4 ? (n == 512 ? 4 : (n == 256 ? 8 : 16)) : (n == 512 ? 2 : (n == 256 ? 4 : 8));
}
template <typename T> int ztx_fast(int n) { return ztx_const<T>(n); }

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

template <typename K> static void allow_smem(K kernel, bool& done)
{
    if (!done) {
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        done = true;
    }
}

template <typename T, typename Tc, int MF> static void xfwd_launch(const XfwdArgs<T, Tc>& a, int guard, cudaStream_t st)
{
    const int grid = xpass_grid(a.g, a.lines_per_block);
    const size_t sm = xpass_smem(a.g, a.lines_per_block, sizeof(cx<T>));
    static bool attr = false;
    allow_smem(k_xfwd<T, Tc, MF>, attr);
    k_xfwd<T, Tc, MF><<<grid, 256, sm, st>>>(a, guard);
}

template <typename T, typename Tc> void launch_xfwd(const XfwdArgs<T, Tc>& a, int guard, cudaStream_t st)
{
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

template <typename T, typename Tc> void launch_xinv(const XinvArgs<T, Tc>& a, int guard, cudaStream_t st)
{
    switch (a.g.M) {
        case 32: xinv_launch<T, Tc, 32>(a, guard, st); break;
        case 64: xinv_launch<T, Tc, 64>(a, guard, st); break;
        case 128: xinv_launch<T, Tc, 128>(a, guard, st); break;
        case 256: xinv_launch<T, Tc, 256>(a, guard, st); break;
        default: xinv_launch<T, Tc, 0>(a, guard, st); break;
    }
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
    dim3 grid((a.g.nh + TX - 1) / TX, a.g.n2, 3);
    const size_t sm = (size_t)3 * N * TX * sizeof(cx<T>) + 64 * sizeof(double);
    static bool attr = false;
    allow_smem(k_zpass_fast<T, N, TX>, attr);
    k_zpass_fast<T, N, TX><<<grid, 3 * TX * FastPlan<N>::TPL, sm, st>>>(a);
}

template <typename T> void launch_zpass(const ZArgs<T>& a, cudaStream_t st)
{
    switch (a.g.n3) {
        case 64: zpass_fast_launch<T, 64>(a, st); return;
        case 128: zpass_fast_launch<T, 128>(a, st); return;
        case 256: zpass_fast_launch<T, 256>(a, st); return;
        case 512: zpass_fast_launch<T, 512>(a, st); return;
        default: break;
    }
    dim3 grid((a.g.nh + a.tx - 1) / a.tx, a.g.n2, 3);
    const size_t sm = 2 * (size_t)a.g.n3 * 3 * a.tx * sizeof(cx<T>) + 64 * sizeof(double);
    static bool attr = false;
    allow_smem(k_zpass<T>, attr);
    k_zpass<T><<<grid, 256, sm, st>>>(a);
}

template void launch_xfwd<double, double>(const XfwdArgs<double, double>&, int, cudaStream_t);
template void launch_xfwd<double, float>(const XfwdArgs<double, float>&, int, cudaStream_t);
template void launch_xfwd<float, float>(const XfwdArgs<float, float>&, int, cudaStream_t);
template void launch_xinv<double, double>(const XinvArgs<double, double>&, int, cudaStream_t);
template void launch_xinv<double, float>(const XinvArgs<double, float>&, int, cudaStream_t);
template void launch_xinv<float, float>(const XinvArgs<float, float>&, int, cudaStream_t);
template void launch_ypass<double, false>(const YArgs<double>&, cudaStream_t);
template void launch_ypass<double, true>(const YArgs<double>&, cudaStream_t);
template void launch_ypass<float, false>(const YArgs<float>&, cudaStream_t);
template void launch_ypass<float, true>(const YArgs<float>&, cudaStream_t);
template void launch_zpass<double>(const ZArgs<double>&, cudaStream_t);
template void launch_zpass<float>(const ZArgs<float>&, cudaStream_t);

}  // namespace combo
