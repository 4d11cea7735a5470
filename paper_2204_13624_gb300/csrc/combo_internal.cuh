// combo_internal.cuh -- device-side types, FFT core and kernel launchers of
// libcombo.so (GB300, sm_103a).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "dfloat.cuh"

namespace combo {

template <typename T> struct CxT;
template <> struct CxT<float> { typedef float2 type; };
template <> struct CxT<double> { typedef double2 type; };
template <> struct CxT<df32> { typedef df2 type; };
template <typename T> using cx = typename CxT<T>::type;

template <typename V> __device__ __forceinline__ V c_add(V a, V b) { return V{a.x + b.x, a.y + b.y}; }
template <typename V> __device__ __forceinline__ V c_sub(V a, V b) { return V{a.x - b.x, a.y - b.y}; }
template <typename V> __device__ __forceinline__ V c_mul(V a, V b)
{
    return V{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename V> __device__ __forceinline__ V c_conj(V a) { return V{a.x, -a.y}; }
// multiply by -i (forward) or +i (inverse)
template <bool INV, typename V> __device__ __forceinline__ V c_rot(V a)
{
    return INV ? V{-a.y, a.x} : V{a.y, -a.x};
}
template <typename V, typename S> __device__ __forceinline__ V c_scale(V a, S s) { return V{a.x * s, a.y * s}; }

// Staggered grid (App. A): row i of F uses k_iB = i rho_B e^{+i theta_B/2}
// (forward difference) for B = i and i rho_B e^{-i theta_B/2} (backward) for
// B != i, rho_B = (2/h_B) sin(theta_B/2).  Row i of the projection
// k_i (k_i^H X_i) / |k|^2 is then the real projection with k = rho between
// the rotations X_B -> u_B X_B and o_B -> conj(u_B) o_B, u_B = e^{-i theta_B/2}
// for B = i and e^{+i theta_B/2} otherwise.
template <typename V> __device__ __forceinline__ V stag_u(int row, int B, V ph)
{
    return row == B ? c_conj(ph) : ph;
}

// |a|^2 + |b|^2 + |c|^2 for a residual norm: in FP64 from FP32 / FP64 values;
// from the leading FP32 parts of double-float values (a norm used for a
// stopping test needs no more than FP32 accuracy)
template <typename V> __device__ __forceinline__ double sq3(V a, V b, V c)
{
    return (double)a.x * (double)a.x + (double)a.y * (double)a.y + (double)b.x * (double)b.x +
           (double)b.y * (double)b.y + (double)c.x * (double)c.x + (double)c.y * (double)c.y;
}
__device__ __forceinline__ double sq3(df2 a, df2 b, df2 c)
{
    const float s = a.x.hi * a.x.hi + a.y.hi * a.y.hi + b.x.hi * b.x.hi + b.y.hi * b.y.hi + c.x.hi * c.x.hi +
                    c.y.hi * c.y.hi;
    return (double)s;
}

constexpr int kMaxStages = 12;

// Mixed-radix Stockham plan for one line length (product of radices 2,3,4,8).
struct Plan {
    int n;
    int nst;
    int R[kMaxStages];
    int Ns[kMaxStages];  // product of the radices of the stages before this one
};

// A batch of nprob independent problems on equal grids n1 x n2 x n3p is laid
// out as one grid whose z axis holds the problems one after another
// (n3 = nprob * n3p): every x-line, y-column and z-column then belongs to one
// problem, the x- and y-passes need no change, the z-passes transform
// segments of length n3p, and solver scalars are kept per problem.  A single
// solve is the batch of one (nprob = 1, n3p = n3).
struct GridDims {
    int n1, n2, n3;
    int M;     // n1 / 2: complex length of the packed x transform
    int nh;    // M + 1 stored x frequencies (Hermitian half)
    int nhp;   // pitch of the x-frequency axis in the spectrum (>= nh)
    int64_t V;   // voxels (all problems)
    int64_t Vs;  // complex entries per spectrum component: n3 * n2 * nhp
    int nprob;   // stacked problems
    int n3p;     // z planes of one problem
};

// x-pass grids give every problem the same number of blocks gp: block vb of
// vg -> (problem b, index j within the problem's blocks)
__device__ __forceinline__ void prob_block(const GridDims& g, int vb, int vg, int& b, int& j, int& gp)
{
    gp = vg / g.nprob;
    b = vb / gp;
    j = vb - b * gp;
}

// Block index of a pass body: blockIdx / gridDim of a launch of its own, or
// one work item of a grid in a grouped launch over several grids.
struct VBlock {
    int x, y, z, gx, gy, gz;
    __device__ __forceinline__ static VBlock of_launch()
    {
        return VBlock{(int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z,
                      (int)gridDim.x,  (int)gridDim.y,  (int)gridDim.z};
    }
    // item l of a gx x gy x gz grid, x fastest
    __device__ __forceinline__ static VBlock of_item(int l, int gx, int gy, int gz)
    {
        return VBlock{l % gx, (l / gx) % gy, l / (gx * gy), gx, gy, gz};
    }
    __device__ __forceinline__ int linear() const { return x + gx * (y + gy * z); }
};

// Descriptor of item v of a grouped launch (few descriptors: a linear scan)
__device__ __forceinline__ int group_of(const int* __restrict__ vstart, int nd, int v)
{
    int d = 0;
    while (d + 1 < nd && v >= __ldg(vstart + d + 1)) d++;
    return d;
}

// Persistent-grid size of a grouped launch: as many blocks as fit on the
// device at once, at most one per item
int group_grid(const void* kernel, int threads, size_t smem, int items);

// Solver scalars that live on the device between kernels.
struct Scalars {
    double resid2;    // sum over the half spectrum of w |ghat|^2
    double dc[9];     // zero-frequency coefficients of the last residual operand
    double Pbar[9];   // <P> of the last evaluation
    double eps;       // equilibrium residual ||G[P]||_rms / |<P>|
    double rr, rr0, pAp, alpha, beta;
    int32_t outer_iter, outer_done;
    int32_t cg_iter, cg_done;
    int32_t admissible;
    int32_t status;  // first error code (COMBO_E_*) raised by a kernel
    unsigned long long nr_iters, n_backproj, n_lam;
    unsigned long long n_operator, n_operator64;
    unsigned int ticket[4];  // last-block counters of fused reductions
    double ncg_gg;           // nonlinear CG: ||G[P]||^2 of the previous iteration
    double alpha_pending;    // x += alpha_pending p still owed by the last CG update
    // first failed laminate solve: 1 + boxel index (0: none), reason (1 F_box
    // inadmissible, 2 a phase inadmissible, 3 singular Hessian, 4 iteration
    // cap) and its state: F_box (9), N (3), c+ (1), a (3)
    int32_t fail_boxel, fail_reason;
    double fail_state[16];
};

// ---------------------------------------------------------------- FFT core
// Radix-R butterflies, DFT_R(v) with sign -1 (forward) or +1 (inverse).
template <bool INV, typename V> __device__ __forceinline__ void dft2(V* v)
{
    V a = v[0], b = v[1];
    v[0] = c_add(a, b);
    v[1] = c_sub(a, b);
}

template <bool INV, typename V> __device__ __forceinline__ void dft4(V* v)
{
    V t0 = c_add(v[0], v[2]), t1 = c_sub(v[0], v[2]);
    V t2 = c_add(v[1], v[3]), t3 = c_rot<INV>(c_sub(v[1], v[3]));
    v[0] = c_add(t0, t2);
    v[2] = c_sub(t0, t2);
    v[1] = c_add(t1, t3);
    v[3] = c_sub(t1, t3);
}

template <bool INV, typename V> __device__ __forceinline__ void dft3(V* v)
{
    typedef decltype(v[0].x) S;
    const S h = (S)0.86602540378443864676;  // sin(2 pi / 3)
    V s = c_add(v[1], v[2]), d = c_sub(v[1], v[2]);
    V t = V{v[0].x - (S)0.5 * s.x, v[0].y - (S)0.5 * s.y};
    V u = c_rot<INV>(c_scale(d, h));
    v[0] = c_add(v[0], s);
    v[1] = c_add(t, u);
    v[2] = c_sub(t, u);
}

template <bool INV, typename V> __device__ __forceinline__ void dft8(V* v)
{
    typedef decltype(v[0].x) S;
    const S c = (S)0.70710678118654752440;  // cos(pi / 4)
    V e[4] = {v[0], v[2], v[4], v[6]};
    V o[4] = {v[1], v[3], v[5], v[7]};
    dft4<INV>(e);
    dft4<INV>(o);
    // o[k] *= exp(-/+ 2 pi i k / 8)
    V o1 = o[1], o3 = o[3];
    if (!INV) {
        o[1] = V{c * (o1.x + o1.y), c * (o1.y - o1.x)};
        o[2] = V{o[2].y, -o[2].x};
        o[3] = V{c * (o3.y - o3.x), -c * (o3.x + o3.y)};
    } else {
        o[1] = V{c * (o1.x - o1.y), c * (o1.x + o1.y)};
        o[2] = V{-o[2].y, o[2].x};
        o[3] = V{-c * (o3.x + o3.y), c * (o3.x - o3.y)};
    }
#pragma unroll
    for (int k = 0; k < 4; k++) {
        v[k] = c_add(e[k], o[k]);
        v[k + 4] = c_sub(e[k], o[k]);
    }
}

// One self-sorting Stockham stage (decimation in time) over nl lines.
// Element e of line q is at buf[q * ls + e * es].  tw[t] = exp(-2 pi i t / n).
template <typename T, int R, bool INV>
__device__ __forceinline__ void fft_stage(const cx<T>* __restrict__ src, cx<T>* __restrict__ dst, int n, int Ns,
                                          int nl, int ls, int es, const cx<T>* __restrict__ tw, int tid, int nthr)
{
    const int nbut = n / R;
    const int total = nbut * nl;
    const int tstep = n / (Ns * R);
    for (int b = tid; b < total; b += nthr) {
        const int q = b % nl;
        const int j = b / nl;
        const int k = j % Ns;
        cx<T> v[R];
        const cx<T>* s = src + (size_t)q * ls;
#pragma unroll
        for (int t = 0; t < R; t++) v[t] = s[(size_t)(j + t * nbut) * es];
        if (Ns > 1) {
#pragma unroll
            for (int t = 1; t < R; t++) {
                cx<T> w = tw[t * k * tstep];
                if (INV) w.y = -w.y;
                v[t] = c_mul(v[t], w);
            }
        }
        if (R == 2) dft2<INV>(v);
        if (R == 3) dft3<INV>(v);
        if (R == 4) dft4<INV>(v);
        if (R == 8) dft8<INV>(v);
        const int idxD = (j / Ns) * Ns * R + k;
        cx<T>* d = dst + (size_t)q * ls;
#pragma unroll
        for (int t = 0; t < R; t++) d[(size_t)(idxD + t * Ns) * es] = v[t];
    }
}

// Full transform of nl lines: data starts in b0, ends in (nst odd ? b1 : b0).
// Returns the buffer holding the result.  Ends with __syncthreads().
template <typename T, bool INV>
__device__ cx<T>* fft_lines(cx<T>* b0, cx<T>* b1, const Plan& p, int nl, int ls, int es, const cx<T>* tw)
{
    cx<T>* src = b0;
    cx<T>* dst = b1;
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int s = 0; s < p.nst; s++) {
        switch (p.R[s]) {
            case 2: fft_stage<T, 2, INV>(src, dst, p.n, p.Ns[s], nl, ls, es, tw, tid, nthr); break;
            case 3: fft_stage<T, 3, INV>(src, dst, p.n, p.Ns[s], nl, ls, es, tw, tid, nthr); break;
            case 4: fft_stage<T, 4, INV>(src, dst, p.n, p.Ns[s], nl, ls, es, tw, tid, nthr); break;
            default: fft_stage<T, 8, INV>(src, dst, p.n, p.Ns[s], nl, ls, es, tw, tid, nthr); break;
        }
        __syncthreads();
        cx<T>* t = src;
        src = dst;
        dst = t;
    }
    return src;
}

// Block-wide sum of one double per thread (result valid in thread 0).
__device__ __forceinline__ double block_sum(double v, double* red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int i = 0; i < nw; i++) s += red[i];
    }
    return s;
}

__device__ __forceinline__ void raise_status(Scalars* sc, int code)
{
    atomicCAS(&sc->status, 0, code);
}

// all nine entries finite: tells a NaN / Inf deformation (COMBO_E_NAN) from
// det F <= 0 (COMBO_E_INADMISSIBLE) where a stress evaluation fails
__device__ __forceinline__ bool finite9(const double f[9])
{
    bool ok = true;
#pragma unroll
    for (int c = 0; c < 9; c++) ok = ok && isfinite(f[c]);
    return ok;
}

// Deterministic sum of n partials by one block: fixed strided accumulation
// (4 independent chains) then a fixed tree.  red: >= blockDim.x rounded up to
// a power of two doubles (blockDim.x <= 256 with the 256-entry buffers).
// All threads call it; every thread gets the total.
__device__ __forceinline__ double sum_partials_fixed(const double* p, int n, double* red)
{
    const int bd = blockDim.x, tid = threadIdx.x;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int i = tid;
    for (; i + 3 * bd < n; i += 4 * bd) {
        a0 += __ldcg(p + i);
        a1 += __ldcg(p + i + bd);
        a2 += __ldcg(p + i + 2 * bd);
        a3 += __ldcg(p + i + 3 * bd);
    }
    for (; i < n; i += bd) a0 += __ldcg(p + i);
    int pw = 1;  // tree over the next power of two, zero-padded
    while (pw < bd) pw <<= 1;
    __syncthreads();
    red[tid] = (a0 + a1) + (a2 + a3);
    if (tid + bd < pw) red[tid + bd] = 0.0;
    __syncthreads();
    for (int o = pw / 2; o > 0; o >>= 1) {
        if (tid < o) red[tid] += red[tid + o];
        __syncthreads();
    }
    const double s = red[0];
    __syncthreads();
    return s;
}

// True in every thread of the block that finishes last of nblocks blocks
// sharing ticket (after its partial was written by thread 0).  ticket is reset
// by that block.
__device__ __forceinline__ bool last_block(unsigned int* ticket, int* flag_smem, unsigned int nblocks)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int t = atomicAdd(ticket, 1u);
        *flag_smem = (t == nblocks - 1) ? 1 : 0;
        if (*flag_smem) *ticket = 0u;
    }
    __syncthreads();
    const bool last = *flag_smem != 0;
    if (last) __threadfence();
    return last;
}

// CG scalars (called by one thread).  Loss of positive curvature stops CG
// with the current iterate.
// The x update of iteration k (x += alpha_k p_k) is applied by the tangent
// x-pass of iteration k+1, which reads p_k anyway; alpha_pending records the
// update still owed (the F update applies it when CG stops).
__device__ __forceinline__ void cg_alpha(Scalars* sc, double pAp)
{
    sc->pAp = pAp;
    sc->alpha_pending = 0.0;  // the owed update was applied by this pass
    if (!(pAp > 0.0)) {
        sc->cg_done = 1;
        return;
    }
    sc->alpha = sc->rr / pAp;
}

__device__ __forceinline__ void cg_beta(Scalars* sc, double rr_new, double cg_tol, int cg_max, int cg_fixed)
{
    sc->alpha_pending = sc->alpha;
    sc->beta = rr_new / sc->rr;
    sc->rr = rr_new;
    const int j = sc->cg_iter + 1;
    sc->cg_iter = j;
    sc->n_operator += 1;
    bool stop;
    if (cg_fixed > 0)
        stop = j >= cg_fixed;
    else
        stop = (sqrt(rr_new) <= cg_tol * sqrt(sc->rr0)) || j >= cg_max;
    if (stop || rr_new == 0.0) sc->cg_done = 1;
}

// y = A : p for a pure Neo-Hookean voxel from its cache (G = F^{-1}, m):
//   y_iJ = mu p_iJ + lam tr(G p) G_Ji + m (G p G)_Ji
template <typename S>
__device__ __forceinline__ void nh_tangent(const S G[9], S m, S mu, S lam, const S p[9], S y[9])
{
    S Gp[9], GpG[9];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) Gp[3 * i + j] = G[3 * i] * p[j] + G[3 * i + 1] * p[3 + j] + G[3 * i + 2] * p[6 + j];
    const S tr = Gp[0] + Gp[4] + Gp[8];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) GpG[3 * i + j] = Gp[3 * i] * G[j] + Gp[3 * i + 1] * G[3 + j] + Gp[3 * i + 2] * G[6 + j];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) y[3 * i + j] = mu * p[3 * i + j] + lam * tr * G[3 * j + i] + m * GpG[3 * j + i];
}

// ---------------------------------------------------------------- launchers
enum XfwdMode { XF_RESID = 0, XF_TANGENT = 1 };

// Position of entry (r, s) of a symmetric 9x9 matrix in its packed upper
// triangle (45 entries, row-major over r <= s).
__host__ __device__ constexpr int sym_idx(int r, int s)
{
    return r <= s ? 9 * r - r * (r - 1) / 2 + (s - r) : 9 * s - s * (s - 1) / 2 + (r - s);
}
enum XinvMode { XI_FIXEDPOINT = 0, XI_RHS = 1, XI_CG = 2, XI_PLAIN = 3, XI_NCG = 4 };

template <typename T, typename Tc> struct XfwdArgs {
    GridDims g;
    Plan plan;           // length M
    const cx<T>* tw;     // [M] exp(-2 pi i t / M)
    const cx<T>* tw2;    // [M + 1] exp(-2 pi i k / n1)
    cx<T>* spec;         // [9][n3][n2][nhp]
    int lines_per_block;
    int mode;
    const uint8_t* phase;
    const int32_t* vox2box;
    double mu[2], lam[2];
    // XF_RESID
    const double* F;     // [9][V]
    const double* bP;    // [nb][9]
    Tc* tc;              // [10][V] tangent cache (F^{-1}, mu - lam ln J), may be null
    // XF_TANGENT
    const Tc* r;
    Tc* p;
    Tc* x;               // receives the previous iteration's x += alpha p
    const double* matp;  // [nprob][4] (mu-, mu+, lam-, lam+) per problem, or null: mu, lam
    const Tc* bA;        // [45][nb] packed symmetric boxel tangent, boxels in voxel order
    const int32_t* bvox; // [nb] voxel of the k-th boxel in voxel order
    const int32_t* lofs; // [n2 n3 + 1] first boxel (voxel order) of each x-line
    int64_t nb;
    // plain operand (no constitutive law): X [9][V] real, FP64 (X) or in the
    // Krylov precision (Xc, the doubly-fine tangent's gathered A : p)
    const double* X;
    const Tc* Xc;
    double* partial;     // [gridDim.x] pAp partials
    Scalars* sc;
    int fuse;            // last block turns the pAp partials into alpha
    int cfg;             // launch-shape candidate (autotuner; 0 = default)
    int linear;          // infinitesimal strain: isotropic linear phases (XF_RESID)
};

template <typename T, typename Tc> struct XinvArgs {
    GridDims g;
    Plan plan;
    const cx<T>* tw;
    const cx<T>* tw2;
    const cx<T>* spec;
    int lines_per_block;
    int mode;
    double inv_mu0;
    double* F;       // XI_FIXEDPOINT / XI_NCG
    double* d;       // XI_NCG: the direction [9][V]
    Tc* x;           // XI_RHS / XI_CG
    Tc* r;
    const Tc* p;
    double* Y;       // XI_PLAIN: real output [9][V]
    double* partial;
    Scalars* sc;
    int fuse;        // last block turns the (r, r) partials into beta / stop (XI_CG)
    double cg_tol;
    int cg_max, cg_fixed;
    int cfg;         // launch-shape candidate (autotuner; 0 = default)
    uint32_t wait_cap;  // poll cap of the bulk-copy waits (wait_cap_of: 0 = default)
};

template <typename T> struct YArgs {
    GridDims g;
    Plan plan;
    const cx<T>* tw;
    cx<T>* spec;
    int tx;
    const Scalars* sc;
    int guard;  // 0 none, 1 skip if cg_done, 2 skip if outer_done
    const void* tmap;  // CUtensorMap of spec for the TMA y-pass (FP32), or null
    int cfg;           // launch-shape candidate (autotuner; 0 = default)
    uint32_t wait_cap;  // poll cap of the tile waits (wait_cap_of: 0 = default)
    int disp;           // TMA y-inverse: only components 0, 3, 6 (displacement form)
    // (double-float words, inverse) the transform in FP32 arithmetic on the
    // values rounded to FP32, stored back as double-float with a zero low
    // word: the Newton right-hand side, an FP32 field; tw32: FP32 twiddles
    int inv32;
    const cx<float>* tw32;
};

template <typename T> struct ZArgs {
    GridDims g;
    Plan plan;
    const cx<T>* tw;
    cx<T>* spec;
    int tx;
    const T* sa[3];  // symbol tables: k_j(xi) = sa[j][xi_j] * prod_{m != j} sb[m][xi_m]
    const T* sb[3];
    const cx<T>* ph[3];  // staggered grid: e^{i theta_j / 2} per index (else null)
    T scale;         // 2 / V
    int want_norm;   // accumulate sum w |G X|^2 and the zero frequency
    double* partial; // [gridDim.x * gridDim.y * gridDim.z]
    Scalars* sc;
    int guard;
    const void* tmap;  // CUtensorMap of spec for the TMA z-pass (FP32), or null
    int cfg;           // launch-shape candidate (autotuner; 0 = default)
    uint32_t wait_cap;  // poll cap of the tile waits (wait_cap_of: 0 = default)
    // displacement form of the rotated operator (TMA z-pass only): row i
    // leaves as one spectrum, u_i = -i conj(P) (k . X_i) / |k|^2, into
    // component 3 i, through tmap_u (tile box of one component); rph[j][xi] =
    // e^{i pi xi / n_j}, P = prod_j rph[j][xi_j]
    int disp;
    const void* tmap_u;
    const cx<T>* rph[3];
    // (double-float words) the inverse z transform in FP32 arithmetic, as the
    // y-pass's inv32; the projection and the norm stay double-float
    int inv32;
    const cx<float>* tw32;
};

// Grouped launches: one persistent launch runs the work items of several
// grids (a batch of problems on different grids).  Descriptor d holds the
// arguments of one grid, args[d]; its items are [vstart[d], vstart[d + 1]),
// item l of d standing for block l of the launch that grid would have had
// on its own (y / z passes: a dims[2d] x dims[2d + 1] x gz grid, x fastest),
// so per-problem partial sums, last-block reductions and results are those
// of that launch.  smem: the largest shared memory of any descriptor.
template <typename A> struct GroupTab {
    const A* args = nullptr;   // [nd] (device)
    const int* vstart = nullptr;  // [nd + 1] (device)
    const int* dims = nullptr;    // [2 nd] (device; y / z passes)
    int nd = 0, total = 0;
    size_t smem = 0;
};
template <typename T, typename Tc> void launch_group_xfwd(const GroupTab<XfwdArgs<T, Tc>>& t, bool tangent, int guard,
                                                          cudaStream_t st);
template <typename T, typename Tc> void launch_group_xinv(const GroupTab<XinvArgs<T, Tc>>& t, int guard,
                                                          cudaStream_t st);
template <typename T, bool INV> void launch_group_ypass(const GroupTab<YArgs<T>>& t, cudaStream_t st);
template <typename T> void launch_group_zpass(const GroupTab<ZArgs<T>>& t, cudaStream_t st);
// item grids and shared memory of one descriptor of a grouped y / z pass
void ypass_group_shape(const GridDims& g, int tx, size_t cxbytes, int& gx, int& gy, int& gz, size_t& smem);
void zpass_group_shape(const GridDims& g, int tx, size_t cxbytes, int& gx, int& gy, int& gz, size_t& smem);

template <typename T, typename Tc> void launch_xfwd(const XfwdArgs<T, Tc>& a, int guard, cudaStream_t st);
template <typename T, typename Tc> void launch_xinv(const XinvArgs<T, Tc>& a, int guard, cudaStream_t st);
template <typename T, bool INV> void launch_ypass(const YArgs<T>& a, cudaStream_t st);
template <typename T> void launch_zpass(const ZArgs<T>& a, cudaStream_t st);
size_t xpass_smem(const GridDims& g, int lines, size_t cxbytes);
int xpass_lines(const GridDims& g, size_t cxbytes);
int xpass_grid(const GridDims& g, int lines);  // x-pass blocks (= partial count)
int xpass_partials_max(const GridDims& g);     // upper bound of any x-pass grid
int xpass_gp(const GridDims& g, int lines, int cap);  // x-pass blocks per problem (grid = nprob * gp)
// Newton right-hand side r = -G[P] of the double-float residual, transformed in
// FP32 (xpass.cu); tw32 / tw2_32: the FP32 engine's twiddles of the same grid
bool xinv_rhs32_ok(const GridDims& g);
void launch_xinv_rhs32(const XinvArgs<df32, float>& a, const cx<float>* tw32, const cx<float>* tw2_32, int guard,
                       cudaStream_t st);
int ypass_tx(int n, size_t cxbytes);  // columns per y-pass block (must match the launcher)
int zpass_tx(int n, size_t cxbytes);  // columns per z-pass block (sets the partial count)
int zpass_blocks(const GridDims& g, int tx, size_t cxbytes);  // non-TMA z-pass blocks (= partials) per problem

// FP32 CG x-inverse with streamed (bulk asynchronous, double-buffered)
// inputs, for n1 = 128, 256, 512 (xpass_stream.cu)
bool stream_xpass_ok(const GridDims& g);
// FP32 Krylov z- and y-passes with TMA tiles, n = 64, 128, 256 (zpass_tma.cu)
bool zpass_tma_size(int n3);
// (cand: tile-width candidate; the tensor map must be encoded for the
// candidate the launch's cfg selects)
bool zpass_tma_encode(void* map, const GridDims& g, const void* spec, int cand);
bool zpass_tma_encode_u(void* map, const GridDims& g, const void* spec, int cand);  // one-component box
void launch_zpass_tma(const ZArgs<float>& a, const void* map, cudaStream_t st);
bool ypass_tma_encode(void* map, const GridDims& g, const void* spec, int cand);
template <bool INV> void launch_ypass_tma(const YArgs<float>& a, const void* map, cudaStream_t st);
void launch_xinv_stream(const XinvArgs<float, float>& a, cudaStream_t st);

// Displacement form of the rotated Green operator in the FP32 CG (xdisp.cu):
// after the displacement z-pass and the y-inverse of components 0, 3, 6, the
// x-inverse turns those three spectra into the nodal fields u_i (real,
// [n3][n2][n1] each, at u + i * ustride), and the gradient pass forms the
// HEX8R gradient F_iJ = c_J sum over the 4 voxel edges along J of the
// differences of u_i (c_J = 1 / (4 h_J)) with the CG update r -= alpha F and
// the fused (r, r) reduction of the CG x-inverse.
struct DispArgs {
    GridDims g;
    const cx<float>* tw;   // exp(-2 pi i t / M)
    const cx<float>* tw2;  // exp(-2 pi i k / n1)
    const cx<float>* spec;
    float* u;              // three real fields
    int64_t ustride;       // floats between them
    float* r;              // [9][V]
    float cJ[3];           // 1 / (4 h_J)
    double* partial;
    Scalars* sc;
    int fuse;              // the last block turns the (r, r) partials into beta / stop
    double cg_tol;
    int cg_max, cg_fixed;
    uint32_t wait_cap;
};
// Nodal form of the rotated operator in the FP32 CG (xnodal.cu): G = D (D^T
// D)^+ D^T with D the HEX8R gradient.  The tangent pass assembles the nodal
// forces f_i = D^T (A : p)_i of the direction in real space (three fields
// instead of nine components) and transforms them along x into components
// 0, 3, 6 of the spectrum; the y-passes take those three; the z-pass divides
// by |kr|^2 (D^T D's symbol) between its transforms; the x side is that of
// the displacement form.  The direction p alternates between two buffers
// (p of CG iteration k in p[k & 1]): a block reads its neighbours' old p.
struct NodalArgs {
    GridDims g;
    const cx<float>* tw;   // exp(-2 pi i t / M)
    const cx<float>* tw2;  // exp(-2 pi i k / n1)
    cx<float>* spec;
    const int32_t* vrank;  // [V] boxel voxels: column of their packed tangent (>= 0); else -1 - phase
    const float* r;
    float* p[2];           // p of iteration k in p[k & 1]
    float* x;              // receives the previous iteration's x += alpha p
    const float* tc;       // [10][V] tangent cache (F^{-1}, mu - lam ln J)
    const double* matp;    // [nprob][4] per problem, or null: mu, lam
    double mu[2], lam[2];
    const float* bA;       // [45][nb] packed boxel tangents, boxels in voxel order
    const int32_t* lofs;   // [n2 n3 + 1] first boxel (voxel order) of each x-line (L2 prefetch)
    int64_t nb;
    float cJ[3];           // 1 / (4 h_J)
    int cfg;               // launch-shape candidate (0: even shares, 1: equal plane chunks per column)
    int nch;               // (set by the launcher) plane chunks per column, or 0: even shares
    int pfd;               // (set by the launcher) voxel lines ahead of the L2 prefetch
    double* partial;       // pAp partials
    Scalars* sc;
    int fuse;              // the last block turns the pAp partials into alpha
};
bool nodal_ok(const GridDims& g);  // sizes the nodal tangent pass takes
void launch_xfwd_nodal(NodalArgs a, cudaStream_t st);
int nodal_partials_max();  // largest grid of the nodal tangent pass
// z-pass of the nodal form: one component per tile (components 0, 3, 6),
// forward z FFT, scale / |kr|^2, inverse z FFT (tmap_u: one-component box)
void launch_zpass_scalar(const ZArgs<float>& a, cudaStream_t st);
// its map for tile-width candidate cand (box {16 or 8 (at 512), 1, n3, 1}, halved for cand 1)
bool zpass_scalar_encode(void* map, const GridDims& g, const void* spec, int cand);

bool disp_x_ok(const GridDims& g);  // sizes the two x kernels take
void launch_xinv_disp(const DispArgs& a, cudaStream_t st);
void launch_disp_grad_cg(const DispArgs& a, cudaStream_t st);
int disp_grad_partials_max();  // largest grid of the gradient pass (its partials)
// the two in one pass (the nodal fields stay in shared memory)
bool xinv_grad_ok(const GridDims& g);
void launch_xinv_grad(const DispArgs& a, cudaStream_t st);

// Record msg as the calling thread's last error; returns code.
int set_error(int code, const char* msg);

// ------------------------------------------------ doubly-fine material grid
// Sub-cell l = (l1, l2, l3) in {0,1}^3 (bit k of l is l_{k+1}) of the cell
// (i, j, k) of one problem (voxels base + i + n1 (j + n2 k), field stride V):
// the diagonal of F at the cell, the off-diagonal pairs at the staggered
// positions c + (l1, l2, 0) (F12, F21), c + (l1, 0, l3) (F13, F31) and
// c + (0, l2, l3) (F23, F32), periodic (App. A, Eq. constitutive_law).
__device__ __forceinline__ void dfmg_fsub(const double* __restrict__ F, int64_t V, int64_t base, int n1, int n2,
                                          int n3, int i, int j, int k, int l, double f[9])
{
    const int ip = (l & 1) ? (i + 1 == n1 ? 0 : i + 1) : i;
    const int jp = (l & 2) ? (j + 1 == n2 ? 0 : j + 1) : j;
    const int kp = (l & 4) ? (k + 1 == n3 ? 0 : k + 1) : k;
    const int64_t vc = base + i + (int64_t)n1 * (j + (int64_t)n2 * k);
    const int64_t v12 = base + ip + (int64_t)n1 * (jp + (int64_t)n2 * k);
    const int64_t v13 = base + ip + (int64_t)n1 * (j + (int64_t)n2 * kp);
    const int64_t v23 = base + i + (int64_t)n1 * (jp + (int64_t)n2 * kp);
    f[0] = F[0 * V + vc];
    f[4] = F[4 * V + vc];
    f[8] = F[8 * V + vc];
    f[1] = F[1 * V + v12];
    f[3] = F[3 * V + v12];
    f[2] = F[2 * V + v13];
    f[6] = F[6 * V + v13];
    f[5] = F[5 * V + v23];
    f[7] = F[7 * V + v23];
}

// Neo-Hookean P of F (Sec. 6.1) in FP64; false where det F <= 0
__device__ __forceinline__ bool nh_P64(const double f[9], double mu, double lam, double P[9])
{
    const double c0 = f[4] * f[8] - f[5] * f[7], c1 = f[5] * f[6] - f[3] * f[8], c2 = f[3] * f[7] - f[4] * f[6];
    const double J = f[0] * c0 + f[1] * c1 + f[2] * c2;
    if (!(J > 0.0)) return false;
    const double iJ = 1.0 / J;
    const double G[9] = {c0 * iJ,
                         (f[2] * f[7] - f[1] * f[8]) * iJ,
                         (f[1] * f[5] - f[2] * f[4]) * iJ,
                         c1 * iJ,
                         (f[0] * f[8] - f[2] * f[6]) * iJ,
                         (f[2] * f[3] - f[0] * f[5]) * iJ,
                         c2 * iJ,
                         (f[1] * f[6] - f[0] * f[7]) * iJ,
                         (f[0] * f[4] - f[1] * f[3]) * iJ};
    const double k = lam * log(J) - mu;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) P[3 * i + j] = mu * f[3 * i + j] + k * G[3 * j + i];
    return true;
}

// Infinitesimal strain: sigma = lam tr(H) I + mu (H + H^T), H = F - I (an
// isotropic linear phase; sigma depends on sym(H) only)
__device__ __forceinline__ void lin_sigma(const double f[9], double mu, double lam, double S[9])
{
    const double tr = (f[0] - 1.0) + (f[4] - 1.0) + (f[8] - 1.0);
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const double hij = f[3 * i + j] - (i == j ? 1.0 : 0.0), hji = f[3 * j + i] - (i == j ? 1.0 : 0.0);
            S[3 * i + j] = mu * (hij + hji) + (i == j ? lam * tr : 0.0);
        }
}

// Arguments of the doubly-fine material grid law (dfmg.cu, boxel.cu): the
// field F [9][V] of nprob problems stacked along z (Vp voxels, n1 x n2 x n3
// each); S [72][V] receives, at cell c and row 9 l + comp, component comp of
// the stress of sub-cell l of c; P [9][V] the gathered stress.
struct DfmgArgs {
    const double* F;
    double* S;
    double* P;
    const uint8_t* phase;
    const double* matp;  // [nprob][4] (mu-, mu+, lam-, lam+), or null: mu, lam
    double mu[2], lam[2];
    int64_t V, Vp;
    int n1, n2, n3;
    Scalars* sc;
    int guard;           // 2: skip problems whose outer iteration is done
    int dfloat;          // double-float residual form: the pure-cell laws and the gather in double-float,
                         // S holds (hi, lo) float pairs in place of doubles
};
// doubly-fine Newton-CG (single problem): the CG vectors, the tangent
// operands and results; stage 0 direction update, 1 sub-cell tangents, 2
// gather and alpha (partials: dfmg_cg_blocks(V) doubles)
template <typename Tc> struct DfmgTanArgs {
    const double* F;        // [9][V]
    const uint8_t* phase;
    const int32_t* vox2box;
    const Tc* bAsub;        // [45][8 nb] packed boxel sub-cell tangents
    int64_t nb;
    double mu[2], lam[2];
    const Tc* r;
    Tc* p;
    Tc* x;
    Tc* St;                 // [72][V] sub-cell values of A : p
    Tc* y;                  // [9][V] gathered A : p
    double* partial;
    Scalars* sc;
    int64_t V;
    int n1, n2, n3;
};
template <typename Tc> void launch_dfmg_cg(const DfmgTanArgs<Tc>& a, int stage, cudaStream_t st);
int dfmg_cg_blocks(int64_t V);

// a field X [9][V] at the doubly-fine positions of sub-cell l of cell (i, j, k)
// (one problem), like dfmg_fsub
template <typename S>
__device__ __forceinline__ void dfmg_fsub_t(const S* __restrict__ X, int64_t V, int n1, int n2, int n3, int i, int j,
                                            int k, int l, double f[9])
{
    const int ip = (l & 1) ? (i + 1 == n1 ? 0 : i + 1) : i;
    const int jp = (l & 2) ? (j + 1 == n2 ? 0 : j + 1) : j;
    const int kp = (l & 4) ? (k + 1 == n3 ? 0 : k + 1) : k;
    const int64_t vc = i + (int64_t)n1 * (j + (int64_t)n2 * k);
    const int64_t v12 = ip + (int64_t)n1 * (jp + (int64_t)n2 * k);
    const int64_t v13 = ip + (int64_t)n1 * (j + (int64_t)n2 * kp);
    const int64_t v23 = i + (int64_t)n1 * (jp + (int64_t)n2 * kp);
    f[0] = X[0 * V + vc];
    f[4] = X[4 * V + vc];
    f[8] = X[8 * V + vc];
    f[1] = X[1 * V + v12];
    f[3] = X[3 * V + v12];
    f[2] = X[2 * V + v13];
    f[6] = X[6 * V + v13];
    f[5] = X[5 * V + v23];
    f[7] = X[7 * V + v23];
}

void launch_dfmg_pure(const DfmgArgs& a, cudaStream_t st);
void launch_dfmg_gather(const DfmgArgs& a, cudaStream_t st);
// mean over the 8 sub-cells of the jump vectors ba8 [nb][8][3] -> ba [nb][3]
void launch_dfmg_amean(const double* ba8, double* ba, int64_t nb, cudaStream_t st);

// boxel laminate Newton solve
template <typename Tc> struct BoxelArgs {
    int64_t nb;
    int64_t V;
    const int32_t* bidx;
    const double* bN;
    const double* bc;
    double* ba;    // [nb][3] jump vectors (warm start in, converged out)
    double* bP;    // [nb][9]
    Tc* bA;        // [45][nb] packed symmetric tangent (sym_idx), column rank[b]; or null
    const int32_t* rank;  // position of boxel b in voxel order
    const int32_t* bprob; // problem of boxel b (stacked problems), or null
    const double* matp;   // [nprob][4] (mu-, mu+, lam-, lam+), or null: mu, lam
    const double* F;
    double mu[2], lam[2];
    double tol_rel, tol_abs;
    int max_iter;
    Scalars* sc;
    int guard;
    int dfloat;  // phase states and residual in double-float (refined double-float form)
    int linear;  // infinitesimal strain: the closed-form linear laminate (no Newton)
    // doubly-fine material grid (launch_boxel_dfmg): one laminate per boxel
    // sub-cell, ba holds [nb][8][3], the stress goes to S [72][V]
    double* S;
    int64_t Vp;
    int n1, n2, n3;
    // doubly-fine Newton-CG: packed tangent of every boxel sub-cell,
    // [45][8 nb] (column 8 b + l) in FP32 (sub_f32) or FP64; or null
    void* bAsub;
    int sub_f32;
};
template <typename Tc> void launch_boxel(const BoxelArgs<Tc>& a, cudaStream_t st);
// grouped: items of 128 boxels ((nb + 127) / 128 per descriptor); every
// descriptor has the same form (dfloat, linear)
template <typename Tc> void launch_group_boxel(const GroupTab<BoxelArgs<Tc>>& t, bool dfloat, bool linear,
                                               cudaStream_t st);
void launch_boxel_dfmg(const BoxelArgs<double>& a, cudaStream_t st);

}  // namespace combo

// Library context: a device and the stream every call on it runs on, plus a
// device scratch array grown on demand by the calls that need one (freed
// with the context).
struct combo_ctx {
    int device;
    cudaStream_t stream;
    bool own_stream;
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
};
