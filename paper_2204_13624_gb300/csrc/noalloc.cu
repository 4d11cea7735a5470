// noalloc.cu -- the Green operator Y = G[X] without any device allocation.
//
// For callers that must not allocate device memory: code running where
// cudaMalloc is unavailable or forbidden (inside a caller's own memory
// arena or pool, a real-time loop that may not allocate, a host framework
// that owns all device memory).  They pass device buffers for the input and
// the output; everything else the operator needs -- the half spectrum, the
// reduction partials, the solver scalars and the twiddle / symbol tables --
// lives in one file-scope device array, g_scratch, of kScratchBytes (4 MiB)
// that every GPU which loads this library holds until the process exits.
//
// Same kernels and the same arithmetic as combo_apply_G (FP64).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/combo.h"
#include "combo_internal.cuh"

using namespace combo;

// 4 MiB of device scratch shared by every call on a device (see the header).
static constexpr size_t kScratchBytes = size_t(4) << 20;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

namespace {

constexpr int kMaxSide = 64;
constexpr int kMaxPartials = 4096;

// scratch layout (byte offsets)
constexpr size_t kOffScalars = 0;
constexpr size_t kOffPartials = 1024;
constexpr size_t kOffTables = kOffPartials + kMaxPartials * sizeof(double);
constexpr size_t kTableBytes = 8192;
constexpr size_t kOffSpectrum = (kOffTables + kTableBytes + 255) / 256 * 256;
constexpr size_t kMaxSpectrum = (kScratchBytes - kOffSpectrum) / sizeof(double2);  // complex entries

static_assert(sizeof(Scalars) <= kOffPartials, "scalars do not fit");
static_assert((kMaxSide / 2 + 1 + kMaxSide / 2 + 2 * kMaxSide) * sizeof(double2) + 6 * kMaxSide * sizeof(double) <=
                  kTableBytes,
              "tables do not fit");

std::mutex g_setup_mutex;
void* g_scratch_addr[128] = {nullptr};  // device address of g_scratch, per device ordinal

bool is_23(int n)
{
    if (n < 1) return false;
    while (n % 2 == 0) n /= 2;
    while (n % 3 == 0) n /= 3;
    return n == 1;
}

Plan plan_for(int n)
{
    // radices 8, 4, 2, 3 with the same factor order as the solver's plans
    Plan p{};
    p.n = n;
    int a = 0, b = 0, m = n;
    while (m % 2 == 0) {
        m /= 2;
        a++;
    }
    while (m % 3 == 0) {
        m /= 3;
        b++;
    }
    int R[kMaxStages], k = 0;
    int p8 = a / 3, rem = a % 3;
    if (rem == 1 && p8 >= 1) p8 -= 1;
    for (int i = 0; i < p8; i++) R[k++] = 8;
    if (a % 3 == 1 && a >= 3) {
        R[k++] = 4;
        R[k++] = 4;
    } else if (a % 3 == 1) {
        R[k++] = 2;
    } else if (a % 3 == 2) {
        R[k++] = 4;
    }
    for (int i = 0; i < b; i++) R[k++] = 3;
    p.nst = k;
    int Ns = 1;
    for (int s = 0; s < k; s++) {
        p.R[s] = R[s];
        p.Ns[s] = Ns;
        Ns *= R[s];
    }
    return p;
}

// Per-call set-up on the device (no host copy): clears the solver scalars and
// fills the twiddle tables exp(-2 pi i k / m) and the derivative symbol of
// the requested scheme in product form k_j = sa_j[xi_j] prod_{m != j} sb_m[xi_m]
// (rotated: sa = (2/h) sin(pi xi / n), sb = cos(pi xi / n), 0 at Nyquist;
// spectral: sa = 2 pi xi_signed / l, 0 at Nyquist, sb = 1).  One block.
__global__ void k_noalloc_tables(int n1, int n2, int n3, double l1, double l2, double l3, int kspace, Scalars* sc,
                                 double2* twM, double2* tw2, double2* twy, double2* twz, double* sa, double* sb)
{
    const int M = n1 / 2;
    uint32_t* z = reinterpret_cast<uint32_t*>(sc);
    for (int i = threadIdx.x; i < (int)(sizeof(Scalars) / 4); i += blockDim.x) z[i] = 0u;
    auto tw = [](int k, int m) {
        double s, c;
        sincospi(2.0 * (double)k / (double)m, &s, &c);
        return double2{c, -s};
    };
    const int n[3] = {n1, n2, n3};
    const double l[3] = {l1, l2, l3};
    for (int k = threadIdx.x; k < kMaxSide; k += blockDim.x) {
        if (k < M) twM[k] = tw(k, M);
        if (k <= M) tw2[k] = tw(k, n1);
        if (k < n2) twy[k] = tw(k, n2);
        if (k < n3) twz[k] = tw(k, n3);
        for (int j = 0; j < 3; j++) {
            if (k >= n[j]) continue;
            const bool nyq = (2 * k == n[j]);
            double a, b;
            if (kspace == COMBO_ROTATED) {
                double s, c;
                sincospi((double)k / (double)n[j], &s, &c);
                a = (2.0 * n[j] / l[j]) * s;
                b = nyq ? 0.0 : c;
            } else {
                const int ks = (2 * k > n[j]) ? k - n[j] : k;
                a = nyq ? 0.0 : 2.0 * M_PI * (double)ks / l[j];
                b = 1.0;
            }
            sa[j * kMaxSide + k] = a;
            sb[j * kMaxSide + k] = b;
        }
    }
}

__global__ void k_noalloc_sumsq(Scalars* sc, const double* part, int n)
{
    __shared__ double red[256];
    const double s = sum_partials_fixed(part, n, red);
    if (threadIdx.x == 0) sc->resid2 = s;
}

}  // namespace

extern "C" int combo_apply_G_noalloc(int32_t device, void* stream, const int32_t n[3], const double l[3],
                                     int32_t kspace, const double* X, double* Y, double* sumsq)
{
    if (!n || !l || !X || !Y) return set_error(COMBO_E_INVALID_ARG, "combo_apply_G_noalloc: null argument");
    for (int j = 0; j < 3; j++) {
        if (n[j] < 2 || n[j] > kMaxSide || !is_23(n[j]))
            return set_error(COMBO_E_INVALID_ARG,
                             "combo_apply_G_noalloc: each side must be 2^a 3^b in [2, 64]");
        if (!(l[j] > 0.0)) return set_error(COMBO_E_INVALID_ARG, "combo_apply_G_noalloc: lengths must be positive");
    }
    if (n[0] % 2) return set_error(COMBO_E_INVALID_ARG, "combo_apply_G_noalloc: n1 must be even");
    if (kspace != COMBO_ROTATED && kspace != COMBO_SPECTRAL)
        return set_error(COMBO_E_INVALID_ARG, "combo_apply_G_noalloc: bad kspace");
    if (device < 0 || device >= 128) return set_error(COMBO_E_INVALID_ARG, "combo_apply_G_noalloc: bad device");

    GridDims g{};
    g.n1 = n[0];
    g.n2 = n[1];
    g.n3 = n[2];
    g.n3p = n[2];
    g.nprob = 1;
    g.M = n[0] / 2;
    g.nh = g.M + 1;
    g.nhp = (g.nh + 3) / 4 * 4;
    g.V = (int64_t)n[0] * n[1] * n[2];
    g.Vs = (int64_t)n[2] * n[1] * g.nhp;
    if ((size_t)(9 * g.Vs) > kMaxSpectrum) {
        char msg[256];
        snprintf(msg, sizeof msg,
                 "combo_apply_G_noalloc: grid too large for the 4 MiB scratch (9 n3 n2 (n1/2+1 rounded up to 4) = "
                 "%lld complex entries; at most %zu fit; every grid up to 32^3 fits)",
                 (long long)(9 * g.Vs), kMaxSpectrum);
        return set_error(COMBO_E_INVALID_ARG, msg);
    }

    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess) return set_error(COMBO_E_CUDA, "combo_apply_G_noalloc: no CUDA device");
    if (cudaSetDevice(device) != cudaSuccess) return set_error(COMBO_E_CUDA, "combo_apply_G_noalloc: cannot use device");
    struct Restore {
        int d;
        ~Restore() { cudaSetDevice(d); }
    } restore{prev};

    // X and Y must be device memory the caller owns
    for (const void* ptr : {(const void*)X, (const void*)Y}) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess ||
            (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)) {
            cudaGetLastError();
            return set_error(COMBO_E_INVALID_ARG, "combo_apply_G_noalloc: X and Y must be device pointers");
        }
    }

    // set-up, once per device with that device current: the device address of g_scratch
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_addr[device]) {
            void* ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
            if (e != cudaSuccess || !ptr) return set_error(COMBO_E_CUDA, "combo_apply_G_noalloc: cudaGetSymbolAddress failed");
            g_scratch_addr[device] = ptr;
        }
        base = g_scratch_addr[device];
    }
    unsigned char* s = static_cast<unsigned char*>(base);
    Scalars* sc = reinterpret_cast<Scalars*>(s + kOffScalars);
    double* part = reinterpret_cast<double*>(s + kOffPartials);
    double2* twM = reinterpret_cast<double2*>(s + kOffTables);
    double2* tw2 = twM + kMaxSide / 2;
    double2* twy = tw2 + (kMaxSide / 2 + 1);
    double2* twz = twy + kMaxSide;
    double* sa = reinterpret_cast<double*>(twz + kMaxSide);
    double* sb = sa + 3 * kMaxSide;
    double2* spec = reinterpret_cast<double2*>(s + kOffSpectrum);
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    // the scratch keeps the previous call's contents: the set-up kernel
    // clears the scalars (the spectrum and partials are overwritten in full)
    k_noalloc_tables<<<1, kMaxSide, 0, st>>>(n[0], n[1], n[2], l[0], l[1], l[2], kspace, sc, twM, tw2, twy, twz, sa,
                                             sb);
    if (cudaGetLastError() != cudaSuccess) return set_error(COMBO_E_CUDA, "combo_apply_G_noalloc: set-up failed");

    const Plan pM = plan_for(g.M), py = plan_for(g.n2), pz = plan_for(g.n3);
    XfwdArgs<double, double> xf{};
    xf.g = g;
    xf.plan = pM;
    xf.tw = twM;
    xf.tw2 = tw2;
    xf.spec = spec;
    xf.lines_per_block = xpass_lines(g, sizeof(double2));
    xf.mode = XF_RESID;
    xf.X = X;
    xf.sc = sc;
    if (xpass_grid(g, xf.lines_per_block) > kMaxPartials) return set_error(COMBO_E_INVALID_ARG, "combo_apply_G_noalloc: grid too large");
    launch_xfwd<double, double>(xf, 0, st);

    YArgs<double> y{};
    y.g = g;
    y.plan = py;
    y.tw = twy;
    y.spec = spec;
    y.tx = ypass_tx(g.n2, sizeof(double2));
    y.sc = sc;
    launch_ypass<double, false>(y, st);

    ZArgs<double> z{};
    z.g = g;
    z.plan = pz;
    z.tw = twz;
    z.spec = spec;
    z.tx = zpass_tx(g.n3, sizeof(double2));
    for (int j = 0; j < 3; j++) {
        z.sa[j] = sa + j * kMaxSide;
        z.sb[j] = sb + j * kMaxSide;
    }
    z.scale = 2.0 / (double)g.V;
    z.want_norm = 1;
    z.partial = part;
    z.sc = sc;
    const int zblocks = zpass_blocks(g, z.tx, sizeof(double2));  // the launcher's own block count
    if (zblocks > kMaxPartials) return set_error(COMBO_E_INVALID_ARG, "combo_apply_G_noalloc: grid too large");
    launch_zpass<double>(z, st);
    launch_ypass<double, true>(y, st);

    XinvArgs<double, double> xi{};
    xi.g = g;
    xi.plan = pM;
    xi.tw = twM;
    xi.tw2 = tw2;
    xi.spec = spec;
    xi.lines_per_block = xf.lines_per_block;
    xi.mode = XI_PLAIN;
    xi.Y = Y;
    xi.sc = sc;
    launch_xinv<double, double>(xi, 0, st);

    if (sumsq) {
        k_noalloc_sumsq<<<1, 256, 0, st>>>(sc, part, zblocks);
        double r2 = 0.0;
        if (cudaMemcpyAsync(&r2, &sc->resid2, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return set_error(COMBO_E_CUDA, "combo_apply_G_noalloc: reading the sum of squares failed");
        *sumsq = r2 / (double)g.V;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(COMBO_E_CUDA, cudaGetErrorString(e));
    return COMBO_OK;
}
