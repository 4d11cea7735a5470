// runtime.cu -- C ABI of libcombo.so: contexts, per-solve device state, the
// solver state machine (load steps, fixed point, Newton-CG with FP32 Krylov
// iterations and FP64 residuals) and the small solver kernels.
//
// Paper: arXiv 2204.13624.  Sec. 2 (HOM, Pbar = <P>), Sec. 3 (Lippmann-
// Schwinger equation, Green operator, fixed point / Newton with a fast linear
// solver), Sec. 4 (composite boxels), Sec. 6.1 (Neo-Hookean phases).
#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <condition_variable>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstddef>
#include <type_traits>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/combo.h"
#include "async_copy.cuh"
#include "combo_internal.cuh"

using namespace combo;

// ------------------------------------------------------------------ errors
static thread_local std::string g_err;

static int fail(int code, const std::string& msg)
{
    g_err = msg;
    return code;
}

#define CK(call)                                                                                        \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess) return fail(COMBO_E_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

extern "C" const char* combo_last_error(void) { return g_err.c_str(); }

// ------------------------------------------------------------------ allocation
// Every device allocation of a solve, batch or server goes through
// dev_malloc, which the fault-injection hook (combo_fault_inject_alloc) can
// make fail the way cudaMalloc fails when the device is out of memory.
static std::atomic<int64_t> g_alloc_countdown{-1};

template <typename T> static cudaError_t dev_malloc(T** p, size_t bytes)
{
    int64_t c = g_alloc_countdown.load();
    while (c >= 0 && !g_alloc_countdown.compare_exchange_weak(c, c - 1)) {
    }
    if (c == 0) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(reinterpret_cast<void**>(p), bytes);
}

extern "C" int combo_fault_inject_alloc(int64_t after)
{
    g_alloc_countdown.store(after < 0 ? -1 : after);
    return COMBO_OK;
}

// Lets other translation units of the library report an error message.
int combo::set_error(int code, const char* msg)
{
    g_err = msg;
    return code;
}

// ------------------------------------------------------------------ context
extern "C" int combo_ctx_create(const combo_ctx_opts* o, combo_ctx** out)
{
    if (!out) return fail(COMBO_E_INVALID_ARG, "null output pointer");
    int dev = o ? o->device : 0;
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev));
    if (dev < 0 || dev >= ndev) return fail(COMBO_E_INVALID_ARG, "no such CUDA device");
    CK(cudaSetDevice(dev));
    combo_ctx* c = new combo_ctx();
    c->device = dev;
    if (o && o->stream) {
        c->stream = (cudaStream_t)o->stream;
        c->own_stream = false;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete c;
            return fail(COMBO_E_CUDA, cudaGetErrorString(e));
        }
        c->own_stream = true;
    }
    *out = c;
    return COMBO_OK;
}

extern "C" void combo_ctx_destroy(combo_ctx* c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->scratch) {
        cudaStreamSynchronize(c->stream);
        cudaFree(c->scratch);
    }
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}

extern "C" void combo_options_default(combo_options* o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = COMBO_FP64;
    o->kspace = COMBO_ROTATED;
    o->solver = COMBO_NEWTON_CG;
    o->tol = 1e-8;
    o->max_iter = 0;  // solver default
    o->fixed_iterations = 0;
    o->cg_tol = 1e-3;
    o->cg_max_iter = 2000;
    o->cg_fixed_iterations = 0;
    o->nr_tol_rel = 1e-12;
    o->nr_tol_abs = 1e-14;
    o->nr_max_iter = 50;
    o->c_min = 1e-6;
    o->mu0 = 0.0;
    o->theory = COMBO_FINITE_STRAIN;
    o->wait_poll_cap = 0;
}

// ------------------------------------------------------------------ plans and tables
static bool is_23(int n)
{
    if (n < 1) return false;
    while (n % 2 == 0) n /= 2;
    while (n % 3 == 0) n /= 3;
    return n == 1;
}

static Plan make_plan(int n)
{
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
    std::vector<int> R;
    int p8 = a / 3, rem = a % 3;
    if (rem == 1 && p8 >= 1) {
        p8 -= 1;
        R.push_back(4);
        R.push_back(4);
    } else if (rem == 1) {
        R.push_back(2);
    } else if (rem == 2) {
        R.push_back(4);
    }
    for (int i = 0; i < p8; i++) R.insert(R.begin(), 8);
    for (int i = 0; i < b; i++) R.push_back(3);
    p.nst = (int)R.size();
    int Ns = 1;
    for (int s = 0; s < p.nst; s++) {
        p.R[s] = R[s];
        p.Ns[s] = Ns;
        Ns *= R[s];
    }
    return p;
}

template <typename T> struct DevTables {
    cx<T>* twM = nullptr;   // [M]
    cx<T>* tw2 = nullptr;   // [M + 1]
    cx<T>* twy = nullptr;   // [n2]
    cx<T>* twz = nullptr;   // [n3]
    T* sa[3] = {nullptr, nullptr, nullptr};
    T* sb[3] = {nullptr, nullptr, nullptr};
    cx<T>* ph[3] = {nullptr, nullptr, nullptr};  // staggered grid only
    cx<T>* rph[3] = {nullptr, nullptr, nullptr};  // rotated scheme only: the same e^{i pi xi / n}
};

template <typename T> static int upload_tw(cx<T>** d, int n, int denom)
{
    std::vector<cx<T>> h(std::max(n, 1));
    for (int t = 0; t < n; t++) {
        const double ang = 2.0 * M_PI * (double)t / (double)denom;
        h[t].x = (T)std::cos(ang);
        h[t].y = (T)(-std::sin(ang));
    }
    CK(dev_malloc(d, sizeof(cx<T>) * h.size()));
    CK(cudaMemcpy(*d, h.data(), sizeof(cx<T>) * h.size(), cudaMemcpyHostToDevice));
    return COMBO_OK;
}

// Discrete derivative symbol in product form k_j = sa_j[xi_j] prod_{m != j} sb_m[xi_m].
//   rotated (Willot, HEX8R): sa = (2/h) sin(pi xi / n), sb = cos(pi xi / n), sb := 0 at Nyquist;
//     this is the rotated-scheme symbol up to the common phase i e^{i sum theta/2},
//     which cancels in k k^H / |k|^2.
//   spectral (Moulinec-Suquet): sa = 2 pi xi_signed / l (0 at Nyquist), sb = 1.
//   staggered (App. A): sa = (2/h) sin(pi xi / n), sb = 1, and the phase
//     table ph = e^{i pi xi / n} = e^{i theta/2} of the forward / backward
//     difference symbols i sa e^{+-i theta/2} (rows differ: stag_u).
template <typename T> static int upload_symbols(DevTables<T>& t, const int n[3], const double l[3], int kspace)
{
    for (int j = 0; j < 3; j++) {
        std::vector<T> a(n[j]), b(n[j]);
        std::vector<cx<T>> ph(n[j]);
        const double h = l[j] / n[j];
        for (int x = 0; x < n[j]; x++) {
            const bool nyq = (2 * x == n[j]);
            ph[x].x = (T)std::cos(M_PI * (double)x / n[j]);
            ph[x].y = (T)std::sin(M_PI * (double)x / n[j]);
            if (kspace == COMBO_STAGGERED) {
                a[x] = (T)((2.0 / h) * std::sin(M_PI * (double)x / n[j]));
                b[x] = (T)1;
            } else if (kspace == COMBO_ROTATED) {
                a[x] = (T)((2.0 / h) * std::sin(M_PI * (double)x / n[j]));
                b[x] = nyq ? (T)0 : (T)std::cos(M_PI * (double)x / n[j]);
            } else {
                const int xs = (2 * x > n[j]) ? x - n[j] : x;
                a[x] = nyq ? (T)0 : (T)(2.0 * M_PI * (double)xs / l[j]);
                b[x] = (T)1;
            }
        }
        CK(dev_malloc(&t.sa[j], sizeof(T) * n[j]));
        CK(dev_malloc(&t.sb[j], sizeof(T) * n[j]));
        CK(cudaMemcpy(t.sa[j], a.data(), sizeof(T) * n[j], cudaMemcpyHostToDevice));
        CK(cudaMemcpy(t.sb[j], b.data(), sizeof(T) * n[j], cudaMemcpyHostToDevice));
        if (kspace == COMBO_STAGGERED) {
            CK(dev_malloc(&t.ph[j], sizeof(cx<T>) * n[j]));
            CK(cudaMemcpy(t.ph[j], ph.data(), sizeof(cx<T>) * n[j], cudaMemcpyHostToDevice));
        } else if (kspace == COMBO_ROTATED && sizeof(T) == 4) {
            CK(dev_malloc(&t.rph[j], sizeof(cx<T>) * n[j]));
            CK(cudaMemcpy(t.rph[j], ph.data(), sizeof(cx<T>) * n[j], cudaMemcpyHostToDevice));
        }
    }
    return COMBO_OK;
}

template <typename T> static int make_tables(DevTables<T>& t, const GridDims& g, const double l[3], int kspace)
{
    int rc;
    if ((rc = upload_tw<T>(&t.twM, g.M, g.M))) return rc;
    if ((rc = upload_tw<T>(&t.tw2, g.M + 1, g.n1))) return rc;
    if ((rc = upload_tw<T>(&t.twy, g.n2, g.n2))) return rc;
    if ((rc = upload_tw<T>(&t.twz, g.n3p, g.n3p))) return rc;
    const int n[3] = {g.n1, g.n2, g.n3p};
    return upload_symbols<T>(t, n, l, kspace);
}

template <typename T> static void free_tables(DevTables<T>& t)
{
    cudaFree(t.twM);
    cudaFree(t.tw2);
    cudaFree(t.twy);
    cudaFree(t.twz);
    for (int j = 0; j < 3; j++) {
        cudaFree(t.sa[j]);
        cudaFree(t.sb[j]);
        cudaFree(t.ph[j]);
        cudaFree(t.rph[j]);
    }
}

// grid of nprob stacked problems of n1 x n2 x n3 each (z axis: problem-major)
static GridDims make_dims(const int32_t n[3], int nprob = 1)
{
    GridDims g{};
    g.n1 = n[0];
    g.n2 = n[1];
    g.n3 = n[2] * nprob;
    g.n3p = n[2];
    g.nprob = nprob;
    g.M = n[0] / 2;
    g.nh = g.M + 1;
    g.nhp = (g.nh + 3) / 4 * 4;
    g.V = (int64_t)n[0] * n[1] * g.n3;
    g.Vs = (int64_t)g.n3 * n[1] * g.nhp;
    return g;
}

// ------------------------------------------------------------------ per-kernel timing
// Optional CUDA-event timing of every kernel launch class of a solve, on the
// solve's stream; pairs are read back at the solver's own sync points.
enum KClass {
    K_BOXEL = 0,
    K_XFWD_RESID,
    K_YFWD_64,
    K_ZGAMMA_64,
    K_YINV_64,
    K_XINV_64,
    K_XFWD_TANGENT,
    K_YFWD_C,
    K_ZGAMMA_C,
    K_YINV_C,
    K_XINV_CG,
    K_FINALIZE,
    K_UPDATE,
    K_DFMG_PURE,
    K_DFMG_GATHER,
    K_DFMG_CG,
    K_DISP_GRAD,
    K_XFWD_NODAL,
    K_XINV_GRAD,
    K_NCLASS
};
static const char* kclass_name[K_NCLASS] = {"boxel_laminate", "xfwd_resid_fp64", "yfwd_fp64", "zgamma_fp64",
                                             "yinv_fp64", "xinv_fp64", "xfwd_tangent", "yfwd_krylov",
                                             "zgamma_krylov", "yinv_krylov", "xinv_cg", "finalize", "update_F",
                                             "dfmg_pure", "dfmg_gather", "dfmg_cg_tangent", "grad_cg", "xfwd_nodal", "xinv_grad_cg"};

struct Profiler {
    bool on = false;
    cudaStream_t st = nullptr;
    std::vector<cudaEvent_t> pool;
    struct Rec {
        int k;
        cudaEvent_t a, b;
    };
    std::vector<Rec> pending;
    double ms[K_NCLASS] = {0};
    long long launches[K_NCLASS] = {0};
    int open_k = -1;
    cudaEvent_t open_a = nullptr;
    cudaEvent_t get()
    {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e;
        cudaEventCreate(&e);
        return e;
    }
    // every launch class is also an NVTX range named after it (a no-op
    // unless a profiler that records NVTX is attached)
    void begin(int k)
    {
        nvtxRangePushA(kclass_name[k]);
        if (!on) {
            launches[k]++;
            return;
        }
        open_k = k;
        open_a = get();
        cudaEventRecord(open_a, st);
    }
    void end()
    {
        nvtxRangePop();
        if (!on) return;
        cudaEvent_t b = get();
        cudaEventRecord(b, st);
        pending.push_back({open_k, open_a, b});
        open_k = -1;
    }
    // call after the stream has been synchronised
    void collect()
    {
        for (auto& r : pending) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) ms[r.k] += t;
            launches[r.k]++;
            pool.push_back(r.a);
            pool.push_back(r.b);
        }
        pending.clear();
    }
    void reset()
    {
        for (int k = 0; k < K_NCLASS; k++) {
            ms[k] = 0;
            launches[k] = 0;
        }
    }
    ~Profiler()
    {
        for (auto& r : pending) {
            pool.push_back(r.a);
            pool.push_back(r.b);
        }
        for (auto e : pool) cudaEventDestroy(e);
    }
};

static double wall_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// COMBO_PROFILE set in the environment: batches time every kernel launch
// class with CUDA events and print the table to stderr when they finish
// (eager launches in place of the captured CG graphs)
static bool env_profile()
{
    const char* e = std::getenv("COMBO_PROFILE");
    return e && *e && *e != '0';
}

static void print_profile(const char* what, Profiler& p)
{
    p.collect();
    double tot = 0.0;
    for (int k = 0; k < K_NCLASS; k++) tot += p.ms[k];
    std::fprintf(stderr, "[combo profile] %s: %.3f ms in kernels\n", what, tot);
    for (int k = 0; k < K_NCLASS; k++)
        if (p.launches[k])
            std::fprintf(stderr, "[combo profile]   %-16s %8lld launches %10.3f ms\n", kclass_name[k], p.launches[k],
                         p.ms[k]);
}

// a named NVTX range over a host scope (solve phases)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// ------------------------------------------------------------------ operator engine
// One FFT + Green-operator pipeline in precision T.
template <typename T> struct Engine {
    GridDims g;
    DevTables<T> tab;
    Plan pM, py, pz;
    int lines, txy, txz;
    int lines_fwd;  // x-lines per group of the x-forward (lines: of the x-inverse)
    cx<T>* spec = nullptr;  // not owned
    // TMA views of spec for the FP32 z- and y-passes, one per tile-width candidate
    CUtensorMap zmap[2], ymap[2];
    bool zmap_ok[2] = {false, false}, ymap_ok[2] = {false, false};
    // displacement form of the rotated operator in the FP32 Krylov passes:
    // the z-pass's one-component store maps and the switch (set per solve)
    CUtensorMap zumap[2];
    bool zumap_ok[2] = {false, false};
    int use_disp = 0;
    // nodal form (the tangent pass assembles nodal forces): the scalar
    // z-pass's map and the switch (set per solve)
    CUtensorMap zsmap[2];
    bool zsmap_ok[2] = {false, false};
    int use_nodal = 0;
    // launch-shape candidates chosen by the autotuner: x-forward, y, z, x-inverse
    int cfg_xf = 0, cfg_y = 0, cfg_z = 0, cfg_xi = 0;
    uint32_t wait_cap = 0;  // poll cap of the bulk-copy waits (wait_cap_of; 0 = default)
    void bind_spec(void* s)
    {
        spec = (cx<T>*)s;
        for (int c = 0; c < 2; c++) {
            zmap_ok[c] = (sizeof(T) == 4) && zpass_tma_encode(&zmap[c], g, s, c);
            ymap_ok[c] = (sizeof(T) == 4) && ypass_tma_encode(&ymap[c], g, s, c);
            zumap_ok[c] = (sizeof(T) == 4) && tab.rph[0] && zpass_tma_encode_u(&zumap[c], g, s, c);
        }
        for (int c = 0; c < 2; c++)
            zsmap_ok[c] = (sizeof(T) == 4) && tab.rph[0] && zpass_scalar_encode(&zsmap[c], g, s, c);
        if (!zmap_ok[cfg_z]) cfg_z = 0;
        if (!ymap_ok[cfg_y]) cfg_y = 0;
    }
    int init(const GridDims& gd, const double l[3], int kspace)
    {
        g = gd;
        pM = make_plan(g.M);
        py = make_plan(g.n2);
        pz = make_plan(g.n3p);
        lines = lines_fwd = xpass_lines(g, sizeof(cx<T>));
        if (sizeof(cx<T>) == 16) {
            // x-forward passes in FP64 or double-float words: groups of lines
            // as large (up to 1024 voxels) as two resident blocks per SM allow
            // (the kernel is register-capped for two), so that the FFT phase
            // keeps more of a 256-thread block busy
            while (lines_fwd * g.n1 < 1024 && xpass_smem(g, lines_fwd * 2, sizeof(cx<T>)) <= 110 * 1024 &&
                   (g.n2 * g.n3p) % (lines_fwd * 2) == 0)
                lines_fwd *= 2;
            // and the x-inverse (two blocks per SM by registers): groups of up
            // to 512 voxels within the same shared-memory budget
            while (lines * g.n1 < 512 && xpass_smem(g, lines * 2, sizeof(cx<T>)) <= 110 * 1024 &&
                   (g.n2 * g.n3p) % (lines * 2) == 0)
                lines *= 2;
        }
        txy = ypass_tx(g.n2, sizeof(cx<T>));
        txz = zpass_tx(g.n3p, sizeof(cx<T>));
        return make_tables<T>(tab, g, l, kspace);
    }
    void release() { free_tables<T>(tab); }
    // the displacement form applies: rotated FP32 tables, TMA y- and z-passes
    // at the chosen tile widths and an x side for this grid
    bool disp_capable() const
    {
        return sizeof(T) == 4 && tab.rph[0] && zmap_ok[cfg_z] && zumap_ok[cfg_z] && ymap_ok[cfg_y] && disp_x_ok(g);
    }
    // the nodal fields of the displacement form: components 1, 4, 7 of the
    // FP32 spectrum (free once the z-pass has read them), V floats each
    float* disp_u() const { return reinterpret_cast<float*>(spec + g.Vs); }
    // the nodal form applies on top: its tangent pass and scalar z-pass
    bool nodal_capable() const { return disp_capable() && zsmap_ok[cfg_z] && nodal_ok(g); }
    int64_t disp_ustride() const { return 3 * 2 * g.Vs; }

    template <typename Tc> XfwdArgs<T, Tc> xf() const
    {
        XfwdArgs<T, Tc> a{};
        a.g = g;
        a.plan = pM;
        a.tw = tab.twM;
        a.tw2 = tab.tw2;
        a.spec = spec;
        a.lines_per_block = lines_fwd;
        a.cfg = cfg_xf;
        return a;
    }
    template <typename Tc> XinvArgs<T, Tc> xi() const
    {
        XinvArgs<T, Tc> a{};
        a.g = g;
        a.plan = pM;
        a.tw = tab.twM;
        a.tw2 = tab.tw2;
        a.spec = spec;
        a.lines_per_block = lines;
        a.cfg = cfg_xi;
        a.wait_cap = wait_cap;
        return a;
    }
    YArgs<T> yargs(Scalars* sc, int guard) const
    {
        YArgs<T> y{};
        y.g = g;
        y.plan = py;
        y.tw = tab.twy;
        y.spec = spec;
        y.tx = txy;
        y.sc = sc;
        y.guard = guard;
        y.cfg = cfg_y;
        y.tmap = ymap_ok[cfg_y] ? &ymap[cfg_y] : nullptr;
        y.wait_cap = wait_cap;
        return y;
    }
    ZArgs<T> zargs(Scalars* sc, int guard, bool want_norm, double* partial) const
    {
        ZArgs<T> z{};
        z.g = g;
        z.plan = pz;
        z.tw = tab.twz;
        z.spec = spec;
        z.tx = txz;
        for (int j = 0; j < 3; j++) {
            z.sa[j] = tab.sa[j];
            z.sb[j] = tab.sb[j];
            z.ph[j] = tab.ph[j];
        }
        z.scale = (T)(2.0 * g.nprob / (double)g.V);  // 2 / (voxels of one problem)
        z.want_norm = want_norm ? 1 : 0;
        z.partial = partial;
        z.sc = sc;
        z.guard = guard;
        z.cfg = cfg_z;
        z.tmap = zmap_ok[cfg_z] ? &zmap[cfg_z] : nullptr;
        z.wait_cap = wait_cap;
        if (use_nodal && guard == 1 && !want_norm && zsmap_ok[cfg_z]) {
            z.disp = 2;  // nodal form: scalar z-pass on components 0, 3, 6
            z.tmap_u = &zsmap[cfg_z];
        } else if (use_disp && guard == 1 && !want_norm && z.tmap && zumap_ok[cfg_z]) {
            z.disp = 1;
            z.tmap_u = &zumap[cfg_z];
            for (int j = 0; j < 3; j++) z.rph[j] = tab.rph[j];
        }
        return z;
    }
    // y forward, z forward + projection + z inverse, y inverse
    // inv32 (double-float words): the inverse z and y transforms in FP32
    // arithmetic (the output feeds an FP32 field); tw32y / tw32z: FP32
    // twiddles of the same sides
    void yz(Scalars* sc, int guard, bool want_norm, double* partial, cudaStream_t st, Profiler* pr = nullptr,
            int kbase = 0, bool inv32 = false, const cx<float>* tw32y = nullptr, const cx<float>* tw32z = nullptr) const
    {
        ZArgs<T> z = zargs(sc, guard, want_norm, partial);
        YArgs<T> y = yargs(sc, guard);
        if (inv32 && tw32y && tw32z) {
            z.inv32 = 1;
            z.tw32 = tw32z;
        }
        y.disp = (z.disp == 2) ? 1 : 0;  // the nodal form's forward spectrum: components 0, 3, 6
        if (pr) pr->begin(kbase);
        launch_ypass<T, false>(y, st);
        if (pr) pr->end();
        if (pr) pr->begin(kbase + 1);
        if constexpr (sizeof(T) == 4) {
            if (z.disp == 2)
                launch_zpass_scalar(z, st);
            else
                launch_zpass<T>(z, st);
        } else {
            launch_zpass<T>(z, st);
        }
        if (pr) pr->end();
        YArgs<T> yi = y;
        yi.disp = z.disp ? 1 : 0;  // the displacement and nodal forms leave components 0, 3, 6 only
        if (inv32 && tw32y && tw32z) {
            yi.inv32 = 1;
            yi.tw32 = tw32y;
        }
        if (pr) pr->begin(kbase + 2);
        launch_ypass<T, true>(yi, st);
        if (pr) pr->end();
    }
    int zblocks_p() const { return zpass_blocks(g, txz, sizeof(cx<T>)); }  // z-pass blocks (partials) per problem
    int zblocks() const { return zblocks_p() * g.nprob; }
    int xblocks() const { return xpass_grid(g, lines); }
    int xpartials() const
    {
        return std::max(std::max(xpass_grid(g, lines), xpass_grid(g, lines_fwd)), xpass_partials_max(g));
    }
};

// ------------------------------------------------------------------ small kernels
__global__ void k_fill_identity(double* F, int64_t V)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 9 * V; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i / V);
        F[i] = (c == 0 || c == 4 || c == 8) ? 1.0 : 0.0;
    }
}

struct Mat9 {
    double v[9];
};

// F += d (uniform); stacked problems: dF [nprob][9] per problem of Vp voxels
__global__ void k_add_uniform(double* F, int64_t V, Mat9 d, const double* dF, int64_t Vp)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 9 * V; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = i / V;
        F[i] += dF ? dF[9 * ((i - c * V) / Vp) + c] : d.v[c];
    }
}

__global__ void k_vox2box(int32_t* map, const int32_t* bidx, int64_t nb)
{
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b < nb) map[bidx[b]] = (int32_t)b;
}

// nodal form's voxel map: a boxel voxel's column of the packed tangents (its
// rank in voxel order), else -1 - phase
__global__ void k_vrank(int32_t* vrank, const uint8_t* phase, const int32_t* v2b, const int32_t* rank, int64_t V)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        const int ph = phase[v];
        vrank[v] = ph == 2 ? rank[v2b[v]] : -1 - ph;
    }
}

// deterministic fixed-order sum of n partials by one block
__device__ double sum_partials(const double* p, int n, double* red) { return sum_partials_fixed(p, n, red); }

// residual of the current evaluation; fixed-point bookkeeping (mode 1).
// Block b: problem b, partials part[b n .. b n + n); V voxels per problem.
// skip_done: problems whose outer_done is set were not evaluated.
__global__ void k_fin_resid(Scalars* scs, const double* part_all, int n, double V, double tol, int fixed, int max_iter,
                            int fixed_point, int skip_done = 0, int ncg = 0)
{
    __shared__ double red[256];
    Scalars* sc = scs + blockIdx.x;
    const double* part = part_all + (size_t)blockIdx.x * n;
    if ((fixed_point || skip_done) && sc->outer_done) return;
    const double s = sum_partials(part, n, red);
    if (threadIdx.x != 0) return;
    sc->resid2 = s;
    double pn = 0.0;
    for (int c = 0; c < 9; c++) {
        sc->Pbar[c] = sc->dc[c] / V;
        pn += sc->Pbar[c] * sc->Pbar[c];
    }
    pn = sqrt(pn);
    const double eps = sqrt(s) / V / (pn > 0.0 ? pn : 1.0);
    sc->eps = eps;
    sc->n_operator64 += 1;
    if (!isfinite(eps)) {
        atomicCAS(&sc->status, 0, COMBO_E_NAN);
        sc->outer_done = 1;
        return;
    }
    if (fixed_point) {
        const int it = sc->outer_iter;
        if (fixed > 0 ? it >= fixed : eps <= tol) {
            sc->outer_done = 1;
        } else if (it >= max_iter) {
            atomicCAS(&sc->status, 0, COMBO_E_NOT_CONVERGED);
            sc->outer_done = 1;
        } else {
            sc->outer_iter = it + 1;
            sc->n_operator += 1;
            if (ncg) {  // Fletcher-Reeves beta; 0 at a load step's first iteration
                sc->beta = (it == 0) ? 0.0 : s / sc->ncg_gg;
                sc->ncg_gg = s;
            }
        }
    }
}

// CG start of problem b = block b (partials part[b n ..]); a problem whose
// outer_done is set takes no CG iterations in this round
__global__ void k_fin_rhs(Scalars* scs, const double* part_all, int n, int cg_fixed, int cg_max)
{
    __shared__ double red[256];
    Scalars* sc = scs + blockIdx.x;
    if (sc->outer_done) {
        if (threadIdx.x == 0) sc->cg_done = 1;
        return;
    }
    const double s = sum_partials(part_all + (size_t)blockIdx.x * n, n, red);
    if (threadIdx.x != 0) return;
    sc->rr = s;
    sc->rr0 = s;
    sc->cg_iter = 0;
    sc->beta = 0.0;
    sc->alpha_pending = 0.0;
    const bool stop = (cg_fixed <= 0) && (cg_max <= 0);
    sc->cg_done = (s == 0.0 || stop) ? 1 : 0;
}

// F += d * (x + alpha_pending p) -- the CG solution including the update the
// last CG iteration still owes -- then admissibility (det F > 0) of every voxel
// Stacked problems: dv[b] per problem of Vp voxels (0: F of that problem is
// left unchanged), the pending alpha and the admissibility flag per problem.
template <typename Tc>
__global__ void k_update_F(double* __restrict__ F, const Tc* __restrict__ x, const Tc* __restrict__ p,
                           const Tc* __restrict__ p_odd, double d0, int64_t V, Scalars* scs, const double* dv,
                           int64_t Vp)
{
    // p_odd (nodal form): the direction of odd CG iterations; the owed update
    // is that of the last iteration, cg_iter - 1
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = dv ? v / Vp : 0;
        const double d = dv ? dv[b] : d0;
        if (d == 0.0) continue;
        Scalars* sc = scs + b;
        const Tc ap = (Tc)sc->alpha_pending;
        double f[9];
        Tc xv[9];
        // all loads before the first store
#pragma unroll
        for (int c = 0; c < 9; c++) {
            f[c] = F[c * V + v];
            xv[c] = x[c * V + v];
        }
        if (ap != (Tc)0) {
            const Tc* pl = (p_odd && ((sc->cg_iter - 1) & 1)) ? p_odd : p;
#pragma unroll
            for (int c = 0; c < 9; c++) xv[c] += ap * pl[c * V + v];
        }
#pragma unroll
        for (int c = 0; c < 9; c++) {
            f[c] += d * (double)xv[c];
            F[c * V + v] = f[c];
        }
        const double J = f[0] * (f[4] * f[8] - f[5] * f[7]) - f[1] * (f[3] * f[8] - f[5] * f[6]) +
                         f[2] * (f[3] * f[7] - f[4] * f[6]);
        if (!(J > 0.0)) sc->admissible = 0;
    }
}

// P field of F (pure voxels Neo-Hookean, boxels from the laminate stresses)
// matp [nprob][4] per problem of Vp voxels, or null: mat
__global__ void k_eval_P(const double* F, const uint8_t* phase, const int32_t* vox2box, const double* bP, Mat9 mat,
                         double* P, int64_t V, Scalars* sc, const double* matp, int64_t Vp, int linear)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        const int ph = phase[v];
        if (ph == 2) {
            const int b = vox2box[v];
            for (int c = 0; c < 9; c++) P[c * V + v] = bP[(int64_t)b * 9 + c];
            continue;
        }
        double f[9];
        for (int c = 0; c < 9; c++) f[c] = F[c * V + v];
        const double* mp = matp ? matp + 4 * (v / Vp) : mat.v;
        const double mu = mp[ph], lam = mp[2 + ph];
        if (linear) {
            double S[9];
            lin_sigma(f, mu, lam, S);
            for (int c = 0; c < 9; c++) P[c * V + v] = S[c];
            continue;
        }
        const double c0 = f[4] * f[8] - f[5] * f[7], c1 = f[5] * f[6] - f[3] * f[8], c2 = f[3] * f[7] - f[4] * f[6];
        const double J = f[0] * c0 + f[1] * c1 + f[2] * c2;
        if (!(J > 0.0)) {
            atomicCAS(&sc->status, 0, COMBO_E_INADMISSIBLE);
            continue;
        }
        const double iJ = 1.0 / J;
        double G[9] = {c0 * iJ,
                       (f[2] * f[7] - f[1] * f[8]) * iJ,
                       (f[1] * f[5] - f[2] * f[4]) * iJ,
                       c1 * iJ,
                       (f[0] * f[8] - f[2] * f[6]) * iJ,
                       (f[2] * f[3] - f[0] * f[5]) * iJ,
                       c2 * iJ,
                       (f[1] * f[6] - f[0] * f[7]) * iJ,
                       (f[0] * f[4] - f[1] * f[3]) * iJ};
        const double k = lam * log(J) - mu;
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) P[(3 * i + j) * V + v] = mu * f[3 * i + j] + k * G[3 * j + i];
    }
}

// Phase-wise sums for the phase averages Pbar_- and Pbar_+ of one problem
// (voxels [v0, v1) of a field with stride V, boxels [b0, b1)): pure voxels add
// P(F) and 1 to their phase; a boxel adds c+ P+ and c+ to the inclusion and
// c- P- and c- to the matrix, P+- the laminate phase stresses at
// F+- = F +- a (x) N / c+- (Sec. 4.1).  Per block: 18 sums, 2 volumes.
constexpr int PHASE_SUMS = 20;
constexpr int PHASE_GRID = 152 * 4;

__global__ void __launch_bounds__(256) k_phase_sums(const double* F, int64_t V, const uint8_t* phase, int64_t v0,
                                                    int64_t v1, const int32_t* bidx, const double* bN,
                                                    const double* bc, const double* ba, int64_t b0, int64_t b1,
                                                    Mat9 mat, double* part, Scalars* sc, int linear)
{
    double s[PHASE_SUMS];
#pragma unroll
    for (int k = 0; k < PHASE_SUMS; k++) s[k] = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = v0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < v1; v += stride) {
        const int ph = phase[v];
        if (ph == 2) continue;
        double f[9], P[9];
        for (int c = 0; c < 9; c++) f[c] = F[c * V + v];
        if (linear) {
            lin_sigma(f, mat.v[ph], mat.v[2 + ph], P);
        } else if (!nh_P64(f, mat.v[ph], mat.v[2 + ph], P)) {
            atomicCAS(&sc->status, 0, COMBO_E_INADMISSIBLE);
            continue;
        }
        for (int c = 0; c < 9; c++) s[9 * ph + c] += P[c];
        s[18 + ph] += 1.0;
    }
    for (int64_t b = b0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < b1; b += stride) {
        const int64_t v = bidx[b];
        const double cp = bc[b], cm = 1.0 - cp;
        const double N[3] = {bN[3 * b], bN[3 * b + 1], bN[3 * b + 2]};
        const double a[3] = {ba[3 * b], ba[3 * b + 1], ba[3 * b + 2]};
        double fp[9], fm[9], Pp[9], Pm[9];
        for (int i = 0; i < 3; i++)
            for (int J = 0; J < 3; J++) {
                const double f = F[(3 * i + J) * V + v], aN = a[i] * N[J];
                fp[3 * i + J] = f + aN / cp;
                fm[3 * i + J] = f - aN / cm;
            }
        // (infinitesimal strain: sigma depends on sym(H) only, so a (x) N
        // stands for its symmetric part)
        if (linear) {
            lin_sigma(fp, mat.v[1], mat.v[3], Pp);
            lin_sigma(fm, mat.v[0], mat.v[2], Pm);
        } else if (!nh_P64(fp, mat.v[1], mat.v[3], Pp) || !nh_P64(fm, mat.v[0], mat.v[2], Pm)) {
            atomicCAS(&sc->status, 0, COMBO_E_INADMISSIBLE);
            continue;
        }
        for (int c = 0; c < 9; c++) {
            s[c] += cm * Pm[c];
            s[9 + c] += cp * Pp[c];
        }
        s[18] += cm;
        s[19] += cp;
    }
    // block sum (fixed order) -> part[blockIdx.x][PHASE_SUMS]
    __shared__ double red[8][PHASE_SUMS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < PHASE_SUMS; k++) {
        double x = s[k];
        for (int o = 16; o >= 1; o >>= 1) x += __shfl_down_sync(0xFFFFFFFFu, x, o);
        if (lane == 0) red[warp][k] = x;
    }
    __syncthreads();
    if (threadIdx.x < PHASE_SUMS) {
        double x = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) x += red[w][threadIdx.x];
        part[(int64_t)blockIdx.x * PHASE_SUMS + threadIdx.x] = x;
    }
}

// Phase-wise sums under the doubly-fine material grid: every sub-cell counts
// with volume 1/8 -- a pure sub-cell adds P(F_sub) to its phase, a boxel
// sub-cell adds c+ P+ and c- P- at F_sub +- a_l (x) N / c+- with its own jump
// a_l (Sec. 4.1, App. A).  One problem: voxels [v0, v1) of n1 x n2 x n3.
__global__ void __launch_bounds__(256) k_phase_sums_dfmg(const double* F, int64_t V, const uint8_t* phase,
                                                         int64_t v0, int64_t v1, int n1, int n2, int n3,
                                                         const int32_t* bidx, const double* bN, const double* bc,
                                                         const double* ba8, int64_t b0, int64_t b1, Mat9 mat,
                                                         double* part, Scalars* sc)
{
    double s[PHASE_SUMS];
#pragma unroll
    for (int k = 0; k < PHASE_SUMS; k++) s[k] = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = v0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < v1; v += stride) {
        const int ph = phase[v];
        if (ph == 2) continue;
        const int64_t lv = v - v0;
        const int i = (int)(lv % n1), j = (int)((lv / n1) % n2), k = (int)(lv / ((int64_t)n1 * n2));
        for (int l = 0; l < 8; l++) {
            double f[9], P[9];
            dfmg_fsub(F, V, v0, n1, n2, n3, i, j, k, l, f);
            if (!nh_P64(f, mat.v[ph], mat.v[2 + ph], P)) {
                atomicCAS(&sc->status, 0, COMBO_E_INADMISSIBLE);
                continue;
            }
            for (int c = 0; c < 9; c++) s[9 * ph + c] += 0.125 * P[c];
            s[18 + ph] += 0.125;
        }
    }
    for (int64_t t = 8 * b0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < 8 * b1; t += stride) {
        const int64_t b = t >> 3;
        const int l = (int)(t & 7);
        const int64_t v = bidx[b], lv = v - v0;
        const int i = (int)(lv % n1), j = (int)((lv / n1) % n2), k = (int)(lv / ((int64_t)n1 * n2));
        const double cp = bc[b], cm = 1.0 - cp;
        const double N[3] = {bN[3 * b], bN[3 * b + 1], bN[3 * b + 2]};
        const double* a = ba8 + 24 * b + 3 * l;
        double fs[9], fp[9], fm[9], Pp[9], Pm[9];
        dfmg_fsub(F, V, v0, n1, n2, n3, i, j, k, l, fs);
        for (int r = 0; r < 3; r++)
            for (int J = 0; J < 3; J++) {
                const double aN = a[r] * N[J];
                fp[3 * r + J] = fs[3 * r + J] + aN / cp;
                fm[3 * r + J] = fs[3 * r + J] - aN / cm;
            }
        if (!nh_P64(fp, mat.v[1], mat.v[3], Pp) || !nh_P64(fm, mat.v[0], mat.v[2], Pm)) {
            atomicCAS(&sc->status, 0, COMBO_E_INADMISSIBLE);
            continue;
        }
        for (int c = 0; c < 9; c++) {
            s[c] += 0.125 * cm * Pm[c];
            s[9 + c] += 0.125 * cp * Pp[c];
        }
        s[18] += 0.125 * cm;
        s[19] += 0.125 * cp;
    }
    __shared__ double red[8][PHASE_SUMS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < PHASE_SUMS; k++) {
        double x = s[k];
        for (int o = 16; o >= 1; o >>= 1) x += __shfl_down_sync(0xFFFFFFFFu, x, o);
        if (lane == 0) red[warp][k] = x;
    }
    __syncthreads();
    if (threadIdx.x < PHASE_SUMS) {
        double x = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) x += red[w][threadIdx.x];
        part[(int64_t)blockIdx.x * PHASE_SUMS + threadIdx.x] = x;
    }
}

static int grid_for(int64_t n, int block = 256)
{
    int64_t g = (n + block - 1) / block;
    return (int)std::min<int64_t>(std::max<int64_t>(g, 1), 152 * 16);
}

// ------------------------------------------------------------------ validated host copy of a problem
struct HostProblem {
    int32_t n[3];
    double l[3];
    std::vector<uint8_t> phase;
    std::vector<int32_t> bidx;
    std::vector<double> bN, bc;
    double mu[2], lam[2], Fbar[9];
    int32_t n_steps;
};

static double det9(const double* F)
{
    return F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) + F[2] * (F[3] * F[7] - F[4] * F[6]);
}

static int validate_dims(const int32_t n[3])
{
    for (int j = 0; j < 3; j++)
        if (n[j] < 2 || n[j] > 1024 || !is_23(n[j])) return fail(COMBO_E_INVALID_ARG, "grid sides must be 2^a 3^b in [2, 1024]");
    if (n[0] % 2) return fail(COMBO_E_INVALID_ARG, "n1 must be even");
    if ((int64_t)n[0] * n[1] * n[2] >= (int64_t)1 << 31) return fail(COMBO_E_INVALID_ARG, "grid too large");
    return COMBO_OK;
}

static int load_problem(const combo_problem* p, const combo_options* o, HostProblem& h)
{
    if (!p || !o) return fail(COMBO_E_INVALID_ARG, "null problem or options");
    int rc = validate_dims(p->n);
    if (rc) return rc;
    for (int j = 0; j < 3; j++) {
        h.n[j] = p->n[j];
        h.l[j] = p->l[j];
        if (!(p->l[j] > 0.0)) return fail(COMBO_E_INVALID_ARG, "RVE lengths must be positive");
    }
    for (int i = 0; i < 2; i++) {
        h.mu[i] = p->mu[i];
        h.lam[i] = p->lambda[i];
        if (!(p->mu[i] > 0.0) || !(p->lambda[i] > -2.0 * p->mu[i] / 3.0))
            return fail(COMBO_E_INVALID_ARG, "need mu > 0 and lambda > -2 mu / 3");
    }
    std::memcpy(h.Fbar, p->Fbar, sizeof(h.Fbar));
    if (!(det9(h.Fbar) > 0.0)) return fail(COMBO_E_INVALID_ARG, "det Fbar must be positive");
    if (p->n_steps < 1) return fail(COMBO_E_INVALID_ARG, "n_steps must be >= 1");
    h.n_steps = p->n_steps;
    const int64_t V = (int64_t)p->n[0] * p->n[1] * p->n[2];
    const int64_t nb = p->n_boxels;
    if (nb < 0 || nb > V) return fail(COMBO_E_INVALID_ARG, "bad n_boxels");
    if (!p->phase || (nb > 0 && (!p->boxel_idx || !p->boxel_N || !p->boxel_c)))
        return fail(COMBO_E_INVALID_ARG, "null problem array");
    h.phase.resize(V);
    std::vector<int64_t> idx(nb);
    std::vector<double> N(3 * nb), c(nb);
    const cudaMemcpyKind kind = (p->mem == COMBO_MEM_DEVICE) ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
    CK(cudaMemcpy(h.phase.data(), p->phase, V, kind));
    if (nb > 0) {
        CK(cudaMemcpy(idx.data(), p->boxel_idx, 8 * nb, kind));
        CK(cudaMemcpy(N.data(), p->boxel_N, 24 * nb, kind));
        CK(cudaMemcpy(c.data(), p->boxel_c, 8 * nb, kind));
    }
    int64_t cnt2 = 0;
    for (int64_t v = 0; v < V; v++) {
        const uint8_t ph = h.phase[v];
        if (ph > 2) return fail(COMBO_E_INVALID_ARG, "phase codes must be 0, 1 or 2");
        cnt2 += (ph == 2);
    }
    if (cnt2 != nb) return fail(COMBO_E_INVALID_ARG, "n_boxels differs from the number of phase-2 voxels");
    h.bidx.reserve(nb);
    h.bN.reserve(3 * nb);
    h.bc.reserve(nb);
    for (int64_t b = 0; b < nb; b++) {
        if (idx[b] < 0 || idx[b] >= V || (b > 0 && idx[b] <= idx[b - 1]))
            return fail(COMBO_E_INVALID_ARG, "boxel_idx must be strictly increasing voxel indices");
        if (h.phase[idx[b]] != 2) return fail(COMBO_E_INVALID_ARG, "boxel_idx points at a non-boxel voxel");
        const double nn = std::sqrt(N[3 * b] * N[3 * b] + N[3 * b + 1] * N[3 * b + 1] + N[3 * b + 2] * N[3 * b + 2]);
        if (!(nn >= 1e-12)) return fail(COMBO_E_INVALID_ARG, "boxel normal of zero length");
        const double cb = c[b];
        if (!(cb > 0.0 && cb < 1.0)) return fail(COMBO_E_INVALID_ARG, "boxel volume fraction outside (0, 1)");
        if (cb < o->c_min) {
            h.phase[idx[b]] = 0;  // evaluated as the pure matrix
            continue;
        }
        if (cb > 1.0 - o->c_min) {
            h.phase[idx[b]] = 1;  // evaluated as the pure inclusion
            continue;
        }
        h.bidx.push_back((int32_t)idx[b]);
        for (int i = 0; i < 3; i++) h.bN.push_back(N[3 * b + i] / nn);
        h.bc.push_back(cb);
    }
    return COMBO_OK;
}

static int check_options(combo_options& o)
{
    if (o.precision != COMBO_FP64 && o.precision != COMBO_FP32_REFINED && o.precision != COMBO_FP32_REFINED_DF)
        return fail(COMBO_E_INVALID_ARG, "bad precision");
    if (o.kspace != COMBO_ROTATED && o.kspace != COMBO_SPECTRAL && o.kspace != COMBO_STAGGERED &&
        o.kspace != COMBO_STAGGERED_DFMG)
        return fail(COMBO_E_INVALID_ARG, "bad kspace");
    if (o.solver != COMBO_FIXED_POINT && o.solver != COMBO_NEWTON_CG && o.solver != COMBO_NONLINEAR_CG)
        return fail(COMBO_E_INVALID_ARG, "bad solver");
    if (o.solver != COMBO_NEWTON_CG && o.precision == COMBO_FP32_REFINED)
        return fail(COMBO_E_INVALID_ARG,
                    "the fixed point and nonlinear CG run in FP64 or the double-float residual form");
    if (o.theory != COMBO_FINITE_STRAIN && o.theory != COMBO_INFINITESIMAL_STRAIN)
        return fail(COMBO_E_INVALID_ARG, "bad theory");
    if (o.kspace == COMBO_STAGGERED_DFMG && o.theory == COMBO_INFINITESIMAL_STRAIN)
        return fail(COMBO_E_INVALID_ARG, "the doubly-fine material grid is built for finite strain only");
    if (o.max_iter <= 0) o.max_iter = (o.solver == COMBO_NEWTON_CG) ? 200 : 100000;
    if (!(o.tol >= 0.0) || !(o.cg_tol >= 0.0)) return fail(COMBO_E_INVALID_ARG, "negative tolerance");
    if (o.nr_max_iter <= 0) o.nr_max_iter = 50;
    if (!(o.c_min >= 0.0 && o.c_min < 0.5)) return fail(COMBO_E_INVALID_ARG, "c_min outside [0, 0.5)");
    if (o.wait_poll_cap < -1) return fail(COMBO_E_INVALID_ARG, "wait_poll_cap below -1");
    return COMBO_OK;
}

// ------------------------------------------------------------------ autotuner store
struct TuneKey {
    int word, n1, n2, n3p, nprob;
    int nodal;  // pass 0 is the nodal form's tangent pass
    bool operator<(const TuneKey& o) const
    {
        return std::tie(word, n1, n2, n3p, nprob, nodal) < std::tie(o.word, o.n1, o.n2, o.n3p, o.nprob, o.nodal);
    }
};
struct TuneRec {
    int cfg[4] = {0, 0, 0, 0};  // x-forward, y, z, x-inverse
    float ms[4][2] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};  // 3 launches of each candidate
};
static std::mutex g_tune_mu;
static std::map<TuneKey, TuneRec> g_tune;
static std::atomic<int> g_tune_enabled{1};
// most reduced form of the rotated Krylov operator a solve set up from now on
// may use (COMBO_KRYLOV_NINE / _DISPLACEMENT / _NODAL), where it applies
static std::atomic<int> g_krylov_form{COMBO_KRYLOV_NODAL};
static std::atomic<int> g_tune_force[4] = {{-1}, {-1}, {-1}, {-1}};  // per pass: forced candidate or -1

static void tune_store(const TuneKey& k, const TuneRec& r)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[k] = r;
}

// the decisions for this grid into an engine; false if none yet
template <typename T> static bool tune_lookup(const TuneKey& k, Engine<T>& e)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(k);
    if (it == g_tune.end()) return false;
    e.cfg_xf = it->second.cfg[0];
    e.cfg_y = e.ymap_ok[it->second.cfg[1]] ? it->second.cfg[1] : 0;
    e.cfg_z = e.zmap_ok[it->second.cfg[2]] ? it->second.cfg[2] : 0;
    e.cfg_xi = it->second.cfg[3];
    return true;
}

// forced candidates (tests of every launch shape) override the decisions
template <typename T> static void tune_force(Engine<T>& e)
{
    int f;
    if ((f = g_tune_force[0].load()) >= 0) e.cfg_xf = f;
    if ((f = g_tune_force[1].load()) >= 0) e.cfg_y = e.ymap_ok[f] ? f : 0;
    if ((f = g_tune_force[2].load()) >= 0) e.cfg_z = e.zmap_ok[f] ? f : 0;
    if ((f = g_tune_force[3].load()) >= 0) e.cfg_xi = f;
}

// ------------------------------------------------------------------ solve state
struct SolveBase {
    virtual ~SolveBase() {}
    virtual int advance(int64_t max_ops) = 0;
    virtual int finish(combo_result* r) = 0;
    virtual int run_batch() = 0;
    virtual int batch_results(combo_result* rs) = 0;
    virtual Profiler& profiler() = 0;
    virtual void request_cancel() = 0;
    virtual int advance_steps(int32_t k) = 0;
    virtual int advance_newton(int64_t min_ops) = 0;
    virtual int export_state(void* buf, int64_t* bytes) = 0;
    virtual int import_state(const void* buf, int64_t bytes) = 0;
};

struct combo_solve_state {
    SolveBase* impl;
};

// Tc: Krylov precision (float or double); Rt: arithmetic of the residual
// transforms (double, or df32 double-float for the refined form)
template <typename Tc, typename Rt = double> struct Solve : SolveBase {
    combo_ctx* ctx;
    combo_options opt;
    HostProblem hp;
    GridDims g;
    int64_t nb = 0;
    cudaStream_t st;
    Engine<Rt> e64;  // residual operator G[P(F)] (P in FP64)
    Engine<Tc> ec;   // Krylov operator
    // device memory
    uint8_t* d_phase = nullptr;
    int32_t* d_v2b = nullptr;
    int32_t* d_bidx = nullptr;
    int32_t *d_rank = nullptr, *d_bvox = nullptr, *d_lofs = nullptr;  // boxels in voxel order
    double *d_bN = nullptr, *d_bc = nullptr, *d_ba = nullptr, *d_bP = nullptr;
    Tc* d_bA = nullptr;
    double* d_F = nullptr;
    void* d_spec = nullptr;
    Tc *d_tc = nullptr, *d_x = nullptr, *d_r = nullptr, *d_p = nullptr;
    Tc* d_p2 = nullptr;  // nodal form: p of odd CG iterations
    int32_t* d_vrank = nullptr;  // nodal form: packed-tangent column of boxel voxels, else -1 - phase
    double* d_part = nullptr;
    Scalars* d_sc = nullptr;  // [B]
    double* d_phpart = nullptr;  // [PHASE_GRID][PHASE_SUMS] phase-average partials
    double* d_dir = nullptr;     // nonlinear CG direction [9][V]
    double mu0 = 0.0;
    // stacked problems (a batch of B equal grids along z; B = 1 for one solve)
    int B = 1;
    int64_t Vp = 0;                    // voxels of one problem
    std::vector<HostProblem> hps;      // the problems of a batch (empty for one solve)
    std::vector<int64_t> boff;         // boxels of problem b: [boff[b], boff[b + 1])
    double* d_S = nullptr;             // doubly-fine material grid: [72][V] sub-cell stresses
    double* d_Pd = nullptr;            //   [9][V] gathered stress
    double* d_ba8 = nullptr;           //   [nb][8][3] sub-cell jump vectors
    Tc* d_bA8 = nullptr;               //   Newton-CG: [45][8 nb] packed sub-cell boxel tangents
    Tc* d_St = nullptr;                //   Newton-CG: [72][V] sub-cell values of A : p
    Tc* d_yd = nullptr;                //   Newton-CG: [9][V] gathered A : p
    double* d_mat = nullptr;           // [B][4] materials (batch only)
    double* d_dF = nullptr;            // [B][9] load-step increments (batch only)
    double* d_dv = nullptr;            // [B] F-update factors (batch only)
    int32_t* d_bprob = nullptr;        // problem of each boxel (batch only)
    Profiler prof;
    static constexpr int kCgChunk = 8;
    cudaGraphExec_t cg_exec = nullptr;
    int64_t cg_chunks_run = 0;
    volatile int cancel_requested = 0;  // set by the server; checked between chunks
    // host state machine
    enum { ST_STEP, ST_RESID, ST_CG, ST_UPDATE, ST_FP, ST_DONE } state = ST_STEP;
    int step = 0;  // completed load steps
    int outer = 0;
    int cg_step_total = 0;
    double Fprev[9];
    std::vector<double> Pbar, resid;
    std::vector<double> Pphase;  // [n_steps][2][9] phase averages Pbar_-, Pbar_+
    std::vector<int32_t> iters, cg_iters;
    int64_t ops_done = 0;
    int64_t step_target = -1;  // advance_steps: stop between load steps once step reaches it
    // member of a batch over several grids (MixSolve): batch-form per-problem
    // arrays even for one problem, scalars in the batch's shared array, no
    // launch-shape tuning (the batch runs grouped launches)
    bool member = false;
    bool own_launches = false;  // a member that runs its own (tuned, specialised) launch sequences
    Scalars* ext_sc = nullptr;
    bool whole_newton = false;  // advance_newton: a reached limit stops only between Newton steps
    int error = 0;

    ~Solve() override
    {
        cudaFree(d_phase);
        cudaFree(d_v2b);
        cudaFree(d_bidx);
        cudaFree(d_rank);
        cudaFree(d_bvox);
        cudaFree(d_lofs);
        cudaFree(d_bN);
        cudaFree(d_bc);
        cudaFree(d_ba);
        cudaFree(d_bP);
        cudaFree(d_bA);
        cudaFree(d_F);
        cudaFree(d_spec);
        cudaFree(d_tc);
        cudaFree(d_x);
        cudaFree(d_r);
        cudaFree(d_p);
        cudaFree(d_p2);
        cudaFree(d_vrank);
        cudaFree(d_part);
        if (!ext_sc) cudaFree(d_sc);
        cudaFree(d_phpart);
        cudaFree(d_dir);
        cudaFree(d_S);
        cudaFree(d_Pd);
        cudaFree(d_ba8);
        cudaFree(d_bA8);
        cudaFree(d_St);
        cudaFree(d_yd);
        cudaFree(d_mat);
        cudaFree(d_dF);
        cudaFree(d_dv);
        cudaFree(d_bprob);
        if (cg_exec) cudaGraphExecDestroy(cg_exec);
        e64.release();
        ec.release();
    }

    bool newton() const { return opt.solver == COMBO_NEWTON_CG; }
    bool dfmg() const { return opt.kspace == COMBO_STAGGERED_DFMG; }
    bool linear() const { return opt.theory == COMBO_INFINITESIMAL_STRAIN; }

    int init(combo_ctx* c, HostProblem&& h, const combo_options& o)
    {
        std::vector<HostProblem> one;
        one.push_back(std::move(h));
        return init(c, std::move(one), o);
    }

    // B >= 1 problems of equal grid n and cell size l: stacked along z; the
    // phase fields, boxel lists and materials are concatenated per problem
    int init(combo_ctx* c, std::vector<HostProblem>&& hs, const combo_options& o)
    {
        ctx = c;
        st = c->stream;
        prof.st = st;
        opt = o;
        B = (int)hs.size();
        if (B == 1 && !member) {
            hp = std::move(hs[0]);
        } else {
            hps = std::move(hs);
            hp.n[0] = hps[0].n[0], hp.n[1] = hps[0].n[1], hp.n[2] = hps[0].n[2];
            for (int j = 0; j < 3; j++) hp.l[j] = hps[0].l[j];
            for (int i = 0; i < 2; i++) hp.mu[i] = hps[0].mu[i], hp.lam[i] = hps[0].lam[i];
            std::memcpy(hp.Fbar, hps[0].Fbar, sizeof hp.Fbar);
            hp.n_steps = hps[0].n_steps;
            Vp = (int64_t)hp.n[0] * hp.n[1] * hp.n[2];
            hp.phase.resize((size_t)B * Vp);
            boff.assign(B + 1, 0);
            for (int b = 0; b < B; b++) {
                std::memcpy(hp.phase.data() + (size_t)b * Vp, hps[b].phase.data(), Vp);
                boff[b + 1] = boff[b] + (int64_t)hps[b].bidx.size();
                for (size_t k = 0; k < hps[b].bidx.size(); k++) hp.bidx.push_back((int32_t)(b * Vp + hps[b].bidx[k]));
                hp.bN.insert(hp.bN.end(), hps[b].bN.begin(), hps[b].bN.end());
                hp.bc.insert(hp.bc.end(), hps[b].bc.begin(), hps[b].bc.end());
                std::vector<uint8_t>().swap(hps[b].phase);  // uploaded with the batch
            }
        }
        g = make_dims(hp.n, B);
        if (B == 1) Vp = g.V;
        nb = (int64_t)hp.bidx.size();
        const int64_t V = g.V;
        int rc;
        // the doubly-fine material grid changes the law, not the operator
        const int kop = dfmg() ? COMBO_STAGGERED : opt.kspace;
        if ((rc = e64.init(g, hp.l, kop))) return rc;
        if ((rc = ec.init(g, hp.l, kop))) return rc;
        e64.wait_cap = ec.wait_cap = (opt.wait_poll_cap < 0) ? kWaitNone : (uint32_t)opt.wait_poll_cap;
        CK(dev_malloc(&d_phase, V));
        CK(dev_malloc(&d_v2b, 4 * V));
        CK(dev_malloc(&d_F, 8 * 9 * V));
        CK(dev_malloc(&d_spec, sizeof(double2) * 9 * g.Vs));
        CK(cudaMemsetAsync(d_spec, 0, sizeof(double2) * 9 * g.Vs, st));
        int nbuf = std::max(std::max(e64.xpartials(), e64.zblocks()), std::max(ec.xpartials(), ec.zblocks()));
        if (dfmg()) nbuf = std::max(nbuf, dfmg_cg_blocks(V));
        nbuf = std::max(nbuf, disp_grad_partials_max() + g.nprob);  // the displacement form's gradient pass
        nbuf = std::max(nbuf, nodal_partials_max() + g.nprob);      // the nodal form's tangent pass
        CK(dev_malloc(&d_part, 8 * (size_t)nbuf));
        if (ext_sc)
            d_sc = ext_sc;
        else
            CK(dev_malloc(&d_sc, sizeof(Scalars) * B));
        CK(dev_malloc(&d_phpart, sizeof(double) * PHASE_GRID * PHASE_SUMS));
        if (opt.solver == COMBO_NONLINEAR_CG) {
            CK(dev_malloc(&d_dir, sizeof(double) * 9 * (size_t)g.V));
            CK(cudaMemsetAsync(d_dir, 0, sizeof(double) * 9 * (size_t)g.V, st));
        }
        if (dfmg() && newton()) {
            CK(dev_malloc(&d_bA8, sizeof(Tc) * 45 * 8 * (size_t)std::max<int64_t>(nb, 1)));
            CK(dev_malloc(&d_St, sizeof(Tc) * 72 * (size_t)g.V));
            CK(dev_malloc(&d_yd, sizeof(Tc) * 9 * (size_t)g.V));
        }
        if (dfmg()) {
            CK(dev_malloc(&d_S, sizeof(double) * 72 * (size_t)g.V));
            CK(dev_malloc(&d_Pd, sizeof(double) * 9 * (size_t)g.V));
            CK(dev_malloc(&d_ba8, sizeof(double) * 24 * (size_t)std::max<int64_t>(nb, 1)));
            CK(cudaMemsetAsync(d_ba8, 0, sizeof(double) * 24 * (size_t)std::max<int64_t>(nb, 1), st));
        }
        CK(cudaMemsetAsync(d_sc, 0, sizeof(Scalars) * B, st));
        if (B > 1 || member) {
            std::vector<double> mat(4 * B);
            std::vector<int32_t> bprob(std::max<int64_t>(nb, 1), 0);
            for (int b = 0; b < B; b++) {
                mat[4 * b + 0] = hps[b].mu[0];
                mat[4 * b + 1] = hps[b].mu[1];
                mat[4 * b + 2] = hps[b].lam[0];
                mat[4 * b + 3] = hps[b].lam[1];
                for (int64_t k = boff[b]; k < boff[b + 1]; k++) bprob[k] = b;
            }
            CK(dev_malloc(&d_mat, 8 * mat.size()));
            CK(dev_malloc(&d_dF, 8 * 9 * (size_t)B));
            CK(dev_malloc(&d_dv, 8 * (size_t)B));
            CK(dev_malloc(&d_bprob, 4 * bprob.size()));
            CK(cudaMemcpy(d_mat, mat.data(), 8 * mat.size(), cudaMemcpyHostToDevice));
            CK(cudaMemcpy(d_bprob, bprob.data(), 4 * bprob.size(), cudaMemcpyHostToDevice));
        }
        const size_t nbs = std::max<int64_t>(nb, 1);
        CK(dev_malloc(&d_bidx, 4 * nbs));
        CK(dev_malloc(&d_bN, 24 * nbs));
        CK(dev_malloc(&d_bc, 8 * nbs));
        CK(dev_malloc(&d_ba, 24 * nbs));
        CK(dev_malloc(&d_bP, 72 * nbs));
        if (newton()) {
            CK(dev_malloc(&d_bA, sizeof(Tc) * 45 * nbs));
            CK(dev_malloc(&d_rank, 4 * nbs));
            CK(dev_malloc(&d_bvox, 4 * nbs));
            CK(dev_malloc(&d_lofs, 4 * ((size_t)g.n2 * g.n3 + 1)));
            CK(dev_malloc(&d_tc, sizeof(Tc) * 10 * V));
            CK(dev_malloc(&d_x, sizeof(Tc) * 9 * V));
            CK(dev_malloc(&d_r, sizeof(Tc) * 9 * V));
            CK(dev_malloc(&d_p, sizeof(Tc) * 9 * V));
        }
        e64.bind_spec(d_spec);
        ec.bind_spec(d_spec);
        // the nodal form's second direction buffer, where that form may apply
        if (newton() && !dfmg() && (!member || own_launches) && g_krylov_form.load() >= COMBO_KRYLOV_NODAL &&
            ec.zsmap_ok[0] && nodal_ok(g))
        {
            CK(dev_malloc(&d_p2, sizeof(Tc) * 9 * V));
            CK(dev_malloc(&d_vrank, 4 * V));
        }
        CK(cudaMemcpyAsync(d_phase, hp.phase.data(), V, cudaMemcpyHostToDevice, st));
        CK(cudaMemsetAsync(d_v2b, 0xff, 4 * V, st));
        if (nb > 0) {
            CK(cudaMemcpyAsync(d_bidx, hp.bidx.data(), 4 * nb, cudaMemcpyHostToDevice, st));
            CK(cudaMemcpyAsync(d_bN, hp.bN.data(), 24 * nb, cudaMemcpyHostToDevice, st));
            CK(cudaMemcpyAsync(d_bc, hp.bc.data(), 8 * nb, cudaMemcpyHostToDevice, st));
            CK(cudaMemsetAsync(d_ba, 0, 24 * nb, st));
            k_vox2box<<<(int)((nb + 255) / 256), 256, 0, st>>>(d_v2b, d_bidx, nb);
        }
        if (newton()) {
            // the tangent x-pass visits each x-line's boxels in voxel order
            const int64_t nlines = (int64_t)g.n2 * g.n3;
            std::vector<int32_t> order(nb), rank(std::max<int64_t>(nb, 1)), bvox(std::max<int64_t>(nb, 1)), lofs(nlines + 1);
            for (int64_t b = 0; b < nb; b++) order[b] = (int32_t)b;
            std::stable_sort(order.begin(), order.end(), [&](int32_t u, int32_t w) { return hp.bidx[u] < hp.bidx[w]; });
            for (int64_t k = 0; k < nb; k++) {
                rank[order[k]] = (int32_t)k;
                bvox[k] = hp.bidx[order[k]];
            }
            int64_t k = 0;
            for (int64_t L = 0; L <= nlines; L++) {
                while (k < nb && bvox[k] < L * g.n1) k++;
                lofs[L] = (int32_t)k;
            }
            CK(cudaMemcpyAsync(d_rank, rank.data(), 4 * rank.size(), cudaMemcpyHostToDevice, st));
            CK(cudaMemcpyAsync(d_bvox, bvox.data(), 4 * bvox.size(), cudaMemcpyHostToDevice, st));
            CK(cudaMemcpyAsync(d_lofs, lofs.data(), 4 * lofs.size(), cudaMemcpyHostToDevice, st));
            if (d_vrank) k_vrank<<<grid_for(V), 256, 0, st>>>(d_vrank, d_phase, d_v2b, d_rank, V);
            CK(cudaStreamSynchronize(st));  // the host vectors go out of scope
        }
        k_fill_identity<<<grid_for(9 * V), 256, 0, st>>>(d_F, V);
        CK(cudaGetLastError());
        mu0 = opt.mu0;
        if (!(mu0 > 0.0))
            mu0 = 0.5 * (std::min(hp.mu[0], hp.mu[1]) + std::max(hp.lam[0] + 2 * hp.mu[0], hp.lam[1] + 2 * hp.mu[1]));
        for (int c = 0; c < 9; c++) Fprev[c] = (c == 0 || c == 4 || c == 8) ? 1.0 : 0.0;
        Pbar.assign(9 * (size_t)hp.n_steps, 0.0);
        Pphase.assign(18 * (size_t)hp.n_steps, 0.0);
        resid.assign(hp.n_steps, 0.0);
        iters.assign(hp.n_steps, 0);
        cg_iters.assign(hp.n_steps, 0);
        CK(cudaStreamSynchronize(st));
        if (newton() && (!member || own_launches)) {
            if ((rc = autotune())) return rc;
            tune_force(ec);
            const int form = g_krylov_form.load();
            ec.use_disp = (form >= COMBO_KRYLOV_DISPLACEMENT && ec.disp_capable()) ? 1 : 0;
            ec.use_nodal = (form >= COMBO_KRYLOV_NODAL && ec.use_disp && d_p2 && ec.nodal_capable()) ? 1 : 0;
        }
        return COMBO_OK;
    }

    // ---- launch-shape autotuner: the first solve of a grid (sides, batch
    // size, Krylov precision) times every candidate shape of each Krylov pass
    // on its own, still empty, buffers (3 launches each after one warm-up, no
    // solver scalars touched) and keeps the fastest for every later solve
    // of that grid in the process.
    int autotune()
    {
        if constexpr (sizeof(Tc) != 4) {
            return COMBO_OK;  // the candidates are shapes of the FP32 passes
        } else {
            const int nodal_pass = d_p2 ? 1 : 0;  // the nodal form may run: tune its tangent pass
            const TuneKey key{sizeof(Tc), g.n1, g.n2, g.n3p, g.nprob, nodal_pass};
            if (tune_lookup(key, ec)) return COMBO_OK;
            if (!g_tune_enabled.load()) return COMBO_OK;
            CK(cudaMemsetAsync(d_r, 0, sizeof(Tc) * 9 * g.V, st));
            CK(cudaMemsetAsync(d_p, 0, sizeof(Tc) * 9 * g.V, st));
            CK(cudaMemsetAsync(d_x, 0, sizeof(Tc) * 9 * g.V, st));
            CK(cudaMemsetAsync(d_tc, 0, sizeof(Tc) * 10 * g.V, st));
            cudaEvent_t e0, e1;
            CK(cudaEventCreate(&e0));
            CK(cudaEventCreate(&e1));
            // best of 3 timings of 3 launches (after a warm-up launch); the
            // candidates of a pass are timed alternately so that clock and
            // cache drift affect both alike
            auto time_once = [&](auto&& launch) -> float {
                cudaEventRecord(e0, st);
                for (int k = 0; k < 3; k++) launch();
                cudaEventRecord(e1, st);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                return (cudaGetLastError() == cudaSuccess) ? ms : 1e30f;
            };
            auto time_pair = [&](auto&& l0, auto&& l1, bool has1, float* out) {
                l0();
                if (has1) l1();
                out[0] = out[1] = 1e30f;
                for (int rep = 0; rep < 3; rep++) {
                    out[0] = std::min(out[0], time_once(l0));
                    if (has1) out[1] = std::min(out[1], time_once(l1));
                }
            };
            TuneRec rec;
            // tangent x-forward
            auto xf = ec.template xf<Tc>();
            xf.mode = XF_TANGENT;
            xf.phase = d_phase;
            xf.vox2box = d_v2b;
            for (int i = 0; i < 2; i++) xf.mu[i] = hp.mu[i], xf.lam[i] = hp.lam[i];
            xf.tc = d_tc;
            xf.r = d_r;
            xf.p = d_p;
            xf.x = d_x;
            xf.matp = d_mat;
            xf.bA = d_bA;
            xf.bvox = d_bvox;
            xf.lofs = d_lofs;
            xf.nb = std::max<int64_t>(nb, 1);
            xf.partial = d_part;
            xf.sc = d_sc;
            xf.fuse = 0;
            auto xf1 = xf;
            xf.cfg = 0;
            xf1.cfg = 1;
            if (nodal_pass) {
                // timed as a later iteration (cg_iter 1, a nonzero owed alpha):
                // the previous direction is read and x updated, as in every
                // iteration but the first; all of them zero, and no alpha is
                // formed (fuse 0); the scalars are cleared afterwards
                CK(cudaMemsetAsync(d_p2, 0, sizeof(Tc) * 9 * g.V, st));
                std::vector<Scalars> hs(B);
                for (auto& q : hs) {
                    std::memset(&q, 0, sizeof(Scalars));
                    q.cg_iter = 1;
                    q.alpha_pending = 1e-30;
                }
                CK(cudaMemcpyAsync(d_sc, hs.data(), sizeof(Scalars) * B, cudaMemcpyHostToDevice, st));
                CK(cudaStreamSynchronize(st));
                NodalArgs n0 = nodal_args();
                n0.fuse = 0;
                NodalArgs n1 = n0;
                n0.cfg = 0;
                n1.cfg = 1;
                time_pair([&] { launch_xfwd_nodal(n0, st); }, [&] { launch_xfwd_nodal(n1, st); }, true, rec.ms[0]);
            } else {
                time_pair([&] { launch_xfwd<Tc, Tc>(xf, 0, st); }, [&] { launch_xfwd<Tc, Tc>(xf1, 0, st); }, true,
                          rec.ms[0]);
            }
            // y forward and z (+ projection): tile widths with a valid tensor map
            YArgs<Tc> y0{};
            y0.g = g;
            y0.plan = ec.py;
            y0.tw = ec.tab.twy;
            y0.spec = ec.spec;
            y0.tx = ec.txy;
            y0.sc = d_sc;
            YArgs<Tc> y1 = y0;
            y0.cfg = 0;
            y0.tmap = ec.ymap_ok[0] ? &ec.ymap[0] : nullptr;
            y1.cfg = 1;
            y1.tmap = ec.ymap_ok[1] ? &ec.ymap[1] : nullptr;
            time_pair([&] { launch_ypass<Tc, false>(y0, st); }, [&] { launch_ypass<Tc, false>(y1, st); },
                      y1.tmap != nullptr, rec.ms[1]);
            ZArgs<Tc> z0{};
            z0.g = g;
            z0.plan = ec.pz;
            z0.tw = ec.tab.twz;
            z0.spec = ec.spec;
            z0.tx = ec.txz;
            for (int j = 0; j < 3; j++) z0.sa[j] = ec.tab.sa[j], z0.sb[j] = ec.tab.sb[j], z0.ph[j] = ec.tab.ph[j];
            z0.scale = (Tc)(2.0 * g.nprob / (double)g.V);
            z0.sc = d_sc;
            ZArgs<Tc> z1 = z0;
            z0.cfg = 0;
            z0.tmap = ec.zmap_ok[0] ? &ec.zmap[0] : nullptr;
            z1.cfg = 1;
            z1.tmap = ec.zmap_ok[1] ? &ec.zmap[1] : nullptr;
            if (nodal_pass) {
                // the nodal form's scalar z-pass: its two tile widths
                ZArgs<Tc> s0 = z0, s1 = z1;
                s0.disp = s1.disp = 2;
                s0.tmap_u = ec.zsmap_ok[0] ? &ec.zsmap[0] : nullptr;
                s1.tmap_u = ec.zsmap_ok[1] ? &ec.zsmap[1] : nullptr;
                if (s0.tmap_u)
                    time_pair([&] { launch_zpass_scalar(s0, st); }, [&] { launch_zpass_scalar(s1, st); },
                              s1.tmap_u != nullptr, rec.ms[2]);
            } else {
                time_pair([&] { launch_zpass<Tc>(z0, st); }, [&] { launch_zpass<Tc>(z1, st); }, z1.tmap != nullptr,
                          rec.ms[2]);
            }
            // CG x-inverse
            auto xi = ec.template xi<Tc>();
            xi.mode = XI_CG;
            xi.x = d_x;
            xi.r = d_r;
            xi.p = d_p;
            xi.partial = d_part;
            xi.sc = d_sc;
            xi.fuse = 0;
            auto xi1 = xi;
            xi.cfg = 0;
            xi1.cfg = 1;
            // (guard 1 selects the streamed kernel; cg_done is 0 here)
            time_pair([&] { launch_xinv<Tc, Tc>(xi, 1, st); }, [&] { launch_xinv<Tc, Tc>(xi1, 1, st); }, true,
                      rec.ms[3]);
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            CK(cudaMemsetAsync(d_sc, 0, sizeof(Scalars) * B, st));
            CK(cudaStreamSynchronize(st));
            CK(cudaGetLastError());
            for (int k = 0; k < 4; k++) rec.cfg[k] = rec.ms[k][1] < 0.98f * rec.ms[k][0] ? 1 : 0;  // 2 % margin
            tune_store(key, rec);
            tune_lookup(key, ec);
            return COMBO_OK;
        }
    }

    // --- kernel arguments and sequences
    BoxelArgs<Tc> boxel_args(bool tangent, int guard) const
    {
        BoxelArgs<Tc> a{};
        a.nb = nb;
        a.V = g.V;
        a.bidx = d_bidx;
        a.bN = d_bN;
        a.bc = d_bc;
        a.ba = d_ba;
        a.bP = d_bP;
        a.bA = tangent ? d_bA : nullptr;
        a.rank = d_rank;
        a.bprob = d_bprob;
        a.matp = d_mat;
        a.dfloat = std::is_same<Rt, df32>::value ? 1 : 0;
        a.linear = linear() ? 1 : 0;
        a.F = d_F;
        a.mu[0] = hp.mu[0];
        a.mu[1] = hp.mu[1];
        a.lam[0] = hp.lam[0];
        a.lam[1] = hp.lam[1];
        a.tol_rel = opt.nr_tol_rel;
        a.tol_abs = opt.nr_tol_abs;
        a.max_iter = opt.nr_max_iter;
        a.sc = d_sc;
        a.guard = guard;
        return a;
    }
    void boxels(bool tangent, int guard)
    {
        if (nb == 0) return;
        const BoxelArgs<Tc> a = boxel_args(tangent, guard);
        prof.begin(K_BOXEL);
        launch_boxel<Tc>(a, st);
        prof.end();
    }

    // doubly-fine material grid law (App. A): sub-cell stresses of the pure
    // cells and of the composite boxels into d_S, gathered into d_Pd
    void dfmg_law(int guard, bool tangent = false)
    {
        DfmgArgs d{};
        d.F = d_F;
        d.S = d_S;
        d.P = d_Pd;
        d.phase = d_phase;
        d.matp = d_mat;
        for (int i = 0; i < 2; i++) {
            d.mu[i] = hp.mu[i];
            d.lam[i] = hp.lam[i];
        }
        d.V = g.V;
        d.Vp = (B > 1) ? Vp : g.V;
        d.n1 = hp.n[0];
        d.n2 = hp.n[1];
        d.n3 = hp.n[2];
        d.sc = d_sc;
        d.guard = guard;
        d.dfloat = std::is_same<Rt, df32>::value ? 1 : 0;
        if (nb > 0) {
            BoxelArgs<double> a{};
            a.nb = nb;
            a.V = g.V;
            a.bidx = d_bidx;
            a.bN = d_bN;
            a.bc = d_bc;
            a.ba = d_ba8;
            a.bprob = d_bprob;
            a.matp = d_mat;
            a.F = d_F;
            for (int i = 0; i < 2; i++) {
                a.mu[i] = hp.mu[i];
                a.lam[i] = hp.lam[i];
            }
            a.tol_rel = opt.nr_tol_rel;
            a.tol_abs = opt.nr_tol_abs;
            a.max_iter = opt.nr_max_iter;
            a.sc = d_sc;
            a.guard = guard;
            a.S = d_S;
            a.dfloat = d.dfloat;
            a.Vp = d.Vp;
            a.n1 = d.n1;
            a.n2 = d.n2;
            a.n3 = d.n3;
            a.bAsub = tangent ? (void*)d_bA8 : nullptr;
            a.sub_f32 = sizeof(Tc) == 4 ? 1 : 0;
            prof.begin(K_BOXEL);
            launch_boxel_dfmg(a, st);
            prof.end();
        }
        prof.begin(K_DFMG_PURE);
        launch_dfmg_pure(d, st);
        prof.end();
        prof.begin(K_DFMG_GATHER);
        launch_dfmg_gather(d, st);
        prof.end();
    }

    // FP64 residual operator: G[P(F)]; mode: XI_FIXEDPOINT (update F) or XI_RHS (r = -G[P], x = 0)
    XfwdArgs<Rt, Tc> resid_xf(int xi_mode) const
    {
        auto xf = e64.template xf<Tc>();
        xf.mode = XF_RESID;
        xf.phase = d_phase;
        xf.vox2box = d_v2b;
        for (int i = 0; i < 2; i++) {
            xf.mu[i] = hp.mu[i];
            xf.lam[i] = hp.lam[i];
        }
        xf.F = d_F;
        xf.bP = d_bP;
        xf.X = dfmg() ? d_Pd : nullptr;  // the gathered stress of the doubly-fine material grid
        xf.linear = linear() ? 1 : 0;
        xf.tc = (xi_mode == XI_RHS) ? d_tc : nullptr;
        xf.matp = d_mat;
        xf.nb = nb;
        xf.sc = d_sc;
        return xf;
    }
    XinvArgs<Rt, Tc> resid_xi(int xi_mode) const
    {
        auto xi = e64.template xi<Tc>();
        xi.mode = xi_mode;
        xi.inv_mu0 = 1.0 / mu0;
        xi.F = d_F;
        xi.d = d_dir;
        xi.x = d_x;
        xi.r = d_r;
        xi.partial = d_part;
        xi.sc = d_sc;
        return xi;
    }
    void fin_resid(int xi_mode)
    {
        prof.begin(K_FINALIZE);
        k_fin_resid<<<B, 256, 0, st>>>(d_sc, d_part, e64.zblocks_p(), (double)Vp, opt.tol, opt.fixed_iterations,
                                       opt.max_iter, (xi_mode == XI_FIXEDPOINT || xi_mode == XI_NCG) ? 1 : 0,
                                       (B > 1 || member) ? 1 : 0, xi_mode == XI_NCG ? 1 : 0);
        prof.end();
    }
    void fin_rhs()
    {
        prof.begin(K_FINALIZE);
        k_fin_rhs<<<B, 256, 0, st>>>(d_sc, d_part, e64.xblocks() / B, opt.cg_fixed_iterations, opt.cg_max_iter);
        prof.end();
    }
    void resid_operator(int xi_mode, int guard)
    {
        const auto xf = resid_xf(xi_mode);
        prof.begin(K_XFWD_RESID);
        launch_xfwd<Rt, Tc>(xf, guard, st);
        prof.end();
        // the Newton right-hand side is an FP32 field: in the double-float
        // form its inverse transforms run in FP32 (the norm stays double-float)
        bool inv32 = false;
        if constexpr (std::is_same<Rt, df32>::value && std::is_same<Tc, float>::value)
            inv32 = xi_mode == XI_RHS && xinv_rhs32_ok(g);
        if constexpr (std::is_same<Tc, float>::value)
            e64.yz(d_sc, guard, true, d_part, st, &prof, K_YFWD_64, inv32, ec.tab.twy, ec.tab.twz);
        else
            e64.yz(d_sc, guard, true, d_part, st, &prof, K_YFWD_64);
        fin_resid(xi_mode);
        const auto xi = resid_xi(xi_mode);
        prof.begin(K_XINV_64);
        bool done = false;
        if constexpr (std::is_same<Rt, df32>::value && std::is_same<Tc, float>::value) {
            // the Newton right-hand side is an FP32 field: its transform in FP32
            if (xi_mode == XI_RHS && xinv_rhs32_ok(g)) {
                launch_xinv_rhs32(xi, ec.tab.twM, ec.tab.tw2, guard, st);
                done = true;
            }
        }
        if (!done) launch_xinv<Rt, Tc>(xi, guard, st);
        prof.end();
        if (xi_mode == XI_RHS) fin_rhs();
    }

    XfwdArgs<Tc, Tc> cg_xf() const
    {
        auto xf = ec.template xf<Tc>();
        xf.mode = XF_TANGENT;
        xf.phase = d_phase;
        xf.vox2box = d_v2b;
        for (int i = 0; i < 2; i++) {
            xf.mu[i] = hp.mu[i];
            xf.lam[i] = hp.lam[i];
        }
        xf.tc = d_tc;
        xf.r = d_r;
        xf.p = d_p;
        xf.x = d_x;
        xf.matp = d_mat;
        xf.bA = d_bA;
        xf.bvox = d_bvox;
        xf.lofs = d_lofs;
        xf.nb = std::max<int64_t>(nb, 1);
        xf.partial = d_part;
        xf.sc = d_sc;
        xf.fuse = 1;  // the last block computes alpha
        return xf;
    }
    XinvArgs<Tc, Tc> cg_xi() const
    {
        auto xi = ec.template xi<Tc>();
        xi.mode = XI_CG;
        xi.x = d_x;
        xi.r = d_r;
        xi.p = d_p;
        xi.partial = d_part;
        xi.sc = d_sc;
        xi.fuse = 1;  // the last block computes beta and the stopping test
        xi.cg_tol = opt.cg_tol;
        xi.cg_max = opt.cg_max_iter;
        xi.cg_fixed = opt.cg_fixed_iterations;
        return xi;
    }
    // arguments of the nodal form's tangent pass (Tc = float)
    NodalArgs nodal_args() const
    {
        NodalArgs n{};
        if constexpr (std::is_same<Tc, float>::value) {
            n.g = g;
            n.tw = ec.tab.twM;
            n.tw2 = ec.tab.tw2;
            n.spec = ec.spec;
            n.vrank = d_vrank;
            n.r = d_r;
            n.p[0] = d_p;
            n.p[1] = d_p2;
            n.x = d_x;
            n.tc = d_tc;
            n.matp = d_mat;
            for (int i = 0; i < 2; i++) {
                n.mu[i] = hp.mu[i];
                n.lam[i] = hp.lam[i];
            }
            n.bA = d_bA;
            n.lofs = d_lofs;
            n.nb = std::max<int64_t>(nb, 1);
            edge_weights(n.cJ);
            n.partial = d_part;
            n.sc = d_sc;
            n.fuse = 1;
            n.cfg = ec.cfg_xf;
        }
        return n;
    }
    // the nodal form's direction of odd CG iterations (else null)
    const Tc* p_odd() const { return ec.use_nodal ? d_p2 : nullptr; }
    // 1 / (4 h_J), the HEX8R gradient's edge weights
    void edge_weights(float cJ[3]) const
    {
        const int n[3] = {g.n1, g.n2, g.n3p};
        for (int j = 0; j < 3; j++) cJ[j] = (float)(n[j] / (4.0 * hp.l[j]));
    }

    // the x side of the Krylov operator with the CG update: the CG x-inverse,
    // or, in the displacement form, the x-inverse of the three nodal fields
    // and their gradient with the update
    void krylov_xinv()
    {
        if constexpr (std::is_same<Tc, float>::value) {
            if (ec.use_disp) {
                DispArgs d{};
                d.g = g;
                d.tw = ec.tab.twM;
                d.tw2 = ec.tab.tw2;
                d.spec = ec.spec;
                d.u = ec.disp_u();
                d.ustride = ec.disp_ustride();
                d.r = d_r;
                edge_weights(d.cJ);
                d.partial = d_part;
                d.sc = d_sc;
                d.fuse = 1;
                d.cg_tol = opt.cg_tol;
                d.cg_max = opt.cg_max_iter;
                d.cg_fixed = opt.cg_fixed_iterations;
                d.wait_cap = ec.wait_cap;
                if (xinv_grad_ok(g)) {
                    prof.begin(K_XINV_GRAD);
                    launch_xinv_grad(d, st);
                    prof.end();
                    return;
                }
                prof.begin(K_XINV_CG);
                launch_xinv_disp(d, st);
                prof.end();
                prof.begin(K_DISP_GRAD);
                launch_disp_grad_cg(d, st);
                prof.end();
                return;
            }
        }
        const auto xi = cg_xi();
        prof.begin(K_XINV_CG);
        launch_xinv<Tc, Tc>(xi, 1, st);
        prof.end();
    }

    // one CG iteration in precision Tc, guarded by cg_done
    void cg_iteration()
    {
        if (dfmg()) {
            dfmg_cg_iteration();
            return;
        }
        if constexpr (std::is_same<Tc, float>::value) {
            if (ec.use_nodal) {
                const NodalArgs n = nodal_args();
                prof.begin(K_XFWD_NODAL);
                launch_xfwd_nodal(n, st);
                prof.end();
                ec.yz(d_sc, 1, false, nullptr, st, &prof, K_YFWD_C);
                krylov_xinv();
                return;
            }
        }
        const auto xf = cg_xf();
        prof.begin(K_XFWD_TANGENT);
        launch_xfwd<Tc, Tc>(xf, 1, st);
        prof.end();
        ec.yz(d_sc, 1, false, nullptr, st, &prof, K_YFWD_C);
        krylov_xinv();
    }

    // doubly-fine material grid: the direction update, the sub-cell tangents
    // applied to p and their gather with (p, A : p) -> alpha, then the
    // transforms of A : p and the CG x-inverse
    void dfmg_cg_iteration()
    {
        DfmgTanArgs<Tc> d{};
        d.F = d_F;
        d.phase = d_phase;
        d.vox2box = d_v2b;
        d.bAsub = d_bA8;
        d.nb = std::max<int64_t>(nb, 1);
        for (int i = 0; i < 2; i++) {
            d.mu[i] = hp.mu[i];
            d.lam[i] = hp.lam[i];
        }
        d.r = d_r;
        d.p = d_p;
        d.x = d_x;
        d.St = d_St;
        d.y = d_yd;
        d.partial = d_part;
        d.sc = d_sc;
        d.V = g.V;
        d.n1 = g.n1;
        d.n2 = g.n2;
        d.n3 = g.n3;
        for (int stage = 0; stage < 3; stage++) {
            prof.begin(K_DFMG_CG);
            launch_dfmg_cg<Tc>(d, stage, st);
            prof.end();
        }
        auto xf = ec.template xf<Tc>();
        xf.mode = XF_RESID;
        xf.Xc = d_yd;
        xf.sc = d_sc;
        prof.begin(K_XFWD_TANGENT);
        launch_xfwd<Tc, Tc>(xf, 1, st);
        prof.end();
        ec.yz(d_sc, 1, false, nullptr, st, &prof, K_YFWD_C);
        krylov_xinv();
    }

    // capture one chunk of kCgChunk CG iterations (kernel arguments are fixed
    // for the life of the solve; control flow is on device flags)
    int capture_cg_chunk()
    {
        cudaGraph_t graph = nullptr;
        CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        for (int k = 0; k < kCgChunk; k++) cg_iteration();
        const cudaError_t e = cudaStreamEndCapture(st, &graph);
        if (e != cudaSuccess) return fail(COMBO_E_CUDA, std::string("CG graph capture: ") + cudaGetErrorString(e));
        const cudaError_t e2 = cudaGraphInstantiate(&cg_exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e2 != cudaSuccess) {
            cg_exec = nullptr;
            return fail(COMBO_E_CUDA, std::string("CG graph instantiate: ") + cudaGetErrorString(e2));
        }
        return COMBO_OK;
    }

    // description of the first failed laminate solve, if any
    std::string boxel_failure(const Scalars& s) const
    {
        if (s.fail_boxel <= 0) return "";
        static const char* why[5] = {"", "F_box inadmissible", "a phase inadmissible", "singular Hessian",
                                     "iteration cap"};
        const int r = (s.fail_reason >= 1 && s.fail_reason <= 4) ? s.fail_reason : 0;
        char buf[512];
        const double* q = s.fail_state;
        snprintf(buf, sizeof buf,
                 "; boxel %d (voxel %d): %s; F_box = [%.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g], "
                 "N = [%.17g %.17g %.17g], c+ = %.17g, a = [%.17g %.17g %.17g]",
                 s.fail_boxel - 1, hp.bidx[s.fail_boxel - 1], why[r], q[0], q[1], q[2], q[3], q[4], q[5], q[6], q[7],
                 q[8], q[9], q[10], q[11], q[12], q[13], q[14], q[15]);
        return buf;
    }

    int read_scalars(Scalars& s)
    {
        CK(cudaMemcpyAsync(&s, d_sc, sizeof(Scalars), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        prof.collect();
        return COMBO_OK;
    }

    int set_flag(size_t offset, int32_t value)
    {
        CK(cudaMemcpyAsync((char*)d_sc + offset, &value, 4, cudaMemcpyHostToDevice, st));
        return COMBO_OK;
    }

    int begin_step()
    {
        double Fn[9];
        Mat9 d;
        const double s = (double)(step + 1) / hp.n_steps;
        for (int c = 0; c < 9; c++) {
            const double I = (c == 0 || c == 4 || c == 8) ? 1.0 : 0.0;
            Fn[c] = I + s * (hp.Fbar[c] - I);
            d.v[c] = Fn[c] - Fprev[c];
        }
        std::memcpy(Fprev, Fn, sizeof(Fn));
        prof.begin(K_UPDATE);
        k_add_uniform<<<grid_for(9 * g.V), 256, 0, st>>>(d_F, g.V, d, nullptr, g.V);
        prof.end();
        CK(cudaGetLastError());
        outer = 0;
        cg_step_total = 0;
        int rc;
        if ((rc = set_flag(offsetof(Scalars, outer_done), 0))) return rc;
        if ((rc = set_flag(offsetof(Scalars, outer_iter), 0))) return rc;
        return COMBO_OK;
    }

    // Pbar_- and Pbar_+ of the converged state of one problem (Sec. 6.2 phase
    // averages): out[0..8] the matrix, out[9..17] the inclusion
    int phase_avg(int64_t v0, int64_t v1, int64_t b0, int64_t b1, const double mu[2], const double lam[2],
                  double* out)
    {
        Mat9 m{};
        m.v[0] = mu[0];
        m.v[1] = mu[1];
        m.v[2] = lam[0];
        m.v[3] = lam[1];
        if (dfmg())
            k_phase_sums_dfmg<<<PHASE_GRID, 256, 0, st>>>(d_F, g.V, d_phase, v0, v1, hp.n[0], hp.n[1], hp.n[2], d_bidx,
                                                          d_bN, d_bc, d_ba8, b0, b1, m, d_phpart, d_sc);
        else
            k_phase_sums<<<PHASE_GRID, 256, 0, st>>>(d_F, g.V, d_phase, v0, v1, d_bidx, d_bN, d_bc, d_ba, b0, b1, m,
                                                     d_phpart, d_sc, linear() ? 1 : 0);
        CK(cudaGetLastError());
        std::vector<double> part((size_t)PHASE_GRID * PHASE_SUMS);
        CK(cudaMemcpyAsync(part.data(), d_phpart, 8 * part.size(), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        double tot[PHASE_SUMS] = {0.0};
        for (int blk = 0; blk < PHASE_GRID; blk++)
            for (int k = 0; k < PHASE_SUMS; k++) tot[k] += part[(size_t)blk * PHASE_SUMS + k];
        for (int ph = 0; ph < 2; ph++)
            for (int c = 0; c < 9; c++) out[9 * ph + c] = tot[18 + ph] > 0.0 ? tot[9 * ph + c] / tot[18 + ph] : 0.0;
        return COMBO_OK;
    }

    int record_step(const Scalars& s)
    {
        int rc = phase_avg(0, g.V, 0, nb, hp.mu, hp.lam, Pphase.data() + 18 * (size_t)step);
        if (rc) return rc;
        for (int c = 0; c < 9; c++) Pbar[9 * step + c] = s.Pbar[c];
        resid[step] = s.eps;
        iters[step] = newton() ? outer : s.outer_iter;
        cg_iters[step] = cg_step_total;
        step++;
        return COMBO_OK;
    }

    int advance(int64_t max_ops) override
    {
        if (error) return error;
        const int64_t limit = (max_ops > 0) ? ops_done + max_ops : INT64_MAX;
        CK(cudaSetDevice(ctx->device));
        Scalars s;
        int rc;
        while (true) {
            if (state == ST_DONE) return COMBO_OK;
            if (ops_done >= limit && (!whole_newton || state == ST_RESID || state == ST_STEP || state == ST_FP))
                return COMBO_PENDING;
            if (cancel_requested) return error = fail(COMBO_E_CANCELLED, "solve cancelled");
            switch (state) {
                case ST_STEP:
                    if (step >= hp.n_steps) {
                        state = ST_DONE;
                        break;
                    }
                    if (step_target >= 0 && step >= step_target) return COMBO_PENDING;
                    if ((rc = begin_step())) return error = rc;
                    state = newton() ? ST_RESID : ST_FP;
                    break;
                case ST_FP: {
                    // a chunk of fixed-point iterations; kernels skip once converged
                    const int chunk = 16;
                    for (int k = 0; k < chunk; k++) {
                        if (dfmg())
                            dfmg_law(2);
                        else
                            boxels(false, 2);
                        resid_operator(opt.solver == COMBO_NONLINEAR_CG ? XI_NCG : XI_FIXEDPOINT, 2);
                    }
                    CK(cudaGetLastError());
                    if ((rc = read_scalars(s))) return error = rc;
                    ops_done = (int64_t)s.n_operator;
                    if (s.status) return error = fail(s.status, "fixed point failed" + boxel_failure(s));
                    if (s.outer_done) {
                        if ((rc = record_step(s))) return error = rc;
                        state = ST_STEP;
                    }
                    break;
                }
                case ST_RESID: {
                    const NvtxRange nr("newton_residual");
                    if (dfmg())
                        dfmg_law(0, true);
                    else
                        boxels(true, 0);
                    resid_operator(XI_RHS, 0);
                    CK(cudaGetLastError());
                    if ((rc = read_scalars(s))) return error = rc;
                    if (s.status) return error = fail(s.status, "residual evaluation failed" + boxel_failure(s));
                    const bool conv = (opt.fixed_iterations > 0) ? (outer >= opt.fixed_iterations) : (s.eps <= opt.tol);
                    if (conv) {
                        if ((rc = record_step(s))) return error = rc;
                        state = ST_STEP;
                    } else if (outer >= opt.max_iter) {
                        return error = fail(COMBO_E_NOT_CONVERGED, "Newton did not converge");
                    } else {
                        state = ST_CG;
                    }
                    break;
                }
                case ST_CG: {
                    const NvtxRange nr("cg_chunk");
                    // 8 CG iterations per host round trip; iterations after the
                    // device-side stop test are no-ops.  Without per-kernel
                    // timing the chunk is replayed from a captured CUDA graph.
                    if (prof.on || cg_chunks_run == 0) {
                        for (int k = 0; k < kCgChunk; k++) cg_iteration();
                    } else {
                        if (!cg_exec && (rc = capture_cg_chunk())) return error = rc;
                        CK(cudaGraphLaunch(cg_exec, st));
                    }
                    cg_chunks_run++;
                    CK(cudaGetLastError());
                    if ((rc = read_scalars(s))) return error = rc;
                    ops_done = (int64_t)s.n_operator;
                    if (s.status) return error = fail(s.status, "CG failed");
                    if (s.cg_done) {
                        cg_step_total += s.cg_iter;
                        state = ST_UPDATE;
                    }
                    break;
                }
                case ST_UPDATE: {
                    double d = 1.0;
                    bool ok = false;
                    for (int h = 0; h <= 10; h++) {
                        if ((rc = set_flag(offsetof(Scalars, admissible), 1))) return error = rc;
                        prof.begin(K_UPDATE);
                        k_update_F<Tc><<<grid_for(g.V), 256, 0, st>>>(d_F, d_x, d_p, p_odd(), d, g.V, d_sc, nullptr, g.V);
                        prof.end();
                        if ((rc = read_scalars(s))) return error = rc;
                        if (s.admissible || linear()) {  // (det F is not constrained on small strains)
                            ok = true;
                            break;
                        }
                        d = -std::ldexp(1.0, -(h + 1));  // F_old + 2^-(h+1) x
                    }
                    if (!ok) return error = fail(COMBO_E_INADMISSIBLE, "det F <= 0 after 10 step halvings");
                    outer++;
                    state = ST_RESID;
                    break;
                }
                default:
                    return COMBO_OK;
            }
        }
    }

    // ---- batch of B > 1 problems: Newton-CG in lockstep rounds.  Each round
    // starts the next load step of every problem that has one; its Newton
    // iterations evaluate the residual of the problems still iterating (the
    // others are masked by outer_done), run CG on them until each meets its
    // own stopping test (masked by cg_done), and update their F.
    struct PState {
        int step = 0, outer = 0, cg_total = 0;
        bool active = false;
        double Fprev[9];
        std::vector<double> Pbar, resid, Pphase;
        std::vector<int32_t> iters, cg_iters;
    };
    std::vector<PState> ps;
    std::vector<Scalars> hsc;

    int read_all()
    {
        CK(cudaMemcpyAsync(hsc.data(), d_sc, sizeof(Scalars) * B, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        prof.collect();
        return COMBO_OK;
    }

    int set_flag_of(int b, size_t offset, int32_t value)
    {
        CK(cudaMemcpyAsync((char*)(d_sc + b) + offset, &value, 4, cudaMemcpyHostToDevice, st));
        return COMBO_OK;
    }

    int batch_status(const char* what)
    {
        for (int b = 0; b < B; b++)
            if (hsc[b].status)
                return error = fail(hsc[b].status, std::string(what) + " (problem " + std::to_string(b) + ")" +
                                                       boxel_failure(hsc[b]));
        return COMBO_OK;
    }

    int run_batch() override
    {
        prof.on = env_profile();
        const int rc = run_batch_rounds();
        if (prof.on) {
            cudaStreamSynchronize(st);
            print_profile("stacked batch", prof);
        }
        return rc;
    }
    int run_batch_rounds()
    {
        CK(cudaSetDevice(ctx->device));
        if (!newton()) return error = fail(COMBO_E_INVALID_ARG, "a batch runs the Newton-CG solver");
        ps.assign(B, PState{});
        hsc.resize(B);
        for (int b = 0; b < B; b++) {
            for (int c = 0; c < 9; c++) ps[b].Fprev[c] = (c == 0 || c == 4 || c == 8) ? 1.0 : 0.0;
            const int S = hps[b].n_steps;
            ps[b].Pbar.assign(9 * (size_t)S, 0.0);
            ps[b].Pphase.assign(18 * (size_t)S, 0.0);
            ps[b].resid.assign(S, 0.0);
            ps[b].iters.assign(S, 0);
            ps[b].cg_iters.assign(S, 0);
        }
        std::vector<double> dF(9 * (size_t)B), dv(B);
        int rc;
        while (true) {
            // next load step of every problem that has one
            bool any = false;
            for (int b = 0; b < B; b++) {
                PState& q = ps[b];
                q.active = q.step < hps[b].n_steps;
                for (int c = 0; c < 9; c++) dF[9 * b + c] = 0.0;
                if (q.active) {
                    any = true;
                    const double f = (double)(q.step + 1) / hps[b].n_steps;
                    for (int c = 0; c < 9; c++) {
                        const double I = (c == 0 || c == 4 || c == 8) ? 1.0 : 0.0;
                        const double Fn = I + f * (hps[b].Fbar[c] - I);
                        dF[9 * b + c] = Fn - q.Fprev[c];
                        q.Fprev[c] = Fn;
                    }
                    q.outer = 0;
                    q.cg_total = 0;
                }
                if ((rc = set_flag_of(b, offsetof(Scalars, outer_done), q.active ? 0 : 1))) return error = rc;
                if ((rc = set_flag_of(b, offsetof(Scalars, outer_iter), 0))) return error = rc;
            }
            if (!any) break;
            CK(cudaMemcpyAsync(d_dF, dF.data(), 8 * dF.size(), cudaMemcpyHostToDevice, st));
            Mat9 zero{};
            prof.begin(K_UPDATE);
            k_add_uniform<<<grid_for(9 * g.V), 256, 0, st>>>(d_F, g.V, zero, d_dF, Vp);
            prof.end();
            CK(cudaGetLastError());
            // Newton iterations of this round
            while (true) {
                if (cancel_requested) return error = fail(COMBO_E_CANCELLED, "solve cancelled");
                boxels(true, 2);
                resid_operator(XI_RHS, 2);
                CK(cudaGetLastError());
                if ((rc = read_all())) return error = rc;
                if ((rc = batch_status("residual evaluation failed"))) return rc;
                bool any_cg = false;
                for (int b = 0; b < B; b++) {
                    PState& q = ps[b];
                    if (!q.active) continue;
                    const Scalars& sb = hsc[b];
                    const bool conv = (opt.fixed_iterations > 0) ? (q.outer >= opt.fixed_iterations) : (sb.eps <= opt.tol);
                    if (conv) {
                        if ((rc = phase_avg((int64_t)b * Vp, (int64_t)(b + 1) * Vp, boff[b], boff[b + 1], hps[b].mu,
                                            hps[b].lam, q.Pphase.data() + 18 * (size_t)q.step)))
                            return error = rc;
                        for (int c = 0; c < 9; c++) q.Pbar[9 * q.step + c] = sb.Pbar[c];
                        q.resid[q.step] = sb.eps;
                        q.iters[q.step] = q.outer;
                        q.cg_iters[q.step] = q.cg_total;
                        q.step++;
                        q.active = false;
                        if ((rc = set_flag_of(b, offsetof(Scalars, outer_done), 1))) return error = rc;
                        if ((rc = set_flag_of(b, offsetof(Scalars, cg_done), 1))) return error = rc;
                    } else if (q.outer >= opt.max_iter) {
                        return error = fail(COMBO_E_NOT_CONVERGED,
                                            "Newton did not converge (problem " + std::to_string(b) + ")");
                    } else {
                        any_cg = true;
                    }
                }
                if (!any_cg) break;
                // CG on the problems still iterating, 8 iterations per host round trip
                while (true) {
                    if (prof.on || cg_chunks_run == 0) {
                        for (int k = 0; k < kCgChunk; k++) cg_iteration();
                    } else {
                        if (!cg_exec && (rc = capture_cg_chunk())) return error = rc;
                        CK(cudaGraphLaunch(cg_exec, st));
                    }
                    cg_chunks_run++;
                    CK(cudaGetLastError());
                    if ((rc = read_all())) return error = rc;
                    if ((rc = batch_status("CG failed"))) return rc;
                    bool all = true;
                    for (int b = 0; b < B; b++) all = all && hsc[b].cg_done;
                    if (all) break;
                }
                // F += x with per-problem step halving until every det F > 0
                for (int b = 0; b < B; b++) {
                    dv[b] = ps[b].active ? 1.0 : 0.0;
                    if (ps[b].active) ps[b].cg_total += hsc[b].cg_iter;
                }
                bool ok = false;
                for (int h = 0; h <= 10; h++) {
                    for (int b = 0; b < B; b++)
                        if ((rc = set_flag_of(b, offsetof(Scalars, admissible), 1))) return error = rc;
                    CK(cudaMemcpyAsync(d_dv, dv.data(), 8 * B, cudaMemcpyHostToDevice, st));
                    prof.begin(K_UPDATE);
                    k_update_F<Tc><<<grid_for(g.V), 256, 0, st>>>(d_F, d_x, d_p, p_odd(), 0.0, g.V, d_sc, d_dv, Vp);
                    prof.end();
                    if ((rc = read_all())) return error = rc;
                    bool bad = false;
                    for (int b = 0; b < B; b++) {
                        if (dv[b] != 0.0 && !hsc[b].admissible && !linear()) {
                            dv[b] = -std::ldexp(1.0, -(h + 1));  // F_old + 2^-(h+1) x
                            bad = true;
                        } else {
                            dv[b] = 0.0;
                        }
                    }
                    if (!bad) {
                        ok = true;
                        break;
                    }
                }
                if (!ok) return error = fail(COMBO_E_INADMISSIBLE, "det F <= 0 after 10 step halvings");
                for (int b = 0; b < B; b++)
                    if (ps[b].active) ps[b].outer++;
            }
        }
        int64_t ops = 0;
        for (int b = 0; b < B; b++) ops += (int64_t)hsc[b].n_operator;
        ops_done = ops;
        state = ST_DONE;
        return COMBO_OK;
    }

    // per-problem results of a finished batch (fields sliced out of the stacked grid)
    int batch_results(combo_result* rs) override
    {
        CK(cudaSetDevice(ctx->device));
        double* P = nullptr;
        bool needP = false;
        for (int b = 0; b < B; b++) needP = needP || rs[b].P_out;
        if (needP) {
            CK(dev_malloc(&P, 8 * 9 * (size_t)g.V));
            Mat9 m{};
            k_eval_P<<<grid_for(g.V), 256, 0, st>>>(d_F, d_phase, d_v2b, d_bP, m, P, g.V, d_sc, d_mat, Vp,
                                                    linear() ? 1 : 0);
            CK(cudaGetLastError());
        }
        int rc = COMBO_OK;
        for (int b = 0; b < B && !rc; b++) {
            combo_result* r = rs + b;
            if (!r->Pbar) {
                rc = fail(COMBO_E_INVALID_ARG, "result needs Pbar");
                break;
            }
            const bool dev = (r->mem == COMBO_MEM_DEVICE);
            const cudaMemcpyKind h2x = dev ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
            const cudaMemcpyKind d2x = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
            const PState& q = ps[b];
            CK(cudaMemcpy(r->Pbar, q.Pbar.data(), 8 * q.Pbar.size(), h2x));
            if (r->Pbar_phase) CK(cudaMemcpy(r->Pbar_phase, q.Pphase.data(), 8 * q.Pphase.size(), h2x));
            if (r->iters) CK(cudaMemcpy(r->iters, q.iters.data(), 4 * q.iters.size(), h2x));
            if (r->cg_iters) CK(cudaMemcpy(r->cg_iters, q.cg_iters.data(), 4 * q.cg_iters.size(), h2x));
            if (r->resid) CK(cudaMemcpy(r->resid, q.resid.data(), 8 * q.resid.size(), h2x));
            for (int c = 0; c < 9; c++) {
                if (r->F_out)
                    CK(cudaMemcpyAsync(r->F_out + (size_t)c * Vp, d_F + (size_t)c * g.V + (size_t)b * Vp, 8 * Vp, d2x,
                                       st));
                if (r->P_out)
                    CK(cudaMemcpyAsync(r->P_out + (size_t)c * Vp, P + (size_t)c * g.V + (size_t)b * Vp, 8 * Vp, d2x, st));
            }
            const int64_t nbb = boff[b + 1] - boff[b];
            if (r->a_out && nbb > 0) CK(cudaMemcpyAsync(r->a_out, d_ba + 3 * boff[b], 24 * nbb, d2x, st));
            CK(cudaStreamSynchronize(st));
            r->steps_done = q.step;
            r->nr_iters = (int64_t)hsc[b].nr_iters;
            r->n_backproj = (int64_t)hsc[b].n_backproj;
            r->n_laminate_evals = (int64_t)hsc[b].n_lam;
            r->n_operator = (int64_t)hsc[b].n_operator;
            r->n_operator_fp64 = (int64_t)hsc[b].n_operator64;
        }
        cudaFree(P);
        return rc;
    }

    Profiler& profiler() override { return prof; }
    void request_cancel() override { cancel_requested = 1; }

    int advance_newton(int64_t min_ops) override
    {
        if (min_ops <= 0) return fail(COMBO_E_INVALID_ARG, "advance_newton needs a positive operator count");
        whole_newton = true;
        const int rc = advance(min_ops);
        whole_newton = false;
        return rc;
    }

    int advance_steps(int32_t k) override
    {
        if (k < 0) return fail(COMBO_E_INVALID_ARG, "negative step count");
        step_target = (int64_t)step + k;
        const int rc = advance(0);
        step_target = -1;
        return rc;
    }

    // Checkpoint of a single solve between load steps (host byte image):
    // header, the per-step results so far, the counters, F [9][V] and the
    // boxel jumps (per sub-cell for the doubly-fine grid).  Nothing else
    // carries over a load step: the Krylov vectors, tangent caches and the
    // nonlinear-CG direction restart with every step.
    struct CkptHeader {
        char magic[8];
        int64_t version, V, nb, n_steps, step;
        int32_t kspace, solver, precision, theory;
        double Fprev[9];
        uint64_t nr_iters, n_backproj, n_lam, n_operator, n_operator64;
    };
    int64_t ckpt_bytes() const
    {
        const int64_t S = hp.n_steps;
        return (int64_t)sizeof(CkptHeader) + 8 * (9 * S + 18 * S + S) + 4 * (2 * S) + 8 * 9 * g.V + 8 * 3 * nb +
               (dfmg() ? 8 * 24 * nb : 0);
    }
    void ckpt_fill(CkptHeader& h) const
    {
        std::memset(&h, 0, sizeof h);
        std::memcpy(h.magic, "COMBOCK1", 8);
        h.version = 1;
        h.V = g.V;
        h.nb = nb;
        h.n_steps = hp.n_steps;
        h.step = step;
        h.kspace = opt.kspace;
        h.solver = opt.solver;
        h.precision = opt.precision;
        h.theory = opt.theory;
        std::memcpy(h.Fprev, Fprev, sizeof Fprev);
    }

    int export_state(void* buf, int64_t* bytes) override
    {
        if (!bytes) return fail(COMBO_E_INVALID_ARG, "null size");
        if (B != 1) return fail(COMBO_E_INVALID_ARG, "checkpoints cover single solves");
        if (error) return error;
        if (state != ST_STEP && state != ST_DONE)
            return fail(COMBO_E_INVALID_ARG, "a checkpoint is taken between load steps (combo_solve_advance_steps)");
        const int64_t need = ckpt_bytes();
        if (!buf) {
            *bytes = need;
            return COMBO_OK;
        }
        if (*bytes < need) return fail(COMBO_E_INVALID_ARG, "checkpoint buffer too small");
        CK(cudaSetDevice(ctx->device));
        Scalars sc;
        int rc;
        if ((rc = read_scalars(sc))) return rc;
        CkptHeader h;
        ckpt_fill(h);
        h.nr_iters = sc.nr_iters;
        h.n_backproj = sc.n_backproj;
        h.n_lam = sc.n_lam;
        h.n_operator = sc.n_operator;
        h.n_operator64 = sc.n_operator64;
        char* o = static_cast<char*>(buf);
        auto put = [&](const void* src, size_t n) {
            std::memcpy(o, src, n);
            o += n;
        };
        const size_t S = (size_t)hp.n_steps;
        put(&h, sizeof h);
        put(Pbar.data(), 8 * 9 * S);
        put(Pphase.data(), 8 * 18 * S);
        put(resid.data(), 8 * S);
        put(iters.data(), 4 * S);
        put(cg_iters.data(), 4 * S);
        CK(cudaMemcpyAsync(o, d_F, 8 * 9 * (size_t)g.V, cudaMemcpyDeviceToHost, st));
        o += 8 * 9 * (size_t)g.V;
        if (nb > 0) CK(cudaMemcpyAsync(o, d_ba, 8 * 3 * (size_t)nb, cudaMemcpyDeviceToHost, st));
        o += 8 * 3 * (size_t)nb;
        if (dfmg() && nb > 0) CK(cudaMemcpyAsync(o, d_ba8, 8 * 24 * (size_t)nb, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        *bytes = need;
        return COMBO_OK;
    }

    int import_state(const void* buf, int64_t bytes) override
    {
        if (!buf) return fail(COMBO_E_INVALID_ARG, "null checkpoint");
        if (B != 1) return fail(COMBO_E_INVALID_ARG, "checkpoints cover single solves");
        if (error) return error;
        if (state != ST_STEP || step != 0 || ops_done != 0)
            return fail(COMBO_E_INVALID_ARG, "a checkpoint is imported into a solve that has not advanced");
        if (bytes != ckpt_bytes()) return fail(COMBO_E_INVALID_ARG, "checkpoint size does not match this solve");
        CkptHeader h, mine;
        std::memcpy(&h, buf, sizeof h);
        ckpt_fill(mine);
        if (std::memcmp(h.magic, mine.magic, 8) != 0 || h.version != 1)
            return fail(COMBO_E_INVALID_ARG, "not a checkpoint of this library");
        if (h.V != mine.V || h.nb != mine.nb || h.n_steps != mine.n_steps || h.kspace != mine.kspace ||
            h.solver != mine.solver || h.precision != mine.precision || h.theory != mine.theory)
            return fail(COMBO_E_INVALID_ARG, "checkpoint of another problem or other options");
        if (h.step < 0 || h.step > h.n_steps) return fail(COMBO_E_INVALID_ARG, "checkpoint step out of range");
        CK(cudaSetDevice(ctx->device));
        const char* in = static_cast<const char*>(buf) + sizeof h;
        auto get = [&](void* dst, size_t n) {
            std::memcpy(dst, in, n);
            in += n;
        };
        const size_t S = (size_t)hp.n_steps;
        get(Pbar.data(), 8 * 9 * S);
        get(Pphase.data(), 8 * 18 * S);
        get(resid.data(), 8 * S);
        get(iters.data(), 4 * S);
        get(cg_iters.data(), 4 * S);
        CK(cudaMemcpyAsync(d_F, in, 8 * 9 * (size_t)g.V, cudaMemcpyHostToDevice, st));
        in += 8 * 9 * (size_t)g.V;
        if (nb > 0) CK(cudaMemcpyAsync(d_ba, in, 8 * 3 * (size_t)nb, cudaMemcpyHostToDevice, st));
        in += 8 * 3 * (size_t)nb;
        if (dfmg() && nb > 0) CK(cudaMemcpyAsync(d_ba8, in, 8 * 24 * (size_t)nb, cudaMemcpyHostToDevice, st));
        const uint64_t cnt[5] = {h.nr_iters, h.n_backproj, h.n_lam, h.n_operator, h.n_operator64};
        CK(cudaMemcpyAsync((char*)d_sc + offsetof(Scalars, nr_iters), cnt, sizeof cnt, cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
        std::memcpy(Fprev, h.Fprev, sizeof Fprev);
        step = (int)h.step;
        ops_done = (int64_t)h.n_operator;
        return COMBO_OK;
    }

    int finish(combo_result* r) override
    {
        if (!r || !r->Pbar) return fail(COMBO_E_INVALID_ARG, "result needs Pbar");
        CK(cudaSetDevice(ctx->device));
        Scalars s;
        int rc;
        if ((rc = read_scalars(s))) return rc;
        const bool dev = (r->mem == COMBO_MEM_DEVICE);
        const cudaMemcpyKind h2x = dev ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
        const cudaMemcpyKind d2x = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        CK(cudaMemcpy(r->Pbar, Pbar.data(), 8 * Pbar.size(), h2x));
        if (r->Pbar_phase) CK(cudaMemcpy(r->Pbar_phase, Pphase.data(), 8 * Pphase.size(), h2x));
        if (r->iters) CK(cudaMemcpy(r->iters, iters.data(), 4 * iters.size(), h2x));
        if (r->cg_iters) CK(cudaMemcpy(r->cg_iters, cg_iters.data(), 4 * cg_iters.size(), h2x));
        if (r->resid) CK(cudaMemcpy(r->resid, resid.data(), 8 * resid.size(), h2x));
        const int64_t V = g.V;
        if (r->F_out) CK(cudaMemcpyAsync(r->F_out, d_F, 8 * 9 * V, d2x, st));
        if (r->P_out && dfmg()) {
            // the law at the current F (a solve stopped between an F update
            // and the next residual has a stale gathered stress)
            dfmg_law(0);
            CK(cudaMemcpyAsync(r->P_out, d_Pd, 8 * 9 * V, d2x, st));
        } else if (r->P_out) {
            // F changed since the last laminate solve (a solve stopped between
            // an F update and the next residual): solve the boxels at this F
            if (state == ST_RESID && nb > 0) {
                boxels(false, 0);
                CK(cudaGetLastError());
            }
            double* P = dev ? r->P_out : nullptr;
            if (!dev) CK(dev_malloc(&P, 8 * 9 * V));
            Mat9 m{};
            m.v[0] = hp.mu[0];
            m.v[1] = hp.mu[1];
            m.v[2] = hp.lam[0];
            m.v[3] = hp.lam[1];
            k_eval_P<<<grid_for(V), 256, 0, st>>>(d_F, d_phase, d_v2b, d_bP, m, P, V, d_sc, nullptr, V,
                                                  linear() ? 1 : 0);
            if (!dev) {
                CK(cudaMemcpyAsync(r->P_out, P, 8 * 9 * V, cudaMemcpyDeviceToHost, st));
                CK(cudaStreamSynchronize(st));
                cudaFree(P);
            }
        }
        if (dfmg()) launch_dfmg_amean(d_ba8, d_ba, nb, st);  // reported: the mean of the sub-cell jumps
        if (r->a_out && nb > 0) CK(cudaMemcpyAsync(r->a_out, d_ba, 24 * nb, d2x, st));
        CK(cudaStreamSynchronize(st));
        r->steps_done = step;
        r->nr_iters = (int64_t)s.nr_iters;
        r->n_backproj = (int64_t)s.n_backproj;
        r->n_laminate_evals = (int64_t)s.n_lam;
        r->n_operator = (int64_t)s.n_operator;
        r->n_operator_fp64 = (int64_t)s.n_operator64;
        return error;
    }
};

// ------------------------------------------------------------------ batches over several grids
// Device copy of one grouped launch's table (GroupTab): per descriptor its
// arguments, its first item and its item grid.
template <typename A> struct GroupBuf {
    GroupTab<A> t;
    void* mem = nullptr;
    ~GroupBuf() { cudaFree(mem); }
    int build(const std::vector<A>& args, const std::vector<int>& items, const std::vector<int>& dims, size_t smem,
              cudaStream_t st)
    {
        const int nd = (int)args.size();
        std::vector<int> vs(nd + 1, 0), dm(2 * std::max(nd, 1), 0);
        for (int d = 0; d < nd; d++) vs[d + 1] = vs[d] + items[d];
        for (size_t i = 0; i < dims.size(); i++) dm[i] = dims[i];
        const size_t ab = (sizeof(A) * std::max(nd, 1) + 255) / 256 * 256;
        const size_t vb = (sizeof(int) * vs.size() + 255) / 256 * 256;
        const size_t db = sizeof(int) * dm.size();
        CK(dev_malloc(&mem, ab + vb + db));
        char* b = static_cast<char*>(mem);
        CK(cudaMemcpyAsync(b, args.data(), sizeof(A) * nd, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(b + ab, vs.data(), sizeof(int) * vs.size(), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(b + ab + vb, dm.data(), db, cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));  // the host vectors go out of scope
        t.args = reinterpret_cast<const A*>(b);
        t.vstart = reinterpret_cast<const int*>(b + ab);
        t.dims = reinterpret_cast<const int*>(b + ab + vb);
        t.nd = nd;
        t.total = vs[nd];
        t.smem = smem;
        return COMBO_OK;
    }
};

// A batch of Newton-CG problems on different grids.  The problems of each
// distinct grid (sides and cell size) form one stacked solve (a class); the
// classes advance in lockstep rounds like the stacked batch.  A class whose
// stacked grid has at least kOwnVoxels voxels (enough work to keep its own
// tuned, specialised launches busy) runs them on a stream of its own; for all
// smaller classes every pass
// of every operator application -- laminate solves, x-forward, y, z + Green
// operator, y inverse, x-inverse -- is ONE grouped launch over the work items
// of all of them (grouped x-, y-, z-pass and boxel kernels) on another
// stream, so the small grids run beside the large ones.  Each CG chunk of
// kCgChunk iterations is replayed from one captured CUDA graph whose
// branches are these streams.  A class runs the same pass bodies and
// reductions as its own stacked solve would (grouped classes with the
// engine's default launch shapes), so each result equals its single solve
// within the Krylov rounding.
template <typename Tc, typename Rt> struct MixSolve : SolveBase {
    using Cls = Solve<Tc, Rt>;
    combo_ctx* ctx = nullptr;
    combo_options opt;
    cudaStream_t st = nullptr;
    std::vector<std::unique_ptr<Cls>> cls;
    std::vector<std::vector<int>> members;  // input index of each class's problems
    std::vector<int> off;                   // first problem (in the shared scalars) of each class
    int P = 0;
    Scalars* d_sc = nullptr;  // [P] scalars of every problem, class-major
    std::vector<Scalars> hsc;
    GroupBuf<BoxelArgs<Tc>> g_box;
    GroupBuf<XfwdArgs<Rt, Tc>> g_xf_res;
    GroupBuf<YArgs<Rt>> g_y_res;
    GroupBuf<ZArgs<Rt>> g_z_res;
    GroupBuf<XinvArgs<Rt, Tc>> g_xi_res;
    GroupBuf<XfwdArgs<Tc, Tc>> g_xf_cg;
    GroupBuf<YArgs<Tc>> g_y_cg;
    GroupBuf<ZArgs<Tc>> g_z_cg;
    GroupBuf<XinvArgs<Tc, Tc>> g_xi_cg;
    Profiler prof;  // the grouped launches (on st_group)
    cudaGraphExec_t cg_exec = nullptr;
    int64_t cg_chunks_run = 0;
    volatile int cancel_requested = 0;
    int error = 0;
    static constexpr int kCgChunk = 8;
    static constexpr int64_t kOwnVoxels = int64_t(1) << 20;  // stacked voxels of a class that runs its own launches
    std::vector<char> own;             // class runs its own launch sequences
    cudaStream_t st_group = nullptr;   // the grouped launches
    std::vector<cudaStream_t> sides;   // st_group and the streams of the own-launch classes
    cudaEvent_t ev_fork = nullptr;
    std::vector<cudaEvent_t> ev_join;

    ~MixSolve() override
    {
        if (cg_exec) cudaGraphExecDestroy(cg_exec);
        cls.clear();
        cudaFree(d_sc);
        for (auto s2 : sides) cudaStreamDestroy(s2);
        for (auto e : ev_join) cudaEventDestroy(e);
        if (ev_fork) cudaEventDestroy(ev_fork);
    }
    // every side stream waits for the work queued on st so far; st waits
    // for all of them (the lockstep's host reads and F updates run on st)
    int fork()
    {
        CK(cudaEventRecord(ev_fork, st));
        for (auto s2 : sides) CK(cudaStreamWaitEvent(s2, ev_fork, 0));
        return COMBO_OK;
    }
    int join()
    {
        for (size_t i = 0; i < sides.size(); i++) {
            CK(cudaEventRecord(ev_join[i], sides[i]));
            CK(cudaStreamWaitEvent(st, ev_join[i], 0));
        }
        return COMBO_OK;
    }
    bool linear() const { return opt.theory == COMBO_INFINITESIMAL_STRAIN; }

    int init(combo_ctx* c, std::vector<HostProblem>&& hs, const combo_options& o)
    {
        ctx = c;
        st = c->stream;
        prof.st = st;
        opt = o;
        P = (int)hs.size();
        // classes: problems of equal sides and cell sizes, in order of first appearance
        std::vector<std::vector<HostProblem>> groups;
        for (int i = 0; i < P; i++) {
            int k = 0;
            for (; k < (int)groups.size(); k++) {
                const HostProblem& q = groups[k][0];
                bool same = true;
                for (int j = 0; j < 3; j++) same = same && q.n[j] == hs[i].n[j] && q.l[j] == hs[i].l[j];
                if (same) break;
            }
            if (k == (int)groups.size()) {
                groups.emplace_back();
                members.emplace_back();
            }
            groups[k].push_back(std::move(hs[i]));
            members[k].push_back(i);
        }
        CK(dev_malloc(&d_sc, sizeof(Scalars) * P));
        CK(cudaMemsetAsync(d_sc, 0, sizeof(Scalars) * P, st));
        hsc.resize(P);
        int rc, o0 = 0;
        CK(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
        CK(cudaStreamCreateWithFlags(&st_group, cudaStreamNonBlocking));
        sides.push_back(st_group);
        prof.st = st_group;
        for (size_t k = 0; k < groups.size(); k++) {
            off.push_back(o0);
            auto q = std::make_unique<Cls>();
            q->member = true;
            const int64_t vox = (int64_t)groups[k].size() * groups[k][0].n[0] * groups[k][0].n[1] * groups[k][0].n[2];
            q->own_launches = vox >= kOwnVoxels;
            own.push_back(q->own_launches ? 1 : 0);
            q->ext_sc = d_sc + o0;
            o0 += (int)groups[k].size();
            rc = q->init(c, std::move(groups[k]), o);
            cls.push_back(std::move(q));
            if (rc) return rc;
            Cls& m = *cls.back();
            if (m.own_launches) {
                cudaStream_t s2;
                CK(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
                sides.push_back(s2);
                m.st = s2;
            } else {
                m.st = st_group;
            }
            m.prof.st = m.st;
        }
        ev_join.resize(sides.size(), nullptr);
        for (auto& e : ev_join) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        CK(cudaStreamSynchronize(st));
        return build_groups();
    }

    // the grouped launches' tables: the arguments each class's own launches
    // would take (default launch shapes, guards of the lockstep batch)
    std::vector<int> grouped() const
    {
        std::vector<int> g;
        for (int k = 0; k < (int)cls.size(); k++)
            if (!own[k]) g.push_back(k);
        return g;
    }
    int build_groups()
    {
        const std::vector<int> G = grouped();
        const int K = (int)G.size();
        int rc;
        {
            std::vector<BoxelArgs<Tc>> a;
            std::vector<int> it;
            for (int k : G)
                if (cls[k]->nb > 0) {
                    a.push_back(cls[k]->boxel_args(true, 2));
                    it.push_back((int)((cls[k]->nb + 127) / 128));
                }
            if ((rc = g_box.build(a, it, {}, 0, st))) return rc;
        }
        {
            std::vector<XfwdArgs<Rt, Tc>> a(K);
            std::vector<XinvArgs<Rt, Tc>> b(K);
            std::vector<int> itf(K), iti(K);
            size_t smf = 0, smi = 0;
            for (int i = 0; i < K; i++) {
                const Cls& q = *cls[G[i]];
                a[i] = q.resid_xf(XI_RHS);
                b[i] = q.resid_xi(XI_RHS);
                itf[i] = xpass_grid(q.g, q.e64.lines_fwd);
                iti[i] = q.e64.xblocks();
                smf = std::max(smf, xpass_smem(q.g, q.e64.lines_fwd, sizeof(cx<Rt>)));
                smi = std::max(smi, xpass_smem(q.g, q.e64.lines, sizeof(cx<Rt>)));
            }
            if ((rc = g_xf_res.build(a, itf, {}, smf, st))) return rc;
            if ((rc = g_xi_res.build(b, iti, {}, smi, st))) return rc;
        }
        {
            std::vector<XfwdArgs<Tc, Tc>> a(K);
            std::vector<XinvArgs<Tc, Tc>> b(K);
            std::vector<int> itf(K), iti(K);
            size_t smf = 0, smi = 0;
            for (int i = 0; i < K; i++) {
                const Cls& q = *cls[G[i]];
                a[i] = q.cg_xf();
                b[i] = q.cg_xi();
                itf[i] = xpass_grid(q.g, q.ec.lines_fwd);
                iti[i] = q.ec.xblocks();
                smf = std::max(smf, xpass_smem(q.g, q.ec.lines_fwd, sizeof(cx<Tc>)));
                smi = std::max(smi, xpass_smem(q.g, q.ec.lines, sizeof(cx<Tc>)));
            }
            if ((rc = g_xf_cg.build(a, itf, {}, smf, st))) return rc;
            if ((rc = g_xi_cg.build(b, iti, {}, smi, st))) return rc;
        }
        if ((rc = build_yz<Rt>(g_y_res, g_z_res, true))) return rc;
        return build_yz<Tc>(g_y_cg, g_z_cg, false);
    }

    template <typename T> int build_yz(GroupBuf<YArgs<T>>& gy, GroupBuf<ZArgs<T>>& gz, bool resid)
    {
        const std::vector<int> G = grouped();
        const int K = (int)G.size();
        std::vector<YArgs<T>> ya(K);
        std::vector<ZArgs<T>> za(K);
        std::vector<int> yi(K), zi(K), yd(2 * K), zd(2 * K);
        size_t ysm = 0, zsm = 0;
        for (int k = 0; k < K; k++) {
            Cls& q = *cls[G[k]];
            const Engine<T>& e = engine_of<T>(q, resid);
            ya[k] = e.yargs(q.d_sc, resid ? 2 : 1);
            za[k] = e.zargs(q.d_sc, resid ? 2 : 1, resid, resid ? q.d_part : nullptr);
            ya[k].tmap = nullptr;
            za[k].tmap = nullptr;
            int gx, gyy, gzz;
            size_t sm;
            ypass_group_shape(q.g, ya[k].tx, sizeof(cx<T>), gx, gyy, gzz, sm);
            yi[k] = gx * gyy * gzz;
            yd[2 * k] = gx;
            yd[2 * k + 1] = gyy;
            ysm = std::max(ysm, sm);
            zpass_group_shape(q.g, za[k].tx, sizeof(cx<T>), gx, gyy, gzz, sm);
            zi[k] = gx * gyy * gzz;
            zd[2 * k] = gx;
            zd[2 * k + 1] = gyy;
            zsm = std::max(zsm, sm);
            if (resid && zi[k] / q.B != q.e64.zblocks_p())
                return fail(COMBO_E_CUDA, "grouped z-pass partial count differs from the class's reduction");
        }
        int rc;
        if ((rc = gy.build(ya, yi, yd, ysm, st))) return rc;
        return gz.build(za, zi, zd, zsm, st);
    }
    template <typename T> static const Engine<T>& engine_of(const Cls& q, bool resid)
    {
        if constexpr (std::is_same<T, Rt>::value && std::is_same<T, Tc>::value)
            return resid ? q.e64 : q.ec;
        else if constexpr (std::is_same<T, Rt>::value)
            return q.e64;
        else
            return q.ec;
    }

    // --- launch sequences: the grouped classes on st_group, each own-launch
    // class on its stream, between a fork from and a join into st
    int residual()
    {
        int rc;
        if ((rc = fork())) return rc;
        const cudaStream_t sg = st_group;
        prof.begin(K_BOXEL);
        launch_group_boxel<Tc>(g_box.t, std::is_same<Rt, df32>::value, linear(), sg);
        prof.end();
        prof.begin(K_XFWD_RESID);
        launch_group_xfwd<Rt, Tc>(g_xf_res.t, false, 2, sg);
        prof.end();
        prof.begin(K_YFWD_64);
        launch_group_ypass<Rt, false>(g_y_res.t, sg);
        prof.end();
        prof.begin(K_ZGAMMA_64);
        launch_group_zpass<Rt>(g_z_res.t, sg);
        prof.end();
        prof.begin(K_YINV_64);
        launch_group_ypass<Rt, true>(g_y_res.t, sg);
        prof.end();
        for (int k : grouped()) cls[k]->fin_resid(XI_RHS);
        prof.begin(K_XINV_64);
        launch_group_xinv<Rt, Tc>(g_xi_res.t, 2, sg);
        prof.end();
        for (int k : grouped()) cls[k]->fin_rhs();
        for (size_t k = 0; k < cls.size(); k++)
            if (own[k]) {
                cls[k]->boxels(true, 2);
                cls[k]->resid_operator(XI_RHS, 2);
            }
        return join();
    }
    void group_cg_iteration()
    {
        const cudaStream_t sg = st_group;
        prof.begin(K_XFWD_TANGENT);
        launch_group_xfwd<Tc, Tc>(g_xf_cg.t, true, 1, sg);
        prof.end();
        prof.begin(K_YFWD_C);
        launch_group_ypass<Tc, false>(g_y_cg.t, sg);
        prof.end();
        prof.begin(K_ZGAMMA_C);
        launch_group_zpass<Tc>(g_z_cg.t, sg);
        prof.end();
        prof.begin(K_YINV_C);
        launch_group_ypass<Tc, true>(g_y_cg.t, sg);
        prof.end();
        prof.begin(K_XINV_CG);
        launch_group_xinv<Tc, Tc>(g_xi_cg.t, 1, sg);
        prof.end();
    }
    int cg_chunk()
    {
        int rc;
        if ((rc = fork())) return rc;
        for (int j = 0; j < kCgChunk; j++) group_cg_iteration();
        for (size_t k = 0; k < cls.size(); k++)
            if (own[k])
                for (int j = 0; j < kCgChunk; j++) cls[k]->cg_iteration();
        return join();
    }
    int capture_cg_chunk()
    {
        cudaGraph_t graph = nullptr;
        CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        const int rc = cg_chunk();
        const cudaError_t e = cudaStreamEndCapture(st, &graph);
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) return fail(COMBO_E_CUDA, std::string("CG graph capture: ") + cudaGetErrorString(e));
        const cudaError_t e2 = cudaGraphInstantiate(&cg_exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e2 != cudaSuccess) {
            cg_exec = nullptr;
            return fail(COMBO_E_CUDA, std::string("CG graph instantiate: ") + cudaGetErrorString(e2));
        }
        return COMBO_OK;
    }
    int read_all()
    {
        CK(cudaMemcpyAsync(hsc.data(), d_sc, sizeof(Scalars) * P, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        prof.collect();
        for (size_t k = 0; k < cls.size(); k++)
            std::copy(hsc.begin() + off[k], hsc.begin() + off[k] + cls[k]->B, cls[k]->hsc.begin());
        return COMBO_OK;
    }
    int set_flag_of(int i, size_t offset, int32_t value)
    {
        CK(cudaMemcpyAsync((char*)(d_sc + i) + offset, &value, 4, cudaMemcpyHostToDevice, st));
        return COMBO_OK;
    }
    int status(const char* what)
    {
        for (size_t k = 0; k < cls.size(); k++)
            for (int b = 0; b < cls[k]->B; b++)
                if (hsc[off[k] + b].status)
                    return error = fail(hsc[off[k] + b].status,
                                        std::string(what) + " (problem " + std::to_string(members[k][b]) + ")" +
                                            cls[k]->boxel_failure(hsc[off[k] + b]));
        return COMBO_OK;
    }

    // Newton-CG in lockstep rounds over every problem of every class (the
    // stacked batch's rounds, with grouped launches)
    int run_batch() override
    {
        prof.on = env_profile();
        for (auto& q : cls) q->prof.on = prof.on;
        const int rc = run_rounds();
        if (prof.on) {
            cudaDeviceSynchronize();
            print_profile("batch over several grids: grouped classes", prof);
            for (size_t k = 0; k < cls.size(); k++)
                if (own[k]) {
                    char what[96];
                    std::snprintf(what, sizeof what, "  own-launch class %dx%dx%d x%d", cls[k]->hp.n[0],
                                  cls[k]->hp.n[1], cls[k]->hp.n[2], cls[k]->B);
                    print_profile(what, cls[k]->prof);
                }
        }
        return rc;
    }
    int run_rounds()
    {
        CK(cudaSetDevice(ctx->device));
        if (opt.solver != COMBO_NEWTON_CG) return error = fail(COMBO_E_INVALID_ARG, "a batch runs the Newton-CG solver");
        const int K = (int)cls.size();
        for (auto& q : cls) {
            q->ps.assign(q->B, typename Cls::PState{});
            q->hsc.resize(q->B);
            for (int b = 0; b < q->B; b++) {
                auto& z = q->ps[b];
                for (int c = 0; c < 9; c++) z.Fprev[c] = (c == 0 || c == 4 || c == 8) ? 1.0 : 0.0;
                const int S = q->hps[b].n_steps;
                z.Pbar.assign(9 * (size_t)S, 0.0);
                z.Pphase.assign(18 * (size_t)S, 0.0);
                z.resid.assign(S, 0.0);
                z.iters.assign(S, 0);
                z.cg_iters.assign(S, 0);
            }
        }
        int rc;
        while (true) {
            // next load step of every problem that has one
            bool any = false;
            for (int k = 0; k < K; k++) {
                Cls& q = *cls[k];
                std::vector<double> dF(9 * (size_t)q.B, 0.0);
                for (int b = 0; b < q.B; b++) {
                    auto& z = q.ps[b];
                    z.active = z.step < q.hps[b].n_steps;
                    if (z.active) {
                        any = true;
                        const double f = (double)(z.step + 1) / q.hps[b].n_steps;
                        for (int c = 0; c < 9; c++) {
                            const double I = (c == 0 || c == 4 || c == 8) ? 1.0 : 0.0;
                            const double Fn = I + f * (q.hps[b].Fbar[c] - I);
                            dF[9 * b + c] = Fn - z.Fprev[c];
                            z.Fprev[c] = Fn;
                        }
                        z.outer = 0;
                        z.cg_total = 0;
                    }
                    if ((rc = set_flag_of(off[k] + b, offsetof(Scalars, outer_done), z.active ? 0 : 1))) return error = rc;
                    if ((rc = set_flag_of(off[k] + b, offsetof(Scalars, outer_iter), 0))) return error = rc;
                }
                CK(cudaMemcpyAsync(q.d_dF, dF.data(), 8 * dF.size(), cudaMemcpyHostToDevice, st));
                Mat9 zero{};
                prof.begin(K_UPDATE);
                k_add_uniform<<<grid_for(9 * q.g.V), 256, 0, st>>>(q.d_F, q.g.V, zero, q.d_dF, q.Vp);
                prof.end();
                CK(cudaStreamSynchronize(st));  // dF goes out of scope
            }
            if (!any) break;
            CK(cudaGetLastError());
            // Newton iterations of this round
            while (true) {
                if (cancel_requested) return error = fail(COMBO_E_CANCELLED, "solve cancelled");
                if ((rc = residual())) return error = rc;
                CK(cudaGetLastError());
                if ((rc = read_all())) return error = rc;
                if ((rc = status("residual evaluation failed"))) return rc;
                bool any_cg = false;
                for (int k = 0; k < K; k++) {
                    Cls& q = *cls[k];
                    for (int b = 0; b < q.B; b++) {
                        auto& z = q.ps[b];
                        if (!z.active) continue;
                        const Scalars& sb = hsc[off[k] + b];
                        const bool conv = (opt.fixed_iterations > 0) ? (z.outer >= opt.fixed_iterations) : (sb.eps <= opt.tol);
                        if (conv) {
                            if ((rc = q.phase_avg((int64_t)b * q.Vp, (int64_t)(b + 1) * q.Vp, q.boff[b], q.boff[b + 1],
                                                  q.hps[b].mu, q.hps[b].lam, z.Pphase.data() + 18 * (size_t)z.step)))
                                return error = rc;
                            for (int c = 0; c < 9; c++) z.Pbar[9 * z.step + c] = sb.Pbar[c];
                            z.resid[z.step] = sb.eps;
                            z.iters[z.step] = z.outer;
                            z.cg_iters[z.step] = z.cg_total;
                            z.step++;
                            z.active = false;
                            if ((rc = set_flag_of(off[k] + b, offsetof(Scalars, outer_done), 1))) return error = rc;
                            if ((rc = set_flag_of(off[k] + b, offsetof(Scalars, cg_done), 1))) return error = rc;
                        } else if (z.outer >= opt.max_iter) {
                            return error = fail(COMBO_E_NOT_CONVERGED, "Newton did not converge (problem " +
                                                                         std::to_string(members[k][b]) + ")");
                        } else {
                            any_cg = true;
                        }
                    }
                }
                if (!any_cg) break;
                // CG on every problem still iterating, kCgChunk iterations per host round trip
                while (true) {
                    if (prof.on || cg_chunks_run == 0) {
                        if ((rc = cg_chunk())) return error = rc;
                    } else {
                        if (!cg_exec && (rc = capture_cg_chunk())) return error = rc;
                        CK(cudaGraphLaunch(cg_exec, st));
                    }
                    cg_chunks_run++;
                    CK(cudaGetLastError());
                    if ((rc = read_all())) return error = rc;
                    if ((rc = status("CG failed"))) return rc;
                    bool all = true;
                    for (int i = 0; i < P; i++) all = all && hsc[i].cg_done;
                    if (all) break;
                }
                // F += x with per-problem step halving until every det F > 0
                std::vector<std::vector<double>> dv(K);
                for (int k = 0; k < K; k++) {
                    Cls& q = *cls[k];
                    dv[k].assign(q.B, 0.0);
                    for (int b = 0; b < q.B; b++) {
                        dv[k][b] = q.ps[b].active ? 1.0 : 0.0;
                        if (q.ps[b].active) q.ps[b].cg_total += hsc[off[k] + b].cg_iter;
                    }
                }
                bool ok = false;
                for (int h = 0; h <= 10; h++) {
                    for (int i = 0; i < P; i++)
                        if ((rc = set_flag_of(i, offsetof(Scalars, admissible), 1))) return error = rc;
                    for (int k = 0; k < K; k++) {
                        Cls& q = *cls[k];
                        CK(cudaMemcpyAsync(q.d_dv, dv[k].data(), 8 * q.B, cudaMemcpyHostToDevice, st));
                        prof.begin(K_UPDATE);
                        k_update_F<Tc><<<grid_for(q.g.V), 256, 0, st>>>(q.d_F, q.d_x, q.d_p, q.p_odd(), 0.0, q.g.V, q.d_sc, q.d_dv,
                                                                        q.Vp);
                        prof.end();
                    }
                    if ((rc = read_all())) return error = rc;
                    bool bad = false;
                    for (int k = 0; k < K; k++)
                        for (int b = 0; b < cls[k]->B; b++) {
                            if (dv[k][b] != 0.0 && !hsc[off[k] + b].admissible && !linear()) {
                                dv[k][b] = -std::ldexp(1.0, -(h + 1));  // F_old + 2^-(h+1) x
                                bad = true;
                            } else {
                                dv[k][b] = 0.0;
                            }
                        }
                    if (!bad) {
                        ok = true;
                        break;
                    }
                }
                if (!ok) return error = fail(COMBO_E_INADMISSIBLE, "det F <= 0 after 10 step halvings");
                for (auto& q : cls)
                    for (int b = 0; b < q->B; b++)
                        if (q->ps[b].active) q->ps[b].outer++;
            }
        }
        return COMBO_OK;
    }

    // per-problem results in input order
    int batch_results(combo_result* rs) override
    {
        for (size_t k = 0; k < cls.size(); k++) {
            std::vector<combo_result> sub;
            for (int i : members[k]) sub.push_back(rs[i]);
            const int rc = cls[k]->batch_results(sub.data());
            for (size_t j = 0; j < sub.size(); j++) rs[members[k][j]] = sub[j];
            if (rc) return rc;
        }
        return COMBO_OK;
    }

    Profiler& profiler() override { return prof; }
    void request_cancel() override { cancel_requested = 1; }
    int advance(int64_t) override { return fail(COMBO_E_INVALID_ARG, "a batch over several grids runs as a whole"); }
    int advance_newton(int64_t) override { return advance(0); }
    int advance_steps(int32_t) override { return advance(0); }
    int finish(combo_result*) override { return advance(0); }
    int export_state(void*, int64_t*) override { return fail(COMBO_E_INVALID_ARG, "checkpoints cover single solves"); }
    int import_state(const void*, int64_t) override { return export_state(nullptr, nullptr); }
};

// A solve of the requested precision form: plain FP64; FP32 Krylov with FP64
// residual transforms; FP32 Krylov with double-float residual transforms.
template <class H> static int make_solve(combo_ctx* ctx, H&& h, const combo_options& o, SolveBase** out)
{
    int rc;
    if (o.precision == COMBO_FP64) {
        auto* s = new Solve<double, double>();
        rc = s->init(ctx, std::move(h), o);
        *out = s;
    } else if (o.precision == COMBO_FP32_REFINED) {
        auto* s = new Solve<float, double>();
        rc = s->init(ctx, std::move(h), o);
        *out = s;
    } else {
        auto* s = new Solve<float, df32>();
        rc = s->init(ctx, std::move(h), o);
        *out = s;
    }
    return rc;
}

// A batch over several grids in the requested precision form
static int make_mix(combo_ctx* ctx, std::vector<HostProblem>&& hs, const combo_options& o, SolveBase** out)
{
    int rc;
    if (o.precision == COMBO_FP64) {
        auto* s = new MixSolve<double, double>();
        *out = s;
        rc = s->init(ctx, std::move(hs), o);
    } else if (o.precision == COMBO_FP32_REFINED) {
        auto* s = new MixSolve<float, double>();
        *out = s;
        rc = s->init(ctx, std::move(hs), o);
    } else {
        auto* s = new MixSolve<float, df32>();
        *out = s;
        rc = s->init(ctx, std::move(hs), o);
    }
    return rc;
}

// ------------------------------------------------------------------ C ABI: solves
extern "C" int64_t combo_solve_footprint(const combo_problem* p, const combo_options* o)
{
    if (!p || !o) return -1;
    const int64_t V = (int64_t)p->n[0] * p->n[1] * p->n[2];
    const GridDims g = make_dims(p->n);
    const int64_t nb = std::max<int64_t>(p->n_boxels, 1);
    const int64_t tc = (o->precision == COMBO_FP64) ? 8 : 4;
    int64_t b = V * (1 + 4 + 72) + 16 * 9 * g.Vs + nb * (4 + 24 + 8 + 24 + 72);
    if (o->solver == COMBO_NEWTON_CG) b += tc * (81 * nb + 37 * V);
    if (o->solver == COMBO_NEWTON_CG && tc == 4 && o->kspace == COMBO_ROTATED) b += 40 * V;  // nodal form's second p and voxel map
    if (o->solver == COMBO_NONLINEAR_CG) b += 72 * V;
    if (o->kspace == COMBO_STAGGERED_DFMG) b += 8 * 81 * V + 192 * nb;
    return b;
}

extern "C" int combo_solve_begin(combo_ctx* ctx, const combo_problem* p, const combo_options* o_in,
                                 combo_solve_state** out)
{
    if (!ctx || !out) return fail(COMBO_E_INVALID_ARG, "null context or output");
    combo_options o;
    if (o_in)
        o = *o_in;
    else
        combo_options_default(&o);
    int rc = check_options(o);
    if (rc) return rc;
    CK(cudaSetDevice(ctx->device));
    HostProblem h;
    const NvtxRange nr("solve_setup");
    if ((rc = load_problem(p, &o, h))) return rc;
    SolveBase* impl = nullptr;
    rc = make_solve(ctx, std::move(h), o, &impl);
    if (rc) {
        std::string msg = g_err;
        delete impl;
        cudaGetLastError();
        g_err = msg;
        return (rc == COMBO_E_CUDA && msg.find("memory") != std::string::npos) ? COMBO_E_OOM : rc;
    }
    *out = new combo_solve_state{impl};
    return COMBO_OK;
}

extern "C" int combo_solve_advance(combo_solve_state* s, int64_t max_ops)
{
    if (!s) return fail(COMBO_E_INVALID_ARG, "null solve");
    return s->impl->advance(max_ops);
}

extern "C" int combo_solve_advance_newton(combo_solve_state* s, int64_t min_operator)
{
    if (!s) return fail(COMBO_E_INVALID_ARG, "null solve");
    return s->impl->advance_newton(min_operator);
}

extern "C" int combo_solve_advance_steps(combo_solve_state* s, int32_t k)
{
    if (!s) return fail(COMBO_E_INVALID_ARG, "null solve");
    return s->impl->advance_steps(k);
}

extern "C" int combo_state_export(combo_solve_state* s, void* buf, int64_t* bytes)
{
    if (!s) return fail(COMBO_E_INVALID_ARG, "null solve");
    return s->impl->export_state(buf, bytes);
}

extern "C" int combo_state_import(combo_solve_state* s, const void* buf, int64_t bytes)
{
    if (!s) return fail(COMBO_E_INVALID_ARG, "null solve");
    return s->impl->import_state(buf, bytes);
}

extern "C" int combo_solve_finish(combo_solve_state* s, combo_result* r)
{
    if (!s) return fail(COMBO_E_INVALID_ARG, "null solve");
    return s->impl->finish(r);
}

extern "C" int combo_solve_profile(combo_solve_state* s, int32_t enable)
{
    if (!s) return fail(COMBO_E_INVALID_ARG, "null solve");
    Profiler& p = s->impl->profiler();
    p.collect();
    p.reset();
    p.on = enable != 0;
    return COMBO_OK;
}

extern "C" int combo_solve_profile_read(combo_solve_state* s, int32_t max_classes, char* names, double* ms,
                                        int64_t* launches)
{
    if (!s) return fail(COMBO_E_INVALID_ARG, "null solve");
    Profiler& p = s->impl->profiler();
    CK(cudaStreamSynchronize(p.st));
    p.collect();
    const int n = std::min<int>(max_classes, K_NCLASS);
    for (int k = 0; k < n; k++) {
        if (names) {
            std::strncpy(names + 32 * k, kclass_name[k], 31);
            names[32 * k + 31] = 0;
        }
        if (ms) ms[k] = p.ms[k];
        if (launches) launches[k] = p.launches[k];
    }
    return K_NCLASS;
}

extern "C" void combo_solve_end(combo_solve_state* s)
{
    if (!s) return;
    delete s->impl;
    delete s;
}

extern "C" int combo_solve(combo_ctx* ctx, const combo_problem* p, const combo_options* o, combo_result* r)
{
    combo_solve_state* s = nullptr;
    int rc = combo_solve_begin(ctx, p, o, &s);
    if (rc) return rc;
    rc = combo_solve_advance(s, 0);
    const std::string msg = g_err;
    const int rc2 = combo_solve_finish(s, r);
    combo_solve_end(s);
    if (rc) {
        g_err = msg;
        return rc;
    }
    return rc2;
}

extern "C" void combo_autotune_enable(int32_t enable) { g_tune_enabled.store(enable ? 1 : 0); }

extern "C" int combo_krylov_form(int32_t form)
{
    if (form < COMBO_KRYLOV_NINE || form > COMBO_KRYLOV_NODAL)
        return fail(COMBO_E_INVALID_ARG, "Krylov operator form outside 0..2");
    g_krylov_form.store(form);
    return COMBO_OK;
}

extern "C" int combo_autotune_force(int32_t pass, int32_t cand)
{
    if (pass < 0 || pass > 3 || cand < -1 || cand > 1) return fail(COMBO_E_INVALID_ARG, "bad pass or candidate");
    g_tune_force[pass].store(cand);
    return COMBO_OK;
}

extern "C" int64_t combo_autotune_report(char* buf, int64_t len)
{
    std::string out;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        static const char* pass[4] = {"x-forward", "y", "z", "x-inverse"};
        for (const auto& kv : g_tune) {
            char line[512];
            int n = snprintf(line, sizeof line, "%dx%dx%d x%d FP%d%s:", kv.first.n1, kv.first.n2, kv.first.n3p,
                             kv.first.nprob, kv.first.word * 8, kv.first.nodal ? " nodal" : "");
            for (int k = 0; k < 4; k++)
                n += snprintf(line + n, sizeof line - n, " %s=%d (%.3f/%.3f ms)", pass[k], kv.second.cfg[k],
                              kv.second.ms[k][0] / 3.0, kv.second.ms[k][1] >= 1e29f ? -1.0 : kv.second.ms[k][1] / 3.0);
            out += line;
            out += "\n";
        }
    }
    if (buf && len > 0) {
        const size_t m = std::min<size_t>((size_t)len - 1, out.size());
        std::memcpy(buf, out.data(), m);
        buf[m] = 0;
    }
    return (int64_t)out.size();
}

extern "C" int combo_solve_batch(combo_ctx* ctx, int32_t n_problems, const combo_problem* problems,
                                 const combo_options* o_in, combo_result* results)
{
    if (!ctx || !problems || !results || n_problems <= 0) return fail(COMBO_E_INVALID_ARG, "bad batch arguments");
    combo_options o;
    if (o_in)
        o = *o_in;
    else
        combo_options_default(&o);
    int rc = check_options(o);
    if (rc) return rc;
    if (n_problems > 1 && o.solver != COMBO_NEWTON_CG)
        return fail(COMBO_E_INVALID_ARG, "a batch runs the Newton-CG solver");
    if (n_problems > 1 && o.kspace == COMBO_STAGGERED_DFMG)
        return fail(COMBO_E_INVALID_ARG, "the doubly-fine material grid runs as single solves");
    CK(cudaSetDevice(ctx->device));
    std::vector<HostProblem> hs(n_problems);
    bool same = true;
    int64_t vmax = 0;
    for (int b = 0; b < n_problems; b++) {
        if ((rc = load_problem(problems + b, &o, hs[b]))) return rc;
        for (int j = 0; j < 3; j++) same = same && hs[b].n[j] == hs[0].n[j] && hs[b].l[j] == hs[0].l[j];
        vmax = std::max(vmax, (int64_t)hs[b].n[0] * hs[b].n[1] * hs[b].n[2]);
    }
    if (vmax * n_problems >= (int64_t)1 << 31) return fail(COMBO_E_INVALID_ARG, "batch too large");
    if (!same) {
        // problems on several grids: one stacked class per grid, grouped launches
        SolveBase* impl = nullptr;
        const double t0 = wall_s();
        rc = make_mix(ctx, std::move(hs), o, &impl);
        const double t1 = wall_s();
        if (!rc) rc = impl->run_batch();
        const double t2 = wall_s();
        const std::string msg = g_err;
        if (!rc) rc = impl->batch_results(results);
        delete impl;
        if (env_profile())
            std::fprintf(stderr, "[combo profile] set-up %.3f s, rounds %.3f s, results and release %.3f s\n",
                         t1 - t0, t2 - t1, wall_s() - t2);
        if (rc) {
            cudaGetLastError();
            g_err = msg.empty() ? g_err : msg;
            return (rc == COMBO_E_CUDA && g_err.find("memory") != std::string::npos) ? COMBO_E_OOM : rc;
        }
        return COMBO_OK;
    }
    if (n_problems == 1) {
        // a batch of one is a plain solve
        SolveBase* impl = nullptr;
        rc = make_solve(ctx, std::move(hs[0]), o, &impl);
        if (!rc) rc = impl->advance(0);
        const std::string msg = g_err;
        const int rc2 = impl ? impl->finish(results) : rc;
        delete impl;
        if (rc) {
            g_err = msg;
            return rc;
        }
        return rc2;
    }
    SolveBase* impl = nullptr;
    rc = make_solve(ctx, std::move(hs), o, &impl);
    if (!rc) rc = impl->run_batch();
    const std::string msg = g_err;
    if (!rc) rc = impl->batch_results(results);
    delete impl;
    if (rc) {
        cudaGetLastError();
        g_err = msg.empty() ? g_err : msg;
        return (rc == COMBO_E_CUDA && g_err.find("memory") != std::string::npos) ? COMBO_E_OOM : rc;
    }
    return COMBO_OK;
}

// ------------------------------------------------------------------ C ABI: unit entry points
template <typename T> static int apply_G_impl(combo_ctx* ctx, const int32_t n[3], const double l[3], int kspace,
                                              const double* X, double* Y, double* sumsq, int mem)
{
    const GridDims g = make_dims(n);
    const int64_t V = g.V;
    Engine<T> e;
    int rc = e.init(g, l, kspace);
    if (rc) return rc;
    cudaStream_t st = ctx->stream;
    double *dX = nullptr, *dY = nullptr, *part = nullptr;
    void* spec = nullptr;
    Scalars* sc = nullptr;
    const bool dev = (mem == COMBO_MEM_DEVICE);
    auto cleanup = [&]() {
        if (!dev) {
            cudaFree(dX);
            cudaFree(dY);
        }
        cudaFree(part);
        cudaFree(spec);
        cudaFree(sc);
        e.release();
    };
#define CKC(call)                                                                                             \
    do {                                                                                                      \
        cudaError_t e_ = (call);                                                                              \
        if (e_ != cudaSuccess) {                                                                              \
            cleanup();                                                                                        \
            return fail(COMBO_E_CUDA, std::string(#call ": ") + cudaGetErrorString(e_));                     \
        }                                                                                                     \
    } while (0)
    if (dev) {
        dX = const_cast<double*>(X);
        dY = Y;
    } else {
        CKC(dev_malloc(&dX, 72 * V));
        CKC(dev_malloc(&dY, 72 * V));
        CKC(cudaMemcpyAsync(dX, X, 72 * V, cudaMemcpyHostToDevice, st));
    }
    CKC(dev_malloc(&spec, sizeof(cx<T>) * 9 * g.Vs));
    CKC(cudaMemsetAsync(spec, 0, sizeof(cx<T>) * 9 * g.Vs, st));
    CKC(dev_malloc(&part, 8 * (size_t)std::max(e.xblocks(), e.zblocks())));
    CKC(dev_malloc(&sc, sizeof(Scalars)));
    CKC(cudaMemsetAsync(sc, 0, sizeof(Scalars), st));
    e.bind_spec(spec);
    // (the Krylov word type only matters for the solver modes of the x-passes)
    typedef typename std::conditional<std::is_same<T, df32>::value, float, T>::type Tk;
    auto xf = e.template xf<Tk>();
    xf.X = dX;
    xf.sc = sc;
    launch_xfwd<T, Tk>(xf, 0, st);
    e.yz(sc, 0, true, part, st);
    k_fin_resid<<<1, 256, 0, st>>>(sc, part, e.zblocks(), (double)V, 0.0, 0, 0, 0);
    auto xi = e.template xi<Tk>();
    xi.mode = XI_PLAIN;
    xi.Y = dY;
    xi.sc = sc;
    launch_xinv<T, Tk>(xi, 0, st);
    CKC(cudaGetLastError());
    Scalars s;
    CKC(cudaMemcpyAsync(&s, sc, sizeof(Scalars), cudaMemcpyDeviceToHost, st));
    if (!dev) CKC(cudaMemcpyAsync(Y, dY, 72 * V, cudaMemcpyDeviceToHost, st));
    CKC(cudaStreamSynchronize(st));
    if (sumsq) *sumsq = s.resid2 / (double)V;
    cleanup();
#undef CKC
    return COMBO_OK;
}

extern "C" int combo_apply_G(combo_ctx* ctx, const int32_t n[3], const double l[3], int32_t kspace, int32_t precision,
                             const double* X, double* Y, double* sumsq, int32_t mem)
{
    if (!ctx || !n || !l || !X || !Y) return fail(COMBO_E_INVALID_ARG, "null argument");
    int rc = validate_dims(n);
    if (rc) return rc;
    if (kspace != COMBO_ROTATED && kspace != COMBO_SPECTRAL && kspace != COMBO_STAGGERED)
        return fail(COMBO_E_INVALID_ARG, "bad kspace");
    CK(cudaSetDevice(ctx->device));
    if (precision == COMBO_FP64) return apply_G_impl<double>(ctx, n, l, kspace, X, Y, sumsq, mem);
    if (precision == COMBO_FP32_REFINED) return apply_G_impl<float>(ctx, n, l, kspace, X, Y, sumsq, mem);
    if (precision == COMBO_FP32_REFINED_DF) return apply_G_impl<df32>(ctx, n, l, kspace, X, Y, sumsq, mem);
    return fail(COMBO_E_INVALID_ARG, "bad precision");
}

// One Neo-Hookean evaluation (Sec. 6.1) with its tangent
// A_iJkL = mu d_ik d_JL + lam G_Ji G_Lk + (mu - lam ln J) G_Jk G_Li, G = F^{-1}.
__global__ void k_nh_eval(const double* F, double mu, double lam, double* P, double* A, int* ok)
{
    const double* f = F;
    const double c0 = f[4] * f[8] - f[5] * f[7], c1 = f[5] * f[6] - f[3] * f[8], c2 = f[3] * f[7] - f[4] * f[6];
    const double J = f[0] * c0 + f[1] * c1 + f[2] * c2;
    if (!nh_P64(f, mu, lam, P)) {
        *ok = 0;
        return;
    }
    const double iJ = 1.0 / J;
    const double G[9] = {c0 * iJ, (f[2] * f[7] - f[1] * f[8]) * iJ, (f[1] * f[5] - f[2] * f[4]) * iJ,
                         c1 * iJ, (f[0] * f[8] - f[2] * f[6]) * iJ, (f[2] * f[3] - f[0] * f[5]) * iJ,
                         c2 * iJ, (f[1] * f[6] - f[0] * f[7]) * iJ, (f[0] * f[4] - f[1] * f[3]) * iJ};
    const double m = mu - lam * log(J);
    for (int i = 0; i < 3; i++)
        for (int Jx = 0; Jx < 3; Jx++)
            for (int k = 0; k < 3; k++)
                for (int L = 0; L < 3; L++)
                    A[9 * (3 * i + Jx) + 3 * k + L] = ((i == k && Jx == L) ? mu : 0.0) +
                                                      lam * G[3 * Jx + i] * G[3 * L + k] +
                                                      m * G[3 * Jx + k] * G[3 * L + i];
    *ok = 1;
}

extern "C" int combo_neohooke_eval(combo_ctx* ctx, const double F[9], double mu, double lam, double P[9],
                                   double A[81])
{
    if (!ctx || !F || !P) return fail(COMBO_E_INVALID_ARG, "null argument");
    CK(cudaSetDevice(ctx->device));
    double* d = nullptr;
    int* dok = nullptr;
    CK(dev_malloc(&d, 8 * (9 + 9 + 81)));
    CK(dev_malloc(&dok, 4));
    int rc = COMBO_OK, ok = 0;
    double hP[9], hA[81];
    if (cudaMemcpyAsync(d, F, 72, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess) rc = COMBO_E_CUDA;
    if (!rc) {
        k_nh_eval<<<1, 1, 0, ctx->stream>>>(d, mu, lam, d + 9, d + 18, dok);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(hP, d + 9, 72, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
            cudaMemcpyAsync(hA, d + 18, 648, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
            cudaMemcpyAsync(&ok, dok, 4, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
            cudaStreamSynchronize(ctx->stream) != cudaSuccess)
            rc = COMBO_E_CUDA;
    }
    cudaFree(d);
    cudaFree(dok);
    if (rc) return fail(rc, "combo_neohooke_eval: CUDA error");
    if (!ok) return fail(COMBO_E_INADMISSIBLE, "det F <= 0");
    std::memcpy(P, hP, 72);
    if (A) std::memcpy(A, hA, 648);
    return COMBO_OK;
}

// One composite boxel through the solver's own laminate kernel (FP64,
// Algorithms 1 and 2, the tangent of Eq. Peff:Seff unpacked from its packed
// upper triangle).  mat = {mu-, lam-, mu+, lam+}.
extern "C" int combo_laminate_eval(combo_ctx* ctx, const double F[9], const double N[3], double c,
                                   const double mat[4], double a_io[3], double P[9], double A[81], int32_t* iters)
{
    if (!ctx || !F || !N || !mat || !a_io || !P) return fail(COMBO_E_INVALID_ARG, "null argument");
    if (!(c > 0.0 && c < 1.0)) return fail(COMBO_E_INVALID_ARG, "volume fraction outside (0, 1)");
    const double nn = std::sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
    if (!(nn >= 1e-12)) return fail(COMBO_E_INVALID_ARG, "normal of zero length");
    CK(cudaSetDevice(ctx->device));
    // device block: F 9 | N 3 | c 1 | a 3 | P 9 | A packed 45, then the boxel index and the scalars
    double h[70];
    std::memcpy(h, F, 72);
    for (int i = 0; i < 3; i++) h[9 + i] = N[i] / nn;
    h[12] = c;
    std::memcpy(h + 13, a_io, 24);
    double* d = nullptr;
    int32_t* didx = nullptr;
    Scalars* dsc = nullptr;
    CK(dev_malloc(&d, sizeof h));
    CK(dev_malloc(&didx, 4));
    CK(dev_malloc(&dsc, sizeof(Scalars)));
    int rc = COMBO_OK;
    const int32_t zero = 0;
    Scalars sc{};
    if (cudaMemcpyAsync(d, h, sizeof h, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess ||
        cudaMemcpyAsync(didx, &zero, 4, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess ||
        cudaMemsetAsync(dsc, 0, sizeof(Scalars), ctx->stream) != cudaSuccess)
        rc = COMBO_E_CUDA;
    if (!rc) {
        BoxelArgs<double> b{};
        b.nb = 1;
        b.V = 1;
        b.bidx = didx;
        b.bN = d + 9;
        b.bc = d + 12;
        b.ba = d + 13;
        b.bP = d + 16;
        b.bA = A ? d + 25 : nullptr;
        b.F = d;
        b.mu[0] = mat[0];
        b.lam[0] = mat[1];
        b.mu[1] = mat[2];
        b.lam[1] = mat[3];
        b.tol_rel = 1e-12;
        b.tol_abs = 1e-14;
        b.max_iter = 50;
        b.sc = dsc;
        launch_boxel<double>(b, ctx->stream);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(h, d, sizeof h, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
            cudaMemcpyAsync(&sc, dsc, sizeof(Scalars), cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
            cudaStreamSynchronize(ctx->stream) != cudaSuccess)
            rc = COMBO_E_CUDA;
    }
    cudaFree(d);
    cudaFree(didx);
    cudaFree(dsc);
    if (rc) return fail(rc, "combo_laminate_eval: CUDA error");
    if (sc.status) return fail(sc.status, "laminate solve failed");
    std::memcpy(a_io, h + 13, 24);
    std::memcpy(P, h + 16, 72);
    if (A)
        for (int r = 0; r < 9; r++)
            for (int q = 0; q < 9; q++) A[9 * r + q] = h[25 + sym_idx(r, q)];
    if (iters) *iters = (int32_t)sc.nr_iters;
    return COMBO_OK;
}

__global__ void k_df_log(const double* x, double* y, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = (double)df_log(df32(x[i]));
}

extern "C" int combo_df_log(combo_ctx* ctx, const double* x, double* y, int64_t n)
{
    if (!ctx || n < 0 || (n > 0 && (!x || !y))) return fail(COMBO_E_INVALID_ARG, "null argument");
    for (int64_t i = 0; i < n; i++)
        if (!(x[i] >= 1.1754944e-38 && x[i] <= 3.4e38)) return fail(COMBO_E_INVALID_ARG, "x outside the FP32 normal range");
    if (n == 0) return COMBO_OK;
    CK(cudaSetDevice(ctx->device));
    double *dx = nullptr, *dy = nullptr;
    CK(dev_malloc(&dx, 8 * n));
    CK(dev_malloc(&dy, 8 * n));
    int rc = COMBO_OK;
    if (cudaMemcpyAsync(dx, x, 8 * n, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess) rc = COMBO_E_CUDA;
    if (!rc) {
        k_df_log<<<(int)((n + 255) / 256), 256, 0, ctx->stream>>>(dx, dy, n);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(y, dy, 8 * n, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
            cudaStreamSynchronize(ctx->stream) != cudaSuccess)
            rc = COMBO_E_CUDA;
    }
    cudaFree(dx);
    cudaFree(dy);
    return rc ? fail(rc, "combo_df_log: CUDA error") : COMBO_OK;
}

// Arithmetic-rate probe: every thread runs 8 independent chains of dependent
// FMAs x <- x b + c (b < 1, so the chains stay bounded); the result is stored
// only under a condition that never holds, which keeps the chains live
// without memory traffic.  FLOPs = 2 * 8 * 16 * iters per thread.
template <typename T> __global__ void __launch_bounds__(256) k_fma_rate(T* out, int iters, T b, T c)
{
    T x[8];
#pragma unroll
    for (int k = 0; k < 8; k++) x[k] = (T)(threadIdx.x & 7) + (T)k;
#pragma unroll 1
    for (int i = 0; i < iters; i++)
#pragma unroll
        for (int u = 0; u < 16; u++)
#pragma unroll
            for (int k = 0; k < 8; k++) {
                if constexpr (sizeof(T) == 8)
                    x[k] = __fma_rn(x[k], b, c);
                else
                    x[k] = __fmaf_rn(x[k], b, c);
            }
    T s = (T)0;
#pragma unroll
    for (int k = 0; k < 8; k++) s += x[k];
    if (s == (T)-1) out[blockIdx.x] = s;  // the chains stay near c / (1 - b) > 0
}

extern "C" int combo_arith_rates(combo_ctx* ctx, double* tflops)
{
    if (!ctx || !tflops) return fail(COMBO_E_INVALID_ARG, "null argument");
    CK(cudaSetDevice(ctx->device));
    int nsm = 0;
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
    const int grid = 8 * nsm;  // 2048 threads per SM
    double* buf = nullptr;
    CK(dev_malloc(&buf, sizeof(double) * grid));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = COMBO_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = COMBO_E_CUDA;
    // best of three launches after one warm-up, each a few ms long
    auto rate = [&](auto launch, double flops) -> double {
        float best = 0.f;
        for (int r = 0; r < 4 && !rc; r++) {
            if (cudaEventRecord(e0, ctx->stream) != cudaSuccess) rc = COMBO_E_CUDA;
            launch();
            if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, ctx->stream) != cudaSuccess ||
                cudaEventSynchronize(e1) != cudaSuccess)
                rc = COMBO_E_CUDA;
            float ms = 0.f;
            if (!rc && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = COMBO_E_CUDA;
            if (r > 0 && ms > 0.f && (best == 0.f || ms < best)) best = ms;
        }
        return (rc || best <= 0.f) ? 0.0 : flops / (best * 1e-3) / 1e12;
    };
    const double per_iter = 2.0 * 8 * 16 * 256.0 * grid;
    const int it64 = 32, it32 = 2048;
    const double r64 = rate([&] { k_fma_rate<double><<<grid, 256, 0, ctx->stream>>>(buf, it64, 0.999, 1e-3); },
                            per_iter * it64);
    const double r32 = rate(
        [&] { k_fma_rate<float><<<grid, 256, 0, ctx->stream>>>((float*)buf, it32, 0.999f, 1e-3f); },
        per_iter * it32);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(buf);
    if (rc) return fail(rc, "combo_arith_rates: CUDA error");
    tflops[0] = r64;
    tflops[1] = r32;
    return COMBO_OK;
}

extern "C" int combo_constitutive(combo_ctx* ctx, const combo_problem* p, const combo_options* o_in, const double* F,
                                  double* a_io, double* P, int32_t mem)
{
    if (!ctx || !F || !P) return fail(COMBO_E_INVALID_ARG, "null argument");
    combo_options o;
    if (o_in)
        o = *o_in;
    else
        combo_options_default(&o);
    o.precision = COMBO_FP64;
    o.solver = COMBO_FIXED_POINT;
    int rc = check_options(o);
    if (rc) return rc;
    CK(cudaSetDevice(ctx->device));
    HostProblem h;
    if ((rc = load_problem(p, &o, h))) return rc;
    // boxel order after snapping: map back to the caller's boxel list
    const int64_t nb_in = p->n_boxels;
    std::vector<int64_t> idx_in(nb_in);
    if (nb_in > 0)
        CK(cudaMemcpy(idx_in.data(), p->boxel_idx, 8 * nb_in,
                      p->mem == COMBO_MEM_DEVICE ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost));
    Solve<double> s;
    if ((rc = s.init(ctx, std::move(h), o))) return rc;
    const int64_t V = s.g.V;
    const bool dev = (mem == COMBO_MEM_DEVICE);
    const cudaMemcpyKind in = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(s.d_F, F, 72 * V, in, s.st));
    std::vector<double> a_all(3 * std::max<int64_t>(nb_in, 1), 0.0), a_kept(3 * std::max<int64_t>(s.nb, 1), 0.0);
    if (a_io && nb_in > 0) {
        CK(cudaMemcpy(a_all.data(), a_io, 24 * nb_in, dev ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost));
    }
    // kept boxels are the subsequence of idx_in that survived the snap
    std::vector<int64_t> pos(s.nb);
    for (int64_t b = 0, k = 0; b < nb_in && k < s.nb; b++)
        if (idx_in[b] == s.hp.bidx[k]) {
            pos[k] = b;
            for (int i = 0; i < 3; i++) a_kept[3 * k + i] = a_all[3 * b + i];
            k++;
        }
    if (s.nb > 0) CK(cudaMemcpyAsync(s.d_ba, a_kept.data(), 24 * s.nb, cudaMemcpyHostToDevice, s.st));
    // (the doubly-fine material grid evaluates its law in finish, from zero
    // sub-cell jumps; a_io returns the mean of the converged sub-cell jumps)
    if (!s.dfmg()) s.boxels(false, 0);
    combo_result r{};
    std::vector<double> pb(9 * (size_t)s.hp.n_steps);
    r.Pbar = pb.data();
    r.P_out = P;
    r.mem = mem;
    if ((rc = s.finish(&r))) return rc;
    Scalars sc;
    if ((rc = s.read_scalars(sc))) return rc;
    if (sc.status) return fail(sc.status, "constitutive evaluation failed");
    if (a_io && s.nb > 0) {
        CK(cudaMemcpy(a_kept.data(), s.d_ba, 24 * s.nb, cudaMemcpyDeviceToHost));
        for (int64_t k = 0; k < s.nb; k++)
            for (int i = 0; i < 3; i++) a_all[3 * pos[k] + i] = a_kept[3 * k + i];
        CK(cudaMemcpy(a_io, a_all.data(), 24 * nb_in, dev ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost));
    }
    return COMBO_OK;
}

// ------------------------------------------------------------------ serving
// A request loop for many solves of different sizes.  submit() validates and
// copies a problem and queues it; a slot (worker thread with its own CUDA
// stream) admits the oldest queued request whose device footprint fits the
// memory left in the budget, keeps that solve's fields and state resident,
// and runs it to completion; a request that arrives while others run is
// admitted as soon as a slot and memory are free, and the admitted solves'
// kernels overlap on the device through their streams.  Latencies (submit to
// completion) give p50 / p99.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>

namespace {

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int64_t footprint_of(const HostProblem& h, const combo_options& o)
{
    const GridDims g = make_dims(h.n);
    const int64_t V = g.V;
    const int64_t nb = std::max<int64_t>((int64_t)h.bidx.size(), 1);
    const int64_t tc = (o.precision == COMBO_FP64) ? 8 : 4;
    int64_t b = V * (1 + 4 + 72) + 16 * 9 * g.Vs + nb * (4 + 24 + 8 + 24 + 72) + (1 << 20);
    if (o.solver == COMBO_NEWTON_CG) b += tc * (45 * nb + 37 * V) + 8 * nb + 4 * ((int64_t)g.n2 * g.n3 + 1);
    if (o.solver == COMBO_NEWTON_CG && tc == 4 && o.kspace == COMBO_ROTATED) b += 40 * V;  // nodal form's second p and voxel map
    if (o.solver == COMBO_NONLINEAR_CG) b += 72 * V;
    if (o.kspace == COMBO_STAGGERED_DFMG) b += 8 * 81 * V + 192 * nb;
    return b;
}

struct ServeReq {
    int64_t id = 0;
    HostProblem hp;
    combo_options opt;
    int64_t footprint = 0;
    enum { QUEUED, RUNNING, DONE } st = QUEUED;
    int rc = 0;
    std::string err;
    std::vector<double> Pbar, resid, F, P, Pphase;
    std::vector<int32_t> iters, cg;
    combo_result res{};
    double t_submit = 0, t_start = 0, t_done = 0;
    SolveBase* live = nullptr;
    bool cancel = false;
    bool batched = false;  // running in a batch with other requests
};

}  // namespace

struct combo_server {
    int device = 0;
    int slots = 1;
    int64_t budget = 0;
    int keep_fields = 0;
    int batch_max = 1;
    int64_t batch_max_voxels = 0;
    int64_t batches = 0, batched_requests = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<ServeReq*> queue;
    std::map<int64_t, ServeReq*> reqs;
    int64_t next_id = 1, in_use = 0, submitted = 0, completed = 0, failed = 0;
    int running = 0, peak_running = 0;
    bool stopping = false;
    std::vector<double> latency;
    std::vector<std::thread> workers;
};

static ServeReq* pick_request(combo_server* S)
{
    for (auto it = S->queue.begin(); it != S->queue.end(); ++it) {
        ServeReq* r = *it;
        if (S->in_use + r->footprint <= S->budget || S->running == 0) {
            S->queue.erase(it);
            return r;
        }
    }
    return nullptr;
}

static bool batchable(const combo_server* S, const ServeReq* r)
{
    const int64_t V = (int64_t)r->hp.n[0] * r->hp.n[1] * r->hp.n[2];
    return S->batch_max >= 2 && r->opt.solver == COMBO_NEWTON_CG && r->opt.kspace != COMBO_STAGGERED_DFMG &&
           !r->cancel && V <= S->batch_max_voxels;
}

// a request that may share a batch with `first`: same grid, cell size and options
static bool compatible(const ServeReq* first, const ServeReq* r)
{
    for (int j = 0; j < 3; j++)
        if (r->hp.n[j] != first->hp.n[j] || r->hp.l[j] != first->hp.l[j]) return false;
    return std::memcmp(&r->opt, &first->opt, sizeof(combo_options)) == 0;
}

// the admitted request plus the queued requests it can be batched with
// (called with S->mu held; r already left the queue, its footprint is not yet counted)
static void gather_batch(combo_server* S, ServeReq* r, std::vector<ServeReq*>& batch)
{
    batch.assign(1, r);
    if (!batchable(S, r)) return;
    int64_t mem = S->in_use + r->footprint;
    for (auto it = S->queue.begin(); it != S->queue.end() && (int)batch.size() < S->batch_max;) {
        ServeReq* q = *it;
        if (batchable(S, q) && compatible(r, q) && mem + q->footprint <= S->budget) {
            mem += q->footprint;
            batch.push_back(q);
            it = S->queue.erase(it);
        } else {
            ++it;
        }
    }
}

// result buffers of a request and its combo_result pointing at them
static combo_result request_buffers(ServeReq* r, int32_t n_steps, int64_t V, bool fields)
{
    r->Pbar.assign(9 * (size_t)n_steps, 0.0);
    r->Pphase.assign(18 * (size_t)n_steps, 0.0);
    r->resid.assign(n_steps, 0.0);
    r->iters.assign(n_steps, 0);
    r->cg.assign(n_steps, 0);
    combo_result res{};
    res.Pbar = r->Pbar.data();
    res.Pbar_phase = r->Pphase.data();
    res.resid = r->resid.data();
    res.iters = r->iters.data();
    res.cg_iters = r->cg.data();
    res.mem = COMBO_MEM_HOST;
    if (fields) {
        r->F.assign(9 * (size_t)V, 0.0);
        r->P.assign(9 * (size_t)V, 0.0);
        res.F_out = r->F.data();
        res.P_out = r->P.data();
    }
    return res;
}

static void keep_result(ServeReq* r, const combo_result& res)
{
    r->res = res;
    r->res.Pbar = nullptr;
    r->res.Pbar_phase = nullptr;
    r->res.F_out = r->res.P_out = nullptr;
    r->res.resid = nullptr;
    r->res.iters = r->res.cg_iters = nullptr;
}

static void run_request(ServeReq* r, combo_ctx* wctx, combo_server* S)
{
    SolveBase* impl = nullptr;
    int rc;
    const int32_t n_steps = r->hp.n_steps;
    const int64_t V = (int64_t)r->hp.n[0] * r->hp.n[1] * r->hp.n[2];
    rc = make_solve(wctx, std::move(r->hp), r->opt, &impl);
    const bool inited = (rc == 0);
    if (inited) {
        {
            std::lock_guard<std::mutex> lk(S->mu);
            r->live = impl;
            if (r->cancel) impl->request_cancel();
        }
        rc = impl->advance(0);
    }
    const std::string msg = g_err;
    combo_result res = request_buffers(r, n_steps, V, S->keep_fields && !rc);
    const int rc2 = inited ? impl->finish(&res) : rc;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        r->live = nullptr;
    }
    delete impl;
    keep_result(r, res);
    r->rc = rc ? rc : (rc2 < 0 ? rc2 : 0);
    r->err = rc ? msg : g_err;
    if (rc == COMBO_E_CUDA && msg.find("memory") != std::string::npos) r->rc = COMBO_E_OOM;
}

// requests of one batch (>= 2) solved together by one combo_solve_batch
static void run_batch_requests(std::vector<ServeReq*>& batch, combo_ctx* wctx, combo_server* S)
{
    const int B = (int)batch.size();
    std::vector<HostProblem> hs(B);
    std::vector<int32_t> steps(B);
    const int64_t V = (int64_t)batch[0]->hp.n[0] * batch[0]->hp.n[1] * batch[0]->hp.n[2];
    for (int b = 0; b < B; b++) {
        steps[b] = batch[b]->hp.n_steps;
        hs[b] = std::move(batch[b]->hp);
    }
    SolveBase* impl = nullptr;
    int rc = make_solve(wctx, std::move(hs), batch[0]->opt, &impl);
    if (!rc) {
        {
            std::lock_guard<std::mutex> lk(S->mu);
            for (ServeReq* r : batch) r->live = impl;
        }
        rc = impl->run_batch();
    }
    std::string msg = g_err;
    std::vector<combo_result> res(B);
    for (int b = 0; b < B; b++) res[b] = request_buffers(batch[b], steps[b], V, S->keep_fields && !rc);
    if (!rc) {
        rc = impl->batch_results(res.data());
        if (rc) msg = g_err;
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        for (ServeReq* r : batch) r->live = nullptr;
    }
    delete impl;
    for (int b = 0; b < B; b++) {
        ServeReq* r = batch[b];
        keep_result(r, res[b]);
        r->rc = rc;
        r->err = rc ? msg : "";
        if (rc == COMBO_E_CUDA && msg.find("memory") != std::string::npos) r->rc = COMBO_E_OOM;
        if (!rc && r->cancel) {
            r->rc = COMBO_E_CANCELLED;
            r->err = "request cancelled";
        }
    }
}

static void server_worker(combo_server* S)
{
    cudaSetDevice(S->device);
    combo_ctx wctx;
    wctx.device = S->device;
    wctx.own_stream = true;
    if (cudaStreamCreateWithFlags(&wctx.stream, cudaStreamNonBlocking) != cudaSuccess) wctx.stream = nullptr;
    std::vector<ServeReq*> batch;
    for (;;) {
        ServeReq* r = nullptr;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] {
                if (S->stopping) return true;
                r = pick_request(S);
                return r != nullptr;
            });
            if (!r) break;  // stopping
            gather_batch(S, r, batch);
            for (ServeReq* q : batch) {
                q->st = ServeReq::RUNNING;
                q->batched = batch.size() > 1;
                q->t_start = now_s();
                S->in_use += q->footprint;
                S->running++;
            }
            S->peak_running = std::max(S->peak_running, S->running);
            if (batch.size() > 1) {
                S->batches++;
                S->batched_requests += (int64_t)batch.size();
            }
        }
        if (batch.size() > 1)
            run_batch_requests(batch, &wctx, S);
        else
            run_request(r, &wctx, S);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            for (ServeReq* q : batch) {
                q->st = ServeReq::DONE;
                q->t_done = now_s();
                S->in_use -= q->footprint;
                S->running--;
                if (q->rc == 0) {
                    S->completed++;
                    S->latency.push_back(q->t_done - q->t_submit);
                } else {
                    S->failed++;
                }
            }
        }
        S->cv_done.notify_all();
        S->cv_work.notify_all();
    }
    if (wctx.stream) cudaStreamDestroy(wctx.stream);
}

extern "C" int combo_server_create(combo_ctx* ctx, const combo_server_opts* o, combo_server** out)
{
    if (!ctx || !out) return fail(COMBO_E_INVALID_ARG, "null context or output");
    CK(cudaSetDevice(ctx->device));
    combo_server* S = new combo_server();
    S->device = ctx->device;
    S->slots = (o && o->max_slots > 0) ? o->max_slots : 4;
    S->keep_fields = o ? o->keep_fields : 0;
    S->batch_max = (o && o->batch_max > 1) ? o->batch_max : 1;
    S->batch_max_voxels = (o && o->batch_max_voxels > 0) ? o->batch_max_voxels : (int64_t)96 * 96 * 96;
    if (o && o->hbm_budget_bytes > 0) {
        S->budget = o->hbm_budget_bytes;
    } else {
        size_t fr = 0, tot = 0;
        CK(cudaMemGetInfo(&fr, &tot));
        S->budget = (int64_t)(0.85 * (double)fr);
    }
    for (int i = 0; i < S->slots; i++) S->workers.emplace_back(server_worker, S);
    *out = S;
    return COMBO_OK;
}

extern "C" void combo_server_destroy(combo_server* S)
{
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
        for (ServeReq* r : S->queue) {
            r->st = ServeReq::DONE;
            r->rc = COMBO_E_CANCELLED;
        }
        S->queue.clear();
        for (auto& kv : S->reqs)
            if (kv.second->live) kv.second->live->request_cancel();
    }
    S->cv_work.notify_all();
    for (auto& t : S->workers) t.join();
    for (auto& kv : S->reqs) delete kv.second;
    delete S;
}

extern "C" int combo_submit(combo_server* S, const combo_problem* p, const combo_options* o_in, int64_t* ticket)
{
    if (!S || !ticket) return fail(COMBO_E_INVALID_ARG, "null server or ticket");
    combo_options o;
    if (o_in)
        o = *o_in;
    else
        combo_options_default(&o);
    int rc = check_options(o);
    if (rc) return rc;
    ServeReq* r = new ServeReq();
    if ((rc = load_problem(p, &o, r->hp))) {
        delete r;
        return rc;
    }
    r->opt = o;
    r->footprint = footprint_of(r->hp, o);
    if (r->footprint > S->budget) {
        delete r;
        return fail(COMBO_E_OOM, "the solve does not fit the server's device-memory budget");
    }
    r->t_submit = now_s();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stopping) {
            delete r;
            return fail(COMBO_E_INVALID_ARG, "server is stopping");
        }
        r->id = S->next_id++;
        S->reqs[r->id] = r;
        S->queue.push_back(r);
        S->submitted++;
        *ticket = r->id;
    }
    S->cv_work.notify_one();
    return COMBO_OK;
}

// copy a finished request into the caller's result (host memory) and release it
static int collect(combo_server* S, ServeReq* r, combo_result* out)
{
    int rc = r->rc;
    if (out) {
        const int32_t ns = (int32_t)r->iters.size();
        if (out->Pbar && !r->Pbar.empty()) std::memcpy(out->Pbar, r->Pbar.data(), 8 * r->Pbar.size());
        if (out->Pbar_phase && !r->Pphase.empty())
            std::memcpy(out->Pbar_phase, r->Pphase.data(), 8 * r->Pphase.size());
        if (out->iters && ns) std::memcpy(out->iters, r->iters.data(), 4 * (size_t)ns);
        if (out->cg_iters && ns) std::memcpy(out->cg_iters, r->cg.data(), 4 * (size_t)ns);
        if (out->resid && ns) std::memcpy(out->resid, r->resid.data(), 8 * (size_t)ns);
        if (out->F_out && !r->F.empty()) std::memcpy(out->F_out, r->F.data(), 8 * r->F.size());
        if (out->P_out && !r->P.empty()) std::memcpy(out->P_out, r->P.data(), 8 * r->P.size());
        out->steps_done = r->res.steps_done;
        out->nr_iters = r->res.nr_iters;
        out->n_backproj = r->res.n_backproj;
        out->n_laminate_evals = r->res.n_laminate_evals;
        out->n_operator = r->res.n_operator;
        out->n_operator_fp64 = r->res.n_operator_fp64;
    }
    if (rc) g_err = r->err.empty() ? "request failed" : r->err;
    S->reqs.erase(r->id);
    delete r;
    return rc;
}

extern "C" int combo_poll(combo_server* S, int64_t ticket, combo_result* out)
{
    if (!S) return fail(COMBO_E_INVALID_ARG, "null server");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(COMBO_E_INVALID_ARG, "unknown ticket");
    if (it->second->st != ServeReq::DONE) return COMBO_PENDING;
    return collect(S, it->second, out);
}

extern "C" int combo_wait(combo_server* S, int64_t ticket, int64_t timeout_ms, combo_result* out)
{
    if (!S) return fail(COMBO_E_INVALID_ARG, "null server");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(COMBO_E_INVALID_ARG, "unknown ticket");
    ServeReq* r = it->second;
    auto done = [&] { return r->st == ServeReq::DONE; };
    if (timeout_ms < 0)
        S->cv_done.wait(lk, done);
    else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done))
        return fail(COMBO_E_TIMEOUT, "request not finished within the timeout");
    return collect(S, r, out);
}

extern "C" int combo_cancel(combo_server* S, int64_t ticket)
{
    if (!S) return fail(COMBO_E_INVALID_ARG, "null server");
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->reqs.find(ticket);
        if (it == S->reqs.end()) return fail(COMBO_E_INVALID_ARG, "unknown ticket");
        ServeReq* r = it->second;
        if (r->st == ServeReq::QUEUED) {
            for (auto q = S->queue.begin(); q != S->queue.end(); ++q)
                if (*q == r) {
                    S->queue.erase(q);
                    break;
                }
            r->st = ServeReq::DONE;
            r->rc = COMBO_E_CANCELLED;
            r->err = "cancelled before it started";
            S->failed++;
        } else if (r->st == ServeReq::RUNNING) {
            r->cancel = true;
            // a batch is not stopped for one of its requests: that request's
            // result is discarded when the batch ends
            if (r->live && !r->batched) r->live->request_cancel();
        }
    }
    S->cv_done.notify_all();
    return COMBO_OK;
}

extern "C" int combo_server_stats(combo_server* S, combo_serving_stats* st)
{
    if (!S || !st) return fail(COMBO_E_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> lk(S->mu);
    std::memset(st, 0, sizeof(*st));
    st->submitted = S->submitted;
    st->completed = S->completed;
    st->failed = S->failed;
    st->queued = (int64_t)S->queue.size();
    st->running = S->running;
    st->peak_running = S->peak_running;
    st->in_use_bytes = S->in_use;
    st->budget_bytes = S->budget;
    st->batches = S->batches;
    st->batched_requests = S->batched_requests;
    if (!S->latency.empty()) {
        std::vector<double> l = S->latency;
        std::sort(l.begin(), l.end());
        auto pct = [&](double q) {
            const double pos = q * (double)(l.size() - 1);
            const size_t i = (size_t)pos;
            const double f = pos - (double)i;
            return (i + 1 < l.size()) ? l[i] * (1 - f) + l[i + 1] * f : l[i];
        };
        st->p50_seconds = pct(0.5);
        st->p99_seconds = pct(0.99);
        double s = 0;
        for (double v : l) s += v;
        st->mean_seconds = s / (double)l.size();
    }
    return COMBO_OK;
}
