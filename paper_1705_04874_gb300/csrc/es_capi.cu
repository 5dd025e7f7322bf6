// Host side of libes.so: the C ABI declared in include/es.h.
//
// A model owns, in one device allocation, the nine field totals (vx vy vz
// sxx syy szz sxy sxz syz), eight FP32 material arrays and, for each axis,
// the split part of every field driven by that axis's derivatives -- but only
// inside that axis's PML slabs ([0, L) and [n-1-L, n)), the only cells where a
// split evolves differently from the total (Sec. II-B split-field PML).
// A time step (Sec. II-A leapfrog) is 3 velocity passes + 3 stress passes
// (fft_pass.cuh), point-source injection and 4C recording; es_run captures it
// as a CUDA graph and replays it.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <mutex>
#include <new>
#include <sstream>
#include <string>
#include <thread>
#include <vector>

#include <sys/stat.h>

#include <nvtx3/nvToolsExt.h>

#include "../../include/es.h"
#include "es_internal.h"

using namespace es;

namespace {

thread_local char g_err[512] = "";

int cuda_fail(cudaError_t e, const char* what)
{
    snprintf(g_err, sizeof g_err, "%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? ES_ERR_OOM : ES_ERR_CUDA;
}

#define CK(call)                                                        \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);             \
    } while (0)


// NVTX range over a scope (header-only NVTX v3: a no-op unless a profiler
// injects itself).  The solver's API calls and the phases of es_run carry
// ranges; inside a time step, each pass launch is marked while the step is
// captured into its CUDA graph (graph replays run without host calls).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Every device allocation of the solver goes through dev_alloc / dev_free: they
// count the allocations the library holds (es_debug_live_allocations) and,
// for testing the error paths, can make the n-th allocation from a chosen
// point fail as an out-of-memory error before cudaMalloc is called
// (es_fault_inject_alloc, or ES_FAULT_ALLOC=n from the first allocation).
std::atomic<long long> g_alloc_countdown{0};
std::atomic<long long> g_live_allocs{0};
std::once_flag g_fault_env_once;

template <class T>
cudaError_t dev_alloc(T** p, size_t bytes)
{
    std::call_once(g_fault_env_once, [] {
        if (const char* v = std::getenv("ES_FAULT_ALLOC")) g_alloc_countdown = std::atoll(v);
    });
    if (g_alloc_countdown.load() > 0 && g_alloc_countdown.fetch_sub(1) == 1) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    void* q = nullptr;
    const cudaError_t e = cudaMalloc(&q, bytes);
    *p = static_cast<T*>(q);
    if (e == cudaSuccess && q) ++g_live_allocs;
    return e;
}

template <class T>
void dev_free(T* p)
{
    if (!p) return;
    cudaFree(const_cast<void*>(static_cast<const void*>(p)));
    --g_live_allocs;
}

bool is_device_ptr(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// copy n elements of T from host or device memory into a host vector
template <class T>
int fetch(const T* src, size_t n, std::vector<T>& out, cudaStream_t st)
{
    out.resize(n);
    if (n == 0) return ES_OK;
    if (is_device_ptr(src)) {
        CK(cudaMemcpyAsync(out.data(), src, n * sizeof(T), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    } else {
        std::memcpy(out.data(), src, n * sizeof(T));
    }
    return ES_OK;
}

// Runs f(lo, hi) over [0, n) split into contiguous blocks of at least `grain`
// items on the host's cores (model setup: the input checks; no shared writes
// between blocks).
template <class F>
void parallel_for(size_t n, F f, size_t grain = 1)
{
    const unsigned hw = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    const size_t nt = std::min<size_t>(hw, std::max<size_t>(1, n / std::max<size_t>(1, grain)));
    if (nt <= 1) {
        f((size_t)0, n);
        return;
    }
    std::vector<std::thread> th;
    th.reserve(nt);
    for (size_t t = 0; t < nt; ++t) th.emplace_back(f, n * t / nt, n * (t + 1) / nt);
    for (auto& x : th) x.join();
}

int g_prepared_dev = -1;

// On-disk cache of autotuned FFT plans: lines "device|kind|n|ra|rb" in
// $ES_TUNE_CACHE, else $HOME/.cache/es_fft_plans.txt.
std::string plan_cache_path()
{
    if (const char* p = std::getenv("ES_TUNE_CACHE")) return p;
    if (const char* h = std::getenv("HOME")) return std::string(h) + "/.cache/es_fft_plans.txt";
    return "";
}

std::string device_name()
{
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
    std::string n = prop.name;
    for (char& c : n)
        if (c == '|' || c == '\n') c = ' ';
    return n;
}

void load_plan_cache()
{
    const std::string path = plan_cache_path();
    if (path.empty()) return;
    std::ifstream in(path);
    const std::string dev = device_name();
    std::string line;
    while (std::getline(in, line)) {
        std::stringstream ss(line);
        std::string d, f;
        int v[4], k = 0;
        if (!std::getline(ss, d, '|') || d != dev) continue;
        while (k < 4 && std::getline(ss, f, '|')) v[k++] = std::atoi(f.c_str());
        if (k == 4) plan_select(v[0], v[1], v[2], v[3]);
    }
}

void store_plan_cache(const std::vector<std::string>& keys, const std::vector<std::string>& lines)
{
    const std::string path = plan_cache_path();
    if (path.empty()) return;
    std::vector<std::string> keep;
    {
        std::ifstream in(path);
        std::string line;
        while (std::getline(in, line)) {
            bool replaced = false;
            for (const auto& k : keys) replaced |= line.rfind(k, 0) == 0;
            if (!replaced && !line.empty()) keep.push_back(line);
        }
    }
    for (const auto& l : lines) keep.push_back(l);
    const size_t slash = path.rfind('/');
    if (slash != std::string::npos && slash > 0) mkdir(path.substr(0, slash).c_str(), 0755);  // one missing level
    std::ofstream out(path, std::ios::trunc);
    for (const auto& l : keep) out << l << "\n";
}

int ensure_prepared()
{
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (g_prepared_dev != dev) {
        CK(prepare_pass_kernels());
        load_plan_cache();
        g_prepared_dev = dev;
    }
    if (!bounds_init()) return cuda_fail(cudaErrorMemoryAllocation, "bounds word");
    return ES_OK;
}

// Axis lengths: an FFT plan (pass_plans.h), else the circulant pass up to
// CIRC_MAX_N (circ_pass.cu).  With an odd nx the y and z FFT passes move their
// x-adjacent pencil pairs as single floats (pass_kernels_odd.cu).
bool fft_plan(int n) { int a, b; return plan_radices(n, &a, &b) != 0; }
bool axis_ok(int n) { return n >= 3 && n <= CIRC_MAX_N; }
bool fft_axis(int n, int) { return fft_plan(n); }

// exp(-2 pi i m / n) and the staggered multipliers H = i kappa exp(sign i kappa d / 2) of
// an axis, in FP64 then rounded.  The FFT passes evaluate D = N + far (es_internal.h):
// g (gp for D(+), gm for D(-)) are the NEAR_TAPS kernel entries c_l at offsets
// near_ofs(sign) .. +NEAR_TAPS-1 rounded to FP32, and the tables hold
// (H - sum_t g_t exp(2 pi i m (near_ofs + t) / n)) / n, the FP32 taps subtracted so that
// near + far equals D exactly up to the rounding of the tables.  Axes of NEAR_TAPS cells
// or fewer keep the whole multiplier (g = 0).  For a circulant axis also the kernels
// c_l = sum_m H_m / n exp(2 pi i m l / n) (real: H is Hermitian, Nyquist included).
void axis_tables(int n, double d, std::vector<float2>& tw, std::vector<float2>& hp, std::vector<float2>& hm,
                 float* gp, float* gm, std::vector<double>* ckp = nullptr, std::vector<double>* ckm = nullptr)
{
    const double pi = 3.14159265358979323846;
    tw.resize(n);
    hp.resize(n);
    hm.resize(n);
    std::vector<double> hr[2], hi[2];
    for (int s = 0; s < 2; ++s) {
        hr[s].resize(n);
        hi[s].resize(n);
    }
    for (int m = 0; m < n; ++m) {
        const double a = 2.0 * pi * (double)m / (double)n;
        tw[m] = make_float2((float)std::cos(a), (float)(-std::sin(a)));
        const int mk = (2 * m < n) ? m : m - n;  // even n: bin n/2 -> -n/2
        const double kap = 2.0 * pi * (double)mk / ((double)n * d);
        for (int s = 0; s < 2; ++s) {
            const double ph = (s == 0 ? 0.5 : -0.5) * kap * d;
            hr[s][m] = -kap * std::sin(ph) / n;
            hi[s][m] = kap * std::cos(ph) / n;
        }
    }
    // c_l of D(+) (s = 0) or D(-) (s = 1), angles reduced exactly in integers
    auto kernel_entry = [&](int s, int l) {
        double acc = 0.0;
        for (int m = 0; m < n; ++m) {
            const long long ml = ((long long)m * l) % n;
            const double a = 2.0 * pi * (double)ml / (double)n;
            acc += hr[s][m] * std::cos(a) - hi[s][m] * std::sin(a);
        }
        return acc;
    };
    for (int s = 0; s < 2; ++s) {
        float* g = s == 0 ? gp : gm;
        const int ofs = near_ofs(s == 0 ? +1 : -1);
        std::vector<double> nr(n, 0.0), ni(n, 0.0);  // H_near / n
        // the taps in antisymmetric pairs, g[NEAR_TAPS - 1 - t] = -g[t] (exact for the staggered
        // kernel up to FP64 roundoff; enforced here so the passes can sum differences)
        for (int t = 0; t < NEAR_PAIRS; ++t) {
            g[t] = g[NEAR_TAPS - 1 - t] = 0.f;
            if (n <= NEAR_TAPS) continue;
            const double lo = kernel_entry(s, ((-(ofs + t)) % n + n) % n);  // (D f)_i = sum_l c_l f_{i - l}
            const double hi = kernel_entry(s, ((-(ofs + NEAR_TAPS - 1 - t)) % n + n) % n);
            g[t] = (float)(0.5 * (lo - hi));
            g[NEAR_TAPS - 1 - t] = -g[t];
        }
        for (int t = 0; t < NEAR_TAPS; ++t) {
            if (n <= NEAR_TAPS) continue;
            const int delta = ofs + t;                      // (N f)_i gains g_t f_{i + delta}
            for (int m = 0; m < n; ++m) {
                const long long md = (((long long)m * delta) % n + n) % n;
                const double a = 2.0 * pi * (double)md / (double)n;
                nr[m] += (double)g[t] * std::cos(a) / n;
                ni[m] += (double)g[t] * std::sin(a) / n;
            }
        }
        for (int m = 0; m < n; ++m)
            (s == 0 ? hp : hm)[m] = make_float2((float)(hr[s][m] - nr[m]), (float)(hi[s][m] - ni[m]));
    }
    if (!ckp || !ckm) return;
    ckp->resize(n);
    ckm->resize(n);
    for (int l = 0; l < n; ++l) {
        (*ckp)[l] = kernel_entry(0, l);
        (*ckm)[l] = kernel_entry(1, l);
    }
}

struct Src {
    int kind;
    int smooth = 0;
    int sim;
    int pos[3];
    double m[6];
    float* d_w;
    int nw;
};

const int KPS_MAX = 10;  // kernels per step (8, +1 with force sources, +1 with viscosity)

}  // namespace

struct es_model {
    int nx, ny, nz;
    size_t ncell;
    double d[3];
    int L;
    double alpha0 = 2.0, cref = 0.0;
    cudaStream_t stream = nullptr;
    std::vector<float> rho, cs;  // host copies (seabed rule, force scaling)
    float cp_max = 0.f;
    char* pool = nullptr;   // materials, tables, counters
    int nsim = 1;           // independent simulations sharing the materials
    char* fpool = nullptr;  // field totals and slab splits, [field][sim][cell]
    float* f[NFIELD] = {};
    float* slab[3][NFIELD] = {};
    float* mat[NMAT] = {};
    float** d_fields = nullptr;
    float2 *tw[3] = {}, *hp[3] = {}, *hm[3] = {};
    float gp[3][NEAR_TAPS] = {}, gm[3][NEAR_TAPS] = {};  // near taps of D(+), D(-) per axis (FFT passes)
    float *ckp[3] = {}, *ckm[3] = {};  // circulant kernels (axes without an FFT pass)
    float *ckp_lo[3] = {}, *ckm_lo[3] = {};  // their low parts (compensated mode)
    __nv_bfloat16* ctc[3] = {};               // long circulant axes: kernel matrices split in three BF16 parts
    float* ctc_scratch = nullptr;             // their z pass's derivatives [job][sim][cell] (circ_tc.cu)
    int prec = ES_PREC_FP32;
    // Kelvin-Voigt viscosity (chi = tau lambda, eta = tau mu): v^{n-1/2} kept per velocity
    // component and the stress passes' combined source w = (dt + tau) v^{n+1/2} - tau v^{n-1/2},
    // [3][sim][cell] each, allocated with the first viscous run
    double tau = 0.0;
    char* vpool = nullptr;
    int vpool_nsim = 0;
    float* vold = nullptr;
    float* wv = nullptr;
    float *pc[3] = {}, *ps[3] = {};
    int* d_int = nullptr;  // [0] step counter, [1] current step, [2] non-finite flag
    std::vector<Src> srcs;
    SourceDev* d_src = nullptr;
    int d_src_cap = 0;
    float* d_rec = nullptr;
    size_t rec_cap = 0;
    float* d_out = nullptr;
    size_t out_cap = 0;
    long long* d_rcv = nullptr;
    int rcv_cap = 0;
    long long steps_done = 0;
    // fused point sources and receivers (FFT passes only): per-CTA cell lists of the velocity z,
    // stress y and stress z passes, one device buffer (build_special)
    bool fused = false;
    char* d_sp = nullptr;
    size_t sp_cap = 0;
    const int* sp_off[3] = {};
    const SpecialCell* sp_cells[3] = {};
    int sp_n[3] = {};  // entries of each list
    cudaEvent_t ev[2 * KPS_MAX] = {};
    float last_ms[KPS_MAX] = {};
    int n_last = 0;
};

namespace {

bool has_split(int f, int a)
{
    return !((f == SXY && a == 2) || (f == SXZ && a == 1) || (f == SYZ && a == 0));
}
bool stag_along(int f, int a)
{
    switch (f) {
    case VX: return a == 0;
    case VY: return a == 1;
    case VZ: return a == 2;
    case SXY: return a == 0 || a == 1;
    case SXZ: return a == 0 || a == 2;
    case SYZ: return a == 1 || a == 2;
    default: return false;
    }
}
int axis_len(const es_model* m, int a) { return a == 0 ? m->nx : (a == 1 ? m->ny : m->nz); }
size_t slab_count(const es_model* m, int a) { return m->L > 0 ? m->ncell / axis_len(m, a) * (2 * m->L + 1) : 0; }

int upload_sources(es_model* m, double dt)
{
    std::vector<SourceDev> h(m->srcs.size());
    const double vol = m->d[0] * m->d[1] * m->d[2];
    for (size_t e = 0; e < m->srcs.size(); ++e) {
        const Src& s = m->srcs[e];
        SourceDev& d = h[e];
        d.kind = s.kind;
        d.smooth = s.smooth;
        d.sim = s.sim;
        d.cell = (long long)s.pos[0] + (long long)m->nx * ((long long)s.pos[1] + (long long)m->ny * s.pos[2]);
        d.w = s.d_w;
        d.nw = s.nw;
        for (int c = 0; c < 6; ++c) d.m[c] = 0.f;
        if (s.kind == 0) {
            for (int c = 0; c < 6; ++c) d.m[c] = (float)s.m[c];
        } else {
            // dt f_c / (rho at v_c's staggered point * dx dy dz)
            for (int c = 0; c < 3; ++c) {
                int p1[3] = {s.pos[0], s.pos[1], s.pos[2]};
                p1[c] = (p1[c] + 1) % axis_len(m, c);
                const size_t q0 = (size_t)d.cell;
                const size_t q1 = (size_t)p1[0] + (size_t)m->nx * ((size_t)p1[1] + (size_t)m->ny * p1[2]);
                const double b = 2.0 / ((double)m->rho[q0] + (double)m->rho[q1]);
                d.m[c] = (float)(dt * s.m[c] * b / vol);
            }
        }
    }
    if ((int)h.size() > m->d_src_cap) {
        dev_free(m->d_src);
        m->d_src = nullptr;
        m->d_src_cap = 0;
        CK(dev_alloc(&m->d_src, sizeof(SourceDev) * h.size()));
        m->d_src_cap = (int)h.size();
    }
    if (!h.empty()) {
        CK(cudaMemcpyAsync(m->d_src, h.data(), sizeof(SourceDev) * h.size(), cudaMemcpyHostToDevice, m->stream));
        CK(cudaStreamSynchronize(m->stream));
    }
    return ES_OK;
}

// whether the point sources and receivers of a run go into the passes (every axis an FFT pass,
// no smoothed source) or through the separate injection and recording kernels
bool fused_sources(const es_model* m);

// twiddles, spectral multipliers and (for a circulant axis) the kernels of axis a
// whether axis a of the model runs through the circulant passes
bool circ_axis(const es_model* m, int a) { return m->prec == ES_PREC_COMPENSATED || !fft_axis(axis_len(m, a), m->nx); }

// twiddles, spectral multipliers and (for a circulant axis) the kernels of axis
// a, the latter as FP32 high parts and FP32 low parts (c - (float)c)
cudaError_t upload_axis_tables(es_model* m, int a)
{
    const int n = axis_len(m, a);
    std::vector<float2> tw, hp, hm;
    std::vector<double> ckp, ckm;
    const bool circ = circ_axis(m, a);
    axis_tables(n, m->d[a], tw, hp, hm, m->gp[a], m->gm[a], circ ? &ckp : nullptr, circ ? &ckm : nullptr);
    cudaError_t e = cudaMemcpy(m->tw[a], tw.data(), tw.size() * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->hp[a], hp.data(), hp.size() * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->hm[a], hm.data(), hm.size() * 8, cudaMemcpyHostToDevice);
    if (circ) {
        std::vector<float> hi(4 * (size_t)n);
        for (int l = 0; l < n; ++l) {
            const float p = (float)ckp[l], q = (float)ckm[l];
            hi[l] = p;
            hi[n + l] = q;
            hi[2 * n + l] = (float)(ckp[l] - (double)p);
            hi[3 * n + l] = (float)(ckm[l] - (double)q);
        }
        if (e == cudaSuccess) e = cudaMemcpy(m->ckp[a], hi.data(), n * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(m->ckm[a], hi.data() + n, n * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(m->ckp_lo[a], hi.data() + 2 * n, n * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(m->ckm_lo[a], hi.data() + 3 * n, n * 4, cudaMemcpyHostToDevice);
        // long axes on the tensor cores (ES_PREC_FP32_TC): the dense matrices C[o][i] =
        // c[(o - i) mod n] of the far parts of D+ and D- (the kernel less its FP32 near taps, which
        // the update kernel adds in FP32), padded to whole 64-row boxes and split into three BF16
        // parts (c = c0 + c1 + c2 to about 2^-24)
        if (e == cudaSuccess && m->prec == ES_PREC_FP32_TC && n >= CIRC_TC_N && n <= CIRC_MAX_N) {
            const int np = (n + 63) / 64 * 64;
            const size_t mat = (size_t)np * np;
            std::vector<__nv_bfloat16> sp(6 * mat, __float2bfloat16(0.f));
            for (int sgn = 0; sgn < 2; ++sgn) {
                std::vector<double> ck = sgn == 0 ? ckp : ckm;
                const float* g = sgn == 0 ? m->gp[a] : m->gm[a];
                for (int t = 0; t < NEAR_TAPS; ++t) {
                    const int delta = near_ofs(sgn == 0 ? +1 : -1) + t;  // (N f)_o gains g_t f_{o + delta}
                    ck[(size_t)(((-delta) % n) + n) % n] -= (double)g[t];
                }
                for (int o = 0; o < n; ++o)
                    for (int i = 0; i < n; ++i) {
                        const double x = ck[(size_t)(((o - i) % n + n) % n)];
                        const __nv_bfloat16 h0 = __double2bfloat16(x);
                        const double r1 = x - (double)__bfloat162float(h0);
                        const __nv_bfloat16 h1 = __double2bfloat16(r1);
                        const double r2 = r1 - (double)__bfloat162float(h1);
                        const size_t q = (size_t)o * np + i;
                        sp[(size_t)(3 * sgn) * mat + q] = h0;
                        sp[(size_t)(3 * sgn + 1) * mat + q] = h1;
                        sp[(size_t)(3 * sgn + 2) * mat + q] = __double2bfloat16(r2);
                    }
            }
            if (!m->ctc[a]) e = dev_alloc(&m->ctc[a], sp.size() * sizeof(__nv_bfloat16));
            if (e == cudaSuccess)
                e = cudaMemcpy(m->ctc[a], sp.data(), sp.size() * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice);
        }
    }
    return e;
}

bool fused_sources(const es_model* m)
{
    for (int a = 0; a < 3; ++a)
        if (circ_axis(m, a)) return false;
    return std::none_of(m->srcs.begin(), m->srcs.end(), [](const Src& s) { return s.smooth != 0; });
}

// The per-CTA cell lists of the fused passes (PassParams::sp_off / sp): for the velocity z pass
// (SP_VEL_Z) the point forces, then the receivers; for the stress y pass (SP_STR_Y) the moment
// sources; for the stress z pass (SP_STR_Z) the moment sources, then the receivers.  A y or z pass
// CTA owns 32 consecutive x at one z (y pass) or one y (z pass) of one simulation: blockIdx.x =
// sim + nsim (x / 32 + ntx outer).  Sources keep their order (the order the injection kernel adds
// them in).
int build_special(es_model* m, const std::vector<long long>& rcv_cells)
{
    const int ntx = (m->nx + 31) / 32;
    const int axis_of[3] = {2, 1, 2};
    std::vector<SpecialCell> cells[3];
    std::vector<int> off[3];
    for (int k = 0; k < 3; ++k) {
        const int mode = k + 1, axis = axis_of[k];
        const size_t nb = (size_t)ntx * (axis == 1 ? m->nz : m->ny) * m->nsim;
        auto block_of = [&](long long cell, int sim) {
            const long long x = cell % m->nx, y = (cell / m->nx) % m->ny, z = cell / ((long long)m->nx * m->ny);
            const long long tile = x / 32 + (long long)ntx * (axis == 1 ? z : y);
            return (size_t)sim + (size_t)m->nsim * (size_t)tile;
        };
        std::vector<std::vector<SpecialCell>> per(nb);
        for (size_t e = 0; e < m->srcs.size(); ++e) {
            const Src& s = m->srcs[e];
            if (s.smooth || (mode == SP_VEL_Z ? s.kind != 1 : s.kind != 0)) continue;
            const long long cell = (long long)s.pos[0] + (long long)m->nx * ((long long)s.pos[1] + (long long)m->ny * s.pos[2]);
            per[block_of(cell, s.sim)].push_back(
                {(long long)s.sim * (long long)m->ncell + cell, s.kind == 1 ? SP_FORCE : SP_MOMENT, (int)e, s.sim});
        }
        if (mode != SP_STR_Y)
            for (int sim = 0; sim < m->nsim; ++sim)
                for (size_t r = 0; r < rcv_cells.size(); ++r)
                    per[block_of(rcv_cells[r], sim)].push_back(
                        {(long long)sim * (long long)m->ncell + rcv_cells[r], SP_RECEIVER, (int)r, sim});
        off[k].assign(nb + 1, 0);
        for (size_t b = 0; b < nb; ++b) {
            off[k][b + 1] = off[k][b] + (int)per[b].size();
            cells[k].insert(cells[k].end(), per[b].begin(), per[b].end());
        }
    }
    const size_t A = 256;
    auto up = [&](size_t b) { return (b + A - 1) / A * A; };
    size_t bytes = 0;
    for (int k = 0; k < 3; ++k) bytes += up(std::max<size_t>(1, cells[k].size()) * sizeof(SpecialCell)) + up(off[k].size() * 4);
    if (bytes > m->sp_cap) {
        dev_free(m->d_sp);
        m->d_sp = nullptr;
        m->sp_cap = 0;
        CK(dev_alloc(&m->d_sp, bytes));
        m->sp_cap = bytes;
    }
    char* cur = m->d_sp;
    for (int k = 0; k < 3; ++k) {
        m->sp_n[k] = (int)cells[k].size();
        m->sp_cells[k] = reinterpret_cast<const SpecialCell*>(cur);
        if (!cells[k].empty())
            CK(cudaMemcpyAsync(cur, cells[k].data(), cells[k].size() * sizeof(SpecialCell), cudaMemcpyHostToDevice,
                               m->stream));
        cur += up(std::max<size_t>(1, cells[k].size()) * sizeof(SpecialCell));
        m->sp_off[k] = reinterpret_cast<const int*>(cur);
        CK(cudaMemcpyAsync(cur, off[k].data(), off[k].size() * 4, cudaMemcpyHostToDevice, m->stream));
        cur += up(off[k].size() * 4);
    }
    CK(cudaStreamSynchronize(m->stream));
    return ES_OK;
}

PassParams make_pass(const es_model* m, int axis, bool stress, float dt)
{
    PassParams p;
    std::memset(&p, 0, sizeof p);
    p.nx = m->nx;
    p.ny = m->ny;
    p.nz = m->nz;
    p.axis = axis;
    p.n = axis_len(m, axis);
    p.njobs = 3;
    p.tw = m->tw[axis];
    p.hp = m->hp[axis];
    p.hm = m->hm[axis];
    p.ckp = m->ckp[axis];
    p.ckm = m->ckm[axis];
    p.ckp_lo = m->ckp_lo[axis];
    p.ckm_lo = m->ckm_lo[axis];
    p.ctc = m->prec == ES_PREC_FP32_TC ? m->ctc[axis] : nullptr;
    p.scratch = m->prec == ES_PREC_FP32_TC ? m->ctc_scratch : nullptr;
    p.circ = circ_axis(m, axis) ? 1 : 0;
    p.comp = m->prec == ES_PREC_COMPENSATED ? 1 : 0;
    p.pc = m->pc[axis];
    p.ps = m->ps[axis];
    p.L = m->L;
    p.dt = dt;
    p.nsim = m->nsim;
    p.fstride = (long long)m->ncell;
    p.sstride = (long long)slab_count(m, axis);
    p.ext_f = p.fstride * m->nsim;
    p.ext_s = p.sstride * m->nsim;
    p.ext_c = p.fstride;
    p.bad = bounds_word();
    auto taps = [&](PassJob& J) {
        for (int t = 0; t < NEAR_TAPS; ++t) J.g[t] = J.sign > 0 ? m->gp[axis][t] : m->gm[axis][t];
    };
    auto single = [&](PassJob& J, int src, int sign, int tgt, int coef) {
        J.src = m->f[src];
        J.kind = JOB_SINGLE;
        J.sign = sign;
        taps(J);
        J.tgt[0] = m->f[tgt];
        J.slab[0] = m->slab[axis][tgt];
        J.coef[0] = m->mat[coef];
        J.stag = stag_along(tgt, axis);
    };
    if (!stress) {
        // dv_i/dt = (1/rho) d sigma_ij / dx_j (Eq. (2)), term along `axis`
        static const int src_tab[3][3] = {{SXX, SXY, SXZ}, {SXY, SYY, SYZ}, {SXZ, SYZ, SZZ}};
        for (int i = 0; i < 3; ++i) {
            const int src = src_tab[axis][i];
            const int sign = (i == axis) ? +1 : -1;  // normal stress -> half index: +; shear -> whole: -
            single(p.job[i], src, sign, VX + i, M_BX + i);
        }
    } else {
        // d sigma_ij/dt = lambda delta_ij dv_k/dx_k + mu (dv_i/dx_j + dv_j/dx_i) (Eq. (2))
        PassJob& J = p.job[0];
        J.src = m->f[VX + axis];
        J.kind = JOB_NORMAL;
        J.sign = -1;
        taps(J);
        J.diag = axis;
        for (int t = 0; t < 3; ++t) {
            J.tgt[t] = m->f[SXX + t];
            J.slab[t] = m->slab[axis][SXX + t];
        }
        J.coef[0] = m->mat[M_LAM];
        J.coef[1] = m->mat[M_MU];
        J.stag = 0;
        // shear terms: d v_b / d x_axis feeds sigma_{axis b}
        int k = 1;
        for (int b = 0; b < 3; ++b) {
            if (b == axis) continue;
            const int lo = std::min(axis, b), hi = std::max(axis, b);
            const int tgt = (lo == 0 && hi == 1) ? SXY : ((lo == 0 && hi == 2) ? SXZ : SYZ);
            const int coef = (tgt == SXY) ? M_MUXY : ((tgt == SXZ) ? M_MUXZ : M_MUYZ);
            single(p.job[k++], VX + b, +1, tgt, coef);
        }
    }
    return p;
}

// Enqueues one time step; with `ev` non-null, events bracket every kernel.
int enqueue_step(es_model* m, float dt, int n_rcv, long long start, cudaStream_t st, cudaEvent_t* ev, int* nk)
{
    int k = 0;
    // under stream capture only cudaEventRecordExternal makes a real record node
    auto mark = [&](bool before) {
        if (ev) cudaEventRecordWithFlags(ev[2 * k + (before ? 0 : 1)], st, cudaEventRecordExternal);
    };
    const bool has_force = std::any_of(m->srcs.begin(), m->srcs.end(), [](const Src& s) { return s.kind == 1; });
    static const char* kVel[3] = {"vel-x", "vel-y", "vel-z"};
    static const char* kStr[3] = {"str-x", "str-y", "str-z"};
    const bool fused = m->fused;
    // the fused passes' source / receiver work (PassParams::sp_mode)
    auto fuse = [&](PassParams& p, int mode) {
        if (!fused) return;
        p.step_now = m->d_int;
        p.sp_mode = mode;
        p.sp_off = m->sp_off[mode - 1];
        p.sp = m->sp_cells[mode - 1];
        p.src = m->d_src;
        p.rec = m->d_rec;
        p.rec_start = start;
        p.n_rcv = n_rcv;
        p.ext_sp = m->sp_n[mode - 1];
        p.ext_rec = (long long)m->rec_cap;
    };
    for (int a = 0; a < 3; ++a) {
        NvtxRange r(kVel[a]);
        PassParams p = make_pass(m, a, false, dt);
        p.pdl = a == 0 ? 2 : 1;  // the x pass reads what the stress half wrote; y and z only add after it
        if (fused && a == 0) p.step_counter = m->d_int;  // step index = counter - 1 from here on
        if (a == 2) fuse(p, SP_VEL_Z);                     // point forces, then the velocity samples
        mark(true);
        CK(launch_pass(p, st));
        mark(false);
        ++k;
    }
    if (has_force && !fused) {
        mark(true);
        CK(launch_inject(m->d_fields, (long long)m->ncell, m->d_src, (int)m->srcs.size(), 1, m->nx, m->ny, m->d_int,
                         m->d_int + 1, 0, st));
        mark(false);
        ++k;
    }
    const bool visc = m->tau > 0.0;
    const size_t nv = m->ncell * (size_t)m->nsim;
    if (visc) {
        // w = (dt + tau) v^{n+1/2} - tau v^{n-1/2}, then v^{n-1/2} <- v^{n+1/2}: the stress passes
        // take c D(w) = dt c D(v) + tau c (D(v^{n+1/2}) - D(v^{n-1/2})) (Eq. (2), chi = tau lambda,
        // eta = tau mu, backward difference of the strain rate)
        mark(true);
        CK(launch_visc_combine(m->d_fields, m->vold, m->wv, nv, (float)((double)dt + m->tau), (float)m->tau, st));
        mark(false);
        ++k;
    }
    for (int a = 0; a < 3; ++a) {
        NvtxRange r(kStr[a]);
        PassParams p = make_pass(m, a, true, dt);
        p.pdl = a == 0 ? 2 : 1;
        if (visc) {
            p.dt = 1.f;
            for (int j = 0; j < p.njobs; ++j)
                for (int c = 0; c < 3; ++c)
                    if (p.job[j].src == m->f[VX + c]) p.job[j].src = m->wv + (size_t)c * nv;
        }
        if (a == 1) fuse(p, SP_STR_Y);  // Mxy: sxy's last update is the y pass
        if (a == 2) fuse(p, SP_STR_Z);  // the other moment components, then the pressure samples
        mark(true);
        CK(launch_pass(p, st));
        mark(false);
        ++k;
    }
    if (fused) {
        *nk = k;
        return ES_OK;
    }
    mark(true);
    CK(launch_inject(m->d_fields, (long long)m->ncell, m->d_src, (int)m->srcs.size(), 0, m->nx, m->ny, m->d_int,
                     m->d_int + 1, 1, st));
    mark(false);
    ++k;
    if (n_rcv > 0) {
        mark(true);
        CK(launch_record(m->d_fields, (long long)m->ncell, m->nsim, m->d_rcv, n_rcv, m->d_int + 1, start, m->d_rec,
                         st));
        mark(false);
        ++k;
    }
    *nk = k;
    return ES_OK;
}

int capture(es_model* m, int steps, float dt, int n_rcv, long long start, bool timed, cudaGraphExec_t* exec)
{
    cudaStream_t cap;
    CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    int rc = ES_OK, nk = 0;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaStreamDestroy(cap);
        return cuda_fail(e, "cudaStreamBeginCapture");
    }
    for (int s = 0; s < steps && rc == ES_OK; ++s) rc = enqueue_step(m, dt, n_rcv, start, cap, timed ? m->ev : nullptr, &nk);
    e = cudaStreamEndCapture(cap, &g);
    cudaStreamDestroy(cap);
    if (rc != ES_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    m->n_last = nk;
    return ES_OK;
}

// whether a pass along axis a runs on the tensor cores (ES_PREC_FP32_TC, a circulant axis of
// CIRC_TC_N to CIRC_MAX_N cells)
bool tc_axis(const es_model* m, int a)
{
    const int n = axis_len(m, a);
    return m->prec == ES_PREC_FP32_TC && n >= CIRC_TC_N && n <= CIRC_MAX_N && !fft_axis(n, m->nx);
}

// In ES_PREC_FP32_TC mode with a tensor-core axis: the buffer through which those passes'
// derivatives go to the field-update kernel, [job][sim][cell] (3 jobs)
int alloc_tc_scratch(es_model* m)
{
    const bool tc = tc_axis(m, 0) || tc_axis(m, 1) || tc_axis(m, 2);
    if (!tc || m->ctc_scratch) return ES_OK;
    cudaError_t e = dev_alloc(&m->ctc_scratch, 3 * m->ncell * (size_t)m->nsim * sizeof(float));
    if (e != cudaSuccess) {
        m->ctc_scratch = nullptr;
        return cuda_fail(e, "cudaMalloc(derivative scratch)");
    }
    return ES_OK;
}

// (Re)allocates the field totals and slab splits for nsim simulations:
// field f of simulation k at f[f] + k ncell, its split along axis a at
// slab[a][f] + k slab_count(a).
int alloc_fields(es_model* m, int nsim)
{
    const size_t A = 256;
    auto up = [&](size_t b) { return (b + A - 1) / A * A; };
    size_t bytes = up(m->ncell * 4 * (size_t)nsim) * NFIELD;
    for (int a = 0; a < 3; ++a)
        for (int f = 0; f < NFIELD; ++f)
            if (m->L > 0 && has_split(f, a)) bytes += up(slab_count(m, a) * 4 * (size_t)nsim);
    char* pool = nullptr;
    cudaError_t e = dev_alloc(&pool, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(fields)");
    dev_free(m->fpool);
    m->fpool = pool;
    m->nsim = nsim;
    char* cur = pool;
    auto take = [&](size_t b) { char* p = cur; cur += up(b); return p; };
    for (int f = 0; f < NFIELD; ++f) m->f[f] = (float*)take(m->ncell * 4 * (size_t)nsim);
    for (int a = 0; a < 3; ++a)
        for (int f = 0; f < NFIELD; ++f)
            m->slab[a][f] = (m->L > 0 && has_split(f, a)) ? (float*)take(slab_count(m, a) * 4 * (size_t)nsim) : nullptr;
    CK(cudaMemcpy(m->d_fields, m->f, sizeof(m->f), cudaMemcpyHostToDevice));
    dev_free(m->ctc_scratch);
    m->ctc_scratch = nullptr;
    return alloc_tc_scratch(m);
}

int run_checked_args(es_model* m, int nt, double dt, int n_rcv)
{
    if (!m || nt < 0 || n_rcv < 0) return ES_ERR_ARG;
    (void)dt;
    return ES_OK;
}

bool aligned16(const void* q) { return ((uintptr_t)q & 15) == 0; }

}  // namespace

// The device word of the bounds-checked build, allocated (outside the counted
// allocations: it lives as long as the process) by ensure_prepared, which
// every entry point calls before it launches or captures anything.
namespace es {
#if ES_BOUNDS
static unsigned long long* g_bounds_word = nullptr;
bool bounds_init()
{
    if (!g_bounds_word) {
        if (cudaMalloc(&g_bounds_word, sizeof(unsigned long long)) != cudaSuccess) {
            g_bounds_word = nullptr;
            return false;
        }
        if (cudaMemset(g_bounds_word, 0, sizeof(unsigned long long)) != cudaSuccess) return false;
    }
    return true;
}
unsigned long long* bounds_word() { return g_bounds_word; }
#else
bool bounds_init() { return true; }
unsigned long long* bounds_word() { return nullptr; }
#endif
}  // namespace es

namespace {

// One staggered derivative of a plain [nz][ny][nx] array along `axis`, with
// its own tables: out = D f (acc == nullptr) or out += acc * D f (acc: a
// per-cell coefficient array, e.g. ones).  Stream-ordered; tables freed after
// the stream reaches them.
cudaError_t derivative_pass(const float* f, int nx, int ny, int nz, int axis, double d, int shift, float* out,
                            const float* acc, cudaStream_t st)
{
    const int n = axis == 0 ? nx : (axis == 1 ? ny : nz);
    const bool circ = !fft_axis(n, nx);
    std::vector<float2> tw, hp, hm;
    std::vector<double> ckp64, ckm64;
    float gp[NEAR_TAPS], gm[NEAR_TAPS];
    axis_tables(n, d, tw, hp, hm, gp, gm, circ ? &ckp64 : nullptr, circ ? &ckm64 : nullptr);
    std::vector<float> ckp(ckp64.begin(), ckp64.end()), ckm(ckm64.begin(), ckm64.end());
    float2* tab = nullptr;
    cudaError_t e = dev_alloc(&tab, 3 * n * 8 + 2 * n * 4);
    if (e != cudaSuccess) return e;
    float* ck = reinterpret_cast<float*>(tab + 3 * n);
    e = cudaMemcpy(tab, tw.data(), n * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(tab + n, hp.data(), n * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(tab + 2 * n, hm.data(), n * 8, cudaMemcpyHostToDevice);
    if (circ && e == cudaSuccess) e = cudaMemcpy(ck, ckp.data(), n * 4, cudaMemcpyHostToDevice);
    if (circ && e == cudaSuccess) e = cudaMemcpy(ck + n, ckm.data(), n * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        PassParams p;
        std::memset(&p, 0, sizeof p);
        p.nx = nx;
        p.ny = ny;
        p.nz = nz;
        p.axis = axis;
        p.n = n;
        p.njobs = 1;
        p.nsim = 1;
        p.dt = 1.f;
        p.tw = tab;
        p.hp = tab + n;
        p.hm = tab + 2 * n;
        p.ckp = ck;
        p.ckm = ck + n;
        p.circ = circ ? 1 : 0;
        p.ext_f = p.ext_c = (long long)nx * ny * nz;
        p.bad = bounds_word();
        p.job[0].src = f;
        p.job[0].tgt[0] = out;
        p.job[0].kind = acc ? JOB_SINGLE : JOB_STORE;
        p.job[0].coef[0] = acc;
        p.job[0].sign = shift;
        for (int t = 0; t < NEAR_TAPS; ++t) p.job[0].g[t] = shift > 0 ? gp[t] : gm[t];
        e = launch_pass(p, st);
    }
    cudaError_t e2 = cudaStreamSynchronize(st);
    dev_free(tab);
    return e != cudaSuccess ? e : e2;
}

}  // namespace

extern "C" {

const char* es_status_string(int s)
{
    switch (s) {
    case ES_OK: return "ok";
    case ES_ERR_ARG: return "invalid argument";
    case ES_ERR_SIZE: return "unsupported grid size";
    case ES_ERR_CUDA: return "CUDA error";
    case ES_ERR_OOM: return "out of device memory";
    case ES_ERR_UNSTABLE: return "unstable (time step too large or non-finite field)";
    case ES_ERR_TIMEOUT: return "device wait timed out";
    case ES_ERR_STATE: return "invalid state";
    default: return "unknown status";
    }
}

const char* es_last_error(void) { return g_err; }

void es_fault_inject_alloc(int n) { g_alloc_countdown = n > 0 ? n : 0; }

long long es_debug_live_allocations(void) { return g_live_allocs.load(); }

int es_debug_bounds(long long* first_bad)
{
    if (!first_bad) return ES_ERR_ARG;
    *first_bad = 0;
#if ES_BOUNDS
    const int rc = ensure_prepared();
    if (rc != ES_OK) return rc;
    unsigned long long* w = bounds_word();
    unsigned long long v = 0;
    if (!w || cudaMemcpy(&v, w, sizeof v, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemset(w, 0, sizeof v) != cudaSuccess)
        return ES_ERR_CUDA;
    *first_bad = (long long)v;
    return ES_OK;
#else
    return ES_ERR_STATE;
#endif
}

void es_model_destroy(es_model* m)
{
    if (!m) return;
    dev_free(m->vpool);
    for (auto& s : m->srcs) dev_free(s.d_w);
    dev_free(m->d_src);
    dev_free(m->d_rec);
    dev_free(m->d_out);
    dev_free(m->d_rcv);
    dev_free(m->pool);
    dev_free(m->fpool);
    for (auto* c : m->ctc) dev_free(c);
    dev_free(m->ctc_scratch);
    dev_free(m->d_sp);
    for (auto& e : m->ev)
        if (e) cudaEventDestroy(e);
    delete m;
}

int es_model_create(const float* rho, const float* cp, const float* cs, int nx, int ny, int nz, double dx, int pml,
                    es_model** out)
{
    NvtxRange nvtx_range("es_model_create");
    if (!out) return ES_ERR_ARG;
    *out = nullptr;
    if (!rho || !cp || !cs || nx < 1 || ny < 1 || nz < 1 || !(dx > 0) || pml < 0) return ES_ERR_ARG;
    if (!axis_ok(nx) || !axis_ok(ny) || !axis_ok(nz)) return ES_ERR_SIZE;
    if (2 * pml + 2 >= nx || 2 * pml + 2 >= ny || 2 * pml + 2 >= nz) return ES_ERR_ARG;
    int rc = ensure_prepared();
    if (rc != ES_OK) return rc;
    const size_t n = (size_t)nx * ny * nz;
    std::vector<float> h_rho, h_cp, h_cs;
    if ((rc = fetch(rho, n, h_rho, nullptr)) != ES_OK) return rc;
    if ((rc = fetch(cp, n, h_cp, nullptr)) != ES_OK) return rc;
    if ((rc = fetch(cs, n, h_cs, nullptr)) != ES_OK) return rc;
    float cpmax = 0.f;
    {
        std::vector<float> bmax(64, 0.f);
        std::vector<char> bad(64, 0);
        const size_t nb = 64;
        parallel_for(nb, [&](size_t b0, size_t b1) {
            for (size_t b = b0; b < b1; ++b)
                for (size_t q = n * b / nb; q < n * (b + 1) / nb; ++q) {
                    const float r = h_rho[q], p = h_cp[q], s = h_cs[q];
                    if (!(r > 0.f) || !(p > 0.f) || !(s >= 0.f) || !std::isfinite(r) || !std::isfinite(p) ||
                        !std::isfinite(s) || (double)p * p - 2.0 * (double)s * s < 0.0)  // lambda >= 0
                        bad[b] = 1;
                    bmax[b] = std::max(bmax[b], p);
                }
        });
        for (size_t b = 0; b < nb; ++b) {
            if (bad[b]) return ES_ERR_ARG;
            cpmax = std::max(cpmax, bmax[b]);
        }
    }
    es_model* m = new (std::nothrow) es_model();
    if (!m) return ES_ERR_OOM;
    m->nx = nx;
    m->ny = ny;
    m->nz = nz;
    m->ncell = n;
    m->d[0] = m->d[1] = m->d[2] = dx;
    m->L = pml;
    m->cp_max = cpmax;
    m->rho = h_rho;
    m->cs = h_cs;

    // one pool: fields, materials, slabs, per-axis tables, counters, pointer table
    const size_t A = 256;
    auto up = [&](size_t b) { return (b + A - 1) / A * A; };
    size_t bytes = up(n * 4) * NMAT;
    for (int a = 0; a < 3; ++a) bytes += 3 * up(axis_len(m, a) * 8) + 6 * up(axis_len(m, a) * 4);
    bytes += up(16) + up(NFIELD * sizeof(float*));
    cudaError_t e = dev_alloc(&m->pool, bytes);
    if (e != cudaSuccess) {
        es_model_destroy(m);
        return cuda_fail(e, "cudaMalloc(model)");
    }
    char* cur = m->pool;
    auto take = [&](size_t b) { char* p = cur; cur += up(b); return p; };
    for (int k = 0; k < NMAT; ++k) m->mat[k] = (float*)take(n * 4);
    for (int a = 0; a < 3; ++a) {
        m->tw[a] = (float2*)take(axis_len(m, a) * 8);
        m->hp[a] = (float2*)take(axis_len(m, a) * 8);
        m->hm[a] = (float2*)take(axis_len(m, a) * 8);
        m->ckp[a] = (float*)take(axis_len(m, a) * 4);
        m->ckm[a] = (float*)take(axis_len(m, a) * 4);
        m->ckp_lo[a] = (float*)take(axis_len(m, a) * 4);
        m->ckm_lo[a] = (float*)take(axis_len(m, a) * 4);
        m->pc[a] = (float*)take(axis_len(m, a) * 4);
        m->ps[a] = (float*)take(axis_len(m, a) * 4);
    }
    m->d_int = (int*)take(16);
    m->d_fields = (float**)take(NFIELD * sizeof(float*));

    // materials (Eq. (4) and the staggered averages) on the device, from rho, cp, cs there: the
    // caller's device arrays as they are, host arrays through one staging buffer
    {
        const bool on_dev = is_device_ptr(rho) && is_device_ptr(cp) && is_device_ptr(cs);
        float* stage = nullptr;
        const float *d_rho = rho, *d_cp = cp, *d_cs = cs;
        if (!on_dev) {
            e = dev_alloc(&stage, 3 * n * sizeof(float));
            if (e == cudaSuccess) e = cudaMemcpy(stage, h_rho.data(), n * 4, cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMemcpy(stage + n, h_cp.data(), n * 4, cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMemcpy(stage + 2 * n, h_cs.data(), n * 4, cudaMemcpyHostToDevice);
            d_rho = stage;
            d_cp = stage + n;
            d_cs = stage + 2 * n;
        }
        MatPtrs mp;
        for (int k = 0; k < NMAT; ++k) mp.p[k] = m->mat[k];
        if (e == cudaSuccess) e = launch_materials(d_rho, d_cp, d_cs, nx, ny, nz, mp, 0);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (stage) dev_free(stage);
    }
    for (int a = 0; a < 3 && e == cudaSuccess; ++a) e = upload_axis_tables(m, a);
    for (int k = 0; k < 2 * KPS_MAX && e == cudaSuccess; ++k) e = cudaEventCreate(&m->ev[k]);
    if (e != cudaSuccess) {
        int r = cuda_fail(e, "es_model_create");
        es_model_destroy(m);
        return r;
    }
    rc = alloc_fields(m, 1);
    if (rc != ES_OK) {
        es_model_destroy(m);
        return rc;
    }
    rc = es_state_reset(m);
    if (rc != ES_OK) {
        es_model_destroy(m);
        return rc;
    }
    *out = m;
    return ES_OK;
}

int es_model_set_viscosity(es_model* m, double tau)
{
    if (!m || !(tau >= 0.0) || !std::isfinite(tau)) return ES_ERR_ARG;
    m->tau = tau;
    return ES_OK;
}

int es_model_set_precision(es_model* m, int mode)
{
    if (!m || (mode != ES_PREC_FP32 && mode != ES_PREC_COMPENSATED && mode != ES_PREC_FP32_TC)) return ES_ERR_ARG;
    m->prec = mode;
    for (int a = 0; a < 3; ++a) CK(upload_axis_tables(m, a));
    return alloc_tc_scratch(m);
}

int es_model_set_spacing(es_model* m, double dx, double dy, double dz)
{
    if (!m || !(dx > 0) || !(dy > 0) || !(dz > 0)) return ES_ERR_ARG;
    m->d[0] = dx;
    m->d[1] = dy;
    m->d[2] = dz;
    for (int a = 0; a < 3; ++a) CK(upload_axis_tables(m, a));
    return ES_OK;
}

int es_model_set_pml(es_model* m, double alpha0, double cref)
{
    if (!m || !(alpha0 >= 0)) return ES_ERR_ARG;
    m->alpha0 = alpha0;
    m->cref = cref;
    return ES_OK;
}

int es_model_set_stream(es_model* m, void* stream)
{
    if (!m) return ES_ERR_ARG;
    m->stream = (cudaStream_t)stream;
    return ES_OK;
}

int es_model_default_dt(const es_model* m, double* dt)
{
    if (!m || !dt) return ES_ERR_ARG;
    *dt = 0.3 * std::min(m->d[0], std::min(m->d[1], m->d[2])) / (double)m->cp_max;  // Eq. (5), CFL 0.3
    return ES_OK;
}

static int add_source(es_model* m, int kind, const int pos[3], const double* v, int nv, const float* w, int nw,
                      int smooth = 0)
{
    if (!m || !pos || !v || nw < 0 || (nw > 0 && !w)) return ES_ERR_ARG;
    const int reach = smooth ? 2 : 0;  // a smoothed source reaches 2 cells out
    for (int a = 0; a < 3; ++a)
        if (pos[a] - reach < m->L || pos[a] + reach > axis_len(m, a) - 2 - m->L) return ES_ERR_ARG;  // outside the PML slabs
    for (int c = 0; c < nv; ++c)
        if (!std::isfinite(v[c])) return ES_ERR_ARG;
    std::vector<float> h;
    int rc = fetch(w, (size_t)nw, h, m->stream);
    if (rc != ES_OK) return rc;
    Src s;
    s.kind = kind;
    s.smooth = smooth;
    s.sim = 0;
    std::memcpy(s.pos, pos, sizeof s.pos);
    for (int c = 0; c < 6; ++c) s.m[c] = c < nv ? v[c] : 0.0;
    s.nw = nw;
    s.d_w = nullptr;
    if (nw > 0) {
        CK(dev_alloc(&s.d_w, sizeof(float) * nw));
        cudaError_t e = cudaMemcpy(s.d_w, h.data(), sizeof(float) * nw, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            dev_free(s.d_w);
            return cuda_fail(e, "cudaMemcpy(wavelet)");
        }
    }
    m->srcs.push_back(s);
    return ES_OK;
}

int es_batch_set(es_model* m, int nb, const int* pos, const double* mt, const float* wavelets, int nw)
{
    if (!m || nb < 1 || !pos || !mt || nw < 0 || (nw > 0 && !wavelets)) return ES_ERR_ARG;
    std::vector<int> hp;
    std::vector<double> hm;
    std::vector<float> hw;
    int rc;
    if ((rc = fetch(pos, (size_t)nb * 3, hp, m->stream)) != ES_OK) return rc;
    if ((rc = fetch(mt, (size_t)nb * 6, hm, m->stream)) != ES_OK) return rc;
    if ((rc = fetch(wavelets, (size_t)nb * nw, hw, m->stream)) != ES_OK) return rc;
    for (int b = 0; b < nb; ++b) {
        for (int a = 0; a < 3; ++a)
            if (hp[3 * b + a] < m->L || hp[3 * b + a] > axis_len(m, a) - 2 - m->L) return ES_ERR_ARG;
        for (int c = 0; c < 6; ++c)
            if (!std::isfinite(hm[6 * b + c])) return ES_ERR_ARG;
    }
    if ((rc = es_source_clear(m)) != ES_OK) return rc;
    if (nb != m->nsim && (rc = alloc_fields(m, nb)) != ES_OK) return rc;
    for (int b = 0; b < nb; ++b) {
        Src s;
        s.kind = 0;
        s.sim = b;
        std::memcpy(s.pos, &hp[3 * b], sizeof s.pos);
        for (int c = 0; c < 6; ++c) s.m[c] = hm[6 * b + c];
        s.nw = nw;
        s.d_w = nullptr;
        if (nw > 0) {
            CK(dev_alloc(&s.d_w, sizeof(float) * nw));
            cudaError_t e = cudaMemcpy(s.d_w, &hw[(size_t)b * nw], sizeof(float) * nw, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                dev_free(s.d_w);
                return cuda_fail(e, "cudaMemcpy(wavelet)");
            }
        }
        m->srcs.push_back(s);
    }
    return es_state_reset(m);
}

int es_source_clear(es_model* m)
{
    if (!m) return ES_ERR_ARG;
    CK(cudaStreamSynchronize(m->stream));
    for (auto& s : m->srcs) dev_free(s.d_w);
    m->srcs.clear();
    return ES_OK;
}

int es_source_set(es_model* m, const int pos[3], const double mt[6], const float* wavelet, int nw)
{
    if (!m) return ES_ERR_ARG;
    int rc = es_source_clear(m);
    if (rc != ES_OK) return rc;
    return add_source(m, 0, pos, mt, 6, wavelet, nw);
}

int es_source_add(es_model* m, const int pos[3], const double mt[6], const float* wavelet, int nw)
{
    return add_source(m, 0, pos, mt, 6, wavelet, nw);
}

int es_source_add_force(es_model* m, const int pos[3], const double f[3], const float* wavelet, int nw)
{
    return add_source(m, 1, pos, f, 3, wavelet, nw);
}

int es_source_add_smoothed(es_model* m, const int pos[3], const double mt[6], const float* wavelet, int nw)
{
    if (m && (m->nx < 5 || m->ny < 5 || m->nz < 5)) return ES_ERR_ARG;
    return add_source(m, 0, pos, mt, 6, wavelet, nw, 1);
}

int es_state_reset(es_model* m)
{
    if (!m) return ES_ERR_ARG;
    const size_t ns = (size_t)m->nsim;
    for (int f = 0; f < NFIELD; ++f) CK(cudaMemsetAsync(m->f[f], 0, m->ncell * 4 * ns, m->stream));
    for (int a = 0; a < 3; ++a)
        for (int f = 0; f < NFIELD; ++f)
            if (m->slab[a][f]) CK(cudaMemsetAsync(m->slab[a][f], 0, slab_count(m, a) * 4 * ns, m->stream));
    CK(cudaMemsetAsync(m->d_int, 0, 16, m->stream));
    if (m->vpool) CK(cudaMemsetAsync(m->vpool, 0, 6 * m->ncell * (size_t)m->vpool_nsim * sizeof(float), m->stream));
    CK(cudaStreamSynchronize(m->stream));
    m->steps_done = 0;
    return ES_OK;
}

int es_state_get(es_model* m, float* fields)
{
    if (!m || !fields) return ES_ERR_ARG;
    const cudaMemcpyKind k = is_device_ptr(fields) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    for (int k2 = 0; k2 < m->nsim; ++k2)
        for (int f = 0; f < NFIELD; ++f)
            CK(cudaMemcpyAsync(fields + ((size_t)k2 * NFIELD + f) * m->ncell, m->f[f] + (size_t)k2 * m->ncell,
                               m->ncell * 4, k, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    return ES_OK;
}

int es_state_set(es_model* m, const float* fields)
{
    if (!m || !fields) return ES_ERR_ARG;
    const cudaMemcpyKind k = is_device_ptr(fields) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    for (int k2 = 0; k2 < m->nsim; ++k2) {
        const size_t fo = (size_t)k2 * m->ncell;
        for (int f = 0; f < NFIELD; ++f)
            CK(cudaMemcpyAsync(m->f[f] + fo, fields + ((size_t)k2 * NFIELD + f) * m->ncell, m->ncell * 4, k, m->stream));
        for (int a = 0; a < 3; ++a)
            for (int f = 0; f < NFIELD; ++f) {
                if (!m->slab[a][f]) continue;
                const int first = has_split(f, 0) ? 0 : 1;  // the split carrying the whole value
                CK(launch_fill_slab(m->f[f] + fo, m->slab[a][f] + (size_t)k2 * slab_count(m, a), a, m->nx, m->ny,
                                    m->nz, m->L, a == first, m->stream));
            }
    }
    // viscous runs: the given velocity also stands for v^{n-1/2} (no strain-rate history)
    if (m->vpool && m->vpool_nsim == m->nsim) {
        const size_t nv = m->ncell * (size_t)m->nsim;
        for (int c = 0; c < 3; ++c)
            CK(cudaMemcpyAsync(m->vold + c * nv, m->f[VX + c], nv * sizeof(float), cudaMemcpyDeviceToDevice,
                               m->stream));
    }
    CK(cudaStreamSynchronize(m->stream));
    return ES_OK;
}

// Validation and per-run set-up of es_run: receivers, buffers, PML factors
// for dt, sources.  dt <= 0 is replaced by the default.
static int run_prepare(es_model* m, int nt, double* pdt, const int* rcv, int n_rcv, float* traces)
{
    int rc = run_checked_args(m, nt, *pdt, n_rcv);
    if (rc != ES_OK) return rc;
    double& dt = *pdt;
    cudaGetLastError();  // launch checks below must not see an earlier, unrelated error
    if (n_rcv > 0 && (!rcv || !traces)) return ES_ERR_ARG;
    if (!(dt > 0)) es_model_default_dt(m, &dt);
    // stability of the staggered pseudo-spectral leapfrog: c dt |kappa_max| <= 2; with the
    // viscous terms every mode needs q (1 + 2 tau / dt) <= 4, q = (c dt |kappa_max|)^2
    const double s = std::sqrt(1.0 / (m->d[0] * m->d[0]) + 1.0 / (m->d[1] * m->d[1]) + 1.0 / (m->d[2] * m->d[2]));
    const double qmax = std::pow((double)m->cp_max * dt * 3.14159265358979323846 * s, 2.0);
    if (qmax * (1.0 + 2.0 * m->tau / dt) > 4.0) return ES_ERR_UNSTABLE;
    if (m->tau > 0.0 && (!m->vpool || m->vpool_nsim != m->nsim)) {
        // first viscous run at this batch size: v^{n-1/2} starts as the current velocity
        const size_t nv = m->ncell * (size_t)m->nsim;
        char* pool = nullptr;
        CK(dev_alloc(&pool, 6 * nv * sizeof(float)));
        dev_free(m->vpool);
        m->vpool = pool;
        m->vpool_nsim = m->nsim;
        m->vold = reinterpret_cast<float*>(pool);
        m->wv = m->vold + 3 * nv;
        for (int c = 0; c < 3; ++c)
            CK(cudaMemcpyAsync(m->vold + c * nv, m->f[VX + c], nv * sizeof(float), cudaMemcpyDeviceToDevice,
                               m->stream));
    }

    std::vector<int> h_rcv;
    if ((rc = fetch(rcv, (size_t)n_rcv * 3, h_rcv, m->stream)) != ES_OK) return rc;
    std::vector<long long> cells(n_rcv);
    for (int r = 0; r < n_rcv; ++r) {
        const int ix = h_rcv[3 * r], iy = h_rcv[3 * r + 1], iz = h_rcv[3 * r + 2];
        if (ix < 0 || ix >= m->nx || iy < 0 || iy >= m->ny || iz < 0 || iz >= m->nz) return ES_ERR_ARG;
        cells[r] = (long long)ix + (long long)m->nx * ((long long)iy + (long long)m->ny * iz);
    }
    if (n_rcv > m->rcv_cap) {
        dev_free(m->d_rcv);
        m->d_rcv = nullptr;
        m->rcv_cap = 0;
        CK(dev_alloc(&m->d_rcv, sizeof(long long) * n_rcv));
        m->rcv_cap = n_rcv;
    }
    const size_t rec_n = (size_t)nt * m->nsim * 4 * n_rcv;
    if (rec_n > m->rec_cap) {
        dev_free(m->d_rec);
        m->d_rec = nullptr;
        m->rec_cap = 0;
        CK(dev_alloc(&m->d_rec, rec_n * 4));
        m->rec_cap = rec_n;
    }
    if (n_rcv > 0) CK(cudaMemcpyAsync(m->d_rcv, cells.data(), sizeof(long long) * n_rcv, cudaMemcpyHostToDevice, m->stream));

    // PML factors for this dt (Sec. II-B; profile alpha0 (cref/d) xi^4)
    const double cref = m->cref > 0 ? m->cref : (double)m->cp_max;
    for (int a = 0; a < 3; ++a) {
        const int n = axis_len(m, a), L = m->L;
        std::vector<float> pc(n), ps(n);
        for (int i = 0; i < n; ++i)
            for (int st = 0; st < 2; ++st) {
                const double x = i + (st ? 0.5 : 0.0);
                double xi = 0.0;
                if (L > 0) {
                    if (x < L) xi = (L - x) / L;
                    else if (x > n - 1 - L) xi = (x - (n - 1 - L)) / L;
                    xi = std::min(xi, 1.0);
                }
                const double alpha = m->alpha0 * (cref / m->d[a]) * xi * xi * xi * xi;
                (st ? ps : pc)[i] = (float)std::exp(-alpha * dt * 0.5);
            }
        CK(cudaMemcpyAsync(m->pc[a], pc.data(), n * 4, cudaMemcpyHostToDevice, m->stream));
        CK(cudaMemcpyAsync(m->ps[a], ps.data(), n * 4, cudaMemcpyHostToDevice, m->stream));
        CK(cudaStreamSynchronize(m->stream));
    }
    if ((rc = upload_sources(m, dt)) != ES_OK) return rc;
    m->fused = fused_sources(m);
    if (m->fused && (rc = build_special(m, cells)) != ES_OK) return rc;
    return ES_OK;
}

// After the steps of a run are queued on st: non-finite check, traces out,
// completion.
static int run_finish(es_model* m, int nt, int n_rcv, float* traces, cudaStream_t st)
{
    CK(cudaMemsetAsync(m->d_int + 2, 0, 4, st));
    CK(launch_nonfinite(m->d_fields, m->ncell * m->nsim, m->d_int + 2, st));
    m->steps_done += nt;
    const size_t rec_n = (size_t)nt * m->nsim * 4 * n_rcv;
    if (n_rcv > 0) {
        const bool dev_out = is_device_ptr(traces);
        float* dst = traces;
        if (!dev_out) {
            if (rec_n > m->out_cap) {
                dev_free(m->d_out);
                m->d_out = nullptr;
                m->out_cap = 0;
                CK(dev_alloc(&m->d_out, rec_n * 4));
                m->out_cap = rec_n;
            }
            dst = m->d_out;
        }
        CK(launch_transpose_traces(m->d_rec, nt, m->nsim * 4 * n_rcv, dst, st));
        if (!dev_out) CK(cudaMemcpyAsync(traces, dst, rec_n * 4, cudaMemcpyDeviceToHost, st));
    }
    int flag = 0;
    CK(cudaMemcpyAsync(&flag, m->d_int + 2, 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    // a bounded wait of a tensor-core pass that ran out left its derivatives unwritten
    if (tc_axis(m, 0) || tc_axis(m, 1) || tc_axis(m, 2)) {
        unsigned status = 0;
        CK(circ_tc_status(&status));
        if (status) {
            snprintf(g_err, sizeof g_err, "tensor-core circulant pass: a bounded wait gave up (status %#x)", status);
            return ES_ERR_TIMEOUT;
        }
    }
    return flag ? ES_ERR_UNSTABLE : ES_OK;
}

int es_run(es_model* m, int nt, double dt, const int* rcv, int n_rcv, float* traces)
{
    NvtxRange whole("es_run");
    int rc;
    {
        NvtxRange r("es_run: prepare");
        rc = run_prepare(m, nt, &dt, rcv, n_rcv, traces);
    }
    if (rc != ES_OK || nt == 0) return rc;
    // graphs: K steps, 1 step, 1 step with per-kernel events (the last step)
    const long long start = m->steps_done;
    const int K = 16;
    cudaGraphExec_t gK = nullptr, g1 = nullptr, gT = nullptr;
    const int body = nt - 1;
    {
        NvtxRange r("es_run: capture");
        if (body >= K) rc = capture(m, K, (float)dt, n_rcv, start, false, &gK);
        if (rc == ES_OK && body % K) rc = capture(m, 1, (float)dt, n_rcv, start, false, &g1);
        if (rc == ES_OK) rc = capture(m, 1, (float)dt, n_rcv, start, true, &gT);
    }
    cudaError_t e = cudaSuccess;
    if (rc == ES_OK) {
        NvtxRange r("es_run: replay");
        for (int i = 0; i < body / K && e == cudaSuccess; ++i) e = cudaGraphLaunch(gK, m->stream);
        for (int i = 0; i < body % K && e == cudaSuccess; ++i) e = cudaGraphLaunch(g1, m->stream);
        if (e == cudaSuccess) e = cudaGraphLaunch(gT, m->stream);
    }
    if (gK) cudaGraphExecDestroy(gK);
    if (g1) cudaGraphExecDestroy(g1);
    if (gT) cudaGraphExecDestroy(gT);
    if (rc != ES_OK) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "es_run launch");
    {
        NvtxRange r("es_run: finish");
        rc = run_finish(m, nt, n_rcv, traces, m->stream);
    }
    if (rc == ES_OK || rc == ES_ERR_UNSTABLE)
        for (int k = 0; k < m->n_last; ++k) CK(cudaEventElapsedTime(&m->last_ms[k], m->ev[2 * k], m->ev[2 * k + 1]));
    return rc;
}

// One graph holding `steps` time steps of every model, each model on its own
// branch forked from and joined back to the capture stream.
static int capture_group(es_model* const* ms, int nmod, int steps, const double* dts, const int* n_rcv,
                         const long long* starts, cudaGraphExec_t* exec)
{
    cudaStream_t root = nullptr;
    std::vector<cudaStream_t> br(nmod, nullptr);
    std::vector<cudaEvent_t> join(nmod, nullptr);
    cudaEvent_t fork = nullptr;
    cudaGraph_t g = nullptr;
    int rc = ES_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&root, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    for (int i = 0; i < nmod && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&br[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaStreamBeginCapture(root, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaEventRecord(fork, root);
        for (int i = 0; i < nmod && rc == ES_OK; ++i) {
            cudaStreamWaitEvent(br[i], fork, 0);
            int nk = 0;
            for (int s = 0; s < steps && rc == ES_OK; ++s)
                rc = enqueue_step(ms[i], (float)dts[i], n_rcv[i], starts[i], br[i], nullptr, &nk);
            cudaEventRecord(join[i], br[i]);
            cudaStreamWaitEvent(root, join[i], 0);
        }
        e = cudaStreamEndCapture(root, &g);
        if (e == cudaSuccess && rc == ES_OK) e = cudaGraphInstantiate(exec, g, 0);
    }
    if (g) cudaGraphDestroy(g);
    for (int i = 0; i < nmod; ++i) {
        if (br[i]) cudaStreamDestroy(br[i]);
        if (join[i]) cudaEventDestroy(join[i]);
    }
    if (fork) cudaEventDestroy(fork);
    if (root) cudaStreamDestroy(root);
    if (rc != ES_OK) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "capture_group");
    return ES_OK;
}

int es_run_group(int nmod, es_model* const* models, int nt, const double* dts, const int* const* rcvs,
                 const int* n_rcvs, float* const* traces)
{
    NvtxRange nvtx_range("es_run_group");
    if (nmod < 1 || !models || !dts || !rcvs || !n_rcvs || !traces || nt < 0) return ES_ERR_ARG;
    for (int i = 0; i < nmod; ++i) {
        if (!models[i]) return ES_ERR_ARG;
        for (int k = 0; k < i; ++k)
            if (models[k] == models[i]) return ES_ERR_ARG;
    }
    std::vector<double> dt(dts, dts + nmod);
    std::vector<long long> starts(nmod);
    for (int i = 0; i < nmod; ++i) {
        int rc = run_prepare(models[i], nt, &dt[i], rcvs[i], n_rcvs[i], traces[i]);
        if (rc != ES_OK) return rc;
        starts[i] = models[i]->steps_done;
    }
    if (nt == 0) return ES_OK;
    cudaStream_t st = models[0]->stream;
    const int K = 16;
    cudaGraphExec_t gK = nullptr, g1 = nullptr;
    int rc = ES_OK;
    if (nt >= K) rc = capture_group(models, nmod, K, dt.data(), n_rcvs, starts.data(), &gK);
    if (rc == ES_OK && nt % K) rc = capture_group(models, nmod, 1, dt.data(), n_rcvs, starts.data(), &g1);
    cudaError_t e = cudaSuccess;
    if (rc == ES_OK) {
        for (int i = 0; i < nt / K && e == cudaSuccess; ++i) e = cudaGraphLaunch(gK, st);
        for (int i = 0; i < nt % K && e == cudaSuccess; ++i) e = cudaGraphLaunch(g1, st);
    }
    if (gK) cudaGraphExecDestroy(gK);
    if (g1) cudaGraphExecDestroy(g1);
    if (rc != ES_OK) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "es_run_group launch");
    int worst = ES_OK;
    for (int i = 0; i < nmod; ++i) {
        const int r = run_finish(models[i], nt, n_rcvs[i], traces[i], st);
        if (r != ES_OK && worst == ES_OK) worst = r;
    }
    return worst;
}

int es_model_autotune(es_model* m, int reps, char* report, int report_len)
{
    NvtxRange nvtx_range("es_model_autotune");
    if (!m || reps < 1) return ES_ERR_ARG;
    double dt = 0.0;
    int rc = run_prepare(m, 1, &dt, nullptr, 0, nullptr);
    if (rc != ES_OK) return rc;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    std::string rep;
    std::vector<std::string> keys, lines;
    const std::string dev = device_name();
    for (int kind = 0; kind < 2 && rc == ES_OK; ++kind) {
        std::vector<int> lens;
        if (kind == 0) lens.push_back(m->nx);
        else {
            lens.push_back(m->ny);
            if (m->nz != m->ny) lens.push_back(m->nz);
        }
        for (int n : lens) {
            int ra[8], rb[8];
            const int nc = plan_candidates(n, ra, rb, 8);
            if (nc < 2 || !fft_axis(n, m->nx) || m->prec != ES_PREC_FP32) continue;
            float best = 1e30f;
            int bi = 0;
            for (int c = 0; c < nc && rc == ES_OK; ++c) {
                plan_select(kind, n, ra[c], rb[c]);
                float total = 0.f;
                for (int a = 0; a < 3; ++a) {
                    if ((kind == 0) != (a == 0) || axis_len(m, a) != n || !fft_axis(n, m->nx)) continue;
                    for (int half = 0; half < 2; ++half) {
                        const PassParams p = make_pass(m, a, half == 1, (float)dt);
                        cudaError_t e = launch_pass(p, m->stream);  // warm-up
                        if (e == cudaSuccess) e = cudaEventRecord(e0, m->stream);
                        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_pass(p, m->stream);
                        if (e == cudaSuccess) e = cudaEventRecord(e1, m->stream);
                        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                        float ms = 0.f;
                        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                        if (e != cudaSuccess) {
                            rc = cuda_fail(e, "es_model_autotune");
                            break;
                        }
                        total += ms / reps;
                    }
                }
                char buf[96];
                snprintf(buf, sizeof buf, "%s n=%d %dx%d %.4f ms\n", kind == 0 ? "x" : "yz", n, ra[c], rb[c], total);
                rep += buf;
                if (total < best) {
                    best = total;
                    bi = c;
                }
            }
            plan_select(kind, n, ra[bi], rb[bi]);
            char key[160], line[200];
            snprintf(key, sizeof key, "%s|%d|%d|", dev.c_str(), kind, n);
            snprintf(line, sizeof line, "%s%d|%d", key, ra[bi], rb[bi]);
            keys.push_back(key);
            lines.push_back(line);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != ES_OK) return rc;
    store_plan_cache(keys, lines);
    if (report && report_len > 0) {
        std::strncpy(report, rep.c_str(), (size_t)report_len - 1);
        report[report_len - 1] = 0;
    }
    return es_state_reset(m);
}

int es_fft_plan_select(int pass_kind, int n, int ra, int rb)
{
    if (pass_kind < 0 || pass_kind > 1) return ES_ERR_ARG;
    return plan_select(pass_kind, n, ra, rb) ? ES_OK : ES_ERR_SIZE;
}

int es_fft_plan(int pass_kind, int n, int* ra, int* rb)
{
    if (!ra || !rb || pass_kind < 0 || pass_kind > 1) return ES_ERR_ARG;
    return plan_current(pass_kind, n, ra, rb) ? ES_OK : ES_ERR_SIZE;
}

int es_last_step_kernel_ms(es_model* m, float* ms, int n)
{
    if (!m || !ms || n < 0) return ES_ERR_ARG;
    const int k = std::min(n, m->n_last);
    for (int i = 0; i < k; ++i) ms[i] = m->last_ms[i];
    return k;
}

int es_kernels_per_step(const es_model* m)
{
    if (!m) return ES_ERR_ARG;
    const bool has_force = std::any_of(m->srcs.begin(), m->srcs.end(), [](const Src& s) { return s.kind == 1; });
    // an axis on the tensor cores adds a field-update kernel to each of its two passes
    int tc = 0;
    for (int a = 0; a < 3; ++a) tc += tc_axis(m, a) ? 2 : 0;
    // fused point sources and receivers: the six passes alone
    if (fused_sources(m)) return 6 + (m->tau > 0.0 ? 1 : 0);
    return 8 + (has_force ? 1 : 0) + (m->tau > 0.0 ? 1 : 0) + tc;
}

int es_seabed_receivers(const es_model* m, int rx, int ry, int* rcv)
{
    if (!m || !rcv || rx < 1 || ry < 1) return ES_ERR_ARG;
    const int nx = m->nx, ny = m->ny, nz = m->nz, L = m->L;
    std::vector<int> out((size_t)rx * ry * 3);
    for (int jy = 0; jy < ry; ++jy)
        for (int jx = 0; jx < rx; ++jx) {
            const int ix = L + ((2 * jx + 1) * (nx - 2 * L)) / (2 * rx);
            const int iy = L + ((2 * jy + 1) * (ny - 2 * L)) / (2 * ry);
            auto at = [&](int z) { return m->cs[(size_t)ix + (size_t)nx * ((size_t)iy + (size_t)ny * z)]; };
            if (at(0) != 0.f) return ES_ERR_ARG;
            int iz = 0;
            while (iz + 1 < nz && at(iz + 1) == 0.f) ++iz;
            const size_t r = (size_t)jx + (size_t)rx * jy;
            out[3 * r] = ix;
            out[3 * r + 1] = iy;
            out[3 * r + 2] = iz;
        }
    std::memcpy(rcv, out.data(), out.size() * sizeof(int));
    return ES_OK;
}

int es_superpose(const float* traces, int n_src, int n_rcv, int nt, const int* src_of_event, const float* amps,
                 const float* t0s, int n_events, double dt, int n_out, float* gather, void* stream)
{
    NvtxRange nvtx_range("es_superpose");
    if (!traces || !gather || n_src < 1 || n_rcv < 1 || nt < 1 || n_events < 0 || n_out < 1 || !(dt > 0))
        return ES_ERR_ARG;
    if (n_events > 0 && (!src_of_event || !amps || !t0s)) return ES_ERR_ARG;
    cudaGetLastError();
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int> ev_src;
    std::vector<float> ev_amp, ev_t0;
    int rc;
    if ((rc = fetch(src_of_event, (size_t)n_events, ev_src, st)) != ES_OK) return rc;
    if ((rc = fetch(amps, (size_t)n_events, ev_amp, st)) != ES_OK) return rc;
    if ((rc = fetch(t0s, (size_t)n_events, ev_t0, st)) != ES_OK) return rc;
    std::vector<int> shift(n_events);
    for (int e = 0; e < n_events; ++e) {
        if (ev_src[e] < 0 || ev_src[e] >= n_src || !std::isfinite(ev_t0[e]) || !std::isfinite(ev_amp[e])) return ES_ERR_ARG;
        const double k = std::floor((double)ev_t0[e] / dt + 0.5);  // k_e in FP64
        shift[e] = (int)std::max(-2e9, std::min(2e9, k));
    }
    const size_t tr_n = (size_t)n_src * 4 * n_rcv * nt, g_n = (size_t)4 * n_rcv * n_out;
    const bool dev_in = is_device_ptr(traces), dev_out = is_device_ptr(gather);
    // one scratch block: events, and staging for host input / output
    const size_t ev_bytes = (size_t)std::max(n_events, 1) * 12;
    const size_t bytes = ev_bytes + (dev_in ? 0 : tr_n * 4 + 256) + (dev_out ? 0 : g_n * 4 + 256);
    char* scratch = nullptr;
    CK(dev_alloc(&scratch, bytes));
    int* d_src = (int*)scratch;
    int* d_k = d_src + std::max(n_events, 1);
    float* d_a = (float*)(d_k + std::max(n_events, 1));
    char* p = scratch + (ev_bytes + 255) / 256 * 256;
    const float* d_tr = traces;
    if (!dev_in) { d_tr = (const float*)p; p += (tr_n * 4 + 255) / 256 * 256; }
    float* d_g = dev_out ? gather : (float*)p;
    cudaError_t e = cudaSuccess;
    if (n_events > 0) {
        e = cudaMemcpyAsync(d_src, ev_src.data(), n_events * 4, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_k, shift.data(), n_events * 4, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_a, ev_amp.data(), n_events * 4, cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess && !dev_in) e = cudaMemcpyAsync((void*)d_tr, traces, tr_n * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_superpose(d_tr, n_src, n_rcv, nt, d_src, d_a, d_k, n_events, n_out, d_g, st);
    if (e == cudaSuccess && !dev_out) e = cudaMemcpyAsync(gather, d_g, g_n * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dev_free(scratch);
    if (e != cudaSuccess) return cuda_fail(e, "es_superpose");
    return ES_OK;
}

int es_derivative(const float* f, int nx, int ny, int nz, int axis, double d, int shift, float* out, void* stream)
{
    if (!f || !out || f == out || axis < 0 || axis > 2 || !(d > 0) || (shift != 1 && shift != -1)) return ES_ERR_ARG;
    if (!axis_ok(nx) || !axis_ok(ny) || !axis_ok(nz)) return ES_ERR_SIZE;
    if (!aligned16(f) || !aligned16(out)) return ES_ERR_ARG;  // the passes move 8- and 16-byte vectors
    if (!is_device_ptr(f) || !is_device_ptr(out)) return ES_ERR_ARG;
    cudaGetLastError();
    int rc = ensure_prepared();
    if (rc != ES_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = derivative_pass(f, nx, ny, nz, axis, d, shift, out, nullptr, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "es_derivative");
    return ES_OK;
}

int es_laplacian(const float* f, int nx, int ny, int nz, double dx, double dy, double dz, float* out, void* stream)
{
    if (!f || !out || f == out || !(dx > 0) || !(dy > 0) || !(dz > 0)) return ES_ERR_ARG;
    if (!axis_ok(nx) || !axis_ok(ny) || !axis_ok(nz)) return ES_ERR_SIZE;
    if (!aligned16(f) || !aligned16(out)) return ES_ERR_ARG;
    if (!is_device_ptr(f) || !is_device_ptr(out)) return ES_ERR_ARG;
    cudaGetLastError();
    int rc = ensure_prepared();
    if (rc != ES_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n = (size_t)nx * ny * nz;
    const size_t n_al = (n + 63) / 64 * 64;  // the second array on a 256-byte boundary
    float* tmp = nullptr;
    CK(dev_alloc(&tmp, (n_al + n) * sizeof(float)));
    float* ones = tmp + n_al;
    const double d[3] = {dx, dy, dz};
    cudaError_t e = launch_fill(ones, n, 1.f, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(out, 0, n * sizeof(float), st);
    // D(+) D(-) along each axis multiplies bin kappa by -kappa^2 (Nyquist included)
    for (int a = 0; a < 3 && e == cudaSuccess; ++a) {
        e = derivative_pass(f, nx, ny, nz, a, d[a], -1, tmp, nullptr, st);
        if (e == cudaSuccess) e = derivative_pass(tmp, nx, ny, nz, a, d[a], +1, out, ones, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dev_free(tmp);
    if (e != cudaSuccess) return cuda_fail(e, "es_laplacian");
    return ES_OK;
}

}  // extern "C"
