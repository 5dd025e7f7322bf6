// es_superpose_noalloc: the superposition of es_superpose for callers that
// cannot allocate device memory.  Its only scratch (one sample shift per
// event and a status word) is a file-scope __device__ array that every GPU
// loading this library holds until the process exits; the caller passes all
// inputs and the output in device memory.  Nothing here allocates: no
// cudaMalloc, cudaFree, cudaMallocAsync or host heap allocation.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/es.h"
#include "es_internal.h"

namespace {

// [0, ES_NOALLOC_MAX_EVENTS): per-event shift; [ES_NOALLOC_MAX_EVENTS]: status
constexpr int kScratchInts = ES_NOALLOC_MAX_EVENTS + 64;
static __device__ __align__(256) int g_noalloc_scratch[kScratchInts];

// Host code cannot use g_noalloc_scratch as an address (its host-side name is
// only a stand-in); the device address is looked up once per device and
// context (cudaGetSymbolAddress with that device current).  The cache is keyed
// on the context's unique id: after cudaDeviceReset the module is loaded again
// into a new primary context, at a new address, and the lookup runs again.
constexpr int kMaxDevices = 64;
struct ScratchEntry {
    unsigned long long ctx_id = 0;
    int* ptr = nullptr;
};
ScratchEntry g_scratch_dev[kMaxDevices];
std::mutex g_scratch_mu;

typedef CUresult (*CtxGetCurrent)(CUcontext*);
typedef CUresult (*CtxGetId)(CUcontext, unsigned long long*);

// the unique id of the calling thread's current context (0 if unknown)
unsigned long long current_context_id()
{
    static CtxGetCurrent get_current = nullptr;
    static CtxGetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrent>(p);
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetId>(p);
        cudaGetLastError();
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

int scratch_address(int** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ES_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return ES_ERR_ARG;
    // id 0 (no context current yet, or no driver entry point): look the address up again
    const unsigned long long id = current_context_id();
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    ScratchEntry& e = g_scratch_dev[dev];
    if (!e.ptr || id == 0 || e.ctx_id != id) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return ES_ERR_CUDA;
        e.ptr = static_cast<int*>(p);
        e.ctx_id = id;
    }
    *out = e.ptr;
    return ES_OK;
}

bool on_device(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// k_e = floor(t0 / dt + 1/2) in FP64 (the same operations es_superpose does on
// the host); status |= 1 for an event with a bad source index or a
// non-finite amplitude or origin time.
__global__ void noalloc_prepare(const int* src, const float* amps, const float* t0s, int n_events, int n_src,
                                double dt, int* shift, int* status)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_events; e += gridDim.x * blockDim.x) {
        const int s = src[e];
        const float t0 = t0s[e], a = amps[e];
        const bool bad = s < 0 || s >= n_src || !isfinite(t0) || !isfinite(a);
        double k = floor((double)t0 / dt + 0.5);
        k = fmax(-2e9, fmin(2e9, k));
        shift[e] = (int)k;
        if (bad) atomicOr(status, 1);
    }
}

}  // namespace

extern "C" int es_superpose_noalloc(const float* traces, int n_src, int n_rcv, int nt, const int* src_of_event,
                                    const float* amps, const float* t0s, int n_events, double dt, int n_out,
                                    float* gather, void* stream)
{
    if (!traces || !gather || n_src < 1 || n_rcv < 1 || nt < 1 || n_events < 0 || n_out < 1 || !(dt > 0))
        return ES_ERR_ARG;
    if (n_events > ES_NOALLOC_MAX_EVENTS) return ES_ERR_ARG;
    if (n_events > 0 && (!src_of_event || !amps || !t0s)) return ES_ERR_ARG;
    if (!on_device(traces) || !on_device(gather)) return ES_ERR_ARG;
    if (n_events > 0 && (!on_device(src_of_event) || !on_device(amps) || !on_device(t0s))) return ES_ERR_ARG;
    cudaGetLastError();
    int* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc != ES_OK) return rc;
    int* shift = scratch;
    int* status = scratch + ES_NOALLOC_MAX_EVENTS;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int h_status = 0;  // host stack, no allocation
    if (n_events > 0) {
        if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return ES_ERR_CUDA;
        noalloc_prepare<<<(n_events + 255) / 256, 256, 0, st>>>(src_of_event, amps, t0s, n_events, n_src, dt, shift,
                                                                status);
        if (cudaGetLastError() != cudaSuccess) return ES_ERR_CUDA;
        if (cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return ES_ERR_CUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) return ES_ERR_CUDA;
        if (h_status) return ES_ERR_ARG;  // nothing written to gather
    }
    if (es::launch_superpose(traces, n_src, n_rcv, nt, src_of_event, amps, shift, n_events, n_out, gather, st) !=
        cudaSuccess)
        return ES_ERR_CUDA;
    return ES_OK;
}
