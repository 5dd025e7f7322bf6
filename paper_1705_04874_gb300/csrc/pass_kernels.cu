// Instantiations, plan choice and launch of the fused derivative passes
// (fft_pass.cuh).
#include <mutex>

#include "fft_pass.cuh"

namespace es {

// Candidate two-stage plans n = RA * RB for every supported axis length (the
// x pass stages float4 chunks in groups of four, so n is a multiple of 16).
// The first candidate is the default; es_model_autotune may pick another.
#define ES_PLANS(X)                                                                                  \
    X(16, 4, 4)                                                                                      \
    X(32, 8, 4) X(32, 4, 8)                                                                          \
    X(48, 12, 4) X(48, 4, 12)                                                                        \
    X(64, 16, 4) X(64, 8, 8) X(64, 4, 16)                                                            \
    X(80, 16, 5) X(80, 5, 16)                                                                        \
    X(96, 16, 6) X(96, 6, 16)                                                                        \
    X(128, 16, 8) X(128, 8, 16)                                                                      \
    X(160, 16, 10) X(160, 10, 16)                                                                    \
    X(192, 16, 12) X(192, 12, 16)                                                                    \
    X(256, 16, 16)

namespace {
struct PlanRow {
    int n, ra, rb;
};
const PlanRow kPlans[] = {
#define ES_ROW(n, a, b) {n, a, b},
    ES_PLANS(ES_ROW)
#undef ES_ROW
};
constexpr int kNumPlans = sizeof(kPlans) / sizeof(kPlans[0]);
// chosen plan index per pass kind (0 = x, 1 = y/z) and axis length
int g_choice[2][257];
std::once_flag g_init;
void init_choice()
{
    for (int k = 0; k < 2; ++k)
        for (int n = 0; n <= 256; ++n) g_choice[k][n] = -1;
    for (int i = kNumPlans - 1; i >= 0; --i) {
        g_choice[0][kPlans[i].n] = i;
        g_choice[1][kPlans[i].n] = i;
    }
}
}  // namespace

int plan_radices(int n, int* ra, int* rb) { return plan_current(1, n, ra, rb); }

int plan_candidates(int n, int* ra, int* rb, int cap)
{
    int k = 0;
    for (int i = 0; i < kNumPlans && k < cap; ++i)
        if (kPlans[i].n == n) {
            ra[k] = kPlans[i].ra;
            rb[k] = kPlans[i].rb;
            ++k;
        }
    return k;
}

int plan_select(int kind, int n, int ra, int rb)
{
    std::call_once(g_init, init_choice);
    for (int i = 0; i < kNumPlans; ++i)
        if (kPlans[i].n == n && kPlans[i].ra == ra && kPlans[i].rb == rb) {
            g_choice[kind][n] = i;
            return 1;
        }
    return 0;
}

int plan_current(int kind, int n, int* ra, int* rb)
{
    std::call_once(g_init, init_choice);
    if (kind < 0 || kind > 1 || n < 1 || n > 256 || g_choice[kind][n] < 0) return 0;
    *ra = kPlans[g_choice[kind][n]].ra;
    *rb = kPlans[g_choice[kind][n]].rb;
    return 1;
}

template <int RA, int RB>
static cudaError_t launch_one(const PassParams& p, cudaStream_t st)
{
    constexpr int threads = pass_threads<RA, RB>();
    if (p.axis == 0) {
        const int lines = p.ny * p.nz;
        dim3 grid((lines + 2 * CP - 1) / (2 * CP) * p.nsim, p.njobs);
        return launch_pass_kernel(pass_x<RA, RB>, grid, threads, pass_smem_x<RA, RB>(), st, p);
    }
    const int ntx = (p.nx + 2 * CP - 1) / (2 * CP);
    const int outer = p.axis == 1 ? p.nz : p.ny;
    dim3 grid(ntx * outer * p.nsim, p.njobs);
    return launch_pass_kernel(pass_strided<RA, RB>, grid, threads, pass_smem_strided<RA, RB>(), st, p);
}

template <int RA, int RB>
static cudaError_t prepare_one()
{
    cudaError_t e = cudaFuncSetAttribute(pass_x<RA, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)pass_smem_x<RA, RB>());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(pass_strided<RA, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)pass_smem_strided<RA, RB>());
}

cudaError_t prepare_pass_kernels()
{
    cudaError_t e;
#define ES_PREP(n, a, b) if ((e = prepare_one<a, b>()) != cudaSuccess) return e;
    ES_PLANS(ES_PREP)
#undef ES_PREP
    return prepare_circ_kernels();
}

cudaError_t launch_pass(const PassParams& p, cudaStream_t st)
{
    if (p.circ) return launch_circ(p, st);
    int ra = 0, rb = 0;
    if (!plan_current(p.axis == 0 ? 0 : 1, p.n, &ra, &rb)) return cudaErrorInvalidValue;
#define ES_CASE(n, a, b) if (ra == a && rb == b) return launch_one<a, b>(p, st);
    ES_PLANS(ES_CASE)
#undef ES_CASE
    return cudaErrorInvalidValue;
}

}  // namespace es
