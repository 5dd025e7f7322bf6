// Instantiations, plan choice and launch of the fused derivative passes
// (fft_pass.cuh).
#include <mutex>

#include "fft_pass.cuh"
#include "pass_plans.h"

namespace es {

namespace {
struct PlanRow {
    int n, ra, rb, rc;
};
const PlanRow kPlans[] = {
#define ES_ROW(n, a, b, c) {n, a, b, c},
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
            rb[k] = kPlans[i].rb * kPlans[i].rc;
            ++k;
        }
    return k;
}

int plan_select(int kind, int n, int ra, int rb)
{
    std::call_once(g_init, init_choice);
    for (int i = 0; i < kNumPlans; ++i)
        if (kPlans[i].n == n && kPlans[i].ra == ra && kPlans[i].rb * kPlans[i].rc == rb) {
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
    *rb = kPlans[g_choice[kind][n]].rb * kPlans[g_choice[kind][n]].rc;
    return 1;
}

template <int RA, int RB, int RC>
static cudaError_t launch_one(const PassParams& p, cudaStream_t st)
{
    constexpr int threads = pass_threads<RA, RB, RC>();
    if (p.axis == 0) {
        const int lines = p.ny * p.nz;
        dim3 grid((lines + 2 * CP - 1) / (2 * CP) * p.nsim, p.njobs);
        return launch_pass_kernel(pass_x<RA, RB, RC>, grid, threads, pass_smem_x<RA, RB, RC>(), st, p);
    }
    const int ntx = (p.nx + 2 * CP - 1) / (2 * CP);
    const int outer = p.axis == 1 ? p.nz : p.ny;
    dim3 grid(ntx * outer * p.nsim, p.njobs);
    if (p.nx % 2) return launch_strided_odd(RA, RB, RC, grid, p, st);
    return launch_pass_kernel(pass_strided<RA, RB, RC, false>, grid, threads, pass_smem_strided<RA, RB, RC>(), st,
                              p);
}

template <int RA, int RB, int RC>
static cudaError_t prepare_one()
{
    cudaError_t e = cudaFuncSetAttribute(pass_x<RA, RB, RC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)pass_smem_x<RA, RB, RC>());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(pass_strided<RA, RB, RC, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)pass_smem_strided<RA, RB, RC>());
}

cudaError_t prepare_pass_kernels()
{
    cudaError_t e;
#define ES_PREP(n, a, b, c) if ((e = prepare_one<a, b, c>()) != cudaSuccess) return e;
    ES_PLANS(ES_PREP)
#undef ES_PREP
    if ((e = prepare_strided_odd()) != cudaSuccess) return e;
    return prepare_circ_kernels();
}

cudaError_t launch_pass(const PassParams& p, cudaStream_t st)
{
    if (p.circ) return launch_circ(p, st);
    std::call_once(g_init, init_choice);
    const int kind = p.axis == 0 ? 0 : 1;
    if (p.n < 1 || p.n > 256 || g_choice[kind][p.n] < 0) return cudaErrorInvalidValue;
    const PlanRow& r = kPlans[g_choice[kind][p.n]];
#define ES_CASE(n, a, b, c) if (r.ra == a && r.rb == b && r.rc == c) return launch_one<a, b, c>(p, st);
    ES_PLANS(ES_CASE)
#undef ES_CASE
    return cudaErrorInvalidValue;
}

}  // namespace es
