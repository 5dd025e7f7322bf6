// The y and z derivative passes for an odd nx (pass_strided<RA, RB, RC, true>),
// in a translation unit of their own so that they compile beside the others.
#include "fft_pass.cuh"
#include "pass_plans.h"

namespace es {

cudaError_t launch_strided_odd(int ra, int rb, int rc, dim3 grid, const PassParams& p, cudaStream_t st)
{
#define ES_CASE(n, a, b, c)                                                                               \
    if (ra == a && rb == b && rc == c)                                                                    \
        return launch_pass_kernel(pass_strided<a, b, c, true>, grid, pass_threads<a, b, c>(),               \
                                  pass_smem_strided<a, b, c>(), st, p);
    ES_PLANS(ES_CASE)
#undef ES_CASE
    return cudaErrorInvalidValue;
}

cudaError_t prepare_strided_odd()
{
    cudaError_t e;
#define ES_PREP(n, a, b, c)                                                                               \
    if ((e = cudaFuncSetAttribute(pass_strided<a, b, c, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                  (int)pass_smem_strided<a, b, c>())) != cudaSuccess)                     \
        return e;
    ES_PLANS(ES_PREP)
#undef ES_PREP
    return cudaSuccess;
}

}  // namespace es
