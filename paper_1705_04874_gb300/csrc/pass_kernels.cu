// Instantiations and launch of the fused derivative passes (fft_pass.cuh).
#include "fft_pass.cuh"

namespace es {

// Two-stage plan n = RA * RB for every supported axis length.  The x pass
// stages float4 chunks in groups of four, so n is a multiple of 16.
int plan_radices(int n, int* ra, int* rb)
{
    static const int table[][3] = {{16, 4, 4},   {32, 8, 4},    {48, 12, 4},   {64, 16, 4},
                                   {80, 16, 5},  {96, 16, 6},   {128, 16, 8},  {160, 16, 10},
                                   {192, 16, 12}, {256, 16, 16}};
    for (auto& t : table)
        if (t[0] == n) {
            *ra = t[1];
            *rb = t[2];
            return 1;
        }
    return 0;
}

template <int RA, int RB>
static cudaError_t launch_one(const PassParams& p, cudaStream_t st)
{
    constexpr int threads = pass_threads<RA, RB>();
    if (p.axis == 0) {
        const int lines = p.ny * p.nz;
        dim3 grid((lines + 2 * CP - 1) / (2 * CP) * p.nsim, p.njobs);
        pass_x<RA, RB><<<grid, threads, pass_smem<RA, RB, CP + 1>(), st>>>(p);
    } else {
        const int ntx = (p.nx + 2 * CP - 1) / (2 * CP);
        const int outer = p.axis == 1 ? p.nz : p.ny;
        dim3 grid(ntx * outer * p.nsim, p.njobs);
        pass_strided<RA, RB><<<grid, threads, pass_smem<RA, RB, CP>(), st>>>(p);
    }
    return cudaGetLastError();
}

template <int RA, int RB>
static cudaError_t prepare_one()
{
    cudaError_t e = cudaFuncSetAttribute(pass_x<RA, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)pass_smem<RA, RB, CP + 1>());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(pass_strided<RA, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)pass_smem<RA, RB, CP>());
}

#define ES_PLANS(X) X(4, 4) X(8, 4) X(12, 4) X(16, 4) X(16, 5) X(16, 6) X(16, 8) X(16, 10) X(16, 12) X(16, 16)

cudaError_t prepare_pass_kernels()
{
    cudaError_t e;
#define ES_PREP(a, b) if ((e = prepare_one<a, b>()) != cudaSuccess) return e;
    ES_PLANS(ES_PREP)
#undef ES_PREP
    return cudaSuccess;
}

cudaError_t launch_pass(const PassParams& p, cudaStream_t st)
{
    int ra = 0, rb = 0;
    if (!plan_radices(p.n, &ra, &rb)) return cudaErrorInvalidValue;
#define ES_CASE(a, b) if (ra == a && rb == b) return launch_one<a, b>(p, st);
    ES_PLANS(ES_CASE)
#undef ES_CASE
    return cudaErrorInvalidValue;
}

}  // namespace es
