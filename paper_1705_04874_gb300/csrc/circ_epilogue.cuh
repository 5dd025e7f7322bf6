// Scalar field-update epilogue shared by the circulant passes (circ_pass.cu on
// the CUDA cores, circ_tc.cu on the tensor cores): the same arithmetic as the
// FFT passes' epilogue_pair (Eq. (2) with the split-field PML in the slabs),
// one cell at a time.
#pragma once
#include "fft_pass.cuh"

namespace es {

// scalar epilogue for one cell (same arithmetic as epilogue_pair)
__device__ __forceinline__ void epilogue_one(const PassParams& p, const PassJob& J, size_t q, int pos, int x, int y,
                                             int z, float d, size_t off, size_t soff)
{
    if (J.kind == JOB_STORE) {
        J.tgt[0][off + q] = d;
        return;
    }
    const float dt = p.dt;
    const bool slab = in_slab(pos, p.n, p.L);
    const int S = 2 * p.L + 1;
    if (J.kind == JOB_SINGLE) {
        float inc = increment(dt, __ldg(J.coef[0] + q), d);
        if (slab) {
            const float P = __ldg((J.stag ? p.ps : p.pc) + pos);
            const size_t si = slab_index(p.axis, x, y, z, slab_pos(pos, p.n, p.L), p.nx, p.ny, S);
            inc = split_delta(J.slab[0], soff + si, P, inc);
        }
        atomicAdd(J.tgt[0] + off + q, inc);
    } else {
        const float lam = __ldg(J.coef[0] + q), mu = __ldg(J.coef[1] + q);
        const float P = slab ? __ldg(p.pc + pos) : 1.f;
        const size_t si = slab ? slab_index(p.axis, x, y, z, slab_pos(pos, p.n, p.L), p.nx, p.ny, S) : 0;
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            float inc = increment(dt, normal_coef(lam, mu, t == J.diag), d);
            if (slab) inc = split_delta(J.slab[t], soff + si, P, inc);
            atomicAdd(J.tgt[t] + off + q, inc);
        }
    }
}

}  // namespace es
