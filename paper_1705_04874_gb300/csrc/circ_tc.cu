// Circulant derivative passes on the fifth-generation tensor cores, for axes
// without an FFT plan of CIRC_TC_N (192) to 512 cells in FP32 mode (the
// 301-cell axis of the paper's 125 x 75 x 301 grid).  Along the axis the
// staggered derivative is the dense contraction out[o][p] = sum_i C[o][i]
// f[i][p] (circulant C, pencils p), so it runs as a tcgen05 GEMM whose A
// operand is a tile of 128 pencils (the field, K = inputs) and whose B operand
// is the kernel matrix (N = outputs, K = inputs).
//
// FP32 accuracy from BF16 products: each field value is split exactly into
// three BF16 parts (f = f0 + f1 + f2, computed in FP32 by the converter
// warps), each kernel value into three BF16 parts on the host (c = c0 + c1 +
// c2 to about 2^-24), and the six products with split orders summing to at
// most 2 are accumulated in FP32 in tensor memory; the three dropped products
// are below 2^-24 of the result, the size of FP32 rounding.
//
// One CTA per tile of 128 pencils and one job, 10 warps:
//   warp 0, one thread: TMA producer of the kernel-matrix splits, in chunks
//       of up to 256 outputs x 64 inputs, through a 3-stage ring;
//   warp 1: allocates tensor memory; one thread issues tcgen05.mma (M 128,
//       N 256 or the remaining outputs, a multiple of 64; K 16) into the
//       accumulator (columns = outputs);
//   warps 2-9: converters -- per k-block of 64 inputs they load the field
//       block (coalesced along the pencils; a thread's 32 loads of a block all
//       in flight at once), split it, and write the three 128 x 64 BF16 tiles
//       in the 128-byte-swizzled K-major layout the MMA reads
//       (double-buffered); then the epilogue (two warps per lane quarter,
//       each half of the output columns): tensor-memory lane =
//       pencil, so each tcgen05.ld gives a thread 32 consecutive outputs of
//       its pencil, and a warp stores 32 consecutive cells of the derivative
//       per instruction into a scratch array (plain stores: nothing to wait
//       for).  The field update with its PML splits then runs as a separate
//       element-wise kernel at full occupancy (circ_tc_update_kernel along z,
//       circ_tc_update_xy_kernel along x and y): done here by the few
//       epilogue warps of one CTA per SM, its dependent coefficient loads made
//       the pass latency-bound.
// Every mbarrier wait is bounded; a wait that runs out records a status bit
// (circ_tc_status) and the CTA finishes.
#include <algorithm>

#include "es_internal.h"
#include "fft_pass.cuh"
#include "tc_ptx.cuh"

namespace es {
namespace {

using namespace tcx;

constexpr int CT_P = 128;                   // pencils per tile (MMA M, tensor-memory lanes)
constexpr int CT_K = 64;                    // inputs per k-block (one 128-byte swizzle row of BF16)
constexpr int CT_OC = 256;                  // outputs per MMA chunk (MMA N)
constexpr int CT_A_SPLIT = CT_P * CT_K * 2;  // 16 KB: one split of a field block
constexpr int CT_A_BUF = 3 * CT_A_SPLIT;    // 48 KB per k-block
constexpr int CT_B_STAGE = CT_OC * CT_K * 2;  // 32 KB: one split of one output chunk
constexpr int CT_B_STAGES = 3;
constexpr int CT_SMEM = 2 * CT_A_BUF + CT_B_STAGES * CT_B_STAGE + 1024;
constexpr int CT_THREADS = 320;
constexpr int CT_CONV = 256;                // converter / epilogue threads (warps 2-9)

__device__ unsigned g_ctc_status;  // bit 0 producer, 1 MMA, 2 converter, 3 epilogue, 4 drain gave up

struct CircMaps {
    CUtensorMap m[6];  // kernel-matrix splits: [sign D+ / D-][split 0..2], rows = outputs, K = inputs
};

// instruction descriptor for kind::f16, D FP32, A and B BF16, both K-major, M 128, N = n
__device__ __forceinline__ uint32_t ct_idesc(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(CT_P >> 4) << 24);
}

// byte offset of element (row r, k) in a 128-byte-swizzled K-major BF16 tile (64 per row)
__device__ __forceinline__ uint32_t sw128_off(int r, int k)
{
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((((k >> 3) ^ (r & 7)) & 7) << 4) + ((k & 7) << 1));
}

// Pencils of a pass along `axis`: z: x + nx y; y: x + nx z; x: the line y + ny z.
__host__ __device__ inline long long pass_pencils(const PassParams& p)
{
    return p.axis == 2 ? (long long)p.nx * p.ny : p.axis == 1 ? (long long)p.nx * p.nz : (long long)p.ny * p.nz;
}
// stride between consecutive positions of a pencil, and the linear index of its position 0
__device__ __forceinline__ size_t pass_stride(const PassParams& p)
{
    return p.axis == 2 ? (size_t)p.nx * p.ny : p.axis == 1 ? (size_t)p.nx : (size_t)1;
}
__device__ __forceinline__ size_t pencil_base(const PassParams& p, long long pl)
{
    if (p.axis == 2) return (size_t)pl;
    if (p.axis == 1) return (size_t)(pl % p.nx) + (size_t)p.nx * p.ny * (size_t)(pl / p.nx);
    return (size_t)pl * p.nx;
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__global__ void __launch_bounds__(CT_THREADS, 1) circ_tc_kernel(const __grid_constant__ PassParams p,
                                                                const __grid_constant__ CircMaps maps)
{
    extern __shared__ uint8_t dyn[];
    __shared__ __align__(8) uint64_t a_full[2], a_empty[2], b_full[CT_B_STAGES], b_empty[CT_B_STAGES], acc_full;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_issued, s_consumed;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t base = (smem_u32(dyn) + 1023u) & ~1023u;
    uint8_t* gbase = dyn + (base - smem_u32(dyn));  // generic pointer to the aligned base
    const uint32_t a_base = base, b_base = base + 2 * CT_A_BUF;

    const int n = p.n, nkb = (n + CT_K - 1) / CT_K;
    const int nop = (n + 63) / 64 * 64;                 // outputs padded to whole 64-row boxes
    const int noc = (nop + CT_OC - 1) / CT_OC;         // output chunks
    const long long P = pass_pencils(p);
    const int ntile = (int)((P + CT_P - 1) / CT_P);
    const int u = blockIdx.x;
    const int job = u / (p.nsim * ntile), rr = u % (p.nsim * ntile);
    const int sim = rr % p.nsim, tile = rr / p.nsim;
    const long long p0 = (long long)tile * CT_P;
    const PassJob& J = p.job[job];
    const size_t est = pass_stride(p);
    const size_t off = (size_t)sim * p.fstride;

    if (threadIdx.x == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(&a_full[s], CT_CONV);
            mbar_init(&a_empty[s], 1);
        }
        for (int s = 0; s < CT_B_STAGES; ++s) {
            mbar_init(&b_full[s], 1);
            mbar_init(&b_empty[s], 1);
        }
        mbar_init(&acc_full, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_issued = 0;
        s_consumed = 0;
    }
    __syncwarp();
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(512u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    pdl_begin(p.pdl);

    if (warp == 0) {
        if (lane == 0) {
            // kernel-matrix splits: for every k-block, split and output chunk in the MMA's order
            const int mb = J.sign > 0 ? 0 : 3;
            int it = 0;
            bool ok = true;
            for (int kb = 0; kb < nkb && ok; ++kb)
                for (int sb = 0; sb < 3 && ok; ++sb)
                    for (int oc = 0; oc < noc; ++oc, ++it) {
                        const int s = it % CT_B_STAGES;
                        if (!mbar_wait(&b_empty[s], ((it / CT_B_STAGES) & 1) ^ 1)) {
                            atomicOr(&g_ctc_status, 1u);
                            ok = false;
                            break;
                        }
                        const int rows = min(CT_OC, nop - oc * CT_OC);  // a multiple of 64
                        mbar_expect_tx(&b_full[s], (unsigned)rows * 128u);
                        for (int bx = 0; bx < rows / 64; ++bx)
                            tma_load_2d(b_base + s * CT_B_STAGE + bx * 8192, &maps.m[mb + sb], &b_full[s], kb * CT_K,
                                        oc * CT_OC + bx * 64);
                    }
            s_issued = it;
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int it = 0;
            bool ok = true;
            for (int kb = 0; kb < nkb && ok; ++kb) {
                const int a = kb & 1;
                if (!mbar_wait(&a_full[a], (kb >> 1) & 1)) {
                    atomicOr(&g_ctc_status, 2u);
                    break;
                }
                tc_fence_after();
                for (int sb = 0; sb < 3 && ok; ++sb)
                    for (int oc = 0; oc < noc; ++oc, ++it) {
                        const int s = it % CT_B_STAGES;
                        if (!mbar_wait(&b_full[s], (it / CT_B_STAGES) & 1)) {
                            atomicOr(&g_ctc_status, 2u);
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const int rows = min(CT_OC, nop - oc * CT_OC);
                        const uint32_t idesc = ct_idesc(rows);
                        const uint64_t db = sw128_desc(b_base + s * CT_B_STAGE);
                        // field splits sa with sa + sb <= 2
                        for (int sa = 0; sa + sb <= 2; ++sa) {
                            const uint64_t da = sw128_desc(a_base + a * CT_A_BUF + sa * CT_A_SPLIT);
#pragma unroll
                            for (int k = 0; k < CT_K / 16; ++k) {
                                const uint64_t step = (uint64_t)((k * 32) >> 4);
                                const bool first = kb == 0 && sb == 0 && sa == 0 && k == 0;
                                tc_mma(tmem + (uint32_t)(oc * CT_OC), da + step, db + step, idesc, first ? 0u : 1u);
                            }
                        }
                        tc_commit(&b_empty[s]);
                    }
                if (ok) tc_commit(&a_empty[a]);
            }
            s_consumed = it;
            if (ok) tc_commit(&acc_full);
        }
    } else {
        // converters: field block (64 inputs x 128 pencils) -> three BF16 tiles [pencil][input]
        const int t = threadIdx.x - 64;
        for (int kb = 0; kb < nkb; ++kb) {
            const int a = kb & 1;
            // one thread waits until the MMAs have released the buffer, the others follow at a named
            // barrier of the converter warps; a wait that runs out (after another role gave up) is
            // recorded and the block is written anyway (the results are then void, nothing hangs)
            if (t == 0 && !mbar_wait(&a_empty[a], ((kb >> 1) & 1) ^ 1)) atomicOr(&g_ctc_status, 4u);
            asm volatile("bar.sync 1, %0;" ::"r"(CT_CONV) : "memory");
            uint8_t* abuf = gbase + a * CT_A_BUF;
            // thread t owns pencil t mod 128 and inputs 32 (t / 128) .. +31 of the block: its 32 loads
            // in flight at once (coalesced over the threads), then each group of 8 consecutive inputs
            // goes out as one 16-byte store per split (one swizzle chunk; the 8 rows of a quarter-warp
            // hit 8 distinct bank groups)
            const int pr = t & (CT_P - 1), half = t >> 7;
            const long long pg = p0 + pr;
            const bool pv = pg < P;
            const float* col = J.src + off + pencil_base(p, pv ? pg : 0);
            float xv[32];
#pragma unroll
            for (int u = 0; u < 32; ++u) {
                const int gi = kb * CT_K + half * 32 + u;
                xv[u] = (pv && gi < n) ? __ldg(col + (size_t)gi * est) : 0.f;
            }
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                uint32_t w0[4], w1[4], w2[4];
#pragma unroll
                for (int u = 0; u < 8; u += 2) {
                    __nv_bfloat16 a0[2], a1[2], a2[2];
#pragma unroll
                    for (int v = 0; v < 2; ++v) {
                        const float x = xv[h * 8 + u + v];
                        a0[v] = __float2bfloat16_rn(x);
                        const float r1 = x - __bfloat162float(a0[v]);
                        a1[v] = __float2bfloat16_rn(r1);
                        a2[v] = __float2bfloat16_rn(r1 - __bfloat162float(a1[v]));
                    }
                    const __nv_bfloat162 p0v = __halves2bfloat162(a0[0], a0[1]);
                    const __nv_bfloat162 p1v = __halves2bfloat162(a1[0], a1[1]);
                    const __nv_bfloat162 p2v = __halves2bfloat162(a2[0], a2[1]);
                    w0[u / 2] = *reinterpret_cast<const uint32_t*>(&p0v);
                    w1[u / 2] = *reinterpret_cast<const uint32_t*>(&p1v);
                    w2[u / 2] = *reinterpret_cast<const uint32_t*>(&p2v);
                }
                const uint32_t o = sw128_off(pr, half * 32 + h * 8);  // start of the 16-byte chunk
                *reinterpret_cast<uint4*>(abuf + o) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
                *reinterpret_cast<uint4*>(abuf + CT_A_SPLIT + o) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
                *reinterpret_cast<uint4*>(abuf + 2 * CT_A_SPLIT + o) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
            }
            fence_proxy_async();  // generic-proxy stores become visible to the tensor cores
            mbar_arrive(&a_full[a]);
        }
        // epilogue: tensor-memory lane = pencil; 32 consecutive outputs per tcgen05.ld
        const int wq = warp & 3;  // the lane quarter this warp may read (warps 2..9 -> 2, 3, 0, 1, 2, ...)
        const int ch = (warp - 2) >> 2;  // which half of the 32-column groups: warps 2-5 and 6-9
        int got = 0;
        if (lane == 0) got = mbar_wait(&acc_full, 0) ? 1 : 0;
        got = __shfl_sync(0xffffffffu, got, 0);
        if (!got) {
            if (lane == 0) atomicOr(&g_ctc_status, 8u);
        } else {
            tc_fence_after();
            const long long pg = p0 + wq * 32 + lane;
            const bool pv = pg < P;
            const size_t pb = pencil_base(p, pv ? pg : 0);
            // the far part of the derivative to the scratch array (the update kernel adds the near part)
            float* dst = p.scratch + (size_t)job * p.nsim * p.fstride + off;
            for (int c0 = ch * 32; c0 < nop; c0 += 64) {
                __syncwarp();
                uint32_t r[32];
                tmem_ld32(tmem + ((uint32_t)(wq * 32) << 16) + (uint32_t)c0, r);
                if (!pv) continue;
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (c0 + j < n) dst[pb + (size_t)(c0 + j) * est] = __uint_as_float(r[j]);
            }
        }
    }

    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
        // copies issued but never consumed (only after a wait gave up) land before the CTA exits
        for (int it = s_consumed; it < s_issued; ++it)
            if (!mbar_wait(&b_full[it % CT_B_STAGES], (it / CT_B_STAGES) & 1)) {
                atomicOr(&g_ctc_status, 16u);
                break;
            }
    }
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u) : "memory");
    }
    // the pass completes only after the previous one (its update kernel then adds in stream order)
    if (p.pdl == 1) pdl_wait();
}

// The field update of the pass from the scratch derivatives (the far part: the GEMM's kernel
// matrices leave out the NEAR_TAPS central entries), plus the near stencil in FP32 from the
// source field, then the same arithmetic as the other passes' epilogues.  Along z the slab
// index is (x + nx y) + nx ny sp, so the pencil offset goes in as x with y = 0 (no division).
constexpr int UPD_Z = 4;

__device__ __forceinline__ void update_cell(const PassParams& p, const PassJob& J, size_t q, int pos, int x, int y,
                                            int z, float d, size_t off, size_t soff)
{
    if (J.kind == JOB_STORE) J.tgt[0][off + q] = d;
    else epilogue_one(p, J, q, pos, x, y, z, d, off, soff);
}

// x and y passes: cell-linear (coalesced), 4 cells per thread spaced by the grid
// size; the coordinates come from the linear index.  The slab index along y is
// x + nx (sp + S z); along x it is sp + S (y + ny z), so the line goes in as y with z = 0.
__global__ void circ_tc_update_xy_kernel(const __grid_constant__ PassParams p)
{
    const int job = blockIdx.y / p.nsim, sim = blockIdx.y % p.nsim;
    const PassJob& J = p.job[job];
    const unsigned cells = (unsigned)p.nx * p.ny * p.nz;
    const size_t off = (size_t)sim * p.fstride, soff = (size_t)sim * p.sstride;
    const float* d = p.scratch + (size_t)job * p.nsim * p.fstride + off;
    const float* f = J.src + off;
    const int ofs = near_ofs(J.sign);
    const unsigned stride = gridDim.x * blockDim.x;
    unsigned q0 = blockIdx.x * blockDim.x + threadIdx.x;
    for (; q0 < cells; q0 += UPD_Z * stride) {
        float dv[UPD_Z];
#pragma unroll
        for (int k = 0; k < UPD_Z; ++k) {
            const unsigned q = q0 + k * stride;
            dv[k] = q < cells ? d[q] : 0.f;
        }
#pragma unroll
        for (int k = 0; k < UPD_Z; ++k) {
            const unsigned q = q0 + k * stride;
            if (q >= cells) break;
            const unsigned x = q % p.nx, line = q / p.nx;
            // near stencil along the pass axis (wrapped), taps in order
            const int pos = p.axis == 0 ? (int)x : (int)(line % p.ny);
            const size_t base = p.axis == 0 ? (size_t)line * p.nx : (size_t)q - (size_t)pos * p.nx;
            const size_t est = p.axis == 0 ? 1 : (size_t)p.nx;
            float v[NEAR_TAPS];
#pragma unroll
            for (int t = 0; t < NEAR_TAPS; ++t) {
                int i = pos + ofs + t;
                i += i < 0 ? p.n : 0;
                i -= i >= p.n ? p.n : 0;
                v[t] = __ldg(f + base + (size_t)i * est);
            }
            float s = 0.f;
#pragma unroll
            for (int t = 0; t < NEAR_PAIRS; ++t) s = __fmaf_rn(J.g[t], __fsub_rn(v[t], v[NEAR_TAPS - 1 - t]), s);
            s = __fadd_rn(dv[k], s);
            if (p.axis == 0)
                update_cell(p, J, q, (int)x, (int)x, (int)line, 0, s, off, soff);
            else
                update_cell(p, J, q, (int)(line % p.ny), (int)x, (int)(line % p.ny), (int)(line / p.ny), s, off, soff);
        }
    }
}

// z passes: blockIdx.x over the pencils (x + nx y), blockIdx.y over groups of UPD_Z
// positions along z, blockIdx.z = job x simulation; the near stencil slides over the
// UPD_Z + NEAR_TAPS - 1 inputs of the group (each read once)
__global__ void circ_tc_update_kernel(const __grid_constant__ PassParams p)
{
    const int job = blockIdx.z / p.nsim, sim = blockIdx.z % p.nsim;
    const PassJob& J = p.job[job];
    const int P = p.nx * p.ny;
    const int pxy = blockIdx.x * blockDim.x + threadIdx.x;
    if (pxy >= P) return;
    const size_t off = (size_t)sim * p.fstride, soff = (size_t)sim * p.sstride;
    const float* d = p.scratch + (size_t)job * p.nsim * p.fstride + off;
    const float* f = J.src + off + pxy;
    const int z0 = blockIdx.y * UPD_Z;
    const int ofs = near_ofs(J.sign);
    float dv[UPD_Z], v[UPD_Z + NEAR_TAPS - 1];
#pragma unroll
    for (int k = 0; k < UPD_Z; ++k) dv[k] = z0 + k < p.n ? d[(size_t)pxy + (size_t)(z0 + k) * P] : 0.f;
#pragma unroll
    for (int m = 0; m < UPD_Z + NEAR_TAPS - 1; ++m) {
        int i = z0 + ofs + m;
        i += i < 0 ? p.n : 0;
        i -= i >= p.n ? p.n : 0;
        v[m] = __ldg(f + (size_t)i * P);
    }
#pragma unroll
    for (int k = 0; k < UPD_Z; ++k) {
        float s = 0.f;
#pragma unroll
        for (int t = 0; t < NEAR_PAIRS; ++t) s = __fmaf_rn(J.g[t], __fsub_rn(v[k + t], v[k + NEAR_TAPS - 1 - t]), s);
        dv[k] = __fadd_rn(dv[k], s);
    }
#pragma unroll
    for (int k = 0; k < UPD_Z; ++k)
        if (z0 + k < p.n) update_cell(p, J, (size_t)pxy + (size_t)(z0 + k) * P, z0 + k, pxy, 0, z0 + k, dv[k], off, soff);
}

}  // namespace

bool circ_tc_eligible(const PassParams& p)
{
    return p.circ && !p.comp && p.n >= CIRC_TC_N && p.n <= CIRC_MAX_N && p.ctc && p.scratch &&
           (long long)p.nx * p.ny * p.nz < (1LL << 31);
}

cudaError_t launch_circ_tc(const PassParams& p, cudaStream_t st)
{
    if (!circ_tc_eligible(p)) return cudaErrorInvalidValue;
    EncodeTiled fn = encode_tiled();
    if (!fn) return cudaErrorNotSupported;
    const int nop = (p.n + 63) / 64 * 64;
    CircMaps maps;
    for (int k = 0; k < 6; ++k)
        if (!make_map(fn, &maps.m[k], p.ctc + (size_t)k * nop * nop, nop, nop, nop, 64))
            return cudaErrorInvalidValue;
    const long long P = pass_pencils(p);
    const long long grid = (long long)p.njobs * p.nsim * ((P + CT_P - 1) / CT_P);
    if (grid > 0x7fffffffLL) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(circ_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, CT_SMEM);
    if (e != cudaSuccess) return e;
    // as launch_pass_kernel, with the tensor maps as a second parameter
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(CT_THREADS);
    cfg.dynamicSmemBytes = CT_SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = p.pdl ? 1 : 0;
    e = cudaLaunchKernelEx(&cfg, circ_tc_kernel, p, maps);
    if (e != cudaSuccess) return e;
    if (p.axis == 2) {
        circ_tc_update_kernel<<<dim3((unsigned)((P + 127) / 128), (unsigned)((p.n + UPD_Z - 1) / UPD_Z),
                                     (unsigned)(p.njobs * p.nsim)),
                                128, 0, st>>>(p);
    } else {
        const long long cells = (long long)p.nx * p.ny * p.nz;
        const long long bx = std::max<long long>(1, std::min<long long>((cells + 256 * UPD_Z - 1) / (256 * UPD_Z), 152 * 16));
        circ_tc_update_xy_kernel<<<dim3((unsigned)bx, (unsigned)(p.njobs * p.nsim)), 256, 0, st>>>(p);
    }
    return cudaGetLastError();
}

cudaError_t circ_tc_status(unsigned* status)
{
    unsigned v = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_ctc_status, sizeof v);
    if (e != cudaSuccess) return e;
    *status = v;
    if (v) {
        const unsigned zero = 0;
        e = cudaMemcpyToSymbol(g_ctc_status, &zero, sizeof zero);
    }
    return e;
}

}  // namespace es
