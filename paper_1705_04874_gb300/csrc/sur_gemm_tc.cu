// BF16-input, FP32-accumulate GEMM on the fifth-generation tensor cores
// (tcgen05) for the K-major storage order of both operands:
//   C[M][N] = alpha * A[M][K] * B[N][K]^T + beta * C
// A row-major [M][K] (lda), B row-major [N][K] (ldb), C FP32 row-major (ldc).
//
// Persistent: one CTA per SM walks the 128 x 256 output tiles (x split_k
// slices of K) with stride gridDim.x, 6 warps:
//   warp 0, one thread: TMA producer -- 64-wide K slabs of A (128 rows) and
//       B (256 rows) into a 4-stage ring of 128-byte-swizzled shared tiles,
//       completion tracked by transaction-count mbarriers; it runs ahead
//       across tile boundaries;
//   warp 1, one thread: issues tcgen05.mma (M 128, N 256, K 16; both
//       operands from shared-memory descriptors) into one of two 256-column
//       FP32 accumulators in tensor memory (512 columns); tcgen05.commit
//       frees each stage and, at the end of a tile, hands the accumulator to
//       the epilogue;
//   warps 2-5: epilogue -- warp w owns TMEM lanes (tile rows)
//       32 (w mod 4) .. +31, reads 32 columns at a time with tcgen05.ld
//       (lane = row), turns the 32 x 32 block around in its own shared
//       buffer so that each store instruction covers four whole 128-byte row
//       segments, and writes alpha * acc + beta * C (split_k > 1: atomically
//       adds alpha * acc onto a C that already holds beta * C), then returns
//       the accumulator; the next tile's MMAs run in the other one meanwhile.
// Rows, columns and K past the matrix edge are zero-filled by TMA and masked
// in the epilogue.  Every mbarrier wait gives up after WAIT_NS of global
// time, records the role that gave up in a device status word (read and
// cleared by gemm_tc_status) and lets the CTA finish: the MMAs issued are
// awaited, TMA copies still in flight are awaited (both bounded) and the
// tensor memory is always freed.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "sur_internal.h"
#include "tc_ptx.cuh"

namespace es {
namespace {

using namespace tcx;

constexpr int TM = 128;  // tile rows = MMA M = TMEM lanes
constexpr int TN = 256;  // tile columns = MMA N = TMEM columns (FP32)
constexpr int TK = 64;   // K per stage: one 128-byte swizzle row of BF16
constexpr int UK = 16;   // K of one tcgen05.mma kind::f16
constexpr int STAGES = 4;
constexpr int A_BYTES = TM * TK * 2;
constexpr int B_BYTES = TN * TK * 2;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int EPI_LD = 36;  // row stride (floats) of an epilogue warp's 32 x 32 staging block: 16-byte rows
constexpr int EPI_BYTES = 4 * 32 * EPI_LD * 4;
// ring + staging + alignment slack for the 1024-byte swizzle atoms
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + EPI_BYTES + 1024;
constexpr int THREADS = 192;
constexpr unsigned TMEM_COLS = 2 * TN;  // two accumulators

static_assert(A_BYTES % 1024 == 0 && STAGE_BYTES % 1024 == 0, "swizzle atoms must stay 1024-byte aligned");
static_assert(TK == 64, "make_map boxes are 64 BF16 wide");

// instruction descriptor for kind::f16: D FP32 (bits 4-5 = 1), A BF16 (bits
// 7-9 = 1), B BF16 (bits 10-12 = 1), both K-major (bits 15, 16 = 0), N / 8 in
// bits 17-22, M / 16 in bits 24-28
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                           ((uint32_t)(TM >> 4) << 24);

__device__ unsigned g_tc_status;  // bit 0 producer, 1 MMA, 2 epilogue, 3 MMA drain, 4 TMA drain, 5 probe gave up

// The timeout path of the bounded waits, on demand: one thread waits, through
// mbar_wait, on the first phase of a fresh barrier that nothing arrives at,
// gives up after limit_ns, records bit 5 of the status word and returns.
__global__ void wait_probe_kernel(unsigned long long limit_ns)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (!mbar_wait(&bar, 0, limit_ns)) atomicOr(&g_tc_status, 32u);
    }
}

__global__ void __launch_bounds__(THREADS, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int M, int N,
                   int nkb, int kb_per, int mt, int ntl, int ntiles, float* __restrict__ C, int ldc, float alpha,
                   float beta, int atomic, float4 alpha4, int span)
{
    extern __shared__ uint8_t dyn[];
    __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], acc_full[2], acc_empty[2], mma_done;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_issued, s_consumed;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t base = (smem_u32(dyn) + 1023u) & ~1023u;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 4);  // one arrival per epilogue warp
        }
        mbar_init(&mma_done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_issued = 0;
        s_consumed = 0;
    }
    __syncwarp();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // producer: every k-block of every tile of this CTA, through the ring
            int it = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                const int mi = t % mt, rest = t / mt;
                const int ni = rest % ntl, kb0 = (rest / ntl) * kb_per;
                const int nk = min(nkb, kb0 + kb_per) - kb0;
                for (int kb = 0; kb < nk; ++kb, ++it) {
                    const int s = it % STAGES;
                    if (!mbar_wait(&empty[s], ((it / STAGES) & 1) ^ 1)) {
                        atomicOr(&g_tc_status, 1u);
                        ok = false;
                        break;
                    }
                    const uint32_t sa = base + s * STAGE_BYTES;
                    mbar_expect_tx(&full[s], STAGE_BYTES);
                    tma_load_2d(sa, &mapA, &full[s], (kb0 + kb) * TK, mi * TM);
                    tma_load_2d(sa + A_BYTES, &mapB, &full[s], (kb0 + kb) * TK, ni * TN);
                }
            }
            s_issued = it;
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer: accumulator b = local tile index mod 2
            int it = 0, lt = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++lt) {
                const int rest = t / mt;
                const int kb0 = (rest / ntl) * kb_per;
                const int nk = min(nkb, kb0 + kb_per) - kb0;
                const int b = lt & 1;
                if (!mbar_wait(&acc_empty[b], ((lt >> 1) & 1) ^ 1)) {
                    atomicOr(&g_tc_status, 2u);
                    break;
                }
                tc_fence_after();
                const uint32_t acc = tmem + (uint32_t)(b * TN);
                for (int kb = 0; kb < nk; ++kb, ++it) {
                    const int s = it % STAGES;
                    if (!mbar_wait(&full[s], (it / STAGES) & 1)) {
                        atomicOr(&g_tc_status, 2u);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = base + s * STAGE_BYTES;
                    const uint64_t da = sw128_desc(sa), db = sw128_desc(sa + A_BYTES);
#pragma unroll
                    for (int k = 0; k < TK / UK; ++k) {
                        const uint64_t step = (uint64_t)((k * UK * 2) >> 4);  // 32 bytes along the swizzled row
                        tc_mma(acc, da + step, db + step, IDESC, (kb | k) != 0);
                    }
                    tc_commit(&empty[s]);
                }
                if (ok) tc_commit(&acc_full[b]);
            }
            s_consumed = it;
            tc_commit(&mma_done);  // arrives when every MMA issued above has completed
        }
    } else {
        // epilogue warps 2..5: TMEM lane quarter q = warp mod 4
        const int q = warp & 3;
        const bool vec = (ldc & 3) == 0 && (reinterpret_cast<uintptr_t>(C) & 15) == 0;
        int lt = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++lt) {
            const int mi = t % mt, ni = (t / mt) % ntl;
            const int b = lt & 1;
            // one lane waits and the warp follows its result: tcgen05.ld below needs the whole warp
            int got = 0;
            if (lane == 0) got = mbar_wait(&acc_full[b], (lt >> 1) & 1) ? 1 : 0;
            got = __shfl_sync(0xffffffffu, got, 0);
            if (!got) {
                if (lane == 0) atomicOr(&g_tc_status, 4u);
                break;
            }
            tc_fence_after();
            const int n0 = ni * TN, row0 = mi * TM + q * 32;
            // this warp's staging block: row r (TMEM lane) at stage + r * EPI_LD
            float* stage = reinterpret_cast<float*>(dyn + (base - smem_u32(dyn)) + STAGES * STAGE_BYTES) +
                           q * 32 * EPI_LD;
            for (int c0 = 0; c0 < TN; c0 += 32) {
                if (n0 + c0 >= N) break;  // uniform over the warp
                __syncwarp();               // the previous block's reads of the staging rows are done
                uint32_t r[32];
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * TN + c0), r);
                float4* srow = reinterpret_cast<float4*>(stage + lane * EPI_LD);
                if (span) {
                    // per-column alpha: columns [c span, (c + 1) span) of C take component c of alpha4
                    float a[32];
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int col = n0 + c0 + j;
                        a[j] = (col < span ? alpha4.x : col < 2 * span ? alpha4.y : col < 3 * span ? alpha4.z
                                                                                                  : alpha4.w) *
                               __uint_as_float(r[j]);
                    }
#pragma unroll
                    for (int j = 0; j < 8; ++j) srow[j] = make_float4(a[4 * j], a[4 * j + 1], a[4 * j + 2], a[4 * j + 3]);
                } else {
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        srow[j] = make_float4(alpha * __uint_as_float(r[4 * j]), alpha * __uint_as_float(r[4 * j + 1]),
                                              alpha * __uint_as_float(r[4 * j + 2]), alpha * __uint_as_float(r[4 * j + 3]));
                }
                __syncwarp();
                // lane l stores columns 4 (l mod 8) .. +3 of row 4 i + l / 8: a warp instruction writes
                // four whole 128-byte row segments
                const int cc = n0 + c0 + 4 * (lane & 7);
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int rr = 4 * i + (lane >> 3), grow = row0 + rr;
                    if (grow >= M || cc >= N) continue;
                    float4 v = *reinterpret_cast<const float4*>(stage + rr * EPI_LD + 4 * (lane & 7));
                    float* p = C + (size_t)grow * ldc + cc;
                    if (vec && cc + 4 <= N) {
                        float4* dst = reinterpret_cast<float4*>(p);
                        if (atomic) {
                            atomicAdd(dst, v);
                        } else {
                            if (beta != 0.f) {
                                const float4 o = *dst;
                                v.x += beta * o.x;
                                v.y += beta * o.y;
                                v.z += beta * o.z;
                                v.w += beta * o.w;
                            }
                            *dst = v;
                        }
                    } else {
                        const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            if (cc + k >= N) break;
                            if (atomic) atomicAdd(p + k, e[k]);
                            else p[k] = beta != 0.f ? e[k] + beta * p[k] : e[k];
                        }
                    }
                }
            }
            // every tcgen05.ld of this warp has completed (tmem_ld32 waits): hand the accumulator back
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[b]);
        }
    }

    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
        if (!mbar_wait(&mma_done, 0)) atomicOr(&g_tc_status, 8u);
        // copies issued but never consumed (only after a wait gave up) must land before the CTA exits
        for (int it = s_consumed; it < s_issued; ++it)
            if (!mbar_wait(&full[it % STAGES], (it / STAGES) & 1)) {
                atomicOr(&g_tc_status, 16u);
                break;
            }
    }
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

}  // namespace

cudaError_t gemm_bf16_tc(int M, int N, int K, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb,
                         float* C, int ldc, float alpha, float beta, int split_k, cudaStream_t st,
                         const float* alpha4, int span)
{
    if (alpha4 && (span < 1 || (long long)4 * span < N)) return cudaErrorInvalidValue;
    const float4 av = alpha4 ? make_float4(alpha4[0], alpha4[1], alpha4[2], alpha4[3]) : make_float4(0.f, 0.f, 0.f, 0.f);
    if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
    if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15) return cudaErrorInvalidValue;
    if (lda % 8 || ldb % 8 || lda < K || ldb < K || ldc < N) return cudaErrorInvalidValue;
    EncodeTiled fn = encode_tiled();
    if (!fn) return cudaErrorNotSupported;
    alignas(64) CUtensorMap mapA, mapB;
    if (!make_map(fn, &mapA, A, M, K, lda, TM) || !make_map(fn, &mapB, B, N, K, ldb, TN))
        return cudaErrorInvalidValue;
    const int nkb = (K + TK - 1) / TK;
    if (split_k < 1) split_k = 1;
    if (split_k > nkb) split_k = nkb;
    const int kb_per = (nkb + split_k - 1) / split_k;
    split_k = (nkb + kb_per - 1) / kb_per;  // no empty slice
    const int mt = (M + TM - 1) / TM, ntl = (N + TN - 1) / TN;
    const long long ntiles = (long long)mt * ntl * split_k;
    if (ntiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    int dev = 0, sms = 0;
    cudaError_t e0 = cudaGetDevice(&dev);
    if (e0 == cudaSuccess) e0 = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e0 != cudaSuccess) return e0;
    const long long grid = ntiles < sms ? ntiles : sms;
    if (split_k > 1 && beta != 1.f) {
        cudaError_t e = scale_f32(C, M, N, ldc, beta, st);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaFuncSetAttribute(gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    gemm_tc_kernel<<<(unsigned)grid, THREADS, SMEM_BYTES, st>>>(mapA, mapB, M, N, nkb, kb_per, mt, ntl, (int)ntiles,
                                                               C, ldc, alpha, beta, split_k > 1 ? 1 : 0, av,
                                                               alpha4 ? span : 0);
    return cudaGetLastError();
}

cudaError_t gemm_wait_probe(double seconds, cudaStream_t st)
{
    if (!(seconds > 0.0) || seconds > 2.0) return cudaErrorInvalidValue;
    wait_probe_kernel<<<1, 32, 0, st>>>((unsigned long long)(seconds * 1e9));
    return cudaGetLastError();
}

cudaError_t gemm_tc_status(unsigned* status)
{
    unsigned v = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_tc_status, sizeof v);
    if (e != cudaSuccess) return e;
    *status = v;
    if (v) {
        const unsigned zero = 0;
        e = cudaMemcpyToSymbol(g_tc_status, &zero, sizeof zero);
    }
    return e;
}

}  // namespace es
