// BF16-input, FP32-accumulate GEMM for the surrogate network:
//   C[M][N] = alpha * op(A)[M][K] op(B)[K][N] + beta * C
// A is row-major [M][K] (lda) or, with a_t, stored [K][M]; B is stored
// [N][K] (b_nk, "column-major") or [K][N].  C is FP32 row-major (ldc).
// With split_k > 1 the K range is cut into slices whose partial products are
// added into C with atomics (C must hold beta * C already; alpha applies).
//
// CTA tile 128 x 128 x 32, 8 warps (2 x 4), warp tile 64 x 32, tensor-core
// mma.sync m16n8k16 bf16 -> f32; operand fragments come from shared memory
// through ldmatrix (transposing on the fly for the [K][M] / [K][N] storage
// orders); global -> shared tiles move with 16-byte cp.async, double
// buffered.  Out-of-range rows and columns are zero-filled.
// The K-major order of both operands (A [M][K], B [N][K]) runs on the
// tcgen05 tensor cores instead (sur_gemm_tc.cu).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "sur_internal.h"

namespace es {
namespace {

constexpr int BM = 128, BN = 128, BK = 32, PAD = 8;
constexpr int THREADS = 256;

__device__ __forceinline__ void cp16(void* dst, const void* src, bool ok)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(src), "r"(ok ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int K>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(K) : "memory"); }

__device__ __forceinline__ void ldsm_x4(unsigned (&r)[4], const void* p)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(s));
}
__device__ __forceinline__ void ldsm_x4_t(unsigned (&r)[4], const void* p)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(s));
}
__device__ __forceinline__ void mma16816(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// shared tiles: A as [BM][BK+PAD] (k contiguous) or [BK][BM+PAD]; B as
// [BN][BK+PAD] or [BK][BN+PAD]
template <bool AT, bool BNK>
struct Smem {
    static constexpr int A_ELEMS = AT ? BK * (BM + PAD) : BM * (BK + PAD);
    static constexpr int B_ELEMS = BNK ? BN * (BK + PAD) : BK * (BN + PAD);
    __nv_bfloat16 a[2][A_ELEMS];
    __nv_bfloat16 b[2][B_ELEMS];
};

template <bool AT, bool BNK>
__global__ void __launch_bounds__(THREADS) gemm_bf16_kernel(int M, int N, int K, const __nv_bfloat16* __restrict__ A,
                                                           int lda, const __nv_bfloat16* __restrict__ B, int ldb,
                                                           float* __restrict__ C, int ldc, float alpha, float beta,
                                                           int k_per_split)
{
    __shared__ __align__(128) Smem<AT, BNK> sm;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 2, wn = warp & 3;  // warp tile 64 x 32
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int kbeg = blockIdx.z * k_per_split;
    const int kend = min(K, kbeg + k_per_split);
    const int ntiles = (kend - kbeg + BK - 1) / BK;

    auto load_tile = [&](int stage, int k0) {
        // A: 512 chunks of 8 bf16
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int c = tid + i * THREADS;
            if (!AT) {
                const int r = c >> 2, kc = (c & 3) * 8;  // row m, 4 chunks per row
                const int gm = m0 + r, gk = k0 + kc;
                const bool ok = gm < M && gk < kend;
                cp16(&sm.a[stage][r * (BK + PAD) + kc], A + (ok ? (size_t)gm * lda + gk : 0), ok);
            } else {
                const int r = c >> 4, mc = (c & 15) * 8;  // row k, 16 chunks per row
                const int gk = k0 + r, gm = m0 + mc;
                const bool ok = gk < kend && gm < M;
                cp16(&sm.a[stage][r * (BM + PAD) + mc], A + (ok ? (size_t)gk * lda + gm : 0), ok);
            }
        }
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int c = tid + i * THREADS;
            if (BNK) {
                const int r = c >> 2, kc = (c & 3) * 8;
                const int gn = n0 + r, gk = k0 + kc;
                const bool ok = gn < N && gk < kend;
                cp16(&sm.b[stage][r * (BK + PAD) + kc], B + (ok ? (size_t)gn * ldb + gk : 0), ok);
            } else {
                const int r = c >> 4, nc = (c & 15) * 8;
                const int gk = k0 + r, gn = n0 + nc;
                const bool ok = gk < kend && gn < N;
                cp16(&sm.b[stage][r * (BN + PAD) + nc], B + (ok ? (size_t)gk * ldb + gn : 0), ok);
            }
        }
        cp_commit();
    };

    float acc[4][4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;

    if (ntiles > 0) load_tile(0, kbeg);
    for (int t = 0; t < ntiles; ++t) {
        const int st = t & 1;
        if (t + 1 < ntiles) {
            load_tile(st ^ 1, kbeg + (t + 1) * BK);
            cp_wait<1>();
        } else {
            cp_wait<0>();
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            unsigned af[4][4], bf[4][2];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int mb = wm * 64 + i * 16;
                if (!AT) {
                    const __nv_bfloat16* p = &sm.a[st][(mb + (lane & 15)) * (BK + PAD) + kk + (lane >> 4) * 8];
                    ldsm_x4(af[i], p);
                } else {
                    const int k = kk + (lane & 7) + ((lane >> 4) << 3);
                    const int m = mb + (((lane >> 3) & 1) << 3);
                    ldsm_x4_t(af[i], &sm.a[st][k * (BM + PAD) + m]);
                }
            }
#pragma unroll
            for (int j = 0; j < 4; j += 2) {  // two n8 tiles per ldmatrix.x4
                const int nb = wn * 32 + j * 8;
                unsigned r[4];
                if (BNK) {
                    // matrices: (n 0-7, k 0-7), (n 0-7, k 8-15), (n 8-15, k 0-7), (n 8-15, k 8-15)
                    const int n = nb + (lane & 7) + ((lane >> 4) << 3);
                    const int k = kk + (((lane >> 3) & 1) << 3);
                    ldsm_x4(r, &sm.b[st][n * (BK + PAD) + k]);
                } else {
                    // stored [k][n]: same four matrices, transposed on load
                    const int k = kk + (lane & 7) + (((lane >> 3) & 1) << 3);
                    const int n = nb + ((lane >> 4) << 3);
                    ldsm_x4_t(r, &sm.b[st][k * (BN + PAD) + n]);
                }
                bf[j][0] = r[0];
                bf[j][1] = r[1];
                bf[j + 1][0] = r[2];
                bf[j + 1][1] = r[3];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma16816(acc[i][j], af[i], bf[j][0], bf[j][1]);
        }
        __syncthreads();
    }

    // accumulator element e of tile (i, j): row = lane/4 (+8 for e >= 2), col = 2 (lane % 4) + (e & 1)
    const bool split = gridDim.z > 1;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int r = m0 + wm * 64 + i * 16 + (lane >> 2) + ((e >> 1) << 3);
                const int c = n0 + wn * 32 + j * 8 + ((lane & 3) << 1) + (e & 1);
                if (r < M && c < N) {
                    float* out = C + (size_t)r * ldc + c;
                    const float v = alpha * acc[i][j][e];
                    if (split) atomicAdd(out, v);
                    else *out = beta == 0.f ? v : v + beta * *out;
                }
            }
}

}  // namespace

cudaError_t gemm_bf16(int M, int N, int K, const __nv_bfloat16* A, int lda, bool a_t, const __nv_bfloat16* B,
                      int ldb, bool b_nk, float* C, int ldc, float alpha, float beta, int split_k, cudaStream_t st)
{
    if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
    if (!a_t && b_nk) return gemm_bf16_tc(M, N, K, A, lda, B, ldb, C, ldc, alpha, beta, split_k, st);
    if (split_k < 1) split_k = 1;
    int kps = (K + split_k - 1) / split_k;
    kps = (kps + BK - 1) / BK * BK;
    split_k = (K + kps - 1) / kps;
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, split_k);
    if (split_k > 1 && beta != 1.f) {
        // atomics add onto C: scale it first
        cudaError_t e = scale_f32(C, M, N, ldc, beta, st);
        if (e != cudaSuccess) return e;
    }
    if (!a_t && !b_nk) gemm_bf16_kernel<false, false><<<grid, THREADS, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, alpha, beta, kps);
    else if (a_t && b_nk) gemm_bf16_kernel<true, true><<<grid, THREADS, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, alpha, beta, kps);
    else gemm_bf16_kernel<true, false><<<grid, THREADS, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, alpha, beta, kps);
    return cudaGetLastError();
}

}  // namespace es
