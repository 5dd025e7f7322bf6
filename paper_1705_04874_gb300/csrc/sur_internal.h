// Internal declarations of the surrogate network's kernels (not public ABI).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace es {

// C[M][N] = alpha op(A) op(B) + beta C (BF16 operands, FP32 accumulate); see
// sur_gemm.cu.  Leading dimensions and K multiples of 8.
cudaError_t gemm_bf16(int M, int N, int K, const __nv_bfloat16* A, int lda, bool a_t, const __nv_bfloat16* B,
                      int ldb, bool b_nk, float* C, int ldc, float alpha, float beta, int split_k, cudaStream_t st);

// the K-major case (A [M][K], B [N][K]) on tcgen05 tensor cores; see sur_gemm_tc.cu.
// alpha4 (host, 4 values) with span > 0: column n of C takes alpha4[n / span] instead of
// alpha (4 span >= N), e.g. one scale per output component of the decoder
cudaError_t gemm_bf16_tc(int M, int N, int K, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb,
                         float* C, int ldc, float alpha, float beta, int split_k, cudaStream_t st,
                         const float* alpha4 = nullptr, int span = 0);
// reads and clears the tcgen05 GEMM's device status word (bits set by waits that gave up)
cudaError_t gemm_tc_status(unsigned* status);
// Launches one kernel whose bounded wait on a barrier nothing completes gives
// up after `seconds` (0 < seconds <= 2) and sets the status word.
cudaError_t gemm_wait_probe(double seconds, cudaStream_t st);
// out[c][r] = in[r][c] for a rows x cols BF16 matrix (row-major both)
cudaError_t transpose_bf16(const __nv_bfloat16* in, long long rows, long long cols, __nv_bfloat16* out,
                           cudaStream_t st);

cudaError_t scale_f32(float* C, int M, int N, int ldc, float s, cudaStream_t st);
cudaError_t cast_bf16(const float* x, __nv_bfloat16* y, size_t n, cudaStream_t st);
// position features: [p, sin(2^j pi p), cos(2^j pi p)], j < nfreq, zero padded to width
cudaError_t sur_features(const float* pos, int B, int nfreq, int width, __nv_bfloat16* X, cudaStream_t st);
// Y = relu(Y + bias) (in place, FP32) and its BF16 copy; relu = false: bias only
cudaError_t sur_bias_act(float* Y, const float* bias, int B, int N, bool relu, __nv_bfloat16* Yb, cudaStream_t st);
// G = G * (H > 0) in place, with its BF16 copy
cudaError_t sur_relu_grad(float* G, const float* H, size_t n, __nv_bfloat16* Gb, cudaStream_t st);
// Z[b][c K + k] = M[b][c] A[b][k] (BF16)
cudaError_t sur_outer(const float* M6, const float* A, int B, int K, __nv_bfloat16* Z, cudaStream_t st);
// dA[b][k] = sum_c M[b][c] dZ[b][c K + k], FP32 and BF16
cudaError_t sur_contract(const float* M6, const float* dZ, int B, int K, float* dA, __nv_bfloat16* dAb,
                         cudaStream_t st);
// outputs [B][4][Dc], y = scale[c] u, tau = t / scale[c]: per sample
// l_b = sum_c |u_c - tau_c|^2 / (sum_c |tau_c|^2 + eps) (squared relative L2 of
// the component-scaled seismogram), loss = mean_b l_b (device float),
// per_sample (optional, device [B]) = l_b, dU = dloss/du in BF16 (skipped when
// null); acc: device scratch of 2 B floats
cudaError_t sur_loss(const float* U, const float* T, const float* scale, int B, long long Dc, float eps,
                     __nv_bfloat16* dU, float* loss, float* acc, float* per_sample, cudaStream_t st);
cudaError_t sur_init_normal(float* p, size_t n, float std, unsigned long long seed, cudaStream_t st);
// ss[c] = sum of squares of component c over n samples [n][4][Dc]
cudaError_t sur_comp_sumsq(const float* T, int n, long long Dc, float* ss, cudaStream_t st);
// out[b] = sum_c mt[b][c] G[loc[b]][c] (G: [n_loc][6][D])
cudaError_t sur_combine(const float* G, long long D, const int* loc, const float* mt, int B, float* out,
                        cudaStream_t st);
// db[n] = sum_b G[b][n]
cudaError_t sur_colsum(const float* G, int B, int N, float* db, cudaStream_t st);
// Adam step (bias-corrected, lr, b1, b2, eps) on FP32 params, refreshing the BF16 copy (may be null)
cudaError_t sur_adam(float* p, const float* g, float* m, float* v, size_t n, float lr, float b1, float b2, float eps,
                     int t, __nv_bfloat16* pb, cudaStream_t st);
// The same step on a row-major [rows][cols] block (the decoder; cols a multiple
// of 4, 16-byte aligned), writing the BF16 copy both row-major (pb) and
// transposed (pt, [cols][rows]) -- one pass over the parameters instead of a
// step plus a transpose.
cudaError_t sur_adam_t(float* p, const float* g, float* m, float* v, long long rows, long long cols, float lr,
                       float b1, float b2, float eps, int t, __nv_bfloat16* pb, __nv_bfloat16* pt, cudaStream_t st);

}  // namespace es
