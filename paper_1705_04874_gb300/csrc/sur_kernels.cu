// Element-wise and reduction kernels of the surrogate network (the GEMMs are
// in sur_gemm.cu).  All arithmetic in FP32; BF16 copies feed the GEMMs.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "sur_internal.h"

namespace es {
namespace {

inline int blocks_for(size_t n, int t = 256)
{
    size_t b = (n + t - 1) / t;
    return (int)(b > 65535 * 8 ? 65535 * 8 : b);
}

__global__ void scale_kernel(float* C, int M, int N, int ldc, float s)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)M * N; i += (size_t)gridDim.x * blockDim.x) {
        const size_t r = i / N, c = i % N;
        C[r * ldc + c] = s == 0.f ? 0.f : C[r * ldc + c] * s;  // s = 0 also clears NaN
    }
}

__global__ void cast_kernel(const float* x, __nv_bfloat16* y, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16(x[i]);
}

__global__ void features_kernel(const float* pos, int B, int nfreq, int width, __nv_bfloat16* X)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    __nv_bfloat16* row = X + (size_t)b * width;
    int k = 0;
    for (int a = 0; a < 3; ++a) row[k++] = __float2bfloat16(pos[3 * b + a]);
    for (int j = 0; j < nfreq; ++j)
        for (int a = 0; a < 3; ++a) {
            float s, c;
            sincospif(ldexpf(pos[3 * b + a], j), &s, &c);  // sin, cos of 2^j pi p
            row[k++] = __float2bfloat16(s);
            row[k++] = __float2bfloat16(c);
        }
    for (; k < width; ++k) row[k] = __float2bfloat16(0.f);
}

__global__ void bias_act_kernel(float* Y, const float* bias, int B, int N, bool relu, __nv_bfloat16* Yb)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)B * N; i += (size_t)gridDim.x * blockDim.x) {
        float v = Y[i] + bias[i % N];
        if (relu) v = fmaxf(v, 0.f);
        Y[i] = v;
        if (Yb) Yb[i] = __float2bfloat16(v);
    }
}

__global__ void relu_grad_kernel(float* G, const float* H, size_t n, __nv_bfloat16* Gb)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float g = H[i] > 0.f ? G[i] : 0.f;
        G[i] = g;
        Gb[i] = __float2bfloat16(g);
    }
}

__global__ void outer_kernel(const float* M6, const float* A, int B, int K, __nv_bfloat16* Z)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)B * 6 * K; i += (size_t)gridDim.x * blockDim.x) {
        const size_t b = i / (6 * (size_t)K), r = i % (6 * (size_t)K);
        const int c = (int)(r / K), k = (int)(r % K);
        Z[i] = __float2bfloat16(M6[6 * b + c] * A[b * K + k]);
    }
}

__global__ void contract_kernel(const float* M6, const float* dZ, int B, int K, float* dA, __nv_bfloat16* dAb)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)B * K; i += (size_t)gridDim.x * blockDim.x) {
        const size_t b = i / K, k = i % K;
        float s = 0.f;
        for (int c = 0; c < 6; ++c) s += M6[6 * b + c] * dZ[b * 6 * K + (size_t)c * K + k];
        dA[i] = s;
        dAb[i] = __float2bfloat16(s);
    }
}

// Loss in component-scaled units: with y = s_c u and tau = t / s_c,
// l_b = sum_c |u_c - tau_c|^2 / (sum_c |tau_c|^2 + eps) -- the relative L2
// error (squared) of the whole 4C seismogram after each component is divided
// by its scale.  Pass 1 (one block per sample and component) accumulates the
// two sums per sample; pass 2 writes l_b, the mean loss and dL/du.
__global__ void loss_sums_kernel(const float* U, const float* T, const float* scale, long long Dc, float* acc)
{
    const int b = blockIdx.x, c = blockIdx.y;
    const size_t base = ((size_t)b * 4 + c) * Dc;
    const float inv = 1.f / scale[c];
    float se = 0.f, st = 0.f;
    for (long long i = threadIdx.x; i < Dc; i += blockDim.x) {
        const float tau = T[base + i] * inv;
        const float d = U[base + i] - tau;
        se += d * d;
        st += tau * tau;
    }
    for (int o = 16; o > 0; o >>= 1) {
        se += __shfl_down_sync(0xffffffffu, se, o);
        st += __shfl_down_sync(0xffffffffu, st, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(acc + 2 * b, se);
        atomicAdd(acc + 2 * b + 1, st);
    }
}

__global__ void loss_grad_kernel(const float* U, const float* T, const float* scale, int B, long long Dc, float eps,
                                 const float* acc, __nv_bfloat16* dU, float* loss, float* per_sample)
{
    const int b = blockIdx.x, c = blockIdx.y;
    const float den = acc[2 * b + 1] + eps;
    if (c == 0 && threadIdx.x == 0) {
        const float lb = acc[2 * b] / den;
        if (per_sample) per_sample[b] = lb;
        atomicAdd(loss, lb / B);
    }
    if (!dU) return;
    const size_t base = ((size_t)b * 4 + c) * Dc;
    const float inv = 1.f / scale[c];
    const float g = 2.f / ((float)B * den);
    for (long long i = threadIdx.x; i < Dc; i += blockDim.x) dU[base + i] = __float2bfloat16(g * (U[base + i] - T[base + i] * inv));
}

// x ~ N(0, std^2) from a counter-based hash (splitmix64 of seed + index) and Box-Muller
__global__ void init_normal_kernel(float* p, size_t n, float std, unsigned long long seed)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (i + 1);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        const float u1 = ((z >> 40) + 1) * (1.0f / 16777217.0f);
        const float u2 = ((z >> 16) & 0xFFFFFF) * (1.0f / 16777216.0f);
        p[i] = std * sqrtf(-2.f * logf(u1)) * cospif(2.f * u2);
    }
}

// ss[c] += sum of t^2 over component c of every sample ([n][4][Dc])
__global__ void comp_sumsq_kernel(const float* T, int n, long long Dc, float* ss)
{
    const int b = blockIdx.x, c = blockIdx.y;
    const float* t = T + ((size_t)b * 4 + c) * Dc;
    float s = 0.f;
    for (long long i = threadIdx.x; i < Dc; i += blockDim.x) s += t[i] * t[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(ss + c, s);
}

// out[b][d] = sum_c mt[b][c] G[loc[b]][c][d]
__global__ void combine_kernel(const float* G, long long D, const int* loc, const float* mt, int B, float* out)
{
    const int b = blockIdx.y;
    const float* g = G + (size_t)loc[b] * 6 * D;
    const float m0 = mt[6 * b], m1 = mt[6 * b + 1], m2 = mt[6 * b + 2], m3 = mt[6 * b + 3], m4 = mt[6 * b + 4],
                m5 = mt[6 * b + 5];
    for (long long d = blockIdx.x * (long long)blockDim.x + threadIdx.x; d < D; d += (long long)gridDim.x * blockDim.x)
        out[(size_t)b * D + d] = m0 * g[d] + m1 * g[D + d] + m2 * g[2 * D + d] + m3 * g[3 * D + d] + m4 * g[4 * D + d] +
                                 m5 * g[5 * D + d];
}

__global__ void colsum_kernel(const float* G, int B, int N, float* db)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += G[(size_t)b * N + n];
    db[n] = s;
}

// one Adam update (bias corrections c1 = 1 - b1^t, c2 = 1 - b2^t); returns the new parameter
__device__ __forceinline__ float adam_one(float& p, float g, float& m, float& v, float lr, float b1, float b2,
                                          float eps, float c1, float c2)
{
    m = b1 * m + (1.f - b1) * g;
    v = b2 * v + (1.f - b2) * g * g;
    p = p - lr * (m / c1) / (sqrtf(v / c2) + eps);
    return p;
}

__global__ void adam_kernel(float* p, const float* g, float* m, float* v, size_t n, float lr, float b1, float b2,
                            float eps, float c1, float c2, __nv_bfloat16* pb)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float pi = p[i], mi = m[i], vi = v[i];
        adam_one(pi, g[i], mi, vi, lr, b1, b2, eps, c1, c2);
        m[i] = mi;
        v[i] = vi;
        p[i] = pi;
        if (pb) pb[i] = __float2bfloat16(pi);
    }
}

__device__ __forceinline__ void adam_four(float4& p, float4 g, float4& m, float4& v, float lr, float b1, float b2,
                                          float eps, float c1, float c2)
{
    adam_one(p.x, g.x, m.x, v.x, lr, b1, b2, eps, c1, c2);
    adam_one(p.y, g.y, m.y, v.y, lr, b1, b2, eps, c1, c2);
    adam_one(p.z, g.z, m.z, v.z, lr, b1, b2, eps, c1, c2);
    adam_one(p.w, g.w, m.w, v.w, lr, b1, b2, eps, c1, c2);
}

__device__ __forceinline__ uint2 pack_bf16x4(float4 p)
{
    const __nv_bfloat162 lo = __floats2bfloat162_rn(p.x, p.y), hi = __floats2bfloat162_rn(p.z, p.w);
    return make_uint2(*reinterpret_cast<const uint32_t*>(&lo), *reinterpret_cast<const uint32_t*>(&hi));
}

// four parameters per thread and iteration (n4 groups of four, 16-byte aligned)
__global__ void adam4_kernel(float4* p, const float4* g, float4* m, float4* v, size_t n4, float lr, float b1,
                             float b2, float eps, float c1, float c2, uint2* pb)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
        float4 pi = p[i], mi = m[i], vi = v[i];
        adam_four(pi, g[i], mi, vi, lr, b1, b2, eps, c1, c2);
        m[i] = mi;
        v[i] = vi;
        p[i] = pi;
        if (pb) pb[i] = pack_bf16x4(pi);
    }
}

// 64 x 64 tiles of a row-major [rows][cols] block: the update and the
// row-major BF16 copy four columns per thread, the transposed copy through a
// shared [column][row] tile, four rows per thread (8-byte stores)
constexpr int AT = 64, AT_LD = AT + 4;
__global__ void adam_t_kernel(float* p, const float* g, float* m, float* v, long long rows, long long cols, float lr,
                              float b1, float b2, float eps, float c1, float c2, __nv_bfloat16* pb,
                              __nv_bfloat16* pt)
{
    __shared__ __align__(16) __nv_bfloat16 tt[AT][AT_LD];
    const long long c0 = (long long)blockIdx.x * AT, r0 = (long long)blockIdx.y * AT;
    const int cq = threadIdx.x & 15, rq = threadIdx.x >> 4;  // 16 column quads x 16 rows per sweep
    for (int i = rq; i < AT; i += 16) {
        const long long r = r0 + i, c = c0 + 4 * cq;
        float4 pi = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r < rows && c < cols) {
            const size_t k = (size_t)r * cols + c;
            pi = *reinterpret_cast<const float4*>(p + k);
            float4 mi = *reinterpret_cast<const float4*>(m + k), vi = *reinterpret_cast<const float4*>(v + k);
            adam_four(pi, *reinterpret_cast<const float4*>(g + k), mi, vi, lr, b1, b2, eps, c1, c2);
            *reinterpret_cast<float4*>(m + k) = mi;
            *reinterpret_cast<float4*>(v + k) = vi;
            *reinterpret_cast<float4*>(p + k) = pi;
            *reinterpret_cast<uint2*>(pb + k) = pack_bf16x4(pi);
        }
        tt[4 * cq][i] = __float2bfloat16(pi.x);
        tt[4 * cq + 1][i] = __float2bfloat16(pi.y);
        tt[4 * cq + 2][i] = __float2bfloat16(pi.z);
        tt[4 * cq + 3][i] = __float2bfloat16(pi.w);
    }
    __syncthreads();
    for (int j = rq; j < AT; j += 16) {
        const long long c = c0 + j, r = r0 + 4 * cq;
        if (c >= cols || r >= rows) continue;
        const uint2 q = *reinterpret_cast<const uint2*>(&tt[j][4 * cq]);
        __nv_bfloat16* dst = pt + (size_t)c * rows + r;
        if (r + 4 <= rows && (rows & 3) == 0) {
            *reinterpret_cast<uint2*>(dst) = q;
        } else {
            const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&q);
            for (int k = 0; k < 4 && r + k < rows; ++k) dst[k] = e[k];
        }
    }
}

}  // namespace

cudaError_t scale_f32(float* C, int M, int N, int ldc, float s, cudaStream_t st)
{
    scale_kernel<<<blocks_for((size_t)M * N), 256, 0, st>>>(C, M, N, ldc, s);
    return cudaGetLastError();
}

// 64 x 64 tiles through shared memory (row padded by 2 elements: the column
// reads of the second half hit 32 distinct banks)
__global__ void transpose_bf16_kernel(const __nv_bfloat16* __restrict__ in, long long rows, long long cols,
                                      __nv_bfloat16* __restrict__ out)
{
    __shared__ __nv_bfloat16 t[64][66];
    const long long c0 = (long long)blockIdx.x * 64, r0 = (long long)blockIdx.y * 64;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int i = ty; i < 64; i += 8)
        for (int j = tx; j < 64; j += 32) {
            const long long r = r0 + i, c = c0 + j;
            t[i][j] = (r < rows && c < cols) ? in[r * cols + c] : __float2bfloat16(0.f);
        }
    __syncthreads();
    for (int i = ty; i < 64; i += 8)
        for (int j = tx; j < 64; j += 32) {
            const long long c = c0 + i, r = r0 + j;
            if (c < cols && r < rows) out[c * rows + r] = t[j][i];
        }
}

cudaError_t transpose_bf16(const __nv_bfloat16* in, long long rows, long long cols, __nv_bfloat16* out,
                           cudaStream_t st)
{
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    const long long gx = (cols + 63) / 64, gy = (rows + 63) / 64;
    if (gx > 0x7fffffffLL || gy > 65535) return cudaErrorInvalidValue;
    transpose_bf16_kernel<<<dim3((unsigned)gx, (unsigned)gy), 256, 0, st>>>(in, rows, cols, out);
    return cudaGetLastError();
}

cudaError_t cast_bf16(const float* x, __nv_bfloat16* y, size_t n, cudaStream_t st)
{
    cast_kernel<<<blocks_for(n), 256, 0, st>>>(x, y, n);
    return cudaGetLastError();
}

cudaError_t sur_features(const float* pos, int B, int nfreq, int width, __nv_bfloat16* X, cudaStream_t st)
{
    if (3 + 6 * nfreq > width) return cudaErrorInvalidValue;
    features_kernel<<<(B + 127) / 128, 128, 0, st>>>(pos, B, nfreq, width, X);
    return cudaGetLastError();
}

cudaError_t sur_bias_act(float* Y, const float* bias, int B, int N, bool relu, __nv_bfloat16* Yb, cudaStream_t st)
{
    bias_act_kernel<<<blocks_for((size_t)B * N), 256, 0, st>>>(Y, bias, B, N, relu, Yb);
    return cudaGetLastError();
}

cudaError_t sur_relu_grad(float* G, const float* H, size_t n, __nv_bfloat16* Gb, cudaStream_t st)
{
    relu_grad_kernel<<<blocks_for(n), 256, 0, st>>>(G, H, n, Gb);
    return cudaGetLastError();
}

cudaError_t sur_outer(const float* M6, const float* A, int B, int K, __nv_bfloat16* Z, cudaStream_t st)
{
    outer_kernel<<<blocks_for((size_t)B * 6 * K), 256, 0, st>>>(M6, A, B, K, Z);
    return cudaGetLastError();
}

cudaError_t sur_contract(const float* M6, const float* dZ, int B, int K, float* dA, __nv_bfloat16* dAb, cudaStream_t st)
{
    contract_kernel<<<blocks_for((size_t)B * K), 256, 0, st>>>(M6, dZ, B, K, dA, dAb);
    return cudaGetLastError();
}

cudaError_t sur_loss(const float* U, const float* T, const float* scale, int B, long long Dc, float eps,
                     __nv_bfloat16* dU, float* loss, float* acc, float* per_sample, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(float), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(acc, 0, 2 * sizeof(float) * B, st);
    if (e != cudaSuccess) return e;
    loss_sums_kernel<<<dim3(B, 4), 256, 0, st>>>(U, T, scale, Dc, acc);
    loss_grad_kernel<<<dim3(B, 4), 256, 0, st>>>(U, T, scale, B, Dc, eps, acc, dU, loss, per_sample);
    return cudaGetLastError();
}

cudaError_t sur_init_normal(float* p, size_t n, float std, unsigned long long seed, cudaStream_t st)
{
    init_normal_kernel<<<blocks_for(n), 256, 0, st>>>(p, n, std, seed);
    return cudaGetLastError();
}

cudaError_t sur_comp_sumsq(const float* T, int n, long long Dc, float* ss, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(ss, 0, 4 * sizeof(float), st);
    if (e != cudaSuccess) return e;
    comp_sumsq_kernel<<<dim3(n, 4), 256, 0, st>>>(T, n, Dc, ss);
    return cudaGetLastError();
}

cudaError_t sur_combine(const float* G, long long D, const int* loc, const float* mt, int B, float* out,
                        cudaStream_t st)
{
    const long long nb = std::min<long long>((D + 255) / 256, 1024);
    combine_kernel<<<dim3((unsigned)nb, B), 256, 0, st>>>(G, D, loc, mt, B, out);
    return cudaGetLastError();
}

cudaError_t sur_colsum(const float* G, int B, int N, float* db, cudaStream_t st)
{
    colsum_kernel<<<(N + 255) / 256, 256, 0, st>>>(G, B, N, db);
    return cudaGetLastError();
}

cudaError_t sur_adam(float* p, const float* g, float* m, float* v, size_t n, float lr, float b1, float b2, float eps,
                     int t, __nv_bfloat16* pb, cudaStream_t st)
{
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    const uintptr_t al = reinterpret_cast<uintptr_t>(p) | reinterpret_cast<uintptr_t>(g) |
                         reinterpret_cast<uintptr_t>(m) | reinterpret_cast<uintptr_t>(v);
    if (n % 4 == 0 && (al & 15) == 0 && (reinterpret_cast<uintptr_t>(pb) & 7) == 0) {
        adam4_kernel<<<blocks_for(n / 4), 256, 0, st>>>(
            reinterpret_cast<float4*>(p), reinterpret_cast<const float4*>(g), reinterpret_cast<float4*>(m),
            reinterpret_cast<float4*>(v), n / 4, lr, b1, b2, eps, c1, c2, reinterpret_cast<uint2*>(pb));
    } else {
        adam_kernel<<<blocks_for(n), 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2, pb);
    }
    return cudaGetLastError();
}

cudaError_t sur_adam_t(float* p, const float* g, float* m, float* v, long long rows, long long cols, float lr,
                       float b1, float b2, float eps, int t, __nv_bfloat16* pb, __nv_bfloat16* pt, cudaStream_t st)
{
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    const uintptr_t al = reinterpret_cast<uintptr_t>(p) | reinterpret_cast<uintptr_t>(g) |
                         reinterpret_cast<uintptr_t>(m) | reinterpret_cast<uintptr_t>(v);
    if (cols % 4 || (al & 15) || (reinterpret_cast<uintptr_t>(pb) & 7) || (reinterpret_cast<uintptr_t>(pt) & 7) ||
        !pb || !pt)
        return cudaErrorInvalidValue;
    const long long gx = (cols + AT - 1) / AT, gy = (rows + AT - 1) / AT;
    if (gx > 0x7fffffffLL || gy > 65535) return cudaErrorInvalidValue;
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    adam_t_kernel<<<dim3((unsigned)gx, (unsigned)gy), 256, 0, st>>>(p, g, m, v, rows, cols, lr, b1, b2, eps, c1, c2,
                                                                     pb, pt);
    return cudaGetLastError();
}

}  // namespace es
