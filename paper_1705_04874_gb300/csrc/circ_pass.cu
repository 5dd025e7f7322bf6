// Staggered spectral derivative passes for axis lengths without an FFT plan
// (odd or non-smooth lengths such as 75, 125 or 301 = 7 * 43, the paper's
// own grid; Sec. III).  Along a periodic axis the operator
//   D(+/-) f = IFFT( i kappa exp(+/- i kappa d / 2) FFT(f) )
// is a real circulant matrix: (D f)_i = sum_j c[(i - j) mod n] f_j with
// c_l = sum_m H_m exp(2 pi i m l / n), computed once on the host in FP64
// (es_capi.cu) and rounded to FP32.  This pass applies that convolution
// directly, with the same field-update epilogues as the FFT passes, so the
// result equals the FFT pass up to rounding.  Work per element is O(n)
// instead of O(log n); the pass is compute-bound for long axes.
//
// One CTA: a tile of 32 pencils (32 consecutive x for the y and z passes,
// 32 consecutive x-lines for the x pass) staged in shared memory as
// [position][pencil] (row stride 33: conflict-free both ways), an output
// tile of the same shape, the doubled kernel row c in shared memory.
// Lane = pencil; a warp computes 16 consecutive outputs at a time with the
// kernel values in a 24-register window over blocks of 8 inputs: 8 shared
// loads plus 6 16-byte broadcast loads per 128 FMAs.  The CTA has as many
// warps (4 to 12) as divide its output chunks most evenly (circ_warps): 19
// chunks of n = 301 take 10 warps in two rounds, 5 chunks of n = 75 take 5.
// The tile and the kernel row arrive by asynchronous 4-byte copies
// (cp.async, zero-filled past the edges): every copy of a thread is in
// flight at once, so staging costs about one memory round trip.
// Accesses are scalar and coalesced (32 consecutive floats per warp), so no
// alignment of nx is assumed; totals take scalar L2 reductions.
//
// Compensated variant (ES_PREC_COMPENSATED): the kernel row is held as
// c_hi + c_lo (both FP32), every product c_hi x is split exactly into p + e
// with one FMA (e = fma(c_hi, x, -p)), the running sum is kept as s_hi + s_lo
// with Knuth's TwoSum, and c_lo x, e and the TwoSum errors go to s_lo; the
// result s_hi + s_lo carries the derivative to about twice FP32's precision,
// so only the FP32 storage of the fields limits accuracy.  Chunks of 8 outputs
// (registers), 10 FP32 operations per multiply-add.
#include <cstdlib>

#include "fft_pass.cuh"

namespace es {
namespace {

constexpr int TP = 32;          // pencils per tile
constexpr int ROW = TP + 1;     // shared row stride
constexpr int OB = 16;          // outputs per warp chunk
constexpr int JB = 8;           // inputs per block
constexpr int KOFF = 16;        // least front padding of the kernel row (the window reaches OB - 1 before it)
constexpr int CMAXW = 12;                // most warps per CTA
constexpr int CTHREADS = 32 * CMAXW;

// warps for a CTA of `chunks` output chunks: the most even split (fewest idle
// warp-rounds), ties to the count nearest 8
inline int circ_warps(int chunks)
{
    int best = 8;
    double be = -1.0;
    for (int w = 4; w <= CMAXW; ++w) {
        const int rounds = (chunks + w - 1) / w;
        const double eff = (double)chunks / (double)(rounds * w);
        if (eff > be + 1e-9 || (eff > be - 1e-9 && std::abs(w - 8) < std::abs(best - 8))) {
            be = eff;
            best = w;
        }
    }
    return best;
}

// asynchronous 4-byte copy global -> shared; ok == false writes a zero and reads nothing
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool ok)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(ok ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__host__ __device__ inline int circ_pad(int n) { return (n + OB - 1) / OB * OB; }

// front padding of the kernel row for axis length n: KOFF plus what makes every
// window start KOFF_n + n + i0 - jb - (JB - 1) (i0, jb multiples of 8) a
// multiple of 4, so the window loads are aligned float4s
__host__ __device__ inline int circ_koff(int n) { return KOFF + (((JB - 1 - KOFF - n) % 4) + 4) % 4; }

// shared floats: the input tile [pad(n)][ROW] (the x pass also an output tile
// of that shape) + the kernel row [2 pad(n) + 2 KOFF + OB + 8] (high and low
// parts in the compensated mode)
__host__ __device__ inline int circ_row_len(int n) { return 2 * circ_pad(n) + 2 * KOFF + OB + 8; }
__host__ __device__ inline size_t circ_smem(int n, bool comp, bool two_tiles)
{
    return sizeof(float) * ((two_tiles ? 2 : 1) * (size_t)circ_pad(n) * ROW + (comp ? 2 : 1) * (size_t)circ_row_len(n));
}

// out[i][lane] = sum_j c[(i - j) mod n] tile[j][lane] for i < n; rows j >= n
// of the tile are zero.  cw[s] = c[(s - koff) mod n], koff = circ_koff(n) in
// [KOFF, KOFF + 3]: the window of chunk i0 (a multiple of OBV) and input block
// jb starts at c[i0 - jb - (JB - 1)], index koff + n + i0 - jb - (JB - 1) >=
// KOFF - (OB - 1) + 1 > 0 since pad(n) - n < OB, a multiple of 4, and its
// OBV + JB entries end at or below koff + n + pad(n) + OB, inside the row
// (circ_row_len).  COMP: cl is the low part of the row (same layout).
template <bool COMP, int OBV, class Emit>
__device__ __forceinline__ void circ_convolve(const float* tile, Emit emit, const float* cw, const float* cl, int n,
                                              int warp, int lane)
{
    constexpr int W = OBV + JB;  // window length, a multiple of 4
    const int np = circ_pad(n), koff = circ_koff(n);
    const int nw = blockDim.x >> 5;
    for (int g = warp; g < np / OBV; g += nw) {
        const int i0 = g * OBV;
        float acc[OBV], lo[OBV];
#pragma unroll
        for (int t = 0; t < OBV; ++t) {
            acc[t] = 0.f;
            lo[t] = 0.f;
        }
        for (int jb = 0; jb < np; jb += JB) {
            float xv[JB];
#pragma unroll
            for (int jj = 0; jj < JB; ++jj) xv[jj] = tile[(jb + jj) * ROW + lane];
            const int w0 = koff + n + i0 - jb - (JB - 1);
            float w[W], wl[COMP ? W : 1];  // w[s] = c[i0 - jb - (JB - 1) + s]
#pragma unroll
            for (int s = 0; s < W / 4; ++s) {
                const float4 v = reinterpret_cast<const float4*>(cw + w0)[s];
                w[4 * s] = v.x;
                w[4 * s + 1] = v.y;
                w[4 * s + 2] = v.z;
                w[4 * s + 3] = v.w;
                if constexpr (COMP) {
                    const float4 u = reinterpret_cast<const float4*>(cl + w0)[s];
                    wl[4 * s] = u.x;
                    wl[4 * s + 1] = u.y;
                    wl[4 * s + 2] = u.z;
                    wl[4 * s + 3] = u.w;
                }
            }
#pragma unroll
            for (int jj = 0; jj < JB; ++jj)
#pragma unroll
                for (int t = 0; t < OBV; ++t) {
                    const float c = w[t - jj + JB - 1];
                    if constexpr (!COMP) {
                        acc[t] = fmaf(c, xv[jj], acc[t]);
                    } else {
                        const float p = __fmul_rn(c, xv[jj]);
                        const float e = fmaf(c, xv[jj], -p);  // c x = p + e exactly
                        const float sum = __fadd_rn(acc[t], p);
                        const float bb = __fsub_rn(sum, acc[t]);
                        const float err = __fadd_rn(__fsub_rn(acc[t], __fsub_rn(sum, bb)), __fsub_rn(p, bb));
                        acc[t] = sum;
                        lo[t] = __fadd_rn(lo[t], __fadd_rn(err, fmaf(wl[t - jj + JB - 1], xv[jj], e)));
                    }
                }
        }
#pragma unroll
        for (int t = 0; t < OBV; ++t)
            if (i0 + t < n) emit(i0 + t, COMP ? __fadd_rn(acc[t], lo[t]) : acc[t]);
    }
}

__device__ __forceinline__ void load_kernel_row(float* cw, const float* c, int n, int tid)
{
    const int len = circ_row_len(n), koff = circ_koff(n);
    for (int s = tid; s < len; s += blockDim.x) {
        int k = (s - koff) % n;
        if (k < 0) k += n;
        cp_async4(cw + s, c + k, true);
    }
}

// Long axes (n >= CIRC_DIRECT_N, es_internal.h) give every warp several 16-output chunks:
// the y and z passes then run the epilogue straight from the registers (no output tile,
// half the shared memory, twice the resident CTAs); shorter axes keep the output tile so
// that all warps share the epilogue.

// y and z passes: blockIdx.x = (tile of 32 consecutive x) x outer x simulation, blockIdx.y = job
template <bool COMP, bool DIRECT>
__global__ void __launch_bounds__(CTHREADS, 2) circ_strided(const __grid_constant__ PassParams p)
{
    extern __shared__ float csm[];
    const int n = p.n, np = circ_pad(n);
    float* tile = csm;
    float* out = tile + (size_t)np * ROW;  // used only without DIRECT
    float* cw = out + (DIRECT ? 0 : (size_t)np * ROW);
    float* cl = cw + circ_row_len(n);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const PassJob& J = p.job[blockIdx.y];
    const int sim = blockIdx.x % p.nsim, t2 = blockIdx.x / p.nsim;
    const size_t off = (size_t)sim * p.fstride, soff = (size_t)sim * p.sstride;
    const int ntx = (p.nx + TP - 1) / TP;
    const int x0 = (t2 % ntx) * TP, outer = t2 / ntx;
    size_t base0, est;
    if (p.axis == 1) {
        base0 = (size_t)x0 + (size_t)p.nx * p.ny * outer;
        est = (size_t)p.nx;
    } else {
        base0 = (size_t)x0 + (size_t)p.nx * outer;
        est = (size_t)p.nx * p.ny;
    }
    pdl_begin(p.pdl);
    load_kernel_row(cw, J.sign > 0 ? p.ckp : p.ckm, n, tid);
    if (COMP) load_kernel_row(cl, J.sign > 0 ? p.ckp_lo : p.ckm_lo, n, tid);
    for (int it = tid; it < np * TP; it += blockDim.x) {
        const int pos = it / TP, c = it % TP;
        const bool ok = pos < n && x0 + c < p.nx;
        cp_async4(tile + pos * ROW + c, J.src + off + (ok ? base0 + c + (size_t)pos * est : 0), ok);
    }
    cp_async_wait_all();
    __syncthreads();
    if constexpr (DIRECT) {
        if (p.pdl == 1) pdl_wait();  // the previous pass's updates of the targets come first
        // lane = x column: the warp's outputs of one position are 32 consecutive cells, so the
        // epilogue runs straight from the registers, coalesced
        const int x = x0 + lane;
        circ_convolve<COMP, COMP ? 8 : OB>(
            tile,
            [&](int pos, float d) {
                if (x >= p.nx) return;
                const int y = p.axis == 1 ? pos : outer, z = p.axis == 1 ? outer : pos;
                epilogue_one(p, J, base0 + lane + (size_t)pos * est, pos, x, y, z, d, off, soff);
            },
            cw, cl, n, warp, lane);
    } else {
        circ_convolve<COMP, COMP ? 8 : OB>(
            tile, [&](int pos, float d) { out[pos * ROW + lane] = d; }, cw, cl, n, warp, lane);
        __syncthreads();
        if (p.pdl == 1) pdl_wait();
        for (int it = tid; it < n * TP; it += blockDim.x) {
            const int pos = it / TP, c = it % TP;
            const int x = x0 + c;
            if (x >= p.nx) continue;
            const int y = p.axis == 1 ? pos : outer, z = p.axis == 1 ? outer : pos;
            epilogue_one(p, J, base0 + c + (size_t)pos * est, pos, x, y, z, out[pos * ROW + c], off, soff);
        }
    }
}

// x pass: blockIdx.x = (tile of 32 consecutive x-lines, line = y + ny z) x simulation, blockIdx.y = job
template <bool COMP>
__global__ void __launch_bounds__(CTHREADS, 2) circ_x(const __grid_constant__ PassParams p)
{
    extern __shared__ float csm[];
    const int n = p.n, np = circ_pad(n);
    float* tile = csm;
    float* out = tile + (size_t)np * ROW;
    float* cw = out + (size_t)np * ROW;
    float* cl = cw + circ_row_len(n);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const PassJob& J = p.job[blockIdx.y];
    const int nlines = p.ny * p.nz;
    const int sim = blockIdx.x % p.nsim;
    const size_t off = (size_t)sim * p.fstride, soff = (size_t)sim * p.sstride;
    const int line0 = (blockIdx.x / p.nsim) * TP;
    const int nl = min(TP, nlines - line0);
    pdl_begin(p.pdl);
    load_kernel_row(cw, J.sign > 0 ? p.ckp : p.ckm, n, tid);
    if (COMP) load_kernel_row(cl, J.sign > 0 ? p.ckp_lo : p.ckm_lo, n, tid);
    // the tile's lines are one contiguous block of nl * n floats
    const float* src = J.src + off + (size_t)line0 * n;
    // zeros where no copy lands (rows past the axis end; lines past the last tile's end), written
    // alongside the copies, which touch only the other elements
    for (int e = tid; e < (np - n) * ROW; e += blockDim.x) tile[n * ROW + e] = 0.f;
    if (nl < TP)
        for (int e = tid; e < n * (TP - nl); e += blockDim.x) tile[(e / (TP - nl)) * ROW + nl + e % (TP - nl)] = 0.f;
    // element e = r n + pos of the block; (r, pos) advance by blockDim.x without a division per element
    const int bd = blockDim.x, dr = bd / n, dp = bd % n;
    for (int r = tid / n, pos = tid % n; r < nl;) {
        cp_async4(tile + pos * ROW + r, src + (size_t)r * n + pos, true);
        pos += dp;
        r += dr;
        if (pos >= n) {
            pos -= n;
            ++r;
        }
    }
    cp_async_wait_all();
    __syncthreads();
    circ_convolve<COMP, COMP ? 8 : OB>(
        tile, [&](int pos, float d) { out[pos * ROW + lane] = d; }, cw, cl, n, warp, lane);
    __syncthreads();
    if (p.pdl == 1) pdl_wait();
    // the slab index along x is sp + S (y + ny z) = sp + S line: the line goes in as y, with z = 0
    for (int r = tid / n, pos = tid % n; r < nl;) {
        const int line = line0 + r;
        epilogue_one(p, J, (size_t)line * n + pos, pos, pos, line, 0, out[pos * ROW + r], off, soff);
        pos += dp;
        r += dr;
        if (pos >= n) {
            pos -= n;
            ++r;
        }
    }
}

}  // namespace


cudaError_t prepare_circ_kernels()
{
    const int maxb = (int)circ_smem(CIRC_MAX_N, true, true);
    cudaError_t e = cudaSuccess;
    auto opt = [&](auto kernel) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, maxb);
    };
    opt(circ_x<false>);
    opt(circ_x<true>);
    opt(circ_strided<false, false>);
    opt(circ_strided<false, true>);
    opt(circ_strided<true, false>);
    opt(circ_strided<true, true>);
    return e;
}

cudaError_t launch_circ(const PassParams& p, cudaStream_t st)
{
    if (circ_tc_eligible(p)) return launch_circ_tc(p, st);
    if (p.n < 2 || p.n > CIRC_MAX_N || !p.ckp || !p.ckm) return cudaErrorInvalidValue;
    if (p.comp && (!p.ckp_lo || !p.ckm_lo)) return cudaErrorInvalidValue;
    const int threads = 32 * circ_warps(circ_pad(p.n) / (p.comp ? 8 : OB));
    if (p.axis == 0) {
        const int lines = p.ny * p.nz;
        dim3 grid((unsigned)((lines + TP - 1) / TP) * p.nsim, p.njobs);
        return launch_pass_kernel(p.comp ? circ_x<true> : circ_x<false>, grid, threads,
                                  circ_smem(p.n, p.comp != 0, true), st, p);
    }
    const int ntx = (p.nx + TP - 1) / TP;
    const int outer = p.axis == 1 ? p.nz : p.ny;
    dim3 grid((unsigned)(ntx * outer) * p.nsim, p.njobs);
    const bool direct = p.n >= CIRC_DIRECT_N;
    const size_t smem = circ_smem(p.n, p.comp != 0, !direct);
    if (direct)
        return launch_pass_kernel(p.comp ? circ_strided<true, true> : circ_strided<false, true>, grid, threads, smem,
                                  st, p);
    return launch_pass_kernel(p.comp ? circ_strided<true, false> : circ_strided<false, false>, grid, threads, smem,
                              st, p);
}

}  // namespace es
