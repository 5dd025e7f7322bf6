// Small kernels around the derivative passes: point-source injection
// (Sec. II-A: point sources at grid points), 4C receiver recording
// (Sec. II-A, Eq. (3); Sec. II-B), superposition of single-event traces
// (Sec. IV), a non-finite scan and slab initialisation.
#include <algorithm>

#include "es_internal.h"

namespace es {

// One thread walks every source in order, so sources sharing a cell add in a
// fixed order.  The step counter lives on the device so that one captured
// step can be replayed: the kernel that runs last in a step (`advance`)
// publishes the step index to `cur` for the recorder and increments it.
// The spatial-frequency Blackman window of one axis, W(m) = 0.42 + 0.5 cos(2 pi m / n)
// + 0.08 cos(4 pi m / n) over the signed wavenumber bins m (1 at m = 0, 0 at the
// Nyquist bin), has the inverse DFT 0.42 at offset 0, 0.25 at +-1, 0.04 at +-2
// and 0 elsewhere (n >= 5): the smoothed point source (Sec. II-A) is exactly the
// product of these three stencils around the source cell.
__constant__ float c_blackman5[5] = {0.04f, 0.25f, 0.42f, 0.25f, 0.04f};

// One block.  Thread 0 adds the point sources in order (deterministic); then
// every thread takes (source, stencil cell) pairs of the smoothed sources and
// adds with reductions (order free only where smoothed stencils of one
// simulation overlap); then thread 0 advances the step counter.
__global__ void inject_kernel(float* const* fields, long long fstride, const SourceDev* src, int nsrc, int kind,
                              int nx, int ny, int* counter, int* cur, int advance)
{
    const int n = *counter;
    if (threadIdx.x == 0) {
        for (int e = 0; e < nsrc; ++e) {
            const SourceDev s = src[e];
            if (s.kind != kind || s.smooth || n >= s.nw) continue;
            const float w = s.w[n];
            const long long q = (long long)s.sim * fstride + s.cell;
            if (kind == 0) {
                // moment tensor: stress component i gains M_i w[n] (Mxx Myy Mzz Mxy Mxz Myz)
                for (int c = 0; c < 6; ++c)
                    if (s.m[c] != 0.f) fields[SXX + c][q] = __fmaf_rn(s.m[c], w, fields[SXX + c][q]);
            } else {
                // point force: m[c] = dt f_c / (rho_c dx dy dz), folded on the host
                for (int c = 0; c < 3; ++c)
                    if (s.m[c] != 0.f) fields[VX + c][q] = __fmaf_rn(s.m[c], w, fields[VX + c][q]);
            }
        }
    }
    __syncthreads();
    if (kind == 0) {
        for (int it = threadIdx.x; it < nsrc * 125; it += blockDim.x) {
            const int e = it / 125, k = it % 125;
            const SourceDev& s = src[e];
            if (!s.smooth || s.kind != 0 || n >= s.nw) continue;
            const int dx = k % 5 - 2, dy = (k / 5) % 5 - 2, dz = k / 25 - 2;
            const float g = c_blackman5[dx + 2] * c_blackman5[dy + 2] * c_blackman5[dz + 2];
            const float w = s.w[n] * g;
            const long long q = (long long)s.sim * fstride + s.cell + dx + (long long)nx * (dy + (long long)ny * dz);
            for (int c = 0; c < 6; ++c)
                if (s.m[c] != 0.f) atomicAdd(fields[SXX + c] + q, s.m[c] * w);
        }
    }
    __syncthreads();
    if (advance && threadIdx.x == 0) {
        *cur = n;
        *counter = n + 1;
    }
}

cudaError_t launch_inject(float* const* fields, long long fstride, const SourceDev* src, int nsrc, int kind,
                          int nx, int ny, int* counter, int* cur, int advance, cudaStream_t st)
{
    inject_kernel<<<1, 256, 0, st>>>(fields, fstride, src, nsrc, kind, nx, ny, counter, cur, advance);
    return cudaGetLastError();
}

// Kelvin-Voigt source of the stress passes: w = a v - b vold, vold <- v, for
// the three velocity components ([c][sim][cell], n = cells x simulations each)
__global__ void visc_combine_kernel(float* const* fields, float* vold, float* w, size_t n, float a, float b)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float v = fields[VX + c][i];
            w[c * n + i] = a * v - b * vold[c * n + i];
            vold[c * n + i] = v;
        }
}

cudaError_t launch_visc_combine(float* const* fields, float* vold, float* w, size_t n, float a, float b,
                                cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const size_t blocks = std::min<size_t>((n + 255) / 256, 152 * 16);
    visc_combine_kernel<<<(unsigned)blocks, 256, 0, st>>>(fields, vold, w, n, a, b);
    return cudaGetLastError();
}

// Material coefficients of one cell per thread (Eq. (4) and the staggered
// averages of the model setup): lambda = rho cp^2 - 2 mu and mu = rho cs^2 at
// the cell, buoyancy 2 / (rho_i + rho_(i+1)) at the half-index point along
// each axis, and the edge shear moduli as the harmonic mean of the four
// surrounding mu (0 if any is 0, i.e. next to water); neighbours wrap
// periodically.  FP64 with explicitly rounded operations (no contraction),
// stored in FP32.
__device__ __forceinline__ double mu_of(const float* rho, const float* cs, size_t p)
{
    const double s = cs[p];
    return __dmul_rn(__dmul_rn(s, s), (double)rho[p]);
}

__device__ __forceinline__ double harmonic4(double a, double b, double c, double d)
{
    if (a == 0.0 || b == 0.0 || c == 0.0 || d == 0.0) return 0.0;
    const double s = __dadd_rn(__dadd_rn(__dadd_rn(__ddiv_rn(1.0, a), __ddiv_rn(1.0, b)), __ddiv_rn(1.0, c)),
                               __ddiv_rn(1.0, d));
    return __ddiv_rn(4.0, s);
}

__global__ void materials_kernel(const float* rho, const float* cp, const float* cs, int nx, int ny, int nz,
                                 MatPtrs out)
{
    const size_t n = (size_t)nx * ny * nz;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(q % nx), j = (int)((q / nx) % ny), k = (int)(q / ((size_t)nx * ny));
        const int ip = i + 1 == nx ? 0 : i + 1, jp = j + 1 == ny ? 0 : j + 1, kp = k + 1 == nz ? 0 : k + 1;
        auto at = [&](int ii, int jj, int kk) { return (size_t)ii + (size_t)nx * ((size_t)jj + (size_t)ny * kk); };
        const size_t qx = at(ip, j, k), qy = at(i, jp, k), qz = at(i, j, kp);
        const double r = rho[q], c = cp[q];
        const double mu = mu_of(rho, cs, q);
        out.p[M_LAM][q] = __double2float_rn(__dsub_rn(__dmul_rn(__dmul_rn(c, c), r), __dmul_rn(2.0, mu)));
        out.p[M_MU][q] = __double2float_rn(mu);
        out.p[M_BX][q] = __double2float_rn(__ddiv_rn(2.0, __dadd_rn(r, (double)rho[qx])));
        out.p[M_BY][q] = __double2float_rn(__ddiv_rn(2.0, __dadd_rn(r, (double)rho[qy])));
        out.p[M_BZ][q] = __double2float_rn(__ddiv_rn(2.0, __dadd_rn(r, (double)rho[qz])));
        const double mx = mu_of(rho, cs, qx), my = mu_of(rho, cs, qy), mz = mu_of(rho, cs, qz);
        out.p[M_MUXY][q] = __double2float_rn(harmonic4(mu, mx, my, mu_of(rho, cs, at(ip, jp, k))));
        out.p[M_MUXZ][q] = __double2float_rn(harmonic4(mu, mx, mz, mu_of(rho, cs, at(ip, j, kp))));
        out.p[M_MUYZ][q] = __double2float_rn(harmonic4(mu, my, mz, mu_of(rho, cs, at(i, jp, kp))));
    }
}

cudaError_t launch_materials(const float* rho, const float* cp, const float* cs, int nx, int ny, int nz,
                             const MatPtrs& out, cudaStream_t st)
{
    const size_t n = (size_t)nx * ny * nz;
    if (n == 0) return cudaSuccess;
    const size_t blocks = std::min<size_t>((n + 255) / 256, 152 * 32);
    materials_kernel<<<(unsigned)blocks, 256, 0, st>>>(rho, cp, cs, nx, ny, nz, out);
    return cudaGetLastError();
}

__global__ void fill_kernel(float* p, size_t n, float v)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = v;
}

cudaError_t launch_fill(float* p, size_t n, float v, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const size_t blocks = std::min<size_t>((n + 255) / 256, 4096);
    fill_kernel<<<(unsigned)blocks, 256, 0, st>>>(p, n, v);
    return cudaGetLastError();
}

// rec[n - start][sim][c][r]: sample n of component c (p, vx, vy, vz) of
// simulation sim at receiver r
__global__ void record_kernel(float* const* fields, long long fstride, int nsim, const long long* rcv_cell, int n_rcv,
                              const int* cur, long long start, float* rec)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_rcv * nsim) return;
    const int r = i % n_rcv, sim = i / n_rcv;
    const long long q = (long long)sim * fstride + rcv_cell[r];
    const size_t row = ((size_t)(*cur - start) * nsim + sim) * 4 * n_rcv;
    const float s = __fadd_rn(__fadd_rn(fields[SXX][q], fields[SYY][q]), fields[SZZ][q]);
    rec[row + r] = __fdiv_rn(-s, 3.f);  // Eq. (3)
    rec[row + n_rcv + r] = fields[VX][q];
    rec[row + 2 * (size_t)n_rcv + r] = fields[VY][q];
    rec[row + 3 * (size_t)n_rcv + r] = fields[VZ][q];
}

cudaError_t launch_record(float* const* fields, long long fstride, int nsim, const long long* rcv_cell, int n_rcv,
                          const int* cur, long long start, float* rec, cudaStream_t st)
{
    if (n_rcv <= 0) return cudaSuccess;
    const int n = n_rcv * nsim;
    record_kernel<<<(n + 127) / 128, 128, 0, st>>>(fields, fstride, nsim, rcv_cell, n_rcv, cur, start, rec);
    return cudaGetLastError();
}

// [rows][cols] -> [cols][rows] through a 32 x 32 shared tile
__global__ void transpose_kernel(const float* in, int rows, int cols, float* out)
{
    __shared__ float tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[i][threadIdx.x] = in[(size_t)r * cols + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (r < rows && c < cols) out[(size_t)c * rows + r] = tile[threadIdx.x][i];
    }
}

cudaError_t launch_transpose_traces(const float* rec, int nt, int cols, float* out, cudaStream_t st)
{
    dim3 grid((cols + 31) / 32, (nt + 31) / 32), block(32, 8);
    transpose_kernel<<<grid, block, 0, st>>>(rec, nt, cols, out);
    return cudaGetLastError();
}

// gather[row][t] = sum_e amp_e traces[src_e][row][t - k_e], rows = 4 n_rcv.
// One thread per output sample; events in order (FP32 accumulation).  The
// events reach shared memory in chunks of SUP_CHUNK, so any number of events
// fits in a fixed 48 KB block without changing the order of the sum.
constexpr int SUP_CHUNK = 4096;

__global__ void superpose_kernel(const float* traces, int n_rcv, int nt, const int* ev_src,
                                 const float* ev_amp, const int* ev_shift, int n_events, int n_out,
                                 float* gather)
{
    __shared__ int s_src[SUP_CHUNK], s_k[SUP_CHUNK];
    __shared__ float s_a[SUP_CHUNK];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const size_t row = blockIdx.y;
    const bool active = t < n_out;
    const size_t rows = 4 * (size_t)n_rcv;
    float acc = 0.f;
    for (int e0 = 0; e0 < n_events; e0 += SUP_CHUNK) {
        const int ne = min(SUP_CHUNK, n_events - e0);
        __syncthreads();  // the previous chunk is no longer read
        for (int i = threadIdx.x; i < ne; i += blockDim.x) {
            s_src[i] = ev_src[e0 + i];
            s_k[i] = ev_shift[e0 + i];
            s_a[i] = ev_amp[e0 + i];
        }
        __syncthreads();
        if (!active) continue;
        for (int e = 0; e < ne; ++e) {
            const long u = (long)t - s_k[e];
            if (u < 0 || u >= nt) continue;
            acc += s_a[e] * __ldg(traces + ((size_t)s_src[e] * rows + row) * nt + u);
        }
    }
    if (active) gather[row * n_out + t] = acc;
}

cudaError_t launch_superpose(const float* traces, int n_src, int n_rcv, int nt, const int* ev_src,
                             const float* ev_amp, const int* ev_shift, int n_events, int n_out, float* gather,
                             cudaStream_t st)
{
    (void)n_src;
    dim3 grid((n_out + 255) / 256, 4 * n_rcv);
    superpose_kernel<<<grid, 256, 0, st>>>(traces, n_rcv, nt, ev_src, ev_amp, ev_shift, n_events, n_out, gather);
    return cudaGetLastError();
}

// flag |= 1 if any field value is NaN or infinite
__global__ void nonfinite_kernel(float* const* fields, size_t n, int* flag)
{
    int bad = 0;
    for (int f = 0; f < NFIELD; ++f) {
        const float* a = fields[f];
        for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
            bad |= !isfinite(a[i]);
    }
    bad = __syncthreads_or(bad);
    if (bad && threadIdx.x == 0) atomicOr(flag, 1);
}

cudaError_t launch_nonfinite(float* const* fields, size_t n, int* flag, cudaStream_t st)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    nonfinite_kernel<<<sms * 4, 256, 0, st>>>(fields, n, flag);
    return cudaGetLastError();
}

// slab[cell in slab] = copy ? total[cell] : 0
__global__ void fill_slab_kernel(const float* total, float* slab, int axis, int nx, int ny, int nz, int L,
                                 int copy)
{
    const int S = 2 * L + 1;
    const int n = axis == 0 ? nx : (axis == 1 ? ny : nz);
    const size_t cnt = (size_t)nx * ny * nz / n * S;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < cnt; i += (size_t)gridDim.x * blockDim.x) {
        int x, y, z, sp;
        if (axis == 0) { sp = (int)(i % S); size_t l = i / S; y = (int)(l % ny); z = (int)(l / ny); x = 0; }
        else if (axis == 1) { x = (int)(i % nx); size_t l = i / nx; sp = (int)(l % S); z = (int)(l / S); y = 0; }
        else { x = (int)(i % nx); size_t l = i / nx; y = (int)(l % ny); sp = (int)(l / ny); z = 0; }
        const int pos = sp < L ? sp : sp - L + (n - 1 - L);
        if (axis == 0) x = pos; else if (axis == 1) y = pos; else z = pos;
        slab[i] = copy ? total[(size_t)x + (size_t)nx * ((size_t)y + (size_t)ny * z)] : 0.f;
    }
}

cudaError_t launch_fill_slab(const float* total, float* slab, int axis, int nx, int ny, int nz, int L, int copy,
                             cudaStream_t st)
{
    fill_slab_kernel<<<1024, 256, 0, st>>>(total, slab, axis, nx, ny, nz, L, copy);
    return cudaGetLastError();
}

}  // namespace es
