// Fused pseudo-spectral derivative passes (Sec. II-A of Das, Chen & Hobson,
// arXiv 1705.04874: Fourier-domain spatial derivatives on a staggered grid).
//
// One CTA owns a tile of 32 real pencils along the pass axis, packed two at a
// time into 16 complex lines (line c = pencil 2c + i * pencil 2c+1).  For
// each job it runs: forward FFT along the axis -> multiply by
// i kappa exp(+/- i kappa d / 2) / n -> inverse FFT -> field-update epilogue.
// Because the multiplier is Hermitian (a real field has a real derivative,
// including at the Nyquist bin, where it is the real number -/+ pi / d), the
// real and imaginary parts of the result are the derivatives of the two
// packed pencils.
//
// The transform of length n = RA * RB is a two-stage Stockham autosort FFT
// (radix RA with stride n/RA, then radix RB with twiddles exp(-2 pi i k r / n)).
// Its last forward stage leaves each thread holding exactly the elements
// b + q n/RB that the first stage of the inverse (run as a forward transform
// of the conjugate, with the radices in reverse order) needs, so the
// multiply and that stage happen in registers; shared memory is touched only
// between stages.  The inverse's last stage ends on the same elements the
// first forward stage loaded, so the epilogue writes where the loads read.
// Three-stage plans (Core3: 125 = 5 x 5 x 5, 75 = 3 x 5 x 5) run their middle
// stages through shared memory and keep the same first / last-stage layout.
//
// Strided passes (y, z): a tile is 32 consecutive x (128-byte rows) by the
// whole pencil; every global access of a warp is a full row segment (an odd
// nx moves the x-adjacent pairs as two floats).  The x pass stages 32 whole
// x-lines (contiguous in memory) through shared memory with float4 accesses
// (float accesses, and a per-line copy of the source for the near stencil,
// when the length is not a multiple of 16) and runs the same FFT core on the
// staged tile.
//
// Each derivative is evaluated as a near part plus a far part (es_internal.h):
// the multiplier tables hold H_far / n, and once the last inverse stage has
// read the shared buffer, the source tile comes back into it (cp.async from
// L2, where the tile's first read left it, with wrap-around copies of the
// first and last rows); the epilogue adds the NEAR_TAPS-point near stencil
// from there (the x pass reads it from the staged lines' L1 / L2 copies, or
// from its per-line copy).  In exact arithmetic the sum is the spectral
// derivative itself; in FP32 the FFT's roundoff, which is spread
// over the whole pencil, is scaled down by |H_far| / |H| (about 1 %), so
// far-away receivers no longer see the FP32 noise of the pencil's largest
// values.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <type_traits>
#include <utility>

#include "es_internal.h"

namespace es {

// ---------------------------------------------------------------------------
// compile-time twiddles W_R^M = exp(-2 pi i M / R)
// ---------------------------------------------------------------------------
__host__ __device__ constexpr double ce_cos_frac(long m, long r)
{
    // cos(2 pi m / r): exact at multiples of pi / 2, Taylor series otherwise
    long mm = ((m % r) + r) % r;
    if ((4 * mm) % r == 0) {
        long q = (4 * mm) / r;
        return q == 0 ? 1.0 : (q == 2 ? -1.0 : 0.0);
    }
    double x = 6.283185307179586476925286766559 * (double)mm / (double)r;
    if (2 * mm > r) x -= 6.283185307179586476925286766559;
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 40; ++k) {
        term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
        sum += term;
    }
    return sum;
}
__host__ __device__ constexpr double ce_sin_frac(long m, long r)
{
    return ce_cos_frac(4 * m - r, 4 * r);  // sin(t) = cos(t - pi/2)
}

template <int R, int M>
__device__ __forceinline__ float2 twc(float2 v)
{
    constexpr int mm = ((M % R) + R) % R;
    if constexpr (mm == 0) {
        return v;
    } else if constexpr ((4 * mm) % R == 0) {
        constexpr int q = (4 * mm) / R;  // rotation by -i q
        if constexpr (q == 1) return make_float2(v.y, -v.x);
        else if constexpr (q == 2) return make_float2(-v.x, -v.y);
        else return make_float2(-v.y, v.x);
    } else {
        constexpr float c = (float)ce_cos_frac(mm, R);
        constexpr float s = (float)(-ce_sin_frac(mm, R));
        return make_float2(c * v.x - s * v.y, c * v.y + s * v.x);
    }
}

template <int... Is, class F>
__device__ __forceinline__ void sfor_impl(std::integer_sequence<int, Is...>, F&& f)
{
    (f(std::integral_constant<int, Is>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void sfor(F&& f)
{
    sfor_impl(std::make_integer_sequence<int, N>{}, f);
}

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 mul_mi(float2 a) { return make_float2(a.y, -a.x); }  // -i a

// Packed FP32 pairs (fma.rn.f32x2 / add.rn.f32x2): two multiply-adds or adds
// in one instruction, each component rounded exactly as fmaf / __fadd_rn
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c)
{
    float2 d;
    asm("{\n.reg .b64 ra, rb, rc, rd;\nmov.b64 ra, {%2, %3};\nmov.b64 rb, {%4, %5};\nmov.b64 rc, {%6, %7};\n"
        "fma.rn.f32x2 rd, ra, rb, rc;\nmov.b64 {%0, %1}, rd;\n}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
// Index check of the bounds-checked build (ES_BOUNDS, es_internal.h): true
// when 0 <= i < n; otherwise the first such index is recorded with the source
// line and the caller skips the access.  Always true in the release build.
__device__ __forceinline__ bool inb(unsigned long long* bad, long long i, long long n, int line)
{
#if ES_BOUNDS
    if (i >= 0 && i < n) return true;
    if (bad) atomicCAS(bad, 0ull, ((unsigned long long)line << 40) | ((unsigned long long)i & 0xFFFFFFFFFFull));
    return false;
#else
    (void)bad;
    (void)i;
    (void)n;
    (void)line;
    return true;
#endif
}
#define ES_INB(p, i, n) inb((p).bad, (long long)(i), (long long)(n), __LINE__)

__device__ __forceinline__ float2 add2(float2 a, float2 b)
{
    float2 d;
    asm("{\n.reg .b64 ra, rb, rd;\nmov.b64 ra, {%2, %3};\nmov.b64 rb, {%4, %5};\n"
        "add.rn.f32x2 rd, ra, rb;\nmov.b64 {%0, %1}, rd;\n}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

// ---------------------------------------------------------------------------
// forward DFTs of small sizes in registers: a[k] <- sum_j a[j] W_R^(jk)
// ---------------------------------------------------------------------------
template <int R> struct Dft;

template <> struct Dft<2> {
    static __device__ __forceinline__ void run(float2* a)
    {
        float2 t = a[0];
        a[0] = cadd(t, a[1]);
        a[1] = csub(t, a[1]);
    }
};

template <> struct Dft<3> {
    static __device__ __forceinline__ void run(float2* a)
    {
        constexpr float h = 0.86602540378443864676f;  // sqrt(3) / 2
        float2 t1 = cadd(a[1], a[2]), t2 = csub(a[1], a[2]);
        float2 m = make_float2(a[0].x - 0.5f * t1.x, a[0].y - 0.5f * t1.y);
        float2 s = mul_mi(make_float2(h * t2.x, h * t2.y));
        a[0] = cadd(a[0], t1);
        a[1] = cadd(m, s);
        a[2] = csub(m, s);
    }
};

template <> struct Dft<4> {
    static __device__ __forceinline__ void run(float2* a)
    {
        float2 s02 = cadd(a[0], a[2]), d02 = csub(a[0], a[2]);
        float2 s13 = cadd(a[1], a[3]), d13 = mul_mi(csub(a[1], a[3]));
        a[0] = cadd(s02, s13);
        a[2] = csub(s02, s13);
        a[1] = cadd(d02, d13);
        a[3] = csub(d02, d13);
    }
};

template <> struct Dft<5> {
    static __device__ __forceinline__ void run(float2* a)
    {
        constexpr float c1 = 0.30901699437494742410f;   // cos(2 pi / 5)
        constexpr float c2 = -0.80901699437494742410f;  // cos(4 pi / 5)
        constexpr float s1 = 0.95105651629515357212f;   // sin(2 pi / 5)
        constexpr float s2 = 0.58778525229247312917f;   // sin(4 pi / 5)
        float2 t1 = cadd(a[1], a[4]), t2 = cadd(a[2], a[3]);
        float2 t3 = csub(a[1], a[4]), t4 = csub(a[2], a[3]);
        float2 b1 = make_float2(a[0].x + c1 * t1.x + c2 * t2.x, a[0].y + c1 * t1.y + c2 * t2.y);
        float2 b2 = make_float2(a[0].x + c2 * t1.x + c1 * t2.x, a[0].y + c2 * t1.y + c1 * t2.y);
        float2 e1 = mul_mi(make_float2(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y));
        float2 e2 = mul_mi(make_float2(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y));
        a[0] = cadd(a[0], cadd(t1, t2));
        a[1] = cadd(b1, e1);
        a[4] = csub(b1, e1);
        a[2] = cadd(b2, e2);
        a[3] = csub(b2, e2);
    }
};

// Composite R = P * Q in registers (Cooley-Tukey):
// X[k1 + P k2] = sum_n2 W_Q^(n2 k2) W_R^(n2 k1) sum_n1 a[Q n1 + n2] W_P^(n1 k1)
template <int P, int Q> struct DftPQ {
    static __device__ __forceinline__ void run(float2* a)
    {
        constexpr int R = P * Q;
        float2 B[Q][P];
        sfor<Q>([&](auto n2) {
            float2 v[P];
            sfor<P>([&](auto n1) { v[n1] = a[Q * n1 + n2]; });
            Dft<P>::run(v);
            sfor<P>([&](auto k1) { B[n2][k1] = twc<R, decltype(n2)::value * decltype(k1)::value>(v[k1]); });
        });
        sfor<P>([&](auto k1) {
            float2 v[Q];
            sfor<Q>([&](auto n2) { v[n2] = B[n2][k1]; });
            Dft<Q>::run(v);
            sfor<Q>([&](auto k2) { a[k1 + P * k2] = v[k2]; });
        });
    }
};
template <> struct Dft<6> : DftPQ<2, 3> {};
template <> struct Dft<8> : DftPQ<2, 4> {};
template <> struct Dft<10> : DftPQ<2, 5> {};
template <> struct Dft<12> : DftPQ<4, 3> {};
template <> struct Dft<15> : DftPQ<3, 5> {};
template <> struct Dft<16> : DftPQ<4, 4> {};
template <> struct Dft<25> : DftPQ<5, 5> {};

// ---------------------------------------------------------------------------
// epilogues
// ---------------------------------------------------------------------------
__device__ __forceinline__ int slab_pos(int pos, int n, int L)
{
    // slab storage covers [0, L) and [n-1-L, n): every point whose whole- or
    // half-index PML factor differs from 1
    return pos < L ? pos : pos - (n - 1 - L) + L;
}
__device__ __forceinline__ bool in_slab(int pos, int n, int L)
{
    return L > 0 && (pos < L || pos >= n - 1 - L);
}

// index of (x, y, z) in the slab array of `axis` (slab coordinate sp)
__device__ __forceinline__ size_t slab_index(int axis, int x, int y, int z, int sp, int nx, int ny, int S)
{
    if (axis == 0) return (size_t)sp + (size_t)S * ((size_t)y + (size_t)ny * z);
    if (axis == 1) return (size_t)x + (size_t)nx * ((size_t)sp + (size_t)S * z);
    return (size_t)x + (size_t)nx * ((size_t)y + (size_t)ny * sp);
}

// Split-field update inside a PML slab: s <- P (P s + inc).  Returns the
// change of the split, which is the change of the field total.  The epilogues
// spell out their roundings (__fmaf_rn / __fmul_rn / __fadd_rn) so that every
// kernel that updates a field does so in the same FP32 operations, whatever
// the compiler would contract around them.
__device__ __forceinline__ float split_delta(float* slab, size_t si, float P, float inc)
{
    const float s = slab[si];
    const float sn = __fmul_rn(P, __fmaf_rn(P, s, inc));
    slab[si] = sn;
    return __fsub_rn(sn, s);
}
// dt c D, rounded after each product
__device__ __forceinline__ float increment(float dt, float c, float d) { return __fmul_rn(__fmul_rn(dt, c), d); }
// lambda + 2 mu (diag) or lambda
__device__ __forceinline__ float normal_coef(float lam, float mu, bool diag) { return diag ? __fmaf_rn(2.f, mu, lam) : lam; }

// Field totals take their increment by a vector reduction in L2 (atomicAdd
// with the result unused): within one pass every total receives exactly one
// increment, and passes are stream-ordered, so the result is the plain
// rounded sum, deterministic, while the epilogue never waits for the old
// value.

// Epilogue for a pair of x-adjacent cells (x even) at position `pos` along
// the axis: q = linear index of the first cell, (x, y, z) its coordinates;
// off / soff = this simulation's offset into the field / slab arrays
// (materials are shared by all simulations).
__device__ __forceinline__ void epilogue_pair(const PassParams& p, const PassJob& J, size_t q, int pos,
                                              int x, int y, int z, float d0, float d1, size_t off, size_t soff)
{
    if (!ES_INB(p, off + q + 1, p.ext_f)) return;
    if (J.kind == JOB_STORE) {
        *reinterpret_cast<float2*>(J.tgt[0] + off + q) = make_float2(d0, d1);
        return;
    }
    if (!ES_INB(p, q + 1, p.ext_c)) return;
    const float dt = p.dt;
    const bool slab = in_slab(pos, p.n, p.L);
    const int S = 2 * p.L + 1;
    if (J.kind == JOB_SINGLE) {
        const float2 c = __ldg(reinterpret_cast<const float2*>(J.coef[0] + q));
        float2 inc = make_float2(increment(dt, c.x, d0), increment(dt, c.y, d1));
        if (slab) {
            const float P = __ldg((J.stag ? p.ps : p.pc) + pos);
            const size_t si = slab_index(p.axis, x, y, z, slab_pos(pos, p.n, p.L), p.nx, p.ny, S);
            if (!ES_INB(p, soff + si + 1, p.ext_s)) return;
            inc.x = split_delta(J.slab[0], soff + si, P, inc.x);
            inc.y = split_delta(J.slab[0], soff + si + 1, P, inc.y);
        }
        atomicAdd(reinterpret_cast<float2*>(J.tgt[0] + off + q), inc);
    } else {
        const float2 lam = __ldg(reinterpret_cast<const float2*>(J.coef[0] + q));
        const float2 mu = __ldg(reinterpret_cast<const float2*>(J.coef[1] + q));
        const float P = slab ? __ldg(p.pc + pos) : 1.f;
        const size_t si = slab ? slab_index(p.axis, x, y, z, slab_pos(pos, p.n, p.L), p.nx, p.ny, S) : 0;
        if (slab && !ES_INB(p, soff + si + 1, p.ext_s)) return;
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            const float2 c = make_float2(normal_coef(lam.x, mu.x, t == J.diag), normal_coef(lam.y, mu.y, t == J.diag));
            float2 inc = make_float2(increment(dt, c.x, d0), increment(dt, c.y, d1));
            if (slab) {
                inc.x = split_delta(J.slab[t], soff + si, P, inc.x);
                inc.y = split_delta(J.slab[t], soff + si + 1, P, inc.y);
            }
            atomicAdd(reinterpret_cast<float2*>(J.tgt[t] + off + q), inc);
        }
    }
}

// Epilogue for 4 x-consecutive cells of one x line (x pass): q0 = linear
// index of the first, pos0 its x, line = y + ny z (the x slabs' row index),
// d[] the derivatives.
__device__ __forceinline__ void epilogue_quad(const PassParams& p, const PassJob& J, size_t q0, int pos0,
                                              int line, const float* d, size_t off, size_t soff)
{
    if (!ES_INB(p, off + q0 + 3, p.ext_f)) return;
    if (J.kind == JOB_STORE) {
        *reinterpret_cast<float4*>(J.tgt[0] + off + q0) = make_float4(d[0], d[1], d[2], d[3]);
        return;
    }
    // the coefficients, and this line's row of the x slabs (S cells)
    if (!ES_INB(p, q0 + 3, p.ext_c)) return;
    if (p.L > 0 && !ES_INB(p, soff + (size_t)(2 * p.L + 1) * (line + 1) - 1, p.ext_s)) return;
    const float dt = p.dt;
    const int S = 2 * p.L + 1;
    const size_t srow = soff + (size_t)S * (size_t)line;  // slab_index(0, ...) without the division
    if (J.kind == JOB_SINGLE) {
        const float4 c4 = __ldg(reinterpret_cast<const float4*>(J.coef[0] + q0));
        const float cv[4] = {c4.x, c4.y, c4.z, c4.w};
        float iv[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int pos = pos0 + e;
            iv[e] = increment(dt, cv[e], d[e]);
            if (in_slab(pos, p.n, p.L))
                iv[e] = split_delta(J.slab[0], srow + slab_pos(pos, p.n, p.L), __ldg((J.stag ? p.ps : p.pc) + pos),
                                    iv[e]);
        }
        atomicAdd(reinterpret_cast<float4*>(J.tgt[0] + off + q0), make_float4(iv[0], iv[1], iv[2], iv[3]));
    } else {
        const float4 l4 = __ldg(reinterpret_cast<const float4*>(J.coef[0] + q0));
        const float4 m4 = __ldg(reinterpret_cast<const float4*>(J.coef[1] + q0));
        const float lv[4] = {l4.x, l4.y, l4.z, l4.w};
        const float mv[4] = {m4.x, m4.y, m4.z, m4.w};
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            float iv[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int pos = pos0 + e;
                iv[e] = increment(dt, normal_coef(lv[e], mv[e], t == J.diag), d[e]);
                if (in_slab(pos, p.n, p.L))
                    iv[e] = split_delta(J.slab[t], srow + slab_pos(pos, p.n, p.L), __ldg(p.pc + pos), iv[e]);
            }
            atomicAdd(reinterpret_cast<float4*>(J.tgt[t] + off + q0), make_float4(iv[0], iv[1], iv[2], iv[3]));
        }
    }
}

// Epilogue for one cell (odd nx in the y / z passes, any length in the x pass,
// the circulant passes): the same arithmetic as epilogue_pair / epilogue_quad,
// one cell at a time.
__device__ __forceinline__ void epilogue_one(const PassParams& p, const PassJob& J, size_t q, int pos, int x, int y,
                                             int z, float d, size_t off, size_t soff)
{
    if (!ES_INB(p, off + q, p.ext_f)) return;
    if (J.kind == JOB_STORE) {
        J.tgt[0][off + q] = d;
        return;
    }
    if (!ES_INB(p, q, p.ext_c)) return;
    const float dt = p.dt;
    const bool slab = in_slab(pos, p.n, p.L);
    const int S = 2 * p.L + 1;
    if (J.kind == JOB_SINGLE) {
        float inc = increment(dt, __ldg(J.coef[0] + q), d);
        if (slab) {
            const float P = __ldg((J.stag ? p.ps : p.pc) + pos);
            const size_t si = slab_index(p.axis, x, y, z, slab_pos(pos, p.n, p.L), p.nx, p.ny, S);
            if (!ES_INB(p, soff + si, p.ext_s)) return;
            inc = split_delta(J.slab[0], soff + si, P, inc);
        }
        atomicAdd(J.tgt[0] + off + q, inc);
    } else {
        const float lam = __ldg(J.coef[0] + q), mu = __ldg(J.coef[1] + q);
        const float P = slab ? __ldg(p.pc + pos) : 1.f;
        const size_t si = slab ? slab_index(p.axis, x, y, z, slab_pos(pos, p.n, p.L), p.nx, p.ny, S) : 0;
        if (slab && !ES_INB(p, soff + si, p.ext_s)) return;
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            float inc = increment(dt, normal_coef(lam, mu, t == J.diag), d);
            if (slab) inc = split_delta(J.slab[t], soff + si, P, inc);
            atomicAdd(J.tgt[t] + off + q, inc);
        }
    }
}

// ---------------------------------------------------------------------------
// FFT core on the shared [pos][line] layout (one buffer, updated in place:
// every stage reads all its inputs, the block synchronises, then it writes)
// ---------------------------------------------------------------------------
template <int RA, int RB, int CPAD>
struct Core {
    static constexpr int N = RA * RB;
    static constexpr int BA = N / RA;   // stage-A butterflies = threads per line
    static constexpr int BB = N / RB;   // stage-B butterflies
    static constexpr int T = BA;
    static constexpr int MB = (BB + T - 1) / T;

    // stage A (radix RA, Stockham Ns = 1): a[] holds elements j + r BA; the
    // result goes to element j RA + q
    static __device__ __forceinline__ void stageA_store(const float2* a, float2* buf, int j, int c)
    {
#pragma unroll
        for (int q = 0; q < RA; ++q) buf[(j * RA + q) * CPAD + c] = a[q];
    }

    // stage B (radix RB, Ns = RA), spectral multiply, conjugate, first inverse
    // stage (radix RB, Ns = 1), all in registers
    static __device__ __forceinline__ void stageB_compute(const float2* buf, float2 (&v)[MB][RB], const float2* tw,
                                                          const float2* H, int j, int c)
    {
#pragma unroll
        for (int m = 0; m < MB; ++m) {
            const int b = j + m * T;
            if (BB % T == 0 || b < BB) {
                const int k = b % RA;
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    const float2 x = buf[(b + r * BB) * CPAD + c];
                    v[m][r] = r == 0 ? x : cmul(x, tw[k * r]);
                }
                Dft<RB>::run(v[m]);
#pragma unroll
                for (int q = 0; q < RB; ++q) {
                    const float2 y = cmul(H[b + q * BB], v[m][q]);
                    v[m][q] = make_float2(y.x, -y.y);
                }
                Dft<RB>::run(v[m]);
            }
        }
    }
    static __device__ __forceinline__ void stageB_store(float2* buf, const float2 (&v)[MB][RB], int j, int c)
    {
#pragma unroll
        for (int m = 0; m < MB; ++m) {
            const int b = j + m * T;
            if (BB % T == 0 || b < BB) {
#pragma unroll
                for (int q = 0; q < RB; ++q) buf[(b * RB + q) * CPAD + c] = v[m][q];
            }
        }
    }

    // last inverse stage (radix RA, Ns = RB): a[q] = conj(result) at element
    // j + q BA, so a[q].x / a[q].y are the derivatives of pencils 2c / 2c+1
    static __device__ __forceinline__ void stageA_inv_load(const float2* buf, const float2* tw, float2* a, int j,
                                                           int c)
    {
        const int k = j % RB;
#pragma unroll
        for (int r = 0; r < RA; ++r) {
            const float2 x = buf[(j + r * BA) * CPAD + c];
            a[r] = r == 0 ? x : cmul(x, tw[k * r]);
        }
    }
    static __device__ __forceinline__ void stageA_inv_finish(float2* a)
    {
        Dft<RA>::run(a);
#pragma unroll
        for (int q = 0; q < RA; ++q) a[q].y = -a[q].y;
    }
    static __device__ __forceinline__ void stageA_inv(const float2* buf, const float2* tw, float2* a, int j, int c)
    {
        stageA_inv_load(buf, tw, a, j, c);
        stageA_inv_finish(a);
    }

    // everything between the first forward and the last inverse stage
    static __device__ __forceinline__ void middle(float2* buf, const float2* tw, const float2* H, int j, int c)
    {
        float2 v[MB][RB];
        stageB_compute(buf, v, tw, H, j, c);
        __syncthreads();
        stageB_store(buf, v, j, c);
    }
};

// Three-stage plan n = R1 R2 R3 (Stockham, as Core): forward stages of radix
// R1, R2, R3, the spectral multiply on the elements the last one leaves in a
// thread's registers, then the inverse (forward DFTs of the conjugate) with
// the radices reversed: R3 on those same elements, R2, and R1, which ends on
// the elements j + q n/R1 the first stage read.  A stage of radix R after
// stages whose radices multiply to Ns: butterfly b (k = b mod Ns) reads
// elements b + r n/R times W_(Ns R)^(k r), runs the R-point DFT and writes
// element (b / Ns) Ns R + k + q Ns.  All stages but the first and the last
// run on the shared buffer; n/R1 threads per line, every butterfly of a
// stage by one thread.
template <int R1, int R2, int R3, int CPAD>
struct Core3 {
    static constexpr int N = R1 * R2 * R3;
    static constexpr int BA = N / R1;  // first / last stage butterflies = threads per line
    static constexpr int T = BA;

    static __device__ __forceinline__ void stageA_store(const float2* a, float2* buf, int j, int c)
    {
#pragma unroll
        for (int q = 0; q < R1; ++q) buf[(j * R1 + q) * CPAD + c] = a[q];
    }

    // one stage of radix R after radices multiplying to NS, shared buffer to
    // shared buffer (reads, block barrier, writes)
    template <int R, int NS>
    static __device__ __forceinline__ void stage(float2* buf, const float2* tw, int j, int c)
    {
        constexpr int B = N / R, M = (B + T - 1) / T, TS = N / (NS * R);
        float2 v[M][R];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const int b = j + m * T;
            if (B % T == 0 || b < B) {
                const int k = b % NS;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const float2 x = buf[(b + r * B) * CPAD + c];
                    v[m][r] = r == 0 ? x : cmul(x, tw[k * r * TS]);
                }
                Dft<R>::run(v[m]);
            }
        }
        __syncthreads();
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const int b = j + m * T;
            if (B % T == 0 || b < B) {
                const int k = b % NS, o = (b / NS) * NS * R + k;
#pragma unroll
                for (int q = 0; q < R; ++q) buf[(o + q * NS) * CPAD + c] = v[m][q];
            }
        }
    }

    static __device__ __forceinline__ void middle(float2* buf, const float2* tw, const float2* H, int j, int c)
    {
        stage<R2, R1>(buf, tw, j, c);
        __syncthreads();
        {
            // last forward stage (radix R3, Ns = n/R3, so k = b), multiply,
            // conjugate, first inverse stage (radix R3, Ns = 1) in registers
            constexpr int B = N / R3, M = (B + T - 1) / T;
            float2 v[M][R3];
#pragma unroll
            for (int m = 0; m < M; ++m) {
                const int b = j + m * T;
                if (B % T == 0 || b < B) {
#pragma unroll
                    for (int r = 0; r < R3; ++r) {
                        const float2 x = buf[(b + r * B) * CPAD + c];
                        v[m][r] = r == 0 ? x : cmul(x, tw[b * r]);
                    }
                    Dft<R3>::run(v[m]);
#pragma unroll
                    for (int q = 0; q < R3; ++q) {
                        const float2 y = cmul(H[b + q * B], v[m][q]);
                        v[m][q] = make_float2(y.x, -y.y);
                    }
                    Dft<R3>::run(v[m]);
                }
            }
            __syncthreads();
#pragma unroll
            for (int m = 0; m < M; ++m) {
                const int b = j + m * T;
                if (B % T == 0 || b < B) {
#pragma unroll
                    for (int q = 0; q < R3; ++q) buf[(b * R3 + q) * CPAD + c] = v[m][q];
                }
            }
        }
        __syncthreads();
        stage<R2, R3>(buf, tw, j, c);
    }

    // last inverse stage (radix R1, Ns = n/R1, so k = j); a[q] = conj(result)
    // at element j + q BA
    static __device__ __forceinline__ void stageA_inv(const float2* buf, const float2* tw, float2* a, int j, int c)
    {
#pragma unroll
        for (int r = 0; r < R1; ++r) {
            const float2 x = buf[(j + r * BA) * CPAD + c];
            a[r] = r == 0 ? x : cmul(x, tw[j * r]);
        }
        Dft<R1>::run(a);
#pragma unroll
        for (int q = 0; q < R1; ++q) a[q].y = -a[q].y;
    }
};

// the FFT core of a plan (RC = 1: two stages)
template <int RA, int RB, int RC, int CPAD>
using CoreOf = std::conditional_t<RC == 1, Core<RA, RB, CPAD>, Core3<RA, RB, RC, CPAD>>;

// asynchronous 8-byte global -> shared copy (cp.async, through L1); no
// register is held while it is in flight
__device__ __forceinline__ void cp_async8(void* dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_all;\n" ::: "memory");
}

constexpr int CP = 16;  // complex lines (pencil pairs) per CTA

template <int RA, int RB, int RC>
__host__ __device__ constexpr int pass_threads() { return RB * RC * CP; }

// blocks per SM the register budget is sized for (about 1024 threads per SM;
// 1200 for the three-stage plans, whose butterflies hold fewer registers)
template <int RA, int RB, int RC>
__host__ __device__ constexpr int pass_min_blocks()
{
    return pass_threads<RA, RB, RC>() >= 1024 ? 1 : (RC == 1 ? 1024 : 1200) / pass_threads<RA, RB, RC>();
}

// rows of wrap-around copies on each side of the strided passes' reloaded
// source tile
constexpr int HALO = 5;
static_assert(-near_ofs(-1) <= HALO && near_ofs(+1) + NEAR_TAPS - 1 <= HALO, "near taps reach beyond the halo");

// shared bytes: one buffer [N + 2 HALO][CP] (FFT, then the source tile) + tables (y, z passes)
template <int RA, int RB, int RC>
__host__ __device__ constexpr size_t pass_smem_strided()
{
    return sizeof(float2) * ((size_t)(RA * RB * RC + 2 * HALO) * CP + 3 * (size_t)RA * RB * RC);
}
// x pass, lengths that are not a multiple of 16: cells per near-stencil item
// (a divisor of n) and the halo of the per-line copy of the source tile
template <int N>
__host__ __device__ constexpr int xseg()
{
    return N % 5 == 0 ? 5 : (N % 4 == 0 ? 4 : (N % 3 == 0 ? 3 : (N % 2 == 0 ? 2 : 1)));
}
constexpr int XHALO = 5;
// FFT buffer [N][CP + 1] + tables (x pass); for a length that is not a
// multiple of 16 also the source tile, line by line with XHALO wrap-around
// copies on each side
template <int RA, int RB, int RC>
__host__ __device__ constexpr size_t pass_smem_x()
{
    constexpr size_t N = (size_t)RA * RB * RC;
    return sizeof(float2) * (N * (CP + 1) + 3 * N) + (N % 16 ? sizeof(float) * 2 * CP * (N + 2 * XHALO) : 0);
}

// Programmatic dependent launch (a pass launched with PDL while the previous
// pass of the same half-step drains): let the next pass launch once every CTA
// of this one has started, and wait for the previous pass to complete (and its
// writes to be visible) before touching what it writes.  Both are no-ops for a
// plain launch.
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Start of a pass.  pdl 2: wait for the previous kernel first, and only then
// let dependents launch, so a dependent that reads early never overtakes a
// kernel this one still waits for.  pdl 1: this pass's early reads are final
// already (it launched after the previous pass had passed its own wait), so
// dependents may launch at once; the epilogue waits (pdl_wait) before adding.
// pdl 0: a plain launch, dependents launch when it completes.
__device__ __forceinline__ void pdl_begin(int pdl)
{
    if (pdl == 2) pdl_wait();
    if (pdl != 0) pdl_launch_dependents();
}

// Launch of a pass kernel, with the programmatic-stream-serialization
// attribute when p.pdl is set (the kernel then waits as p.pdl says).
template <class K>
inline cudaError_t launch_pass_kernel(K kernel, dim3 grid, int threads, size_t smem, cudaStream_t st,
                                      const PassParams& p)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = p.pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, p);
}

// Fused point sources and receivers of this CTA (PassParams::sp_mode): once
// the CTA's own field updates are done (a CTA barrier makes its threads'
// reductions visible to the CTA; the reads go through L2), thread 0 adds the
// sources in their order, and after a second barrier every receiver is
// recorded by a thread of its own -- the arithmetic of the separate injection
// and recording kernels (inject_kernel, record_kernel).  job = the CTA's job
// (blockIdx.y): the velocity z pass's job c updates v_c, the stress y pass's
// job 1 sxy, the stress z pass's job 0 sxx syy szz, job 1 sxz, job 2 syz.
__device__ __forceinline__ void special_phase(const PassParams& p, const PassJob& J, int job)
{
    const int b0 = p.sp_off[blockIdx.x], b1 = p.sp_off[blockIdx.x + 1];
    if (b0 == b1) return;  // the same for every thread of the CTA
    const int n = *p.step_now - 1;
    __syncthreads();
    if (p.sp[b0].kind != SP_RECEIVER) {  // sources come first in the list
        if (threadIdx.x == 0) {
            if (p.pdl == 1) pdl_wait();  // (done already if this thread had cells to update)
            for (int e = b0; e < b1; ++e) {
                if (!ES_INB(p, e, p.ext_sp)) break;
                const SpecialCell c = p.sp[e];
                if (c.kind == SP_RECEIVER) break;
                const SourceDev& s = p.src[c.idx];
                if (n >= s.nw) continue;
                const float w = s.w[n];
                auto add = [&](float* t, float m) {
                    if (m != 0.f && ES_INB(p, c.q, p.ext_f)) *t = __fmaf_rn(m, w, __ldcg(t));
                };
                if (p.sp_mode == SP_VEL_Z) {
                    if (c.kind == SP_FORCE) add(J.tgt[0] + c.q, s.m[job]);
                } else if (c.kind == SP_MOMENT) {
                    if (p.sp_mode == SP_STR_Y) {
                        if (job == 1) add(J.tgt[0] + c.q, s.m[3]);
                    } else if (job == 0) {
                        add(J.tgt[0] + c.q, s.m[0]);
                        add(J.tgt[1] + c.q, s.m[1]);
                        add(J.tgt[2] + c.q, s.m[2]);
                    } else {
                        add(J.tgt[0] + c.q, s.m[job == 1 ? 4 : 5]);
                    }
                }
            }
        }
        __syncthreads();
    }
    if (p.sp_mode == SP_STR_Y || (p.sp_mode == SP_STR_Z && job != 0)) return;
    if (p.pdl == 1) pdl_wait();
    for (int e = b0 + threadIdx.x; e < b1; e += blockDim.x) {
        if (!ES_INB(p, e, p.ext_sp)) break;
        const SpecialCell c = p.sp[e];
        if (c.kind != SP_RECEIVER) continue;
        const size_t row0 = ((size_t)(n - p.rec_start) * p.nsim + c.sim) * 4 * p.n_rcv;
        if (!ES_INB(p, c.q, p.ext_f) || !ES_INB(p, row0 + 4 * (size_t)p.n_rcv - 1, p.ext_rec)) continue;
        float* row = p.rec + row0;
        if (p.sp_mode == SP_VEL_Z) {
            row[(size_t)(job + 1) * p.n_rcv + c.idx] = __ldcg(J.tgt[0] + c.q);
        } else {
            const float s = __fadd_rn(__fadd_rn(__ldcg(J.tgt[0] + c.q), __ldcg(J.tgt[1] + c.q)),
                                      __ldcg(J.tgt[2] + c.q));
            row[c.idx] = __fdiv_rn(-s, 3.f);  // Eq. (3)
        }
    }
}

// warm L2 with a 128-byte line the epilogue will read (no registers held)
__device__ __forceinline__ void prefetch_l2(const void* p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

template <int N>
__device__ __forceinline__ void load_tables(const PassParams& p, float2* s_tw, float2* s_hp, float2* s_hm, int tid,
                                            int nthreads)
{
    for (int i = tid; i < N; i += nthreads) {
        s_tw[i] = p.tw[i];
        s_hp[i] = p.hp[i];
        s_hm[i] = p.hm[i];
    }
}

// y and z passes: blockIdx.x = tile (32 consecutive x at one z (y pass) or
// one y (z pass)), blockIdx.y = job.  ODD: nx is odd, so a pencil pair does not
// start on an 8-byte boundary in every row; the pair then moves as two floats
// (the second one absent at x = nx - 1), with the same arithmetic.
template <int RA, int RB, int RC, bool ODD>
__global__ void __launch_bounds__(pass_threads<RA, RB, RC>(), pass_min_blocks<RA, RB, RC>())
pass_strided(const __grid_constant__ PassParams p)
{
    using C = CoreOf<RA, RB, RC, CP>;
    constexpr int N = C::N, BA = C::BA, T = C::T;
    extern __shared__ float2 smem[];
    float2* buf = smem;  // FFT rows 0 .. N-1; then the source tile at rows HALO + pos (wrapped)
    float2* s_tw = buf + (N + 2 * HALO) * CP;
    float2* s_hp = s_tw + N;
    float2* s_hm = s_hp + N;
    const int tid = threadIdx.x;
    const int c = tid % CP, j = tid / CP;
    const PassJob& J = p.job[blockIdx.y];
    pdl_begin(p.pdl);
    // simulations run fastest in blockIdx.x: the CTAs of one tile are adjacent
    // and read that tile's material rows through L2
    const int sim = blockIdx.x % p.nsim, tile = blockIdx.x / p.nsim;
    const size_t off = (size_t)sim * p.fstride, soff = (size_t)sim * p.sstride;
    const int ntx = (p.nx + 2 * CP - 1) / (2 * CP);
    const int tx = tile % ntx, outer = tile / ntx;
    const int x = tx * 2 * CP + 2 * c;
    const bool valid = x < p.nx;
    const bool valid1 = x + 1 < p.nx;  // the second pencil of the pair (ODD)
    size_t base, est;
    int y = 0, z = 0;
    if (p.axis == 1) {
        z = outer;
        base = (size_t)x + (size_t)p.nx * p.ny * z;
        est = (size_t)p.nx;
    } else {
        y = outer;
        base = (size_t)x + (size_t)p.nx * y;
        est = (size_t)p.nx * p.ny;
    }
    const float* src = J.src + off + base;
    float2 a[RA];
    if constexpr (ODD) {
#pragma unroll
        for (int r = 0; r < RA; ++r) {
            const float* g = src + (size_t)(j + r * BA) * est;
            a[r].x = valid && ES_INB(p, off + base + (size_t)(j + r * BA) * est, p.ext_f) ? __ldg(g) : 0.f;
            a[r].y = valid1 && ES_INB(p, off + base + (size_t)(j + r * BA) * est + 1, p.ext_f) ? __ldg(g + 1) : 0.f;
        }
    } else {
#pragma unroll
        for (int r = 0; r < RA; ++r)
            a[r] = valid && ES_INB(p, off + base + (size_t)(j + r * BA) * est + 1, p.ext_f)
                       ? __ldg(reinterpret_cast<const float2*>(src + (size_t)(j + r * BA) * est))
                       : make_float2(0.f, 0.f);
    }
    // coefficient rows of this tile (128 bytes each) into L2 for the epilogue
    if (tid < N && J.coef[0] && tx * 2 * CP < p.nx) {
        const size_t row = base - 2 * c + (size_t)tid * est;
        if (ES_INB(p, row, p.ext_c)) {
            prefetch_l2(J.coef[0] + row);
            if (J.coef[1]) prefetch_l2(J.coef[1] + row);
        }
    }
    load_tables<N>(p, s_tw, s_hp, s_hm, tid, T * CP);
    Dft<RA>::run(a);
    C::stageA_store(a, buf, j, c);
    __syncthreads();
    C::middle(buf, s_tw, J.sign > 0 ? s_hp : s_hm, j, c);
    __syncthreads();
    C::stageA_inv(buf, s_tw, a, j, c);
    __syncthreads();
    if (valid) {
        const float* g = src + (size_t)j * est;
        float2* sb = buf + (j + HALO) * CP + c;
        const size_t gstep = (size_t)BA * est;
#pragma unroll 1
        for (int r = 0; r < RA; ++r, g += gstep, sb += BA * CP) {
#if ES_BOUNDS
            if (!ES_INB(p, off + base + (size_t)(j + r * BA) * est + (ODD && !valid1 ? 0 : 1), p.ext_f)) {
                *sb = make_float2(0.f, 0.f);
                continue;
            }
#endif
            if constexpr (ODD) {
                cp_async4(&sb->x, g);
                if (valid1) cp_async4(&sb->y, g + 1);
                else sb->y = 0.f;
            } else {
                cp_async8(sb, g);
            }
        }
    }
    for (int i = tid; i < 2 * HALO * CP; i += T * CP) {
        const int h = i / CP, cc = i % CP;
        const int xc = tx * 2 * CP + 2 * cc;
        if (xc >= p.nx) continue;
        const int pos = h < HALO ? N - HALO + h : h - HALO;
        float2* d = buf + (h < HALO ? h : N + h) * CP + cc;
        const float* g = J.src + off + base - 2 * c + 2 * cc + (size_t)pos * est;
#if ES_BOUNDS
        if (!ES_INB(p, off + base - 2 * c + 2 * cc + (size_t)pos * est + (ODD && xc + 1 >= p.nx ? 0 : 1), p.ext_f)) {
            *d = make_float2(0.f, 0.f);
            continue;
        }
#endif
        if constexpr (ODD) {
            cp_async4(&d->x, g);
            if (xc + 1 < p.nx) cp_async4(&d->y, g + 1);
            else d->y = 0.f;
        } else {
            cp_async8(d, g);
        }
    }
    cp_async_commit_wait_all();
    __syncthreads();
    if (valid) {
        // near part: the 10 taps in order from the first offset, then one add to the far part
        const int o = HALO + near_ofs(J.sign);
#pragma unroll
        for (int q = 0; q < RA; ++q) {
            const float2* w = buf + (j + q * BA + o) * CP + c;
            float2 s = make_float2(0.f, 0.f);
#pragma unroll
            for (int t = 0; t < NEAR_TAPS; ++t) s = fma2(make_float2(J.g[t], J.g[t]), w[t * CP], s);
            a[q] = add2(a[q], s);
        }
        if (p.pdl == 1) pdl_wait();  // the previous pass's updates of the targets come first
#pragma unroll
        for (int q = 0; q < RA; ++q) {
            const int pos = j + q * BA;
            if (p.axis == 1) y = pos; else z = pos;
            const size_t qc = base + (size_t)pos * est;
            if constexpr (ODD) {
                epilogue_one(p, J, qc, pos, x, y, z, a[q].x, off, soff);
                if (valid1) epilogue_one(p, J, qc + 1, pos, x + 1, y, z, a[q].y, off, soff);
            } else {
                epilogue_pair(p, J, qc, pos, x, y, z, a[q].x, a[q].y, off, soff);
            }
        }
    }
    if (p.sp_mode != SP_NONE) special_phase(p, J, blockIdx.y);
}

// x pass epilogue: the far derivative from the turned-around FFT buffer (bf,
// [x][line]) plus the near stencil over the source line, read again from
// global memory (L1 / L2: the CTA read the whole tile at its start), then the
// field update, four consecutive x of one line per item.  OFS = first tap
// offset.
template <int N, int CPAD, int OFS, int NT>
__device__ __forceinline__ void pass_x_epilogue(const PassParams& p, const PassJob& J, const float* bf,
                                                const float* src, int line0, int nlines, size_t off, size_t soff)
{
    constexpr int LINES = 2 * CP;
    constexpr int ITEMS = LINES * N / 4;

    // x = xx - 8 .. xx + 11 in five float4 chunks (wrapped along the line); the
    // taps of the four outputs reach xx + OFS .. xx + 3 + OFS + NEAR_TAPS - 1
    static_assert(8 + OFS >= 0 && 8 + 3 + OFS + NEAR_TAPS - 1 < 20, "near taps outside the window");
#pragma unroll 2
    for (int i = 0; i < (ITEMS + NT - 1) / NT; ++i) {
        const int it = (int)threadIdx.x + i * NT;
        if (ITEMS % NT != 0 && it >= ITEMS) break;
        const int lo = it & 3, r = (it >> 2) & (LINES - 1), hi = it >> 7;
        const int xx = (hi * 4 + lo) * 4;
        const int line = line0 + r;
        if (line >= nlines) continue;
        const float* ln = src + (size_t)line * N;
        float w[20];  // w[m] = f at x = xx - 8 + m
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            const int x0 = (xx - 8 + 4 * m + N) % N;
            if (4 * m + 3 < 8 + OFS || 4 * m > 8 + 3 + OFS + NEAR_TAPS - 1) continue;  // chunk unused
#if ES_BOUNDS
            if (!ES_INB(p, off + (size_t)line * N + x0 + 3, p.ext_f)) return;
#endif
            const float4 v = __ldg(reinterpret_cast<const float4*>(ln + x0));
            w[4 * m] = v.x;
            w[4 * m + 1] = v.y;
            w[4 * m + 2] = v.z;
            w[4 * m + 3] = v.w;
        }
        // outputs xx, xx + 1 and xx + 2, xx + 3 as packed pairs
        float2 s01 = make_float2(0.f, 0.f), s23 = make_float2(0.f, 0.f);
#pragma unroll
        for (int t = 0; t < NEAR_TAPS; ++t) {
            const float2 g2 = make_float2(J.g[t], J.g[t]);
            s01 = fma2(g2, make_float2(w[8 + OFS + t], w[9 + OFS + t]), s01);
            s23 = fma2(g2, make_float2(w[10 + OFS + t], w[11 + OFS + t]), s23);
        }
        const float sn[4] = {s01.x, s01.y, s23.x, s23.y};
        float d[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) d[e] = __fadd_rn(bf[((xx + e) * CPAD) * 2 + r], sn[e]);
        epilogue_quad(p, J, (size_t)line * N + xx, xx, line, d, off, soff);
    }
}

// Epilogue for 4 consecutive cells of an x-pass tile in memory order (f0 =
// the first one's offset from the tile start, q0 its linear index, 16-byte
// aligned): a chunk may span two lines, so every cell takes its own x and
// line for the PML split (slab row S line); the arithmetic of epilogue_one.
template <int N>
__device__ __forceinline__ void epilogue_quad_flat(const PassParams& p, const PassJob& J, size_t q0, int f0,
                                                   int line0, float4 d4, size_t off, size_t soff)
{
    if (!ES_INB(p, off + q0 + 3, p.ext_f)) return;
    if (J.kind == JOB_STORE) {
        *reinterpret_cast<float4*>(J.tgt[0] + off + q0) = d4;
        return;
    }
    if (!ES_INB(p, q0 + 3, p.ext_c)) return;
    const float d[4] = {d4.x, d4.y, d4.z, d4.w};
    const float dt = p.dt;
    const int S = 2 * p.L + 1;
    int xs[4];
    size_t srow[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int r = (f0 + e) / N;
        xs[e] = f0 + e - r * N;
        srow[e] = soff + (size_t)S * (size_t)(line0 + r);
        if (p.L > 0 && !ES_INB(p, srow[e] + S - 1, p.ext_s)) return;
    }
    if (J.kind == JOB_SINGLE) {
        const float4 c4 = __ldg(reinterpret_cast<const float4*>(J.coef[0] + q0));
        const float cv[4] = {c4.x, c4.y, c4.z, c4.w};
        float iv[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            iv[e] = increment(dt, cv[e], d[e]);
            if (in_slab(xs[e], p.n, p.L))
                iv[e] = split_delta(J.slab[0], srow[e] + slab_pos(xs[e], p.n, p.L),
                                    __ldg((J.stag ? p.ps : p.pc) + xs[e]), iv[e]);
        }
        atomicAdd(reinterpret_cast<float4*>(J.tgt[0] + off + q0), make_float4(iv[0], iv[1], iv[2], iv[3]));
    } else {
        const float4 l4 = __ldg(reinterpret_cast<const float4*>(J.coef[0] + q0));
        const float4 m4 = __ldg(reinterpret_cast<const float4*>(J.coef[1] + q0));
        const float lv[4] = {l4.x, l4.y, l4.z, l4.w};
        const float mv[4] = {m4.x, m4.y, m4.z, m4.w};
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            float iv[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                iv[e] = increment(dt, normal_coef(lv[e], mv[e], t == J.diag), d[e]);
                if (in_slab(xs[e], p.n, p.L))
                    iv[e] = split_delta(J.slab[t], srow[e] + slab_pos(xs[e], p.n, p.L), __ldg(p.pc + xs[e]), iv[e]);
            }
            atomicAdd(reinterpret_cast<float4*>(J.tgt[t] + off + q0), make_float4(iv[0], iv[1], iv[2], iv[3]));
        }
    }
}

// x pass epilogue for a length that is not a multiple of 16.  The derivative
// of every cell is formed one cell per thread in memory order over the tile
// (the far part from the turned-around buffer, the near taps read one by one
// and wrapped along the line: the arithmetic of pass_x_epilogue), written
// back to the buffer in memory order, and the update then takes four cells
// per thread with 16-byte coefficient loads and reductions (the tile, 32 n
// floats from line 32 k, starts on a 16-byte boundary).
template <int N, int CPAD, int OFS, int NT>
__device__ __forceinline__ void pass_x_epilogue_any(const PassParams& p, const PassJob& J, float* bf,
                                                    const float* srcs, int line0, int nlines, size_t off,
                                                    size_t soff)
{
    static_assert(XHALO + OFS >= 0 && XHALO + OFS + NEAR_TAPS - 1 <= 2 * XHALO, "near taps outside the halo");
    constexpr int LINES = 2 * CP;
    constexpr int XS = xseg<N>(), NS = N / XS, W = N + 2 * XHALO;
    constexpr int ITER = (LINES * NS + NT - 1) / NT;
    static_assert(LINES * N <= 2 * N * CPAD, "the tile's derivatives fit the buffer");
    const int nl = min(LINES, nlines - line0);
    const int nf = nl * N;
    const int tid = threadIdx.x;
    // item = XS consecutive cells of one line: a window of XS + NEAR_TAPS - 1
    // source values from the line's copy, the near taps in order from the
    // first offset, then one add to the far part
    float dv[ITER][XS];
#pragma unroll
    for (int i = 0; i < ITER; ++i) {
        const int it = tid + i * NT;
        const int r = it / NS, x0 = (it - r * NS) * XS;
        if (r < nl) {
            const float* wrow = srcs + r * W + XHALO + OFS + x0;
            float w[XS + NEAR_TAPS - 1];
#pragma unroll
            for (int k = 0; k < XS + NEAR_TAPS - 1; ++k) w[k] = wrow[k];
#pragma unroll
            for (int e = 0; e < XS; ++e) {
                float s = 0.f;
#pragma unroll
                for (int t = 0; t < NEAR_TAPS; ++t) s = fmaf(J.g[t], w[e + t], s);
                dv[i][e] = __fadd_rn(bf[((x0 + e) * CPAD) * 2 + r], s);
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ITER; ++i) {
        const int it = tid + i * NT;
        const int r = it / NS, x0 = (it - r * NS) * XS;
        if (r < nl) {
#pragma unroll
            for (int e = 0; e < XS; ++e) bf[r * N + x0 + e] = dv[i][e];
        }
    }
    __syncthreads();
    const size_t q0 = (size_t)line0 * N;
    // 16-byte chunks need every array they touch on a 16-byte boundary at the
    // tile (the tile's own offset q0 is a multiple of 4 cells): the targets
    // at this simulation's offset (an odd cell count per simulation leaves
    // every other one unaligned) and the coefficient arrays, which a caller
    // may pass at any 4-byte offset
    auto a16 = [](const float* q) { return ((uintptr_t)q & 15) == 0; };
    bool vec = a16(J.tgt[0] + off);
    if (J.kind == JOB_NORMAL) vec = vec && a16(J.tgt[1] + off) && a16(J.tgt[2] + off) && a16(J.coef[1]);
    if (J.kind != JOB_STORE) vec = vec && a16(J.coef[0]);
    const int nq = vec ? nf / 4 : 0;
    for (int i = tid; i < nq; i += NT)
        epilogue_quad_flat<N>(p, J, q0 + 4 * (size_t)i, 4 * i, line0, reinterpret_cast<const float4*>(bf)[i], off,
                              soff);
    // what is left: a last, partial tile's cells past its last full chunk
    for (int f = 4 * nq + tid; f < nf; f += NT) {
        const int r = f / N, x = f - r * N, line = line0 + r;
        epilogue_one(p, J, q0 + f, x, x, line % p.ny, line / p.ny, bf[f], off, soff);
    }
}

// x pass: blockIdx.x = tile of 32 consecutive x-lines (line = y + ny z, so
// the tile is one contiguous block of memory), blockIdx.y = job.  The FFT
// result is turned around in the shared buffer so that a thread owns four
// consecutive x of one line (an item) in the epilogue.
template <int RA, int RB, int RC>
__global__ void __launch_bounds__(pass_threads<RA, RB, RC>(), pass_min_blocks<RA, RB, RC>())
pass_x(const __grid_constant__ PassParams p)
{
    constexpr int CPAD = CP + 1;  // row padding: the staging transposes stay conflict-free
    using C = CoreOf<RA, RB, RC, CPAD>;
    constexpr int N = C::N, BA = C::BA, NT = C::T * CP;
    constexpr int LINES = 2 * CP;
    constexpr int ITEMS = LINES * N / 4;  // float4 chunks in the tile (N a multiple of 16)
    extern __shared__ float2 smem[];
    float2* buf = smem;
    float2* s_tw = buf + N * CPAD;
    float2* s_hp = s_tw + N;
    float2* s_hm = s_hp + N;
    const int tid = threadIdx.x;
    const int c = tid % CP, j = tid / CP;
    const PassJob& J = p.job[blockIdx.y];
    pdl_begin(p.pdl);
    // the first pass of a fused time step advances the step counter
    if (p.step_counter && blockIdx.x == 0 && blockIdx.y == 0 && tid == 0) *p.step_counter += 1;
    const int nlines = p.ny * p.nz;
    const int sim = blockIdx.x % p.nsim;
    const size_t off = (size_t)sim * p.fstride, soff = (size_t)sim * p.sstride;
    const int line0 = (blockIdx.x / p.nsim) * LINES;
    const float* src = J.src + off;
    // chunk it -> line r = (it / 4) % 32, x = 4 (4 (it / 128) + it % 4): a warp
    // covers 8 lines x 64 contiguous bytes, and its shared stores hit 32 banks
    float* bf = reinterpret_cast<float*>(buf);
    // the tile's coefficient lines (contiguous, N lines of 128 bytes) into L2
    if (J.coef[0] && tid < N) {
        const size_t off = (size_t)line0 * N + (size_t)tid * 32;
        if (off < (size_t)nlines * N) {
            prefetch_l2(J.coef[0] + off);
            if (J.coef[1]) prefetch_l2(J.coef[1] + off);
        }
    }
    if constexpr (N % 16 == 0) {
#pragma unroll
        for (int i = 0; i < (ITEMS + NT - 1) / NT; ++i) {
            const int it = tid + i * NT;
            if (ITEMS % NT != 0 && it >= ITEMS) break;
            const int lo = it & 3, r = (it >> 2) & (LINES - 1), hi = it >> 7;
            const int xx = (hi * 4 + lo) * 4;
            const int line = line0 + r;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (line < nlines && ES_INB(p, off + (size_t)line * N + xx + 3, p.ext_f))
                v = __ldg(reinterpret_cast<const float4*>(src + (size_t)line * N + xx));
            bf[((xx + 0) * CPAD) * 2 + r] = v.x;
            bf[((xx + 1) * CPAD) * 2 + r] = v.y;
            bf[((xx + 2) * CPAD) * 2 + r] = v.z;
            bf[((xx + 3) * CPAD) * 2 + r] = v.w;
        }
    } else {
        // any length: the tile is one contiguous run of 32 N floats, read in
        // order; each value also goes to the per-line source copy (row r at
        // r (N + 2 XHALO), x at XHALO + x, the ends wrapped on both sides)
        const float* tile = src + (size_t)line0 * N;
        const int nf = min(LINES, nlines - line0) * N;
        float* srcs = reinterpret_cast<float*>(s_hm + N);
        constexpr int W = N + 2 * XHALO;
        constexpr int ITER = (LINES * N + NT - 1) / NT;
#pragma unroll
        for (int i = 0; i < ITER; ++i) {
            const int f = tid + i * NT;
            if (f < LINES * N) {
                const int r = f / N, xx = f - r * N;
                const float v = f < nf && ES_INB(p, off + (size_t)line0 * N + f, p.ext_f) ? __ldg(tile + f) : 0.f;
                bf[(xx * CPAD) * 2 + r] = v;
                float* row = srcs + r * W + XHALO;
                row[xx] = v;
                if (xx < XHALO) row[N + xx] = v;
                if (xx >= N - XHALO) row[xx - N] = v;
            }
        }
    }
    load_tables<N>(p, s_tw, s_hp, s_hm, tid, NT);
    __syncthreads();
    float2 a[RA];
#pragma unroll
    for (int r = 0; r < RA; ++r) a[r] = buf[(j + r * BA) * CPAD + c];
    Dft<RA>::run(a);
    __syncthreads();
    C::stageA_store(a, buf, j, c);
    __syncthreads();
    C::middle(buf, s_tw, J.sign > 0 ? s_hp : s_hm, j, c);
    __syncthreads();
    C::stageA_inv(buf, s_tw, a, j, c);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < RA; ++q) buf[(j + q * BA) * CPAD + c] = a[q];
    __syncthreads();
    if (p.pdl == 1) pdl_wait();  // the previous pass's updates of the targets come first
    if constexpr (N % 16 == 0) {
        if (J.sign > 0) pass_x_epilogue<N, CPAD, near_ofs(+1), NT>(p, J, bf, src, line0, nlines, off, soff);
        else pass_x_epilogue<N, CPAD, near_ofs(-1), NT>(p, J, bf, src, line0, nlines, off, soff);
    } else {
        const float* srcs = reinterpret_cast<const float*>(s_hm + N);
        if (J.sign > 0) pass_x_epilogue_any<N, CPAD, near_ofs(+1), NT>(p, J, bf, srcs, line0, nlines, off, soff);
        else pass_x_epilogue_any<N, CPAD, near_ofs(-1), NT>(p, J, bf, srcs, line0, nlines, off, soff);
    }
}

}  // namespace es
