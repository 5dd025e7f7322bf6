// Internal declarations shared by the kernel and host translation units of
// libes.so.  Nothing here is part of the public C ABI (include/es.h).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace es {

// Field numbering: velocity components, normal stresses, shear stresses.
enum { VX, VY, VZ, SXX, SYY, SZZ, SXY, SXZ, SYZ, NFIELD };
// Material arrays kept on the device.
enum { M_BX, M_BY, M_BZ, M_LAM, M_MU, M_MUXY, M_MUXZ, M_MUYZ, NMAT };

// What one derivative job does with D = D_axis^(sign) src in its epilogue.
enum JobKind {
    JOB_STORE = 0,   // tgt[0] = D (diagnostic)
    JOB_SINGLE = 1,  // tgt[0] += dt coef[0] D (split-field PML in slabs)
    JOB_NORMAL = 2   // sxx, syy, szz += dt (lambda + 2 mu [t == diag]) D
};

// The FFT passes evaluate each staggered derivative split in two:
//   D f = N f + IFFT(H_far FFT f),  (N f)_i = sum_t g_t f_{i + t + NEAR_OFS(sign)}
// with g the NEAR_TAPS central entries of the operator's circulant kernel and
// H_far = H - FFT(those entries), which in exact arithmetic is D itself.  The
// kernel decays as 1/l^2, so |H_far| is about 1 % of |H|, and the FFT's FP32
// roundoff -- spread over the whole pencil -- shrinks with it; the near part
// rounds locally, like the field storage itself.
constexpr int NEAR_TAPS = 10;
// The kernel is antisymmetric about the staggered point, g[NEAR_TAPS - 1 - t] = -g[t],
// so N f = sum over t < NEAR_PAIRS of g_t (f_{i+o+t} - f_{i+o+NEAR_TAPS-1-t}).
constexpr int NEAR_PAIRS = NEAR_TAPS / 2;
// first tap offset o: D(+) (result at i + 1/2) reads i-4 .. i+5, D(-) reads i-5 .. i+4
__host__ __device__ constexpr int near_ofs(int sign) { return sign > 0 ? -4 : -5; }

struct PassJob {
    const float* src;     // field differentiated (total)
    float* tgt[3];        // target totals
    float* slab[3];       // target split parts along this axis, slab storage
    const float* coef[2]; // JOB_SINGLE: coef[0]; JOB_NORMAL: lambda, mu
    int kind;
    int sign;             // +1: D(+) (result at +d/2), -1: D(-)
    int stag;             // targets sit at half indices along this axis
    int diag;             // JOB_NORMAL: target index receiving lambda + 2 mu
    float g[NEAR_TAPS];   // FFT passes: near taps of D(sign) (the multiplier tables hold H_far / n)
};

struct SourceDev {
    int kind;            // 0 moment, 1 force
    int smooth;          // 1: spread over the 5 x 5 x 5 Blackman stencil (moment sources)
    int sim;             // simulation the source belongs to
    long long cell;      // linear index
    float m[6];          // moment (Mxx Myy Mzz Mxy Mxz Myz) or force scale per component
    const float* w;      // wavelet samples (device)
    int nw;
};

// A cell where a fused pass injects a point source or records a receiver after
// its own field updates: q = linear index including the simulation's offset.
enum { SP_MOMENT = 0, SP_FORCE = 1, SP_RECEIVER = 2 };
struct SpecialCell {
    long long q;
    int kind;   // SP_MOMENT / SP_FORCE: idx = source; SP_RECEIVER: idx = receiver
    int idx;
    int sim;
};
// Which fused work a pass does in its special phase.
enum { SP_NONE = 0, SP_VEL_Z = 1, SP_STR_Y = 2, SP_STR_Z = 3 };

struct PassParams {
    int nx, ny, nz;
    int axis;             // 0 = x, 1 = y, 2 = z
    int n;                // length along the axis
    int njobs;
    PassJob job[3];
    const float2* tw;     // tw[m] = exp(-2 pi i m / n)
    const float2* hp;     // (H - H_near) / n for D(+), H = i kappa exp(+i kappa d/2)
    const float2* hm;     // the same for D(-), H = i kappa exp(-i kappa d/2)
    const float* ckp;     // circulant kernel of D(+) along the axis (lengths without an FFT plan)
    const float* ckm;     // circulant kernel of D(-)
    const float* ckp_lo;  // compensated mode: c - (float)c of the two kernels
    const float* ckm_lo;
    int circ;             // 1: the circulant pass (circ_pass.cu) instead of the FFT pass
    int comp;             // 1: compensated circulant pass (error-free products and sums)
    int pdl;              // programmatic dependent launch: 0 off; 1 sources may be read before the
                          // previous pass finishes (the epilogue waits); 2 wait before any read
    const float* pc;      // PML factors at whole indices along the axis
    const float* ps;      // PML factors at half indices along the axis
    int L;                // PML cells per face (slab width 2L+1, none if 0)
    float dt;
    int nsim;             // independent simulations sharing the materials
    long long fstride;    // elements between consecutive simulations' field arrays
    long long sstride;    // elements between consecutive simulations' slab arrays (this axis)
    const __nv_bfloat16* ctc;  // long circulant axes: the kernel matrices split in three BF16 parts,
                               // [D+, D-][split][outputs][inputs], each pad64(n) x pad64(n) (circ_tc.cu)
    float* scratch;            // that pass's derivatives, [job][sim][cell], before the field update
    // Point sources and receivers fused into the passes (FFT passes only): the first pass of a
    // step advances the device step counter (step_counter); the velocity z pass injects the
    // point forces and records the velocities, the stress y pass injects Mxy, the stress z pass
    // the other moment components and records the pressure.  sp_off[b] .. sp_off[b + 1] are
    // CTA b's (blockIdx.x) cells in sp, in source order, then receivers.  The step index is
    // *step_now - 1; samples go to rec[(n - rec_start) nsim + sim][4][n_rcv].
    int* step_counter;
    const int* step_now;
    int sp_mode;
    const int* sp_off;
    const SpecialCell* sp;
    const SourceDev* src;
    float* rec;
    long long rec_start;
    int n_rcv;
    // Extents for the bounds-checked build (ES_BOUNDS): elements of each field
    // array (all simulations), of each slab array of this axis, of each
    // coefficient array, of the receiver buffer, and entries of sp; bad: where
    // that build records the first index out of range (null otherwise).
    long long ext_f, ext_s, ext_c, ext_rec;
    int ext_sp;
    unsigned long long* bad;
};

// Bounds-checked debug build: compiled with -DES_BOUNDS=1 (libes_bounds.so),
// the pass kernels check each global index of their loads, stores and
// reductions against the array's extent before the access; an index out of
// range is recorded in *PassParams::bad (the first one: source line << 40 |
// the index's low 40 bits) and the access skipped, so the kernel never leaves
// its arrays.  The release build compiles the checks to nothing.
#ifndef ES_BOUNDS
#define ES_BOUNDS 0
#endif
// the device word of the bounds-checked build (null in the release build),
// and its allocation (a no-op in the release build; false if it failed)
unsigned long long* bounds_word();
bool bounds_init();

// Plan of the FFT for an axis length, as (R1, n / R1) (0 if unsupported).
int plan_radices(int n, int* ra, int* rb);
// Candidate plans for n (up to cap), and the plan in use per pass kind
// (0 = x pass, 1 = y/z passes): read and select.
int plan_candidates(int n, int* ra, int* rb, int cap);
int plan_current(int kind, int n, int* ra, int* rb);
int plan_select(int kind, int n, int ra, int rb);
// Launches one pass (all jobs) along p.axis.  Returns a cudaError_t.
cudaError_t launch_pass(const PassParams& p, cudaStream_t st);
// The y / z FFT pass for an odd nx with stage radices ra, rb, rc (rc = 1: two
// stages; pass_kernels_odd.cu), and its shared-memory opt-in.
cudaError_t launch_strided_odd(int ra, int rb, int rc, dim3 grid, const PassParams& p, cudaStream_t st);
cudaError_t prepare_strided_odd();
// Longest axis the circulant pass takes (shared tiles of 2 x 32 x pad(n) floats).
constexpr int CIRC_MAX_N = 512;
// From this length on, the CUDA-core circulant passes along y and z run their epilogue from
// the registers.
constexpr int CIRC_DIRECT_N = 192;
// From this length on, circulant passes in FP32 mode run on the tensor cores (circ_tc.cu):
// below it the CUDA-core pass is faster (measured at 75 and 125 cells: the scratch round trip
// and the separate update kernel cost more than the O(n) multiply-adds they replace).
constexpr int CIRC_TC_N = 192;
cudaError_t launch_circ(const PassParams& p, cudaStream_t st);
// The circulant pass on the tensor cores (long z axes, FP32 mode; circ_tc.cu).
bool circ_tc_eligible(const PassParams& p);
cudaError_t launch_circ_tc(const PassParams& p, cudaStream_t st);
// reads and clears its device status word (bits set by waits that gave up)
cudaError_t circ_tc_status(unsigned* status);
cudaError_t prepare_circ_kernels();
// Opts every pass kernel into the shared memory it needs (once per device).
cudaError_t prepare_pass_kernels();

// ---- auxiliary kernels (aux_kernels.cu) ----
cudaError_t launch_inject(float* const* fields, long long fstride, const SourceDev* src, int nsrc, int kind,
                          int nx, int ny, int* counter, int* cur, int advance, cudaStream_t st);
// rec[n - start][sim][4][n_rcv]
cudaError_t launch_record(float* const* fields, long long fstride, int nsim, const long long* rcv_cell,
                          int n_rcv, const int* cur, long long start, float* rec, cudaStream_t st);
// [nt][cols] -> [cols][nt]
cudaError_t launch_transpose_traces(const float* rec, int nt, int cols, float* out, cudaStream_t st);
cudaError_t launch_superpose(const float* traces, int n_src, int n_rcv, int nt, const int* ev_src,
                             const float* ev_amp, const int* ev_shift, int n_events, int n_out,
                             float* gather, cudaStream_t st);
struct MatPtrs {
    float* p[NMAT];  // the material arrays, indexed by M_BX ... M_MUYZ
};
// model setup on the device: every material array from rho, cp, cs (device, [nz][ny][nx])
cudaError_t launch_materials(const float* rho, const float* cp, const float* cs, int nx, int ny, int nz,
                             const MatPtrs& out, cudaStream_t st);
cudaError_t launch_fill(float* p, size_t n, float v, cudaStream_t st);
cudaError_t launch_visc_combine(float* const* fields, float* vold, float* w, size_t n, float a, float b,
                                cudaStream_t st);
cudaError_t launch_nonfinite(float* const* fields, size_t n, int* flag, cudaStream_t st);
cudaError_t launch_fill_slab(const float* total, float* slab, int axis, int nx, int ny, int nz,
                             int L, int copy, cudaStream_t st);

}  // namespace es
