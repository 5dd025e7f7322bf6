/*
 * es.h -- C ABI of libes.so, a GB300 (sm_103a) solver for the 3D heterogeneous
 * elastic wave equation by the staggered-grid Fourier pseudo-spectral method,
 * recording 4C seabed seismograms, after Das, Chen & Hobson, arXiv 1705.04874.
 *
 * Conventions shared by every call
 * --------------------------------
 * - Grids are [nz][ny][nx] FP32 arrays, x fastest, z = 0 at the sea surface
 *   and increasing with depth.  Linear index = ix + nx * (iy + ny * iz).
 * - Staggering (velocity at half time steps, stress at whole steps):
 *   sxx, syy, szz at (i, j, k); vx at (i+1/2, j, k); vy at (i, j+1/2, k);
 *   vz at (i, j, k+1/2); sxy at (i+1/2, j+1/2, k); sxz at (i+1/2, j, k+1/2);
 *   syz at (i, j+1/2, k+1/2).  Every field is stored at the index of its
 *   lower corner.
 * - Pointer arguments may be host or device memory unless stated otherwise;
 *   the library detects the kind with cudaPointerGetAttributes.  Inputs are
 *   copied (the caller keeps ownership); outputs are caller-owned buffers.
 * - Every call returns ES_OK or a negative status and writes no output on
 *   error.  Work is ordered on the model's stream (default: the legacy
 *   default stream); a call that returns ES_OK into a host buffer has
 *   finished; into a device buffer, it is complete in stream order.
 * - A model is not thread-safe: one thread at a time per model.
 * - Axis lengths run from 3 to 512; anything else is ES_ERR_SIZE.  The
 *   lengths 16, 32, 48, 64, 80, 96, 128, 160, 192 and 256 take the fused FFT
 *   passes (two-stage plans R1 x R2, R1, R2 in {4,5,6,8,10,12,16}; along y
 *   and z only when nx is even); every other length -- odd or non-smooth
 *   ones such as the paper's 125 x 75 x 301 grid (Sec. III) -- takes the
 *   circulant passes, which apply the same staggered spectral derivative as
 *   an exact periodic convolution with O(n) work per element.
 */
#ifndef ES_H
#define ES_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct es_model es_model; /* opaque, library-owned */

enum {
    ES_OK = 0,
    ES_ERR_ARG = -1,      /* bad argument (null, out of range, source in PML, ...) */
    ES_ERR_SIZE = -2,     /* unsupported grid axis length */
    ES_ERR_CUDA = -3,     /* a CUDA call failed (the message is kept, see es_last_error) */
    ES_ERR_OOM = -4,      /* device allocation failed */
    ES_ERR_UNSTABLE = -5, /* time step beyond the stability limit, or a non-finite field */
    ES_ERR_TIMEOUT = -6,  /* a bounded device wait ran out */
    ES_ERR_STATE = -7     /* call not valid in the model's current state */
};

/* Builds a model from density rho [kg/m^3], P velocity cp and S velocity cs
 * [m/s] per grid point (Sec. II-A, Eq. (4): mu = cs^2 rho, lambda + 2 mu =
 * cp^2 rho; water has cs = 0), grid spacing dx [m] on all axes and a PML of
 * `pml` cells inside the grid at every face (Sec. II-B, 10 in the paper).
 * Material parameters, staggered buoyancies (2 / (rho_a + rho_b)) and edge
 * shear moduli (harmonic mean of the 4 surrounding mu, 0 next to water) are
 * computed once in FP64 and stored in FP32; neighbours wrap at the last
 * index.  Requires cs <= cp / sqrt(2) (lambda >= 0), rho > 0, cp > 0,
 * 0 <= pml and 2 * pml + 2 < every axis length.  *out receives the model.
 * Allocates ~ (17 + 24 (2 pml + 1) / n) nx ny nz floats of device memory. */
int es_model_create(const float* rho, const float* cp, const float* cs, int nx, int ny, int nz,
                    double dx, int pml, es_model** out);

/* Arithmetic of the spatial derivatives (the fields are FP32 either way).
 * ES_PREC_FP32 (default): fused FFT passes where an axis has a plan (each
 * derivative as a 10-point near stencil in FP32 plus the FFT of the rest of
 * the operator, which confines FP32 FFT roundoff to about 1 % of its plain
 * size), FP32 circulant passes on the CUDA cores elsewhere.
 * ES_PREC_COMPENSATED: every axis through the circulant passes with
 * error-free transformations (each product split exactly by one FMA, Knuth's
 * TwoSum on the running sum, the kernel row as FP32 high plus low parts), so
 * each derivative is accurate to about twice FP32's precision and only the
 * FP32 storage of the fields limits the traces (O(n) work per element, about
 * 10 FP32 operations per multiply-add).  ES_PREC_FP32_TC: as ES_PREC_FP32, but
 * circulant axes of 192 to 512 cells run as GEMMs on the tensor cores (the
 * field and the kernel matrix split in three BF16 parts each, six products
 * accumulated in FP32; the near stencil stays on the CUDA cores).  The paper
 * has no tensor-core step: this mode is an opt-in speed-up for long odd axes
 * such as the paper's 301.  Applies from the next es_run.  ES_ERR_ARG for any
 * other mode. */
#define ES_PREC_FP32 0
#define ES_PREC_COMPENSATED 1
#define ES_PREC_FP32_TC 2
int es_model_set_precision(es_model* m, int mode);

/* Kelvin-Voigt viscosity (Eq. (1)-(2): the chi and eta terms, zero in the
 * paper's own runs), read as chi = tau lambda and eta = tau mu with one
 * relaxation time tau [s] >= 0, and the time derivative of the strain rate as
 * the backward difference of the velocity derivatives over one step:
 *   sigma^{n+1} = sigma^n + C D(dt v^{n+1/2} + tau (v^{n+1/2} - v^{n-1/2}))
 * (C the elastic stiffness of each term, split-field PML as usual).  tau = 0
 * is the elastic scheme.  For one Fourier mode the amplification z solves
 * z^2 + (q (1 + r) - 2) z + 1 - q r = 0, q = (c dt |kappa|)^2, r = tau / dt:
 * es_run returns ES_ERR_UNSTABLE unless q_max (1 + 2 tau / dt) <= 4.  The
 * first viscous run allocates 6 floats per cell and simulation and starts
 * from v^{n-1/2} = the current velocity; es_state_reset zeroes it and
 * es_state_set sets it to the given velocity.  Adds one kernel per step
 * (after the velocity half, before the stress passes). */
int es_model_set_viscosity(es_model* m, double tau);

/* Anisotropic spacing [m] (the paper's grid is 12.5 / 12.5 / 10 m, Sec. II-B). */
int es_model_set_spacing(es_model* m, double dx, double dy, double dz);

/* PML strength: alpha(xi) = alpha0 (cref / d) xi^4, factor exp(-alpha dt / 2)
 * before and after each split increment.  Defaults alpha0 = 2, cref = max cp
 * (cref <= 0 selects max cp). */
int es_model_set_pml(es_model* m, double alpha0, double cref);

/* Stream for all work of this model: a cudaStream_t passed as void*
 * (e.g. torch.cuda.current_stream().cuda_stream).  NULL = legacy default. */
int es_model_set_stream(es_model* m, void* stream);

/* Default time step from the CFL rule (Sec. II-B, Eq. (5), CFL 0.3):
 * dt = 0.3 min(dx, dy, dz) / max cp. */
int es_model_default_dt(const es_model* m, double* dt);

/* Replaces all sources by one moment-tensor point source (Sec. II-A point
 * sources; Sec. V, Eq. (6)-(7) mechanisms, read as a symmetric tensor).
 * pos = (ix, iy, iz) grid cell, each in [pml, n - 2 - pml] (outside the PML).
 * mt = (Mxx, Myy, Mzz, Mxy, Mxz, Myz) [Pa]; after the stress half of step n
 * every stress component at the source index gains M_ij * wavelet[n]
 * (wavelet[n] = 0 for n >= nw).  wavelet: nw floats, host or device. */
int es_source_set(es_model* m, const int pos[3], const double mt[6], const float* wavelet, int nw);

/* Adds a further moment-tensor source (same meaning as es_source_set). */
int es_source_add(es_model* m, const int pos[3], const double mt[6], const float* wavelet, int nw);

/* Adds a moment-tensor source smoothed in the spatial-frequency domain with a
 * Blackman window, as the paper does to keep a grid-point delta from ringing
 * in the pseudo-spectral derivatives (Sec. II-A).  Reading: the window is the
 * product over the axes of W(m) = 0.42 + 0.5 cos(2 pi m / n) + 0.08 cos(4 pi m / n)
 * on each axis's signed wavenumber bins m (1 at m = 0, 0 at Nyquist); its
 * inverse transform is exactly the stencil (0.04, 0.25, 0.42, 0.25, 0.04) per
 * axis, so after the stress half of step n the stress at cell pos + (i, j, k),
 * |i|, |j|, |k| <= 2, gains M * wavelet[n] * s_i s_j s_k (weights sum to 1).
 * The paper's initial-value source is nw = 1, wavelet = {1}: the smoothed
 * stress distribution appears at the first step.  pos +- 2 must lie outside
 * the PML (each axis at least 5 long), else ES_ERR_ARG. */
int es_source_add_smoothed(es_model* m, const int pos[3], const double mt[6], const float* wavelet, int nw);

/* Adds a point force f = (fx, fy, fz) [N]: after the velocity half of step n,
 * v_i at the source index gains dt f_i wavelet[n] / (rho_i dx dy dz), rho_i
 * the density at v_i's staggered point. */
int es_source_add_force(es_model* m, const int pos[3], const double f[3], const float* wavelet,
                        int nw);

/* Removes every source. */
int es_source_clear(es_model* m);

/* Batched runs of independent sources on one model (the paper runs thousands
 * of single-source simulations on the same velocity model, Sec. III-A):
 * the model then holds nb simulations that share its material arrays, each
 * driven by one moment-tensor point source -- simulation b by pos[3b..3b+2],
 * mt[6b..6b+5] (as in es_source_set) and wavelet
 * wavelets[b nw .. b nw + nw - 1].  Replaces every source, resets the state
 * and, when nb changes, reallocates the fields (9 nb nx ny nz floats plus
 * slabs).  es_run then advances all nb simulations in the same kernel
 * launches and writes traces as [nb][4][n_rcv][nt]; es_state_get/set use
 * [nb][9][nz][ny][nx].  Arrays host or device.  nb = 1 is the plain model. */
int es_batch_set(es_model* m, int nb, const int* pos, const double* mt, const float* wavelets, int nw);

/* Sets every field to zero (the state before the first step). */
int es_state_reset(es_model* m);

/* Field state as 9 [nz][ny][nx] FP32 arrays in the order vx vy vz sxx syy
 * szz sxy sxz syz (velocity at t - dt/2, stress at t).  es_state_set puts
 * each value on the field's x split (y split for syz) inside the PML. */
int es_state_get(es_model* m, float* fields);
int es_state_set(es_model* m, const float* fields);

/* Runs nt time steps of the leapfrog scheme (Sec. II-A) from the model's
 * current state and records 4C traces (Sec. II-A, Eq. (3)):
 *   traces[0][r][n] = p = -(sxx + syy + szz) / 3 at t_{n+1}
 *   traces[1..3][r][n] = vx, vy, vz at t_{n+1/2}
 * at receiver r = (ix, iy, iz) of rcv [n_rcv][3] (each component at its own
 * staggered point, no interpolation).  dt <= 0 selects es_model_default_dt.
 * Returns ES_ERR_UNSTABLE if c_max dt sqrt(1/dx^2 + 1/dy^2 + 1/dz^2) > 2/pi
 * or if a field became non-finite.  traces: [4][n_rcv][nt] floats, host or
 * device; n_rcv may be 0 (traces then unused).  The state carries over to
 * the next call (call es_state_reset for a fresh run). */
int es_run(es_model* m, int nt, double dt, const int* rcv, int n_rcv, float* traces);

/* Runs nt steps of nmod models together, as es_run does for each (models[i]
 * with dts[i], receivers rcvs[i] [n_rcvs[i]][3], traces traces[i]), but
 * captured into one CUDA graph with one branch per model, so models of
 * different grid sizes (batched or not) share the GPU concurrently.  The
 * work is queued on models[0]'s stream.  Models must be distinct.
 * Per-kernel timings (es_last_step_kernel_ms) are not recorded. */
int es_run_group(int nmod, es_model* const* models, int nt, const double* dts, const int* const* rcvs,
                 const int* n_rcvs, float* const* traces);

/* Superposition of single-event traces (Sec. IV): for every event e,
 * k_e = floor(t0s[e] / dt + 1/2) (computed in FP64) and
 *   gather[c][r][t] = sum_e amps[e] * traces[src_of_event[e]][c][r][t - k_e],
 * terms with t - k_e outside [0, nt) being zero (zero padding; negative t0
 * cuts the front).  traces: [n_src][4][n_rcv][nt]; gather: [4][n_rcv][n_out].
 * All arrays host or device; stream as in es_model_set_stream.  FP32 sums in
 * event order. */
int es_superpose(const float* traces, int n_src, int n_rcv, int nt, const int* src_of_event,
                 const float* amps, const float* t0s, int n_events, double dt, int n_out,
                 float* gather, void* stream);

/* The same superposition as es_superpose, for callers that cannot allocate
 * device memory: a caller whose device memory is owned by its own pool
 * allocator (which may leave no headroom, and whose budget a library
 * cudaMalloc would break), or a caller streaming work where the implicit
 * device synchronisation of cudaMalloc / cudaFree would stall its other
 * streams.  This entry point calls no cudaMalloc, cudaFree or other
 * allocating routine.  The paper has no counterpart; it is a service of this
 * library.
 * - traces, src_of_event, amps, t0s and gather must all be device pointers
 *   (ES_ERR_ARG otherwise); layouts and results are those of es_superpose,
 *   and the output matches it exactly.
 * - Scratch: a fixed device array of ES_NOALLOC_MAX_EVENTS + 64 ints
 *   (~256 KB), allocated when the library is loaded and held by every GPU
 *   that loads it until the process exits.  n_events > ES_NOALLOC_MAX_EVENTS
 *   is ES_ERR_ARG.
 * - The first call on a device (in each of its contexts: again after a
 *   cudaDeviceReset) looks up that array's device address; make the first
 *   call on each device before any stream capture.
 * - Every call shares the array (each call clears what it needs): calls that
 *   overlap on the GPU (other streams, other host threads) race; order them.
 * - The call waits for an argument check on the device before launching, so
 *   it returns after queueing the superposition (stream-ordered output); on
 *   ES_ERR_ARG (bad source index, non-finite amplitude or time) nothing is
 *   written to gather. */
#define ES_NOALLOC_MAX_EVENTS 65536
int es_superpose_noalloc(const float* traces, int n_src, int n_rcv, int nt, const int* src_of_event,
                         const float* amps, const float* t0s, int n_events, double dt, int n_out,
                         float* gather, void* stream);

/* Seabed receiver grid (Sec. II-B, Fig. 2): rx * ry receivers over the
 * non-PML interior, ix_i = pml + ((2i+1)(nx - 2 pml)) / (2 rx) (integer
 * division), likewise in y; iz = the last cell of the top run of cs == 0 in
 * that column.  rcv: [rx*ry][3] ints, host memory, r = i + rx * j.
 * ES_ERR_ARG if a chosen column has cs != 0 at the surface. */
int es_seabed_receivers(const es_model* m, int rx, int ry, int* rcv);

/* One staggered spectral derivative (Sec. II-A): out = D_axis^(shift) f,
 * D(+/-) f (x) = f'(x +/- d/2), i.e. forward FFT along the axis, multiply by
 * i kappa exp(+/- i kappa d / 2), inverse FFT, with kappa_m = 2 pi m / (n d),
 * m = -n/2 .. n/2 - 1.  The same fused FFT pass kernels as es_run.  f, out:
 * [nz][ny][nx] device pointers (distinct), each on a 16-byte boundary (the
 * passes move 8- and 16-byte vectors; ES_ERR_ARG otherwise); shift = +1 or
 * -1. */
int es_derivative(const float* f, int nx, int ny, int nz, int axis, double d, int shift, float* out,
                  void* stream);

/* Laplacian of a field (Sec. VI-A, Eq. (8): the paper thresholds the Laplacian
 * of the density to pick event locations on rock interfaces):
 * out = sum over the axes of D(+) D(-) f, which multiplies every wavenumber
 * bin by -kappa^2 (Nyquist included): the spectral Laplacian, with the
 * solver's own derivative passes.  f, out: [nz][ny][nx] device arrays
 * (distinct, each on a 16-byte boundary, else ES_ERR_ARG), spacings dx, dy,
 * dz > 0.  Allocates about 2 n floats of scratch. */
int es_laplacian(const float* f, int nx, int ny, int nz, double dx, double dy, double dz, float* out,
                 void* stream);

/* FFT plan autotuner: for each axis length of this model with more than one
 * plan (radix order R1 x R2, or three stages R1 x R2 x R3; a plan is named
 * (R1, n / R1)), times the model's own velocity and stress passes (reps
 * launches after one warm-up, CUDA events on the model's stream) with every
 * candidate, keeps the fastest per pass kind (x pass, y/z
 * passes) and length for the rest of the process, and records the choice
 * in the plan cache ($ES_TUNE_CACHE, else $HOME/.cache/es_fft_plans.txt,
 * keyed by device name), which every process loads when it creates its first
 * model.  Resets the model's state.  report (optional): the timings, one line
 * per candidate. */
int es_model_autotune(es_model* m, int reps, char* report, int report_len);

/* The plan in use for pass kind 0 (x) or 1 (y/z) and axis length n, as
 * ra = R1 (the first stage's radix) and rb = n / R1: (5, 25) for 125 is the
 * three-stage 5 x 5 x 5, (3, 25) for 75 the three-stage 3 x 5 x 5.  Host-side
 * only; ES_ERR_SIZE if n has no plan. */
int es_fft_plan(int pass_kind, int n, int* ra, int* rb);

/* Pins the plan (ra, rb) (one of the candidates for n, named as above) for
 * pass kind 0 (x) or 1 (y/z) in this process.  ES_ERR_SIZE if it is not a
 * candidate. */
int es_fft_plan_select(int pass_kind, int n, int ra, int rb);

/* Device time [ms] of each kernel of the last time step of the last es_run
 * (CUDA events around each kernel launch of that step), in launch order:
 * vel-x, vel-y, vel-z, [force inject], [viscous combine], str-x, str-y,
 * str-z, inject, record (bracketed ones only when present).  n = capacity;
 * returns the number written (>= 0) or a negative status. */
int es_last_step_kernel_ms(es_model* m, float* ms, int n);

/* Number of kernel launches one time step makes (for launch accounting). */
int es_kernels_per_step(const es_model* m);

void es_model_destroy(es_model* m);

/* Static description of a status code. */
const char* es_status_string(int status);

/* Text of the last CUDA error seen by this thread ("" if none). */
const char* es_last_error(void);

/* Debug aids for the error paths (no counterpart in the paper).
 * es_fault_inject_alloc(n): the n-th device allocation the solver makes from
 * now on fails as if the device were out of memory, before cudaMalloc is
 * called; the call that needed it returns ES_ERR_OOM and releases what it had
 * taken.  n <= 0 disables.  The environment variable ES_FAULT_ALLOC=n does
 * the same from the first allocation of the process.  Host-side only: no
 * kernel is affected.
 * es_debug_live_allocations: the number of device allocations the solver
 * currently holds (models, their run buffers, scratch of running calls). */
void es_fault_inject_alloc(int n);
long long es_debug_live_allocations(void);

/* Bounds-checked debug build (libes_bounds.so, compiled with -DES_BOUNDS=1):
 * the derivative passes check each global index of their loads, stores and
 * reductions against its array's extent, skip an access out of range and
 * record the first one.  es_debug_bounds reads and clears that record:
 * *first_bad = 0 if every index was in range, else (source line << 40) |
 * (the index's low 40 bits).  ES_ERR_STATE in the release build (which checks
 * nothing), ES_ERR_ARG for a null pointer, ES_ERR_CUDA if the device word
 * cannot be read. */
int es_debug_bounds(long long* first_bad);

#ifdef __cplusplus
}
#endif
#endif /* ES_H */
