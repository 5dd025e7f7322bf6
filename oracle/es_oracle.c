/*
 * es_oracle.c -- plain, slow, FP64 CPU oracle for the staggered-grid Fourier
 * pseudo-spectral (PSTD) elastic solver of Das, Chen & Hobson, "Fast GPU-Based
 * Seismogram Simulation from Microseismic Events in Marine Environments Using
 * Heterogeneous Velocity Models" (arXiv 1705.04874).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package smoke check and
 * the benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA path, and the CUDA path never calls
 * it.  Everything is written for a reader checking it against the paper:
 * no blocking, fusion or reordering beyond what each definition states.
 *
 * Passages followed (paper section / equation):
 *   Sec. II-A, Eq. (2)  velocity-stress elastic system, lossless (chi = eta = 0)
 *   Sec. II-A, Eq. (3)  pressure p = -(sxx + syy + szz) / 3
 *   Sec. II-A, Eq. (4)  mu = cs^2 rho, lambda + 2 mu = cp^2 rho
 *   Sec. II-A           Fourier-domain pseudo-spectral spatial derivatives and a
 *                       leapfrog time march on a spatially and temporally
 *                       staggered grid
 *   Sec. II-B, Eq. (5)  CFL = c_max dt / dx
 *   Sec. II-B           absorbing PML of L grid points at every face
 *   Sec. II-A           point sources at grid points; Sec. V Eq. (6)-(7)
 *                       source stress tensors
 *   Sec. II-B           4C receivers at the seabed, where cs first becomes 0
 *   Sec. IV             superposition of single-event traces with amplitude
 *                       scaling and origin-time shift, zero padded
 *
 * Readings of points the paper leaves open (each is listed again where used):
 *   R-stagger  sxx,syy,szz at (i,j,k); vx at (i+1/2,j,k); vy at (i,j+1/2,k);
 *              vz at (i,j,k+1/2); sxy at (i+1/2,j+1/2,k); sxz at
 *              (i+1/2,j,k+1/2); syz at (i,j+1/2,k+1/2).  v lives at half
 *              time steps, stress at whole steps.
 *   R-kappa    wavenumbers kappa_m = 2 pi m / (N d), m = 0..ceil(N/2)-1, then
 *              negative; for even N the Nyquist bin takes m = -N/2.
 *   R-shift    staggered derivative D(+/-) f(x) = f'(x +/- d/2), i.e. the
 *              spectral multiplier i kappa exp(+/- i kappa d / 2).
 *   R-fft      forward DFT unscaled, inverse scaled by 1/N.
 *   R-avg      buoyancy at a staggered point = 2 / (rho_a + rho_b) of its two
 *              neighbours; edge shear modulus = harmonic mean of the four
 *              surrounding mu, 0 when any of them is 0 (water).  Neighbours
 *              wrap periodically at the last index.
 *   R-pml      split-field PML, L cells at each face.  alpha(xi) =
 *              alpha0 * (c_ref / d) * xi^4, xi in (0,1] the depth into the
 *              layer (outermost cell xi = 1), staggered points at i + 1/2,
 *              clamped to 1; factor P = exp(-alpha dt / 2) applied before and
 *              after each split increment: s <- P (P s + dt c D).
 *   R-src      moment source: after the stress half of step n, each stress
 *              component at the source index gains M_ij w[n] (on its x split):
 *              the stress-glut form of a moment tensor whose moment rate is
 *              -(V / dt) M w(t - dt / 2), V = dx dy dz, in Aki & Richards'
 *              sign convention (pinned against the analytic moment-tensor
 *              solution in tests/test_oracle_moment.py).
 *              Force source: after the velocity half of step n, v_i at the
 *              source index gains dt f_i w[n] / (rho_stag dx dy dz).
 *   R-rec      sample n of a trace holds p(t_{n+1}) and v(t_{n+1/2}) at the
 *              receiver's index (each component at its own staggered point).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PI 3.14159265358979323846264338327950288

/* ------------------------------------------------------------------------ */
/* 1. Discrete Fourier transforms (the oracle's own; Sec. II-A names FFT/IFFT) */
/* ------------------------------------------------------------------------ */

/* Root table w[j] = exp(-2 pi i j / n), j in [0, n).  The angle index is
 * reduced exactly in integers before the library cos/sin call. */
static void root_table(int n, double complex *w)
{
    for (int j = 0; j < n; ++j) {
        double a = -2.0 * PI * (double)j / (double)n;
        w[j] = cos(a) + I * sin(a);
    }
}

static int smallest_factor(int n)
{
    for (int p = 2; p * p <= n; ++p)
        if (n % p == 0) return p;
    return n;
}

/* Recursive mixed-radix Cooley-Tukey (decimation in time, any prime factor).
 * Computes y[k] = sum_j x[j*stride] * W^(j k) for the length-n sequence, with
 * W = w_top[wstep] (w_top is the root table of the top-level length, so
 * n * wstep = top length).  tmp holds >= n scratch values. */
static void fft_rec(const double complex *x, int stride, double complex *y, int n,
                    const double complex *w_top, int wstep, double complex *tmp)
{
    if (n == 1) { y[0] = x[0]; return; }
    int p = smallest_factor(n), m = n / p;
    /* p interleaved sub-sequences x[q + p j], each transformed to length m */
    for (int q = 0; q < p; ++q)
        fft_rec(x + (size_t)q * stride, stride * p, y + (size_t)q * m, m, w_top, wstep * p, tmp);
    /* X[k + m s] = sum_q W_n^(q (k + m s)) Y_q[k] */
    for (int k = 0; k < m; ++k)
        for (int s = 0; s < p; ++s) {
            const int step = k + m * s; /* < n */
            double complex acc = y[k];  /* q = 0: W^0 = 1 */
            int e = 0;                  /* e = q * step mod n */
            for (int q = 1; q < p; ++q) {
                e += step;
                if (e >= n) e -= n;
                acc += w_top[(size_t)e * wstep] * y[(size_t)q * m + k];
            }
            tmp[step] = acc;
        }
    memcpy(y, tmp, sizeof(double complex) * (size_t)n);
}

/* Forward (sign = -1) or inverse (sign = +1, scaled by 1/n) DFT of x into y. */
static void fft_1d(const double complex *x, double complex *y, int n, int sign,
                   const double complex *wf, double complex *tmp)
{
    if (sign < 0) {
        fft_rec(x, 1, y, n, wf, 1, tmp);
    } else {
        /* inverse through conjugation: x = conj(DFT(conj(X))) / n */
        double complex *c = tmp + n;
        for (int j = 0; j < n; ++j) c[j] = conj(x[j]);
        fft_rec(c, 1, y, n, wf, 1, tmp);
        for (int j = 0; j < n; ++j) y[j] = conj(y[j]) / (double)n;
    }
}

/* The DFT by its definition, O(n^2): y[k] = sum_j x[j] exp(sign 2 pi i j k / n). */
static void dft_naive(const double complex *x, double complex *y, int n, int sign)
{
    for (int k = 0; k < n; ++k) {
        double complex acc = 0.0;
        for (int j = 0; j < n; ++j) {
            long e = ((long)j * (long)k) % n;
            double a = (double)sign * 2.0 * PI * (double)e / (double)n;
            acc += x[j] * (cos(a) + I * sin(a));
        }
        y[k] = (sign > 0) ? acc / (double)n : acc;
    }
}

/* Exported: 1D transform for the oracle's own tests.  mode 0 = FFT, 1 = naive. */
int orc_fft(int n, const double *re_in, const double *im_in, double *re_out,
            double *im_out, int inverse, int naive)
{
    if (n < 1) return -1;
    double complex *x = malloc(sizeof(double complex) * (size_t)n);
    double complex *y = malloc(sizeof(double complex) * (size_t)n);
    double complex *w = malloc(sizeof(double complex) * (size_t)n);
    double complex *t = malloc(sizeof(double complex) * (size_t)(2 * n));
    for (int j = 0; j < n; ++j) x[j] = re_in[j] + I * (im_in ? im_in[j] : 0.0);
    int sign = inverse ? +1 : -1;
    if (naive) dft_naive(x, y, n, sign);
    else { root_table(n, w); fft_1d(x, y, n, sign, w, t); }
    for (int j = 0; j < n; ++j) { re_out[j] = creal(y[j]); im_out[j] = cimag(y[j]); }
    free(x); free(y); free(w); free(t);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* 2. Staggered spectral derivative along one axis (Sec. II-A; R-kappa,      */
/*    R-shift, R-fft)                                                         */
/* ------------------------------------------------------------------------ */

/* Spectral multiplier for bin k of an n-point axis with spacing d:
 * i kappa exp(i shift kappa d / 2), shift = +1 or -1 (0: plain derivative). */
static double complex multiplier(int k, int n, double d, int shift)
{
    int m = (k <= (n - 1) / 2) ? k : k - n; /* even n: k = n/2 -> m = -n/2 */
    double kappa = 2.0 * PI * (double)m / ((double)n * d);
    double ph = (double)shift * kappa * d * 0.5;
    return I * kappa * (cos(ph) + I * sin(ph));
}

typedef struct { int n, stride, nlines; } axis_geom;

static axis_geom geom(int nx, int ny, int nz, int axis)
{
    axis_geom g;
    if (axis == 0) { g.n = nx; g.stride = 1; g.nlines = ny * nz; }
    else if (axis == 1) { g.n = ny; g.stride = nx; g.nlines = nx * nz; }
    else { g.n = nz; g.stride = nx * ny; g.nlines = nx * ny; }
    return g;
}

/* first element of line l along the axis */
static size_t line_base(int nx, int ny, int axis, int l)
{
    if (axis == 0) return (size_t)nx * (size_t)l;                  /* l = j + ny k */
    if (axis == 1) return (size_t)(l % nx) + (size_t)nx * ny * (l / nx); /* l = i + nx k */
    return (size_t)l;                                              /* l = i + nx j */
}

/* out = D(shift)_axis f, line by line with 1D transforms.  mode 0: FFT,
 * mode 1: naive DFT.  Each line: forward transform, multiply, inverse
 * transform, real part. */
static void deriv_lines(const double *f, double *out, int nx, int ny, int nz, int axis,
                        double d, int shift, int mode, int nthreads)
{
    axis_geom g = geom(nx, ny, nz, axis);
    int n = g.n;
    double complex *H = malloc(sizeof(double complex) * (size_t)n);
    double complex *wf = malloc(sizeof(double complex) * (size_t)n);
    for (int k = 0; k < n; ++k) H[k] = multiplier(k, n, d, shift);
    root_table(n, wf);
    (void)nthreads;
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1)
    {
        double complex *a = malloc(sizeof(double complex) * (size_t)n);
        double complex *b = malloc(sizeof(double complex) * (size_t)n);
        double complex *t = malloc(sizeof(double complex) * (size_t)(2 * n));
#pragma omp for schedule(static)
        for (int l = 0; l < g.nlines; ++l) {
            size_t base = line_base(nx, ny, axis, l);
            for (int j = 0; j < n; ++j) a[j] = f[base + (size_t)j * g.stride];
            if (mode == 1) dft_naive(a, b, n, -1); else fft_1d(a, b, n, -1, wf, t);
            for (int k = 0; k < n; ++k) b[k] *= H[k];
            if (mode == 1) dft_naive(b, a, n, +1); else fft_1d(b, a, n, +1, wf, t);
            for (int j = 0; j < n; ++j) out[base + (size_t)j * g.stride] = creal(a[j]);
        }
        free(a); free(b); free(t);
    }
    free(H); free(wf);
}

/* out = D(shift)_axis f through the full 3D transform: 3D FFT, multiply by the
 * axis's multiplier (which depends only on that axis's index), 3D IFFT, real
 * part.  Identical to deriv_lines in exact arithmetic. */
static void deriv_3d(const double *f, double *out, int nx, int ny, int nz, int axis,
                     double d, int shift)
{
    size_t ncell = (size_t)nx * ny * nz;
    int dims[3] = {nx, ny, nz};
    double complex *c = malloc(sizeof(double complex) * ncell);
    for (size_t q = 0; q < ncell; ++q) c[q] = f[q];
    int maxn = nx > ny ? (nx > nz ? nx : nz) : (ny > nz ? ny : nz);
    double complex *a = malloc(sizeof(double complex) * (size_t)maxn);
    double complex *b = malloc(sizeof(double complex) * (size_t)maxn);
    double complex *t = malloc(sizeof(double complex) * (size_t)(2 * maxn));
    double complex *w = malloc(sizeof(double complex) * (size_t)maxn);
    for (int pass = 0; pass < 2; ++pass) {
        int sign = pass == 0 ? -1 : +1;
        for (int ax = 0; ax < 3; ++ax) {
            axis_geom g = geom(nx, ny, nz, ax);
            root_table(g.n, w);
            for (int l = 0; l < g.nlines; ++l) {
                size_t base = line_base(nx, ny, ax, l);
                for (int j = 0; j < g.n; ++j) a[j] = c[base + (size_t)j * g.stride];
                fft_1d(a, b, g.n, sign, w, t);
                for (int j = 0; j < g.n; ++j) c[base + (size_t)j * g.stride] = b[j];
            }
        }
        if (pass == 0) {
            for (size_t q = 0; q < ncell; ++q) {
                int i = (int)(q % nx), jj = (int)((q / nx) % ny), kk = (int)(q / ((size_t)nx * ny));
                int idx = axis == 0 ? i : (axis == 1 ? jj : kk);
                c[q] *= multiplier(idx, dims[axis], d, shift);
            }
        }
    }
    for (size_t q = 0; q < ncell; ++q) out[q] = creal(c[q]);
    free(c); free(a); free(b); free(t); free(w);
}

/* Exported: mode 0 = 1D FFT per line, 1 = naive DFT per line, 2 = 3D FFT. */
int orc_deriv(const double *f, int nx, int ny, int nz, int axis, double d, int shift,
              double *out, int mode, int nthreads)
{
    if (nx < 1 || ny < 1 || nz < 1 || axis < 0 || axis > 2 || !(d > 0)) return -1;
    if (mode == 2) deriv_3d(f, out, nx, ny, nz, axis, d, shift);
    else deriv_lines(f, out, nx, ny, nz, axis, d, shift, mode, nthreads);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* 3. Material parameters (Sec. II-A Eq. (4); R-avg)                         */
/* ------------------------------------------------------------------------ */

#define IDX(i, j, k) ((size_t)(i) + (size_t)nx * ((size_t)(j) + (size_t)ny * (size_t)(k)))

static double harmonic4(double a, double b, double c, double d)
{
    if (a == 0.0 || b == 0.0 || c == 0.0 || d == 0.0) return 0.0;
    return 4.0 / (1.0 / a + 1.0 / b + 1.0 / c + 1.0 / d);
}

/* lam, mu at cell centres; bx, by, bz buoyancy at the vx, vy, vz points;
 * muxy, muxz, muyz at the sxy, sxz, syz points. */
int orc_materials(const double *rho, const double *cp, const double *cs, int nx, int ny, int nz,
                  double *lam, double *mu, double *bx, double *by, double *bz,
                  double *muxy, double *muxz, double *muyz)
{
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t q = IDX(i, j, k);
                mu[q] = cs[q] * cs[q] * rho[q];                 /* Eq. (4) */
                lam[q] = cp[q] * cp[q] * rho[q] - 2.0 * mu[q];  /* Eq. (4) */
            }
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int i1 = (i + 1) % nx, j1 = (j + 1) % ny, k1 = (k + 1) % nz;
                size_t q = IDX(i, j, k);
                bx[q] = 2.0 / (rho[q] + rho[IDX(i1, j, k)]);
                by[q] = 2.0 / (rho[q] + rho[IDX(i, j1, k)]);
                bz[q] = 2.0 / (rho[q] + rho[IDX(i, j, k1)]);
                muxy[q] = harmonic4(mu[q], mu[IDX(i1, j, k)], mu[IDX(i, j1, k)], mu[IDX(i1, j1, k)]);
                muxz[q] = harmonic4(mu[q], mu[IDX(i1, j, k)], mu[IDX(i, j, k1)], mu[IDX(i1, j, k1)]);
                muyz[q] = harmonic4(mu[q], mu[IDX(i, j1, k)], mu[IDX(i, j, k1)], mu[IDX(i, j1, k1)]);
            }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* 4. PML profile (Sec. II-B; R-pml)                                          */
/* ------------------------------------------------------------------------ */

/* Depth into the PML (0 outside) of the point at position x (grid units). */
static double pml_depth(double x, int n, int L)
{
    if (L <= 0) return 0.0;
    double xi = 0.0;
    if (x < (double)L) xi = ((double)L - x) / (double)L;
    else if (x > (double)(n - 1 - L)) xi = (x - (double)(n - 1 - L)) / (double)L;
    return xi > 1.0 ? 1.0 : xi;
}

/* P[i] = exp(-alpha(xi) dt / 2) at the centred (stag = 0) or staggered
 * (stag = 1, position i + 1/2) points of an n-point axis. */
int orc_pml_profile(int n, int L, double alpha0, double cref, double d, double dt, int stag, double *P)
{
    for (int i = 0; i < n; ++i) {
        double xi = pml_depth((double)i + (stag ? 0.5 : 0.0), n, L);
        double alpha = alpha0 * (cref / d) * xi * xi * xi * xi;
        P[i] = exp(-alpha * dt * 0.5);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* 5. Time stepping (Sec. II-A Eq. (2)-(3); R-stagger, R-pml, R-src, R-rec)   */
/* ------------------------------------------------------------------------ */

enum { VX, VY, VZ, SXX, SYY, SZZ, SXY, SXZ, SYZ, NF };

/* Cell loops run in parallel over z planes; every cell is independent, so
 * the arithmetic is the same as a serial loop. */
#define OMP_PRAGMA(x) _Pragma(#x)
#define OMP_CELLS OMP_PRAGMA(omp parallel for schedule(static) num_threads(nthr))
#define OMP_TOTAL OMP_PRAGMA(omp parallel for schedule(static) num_threads(nthr))

typedef struct {
    int nx, ny, nz;
    double dx, dy, dz;
    int pml;          /* L cells per face, 0 = none */
    double pml_alpha0;
    double pml_cref;  /* <= 0: max cp of the model */
    double dt;
    int nt;
    int deriv_mode;   /* 0: 1D FFT, 1: naive DFT, 2: 3D FFT */
    int nthreads;
    double tau;       /* Kelvin-Voigt relaxation time (chi = tau lambda, eta = tau mu); 0 = elastic */
} orc_params;

typedef struct {
    int kind;          /* 0: moment tensor, 1: point force */
    int ix, iy, iz;
    double m[6];       /* kind 0: Mxx Myy Mzz Mxy Mxz Myz;  kind 1: fx fy fz */
    const double *w;   /* wavelet, sample n used at step n */
    int nw;
    const double *g;   /* kind 0 only: NULL = point source at (ix, iy, iz); else a
                          [nz][ny][nx] spatial distribution (the smoothed source of
                          Sec. II-A), every cell gaining M_ij w[n] g */
} orc_source;

/* whether field f sits at a half-index along axis a (R-stagger) */
static int stag_along(int f, int a)
{
    switch (f) {
    case VX: return a == 0;
    case VY: return a == 1;
    case VZ: return a == 2;
    case SXY: return a == 0 || a == 1;
    case SXZ: return a == 0 || a == 2;
    case SYZ: return a == 1 || a == 2;
    default: return 0;
    }
}

/* One term of Eq. (2) in split form: target field, the axis of the
 * derivative, the field differentiated, the shift of the staggered operator. */
typedef struct { int target, axis, source, shift; } term;

/* Velocity half: dv_i/dt = (1/rho) d sigma_ij / dx_j */
static const term VEL_TERMS[9] = {
    {VX, 0, SXX, +1}, {VX, 1, SXY, -1}, {VX, 2, SXZ, -1},
    {VY, 0, SXY, -1}, {VY, 1, SYY, +1}, {VY, 2, SYZ, -1},
    {VZ, 0, SXZ, -1}, {VZ, 1, SYZ, -1}, {VZ, 2, SZZ, +1},
};
/* Stress half: d sigma_ij/dt = lambda delta_ij dv_k/dx_k + mu (dv_i/dx_j + dv_j/dx_i) */
static const term STR_TERMS[9] = {
    {SXX, 0, VX, -1}, {SYY, 0, VX, -1}, {SZZ, 0, VX, -1},
    {SXX, 1, VY, -1}, {SYY, 1, VY, -1}, {SZZ, 1, VY, -1},
    {SXX, 2, VZ, -1}, {SYY, 2, VZ, -1}, {SZZ, 2, VZ, -1},
};
static const term SHEAR_TERMS[6] = {
    {SXY, 0, VY, +1}, {SXY, 1, VX, +1},
    {SXZ, 0, VZ, +1}, {SXZ, 2, VX, +1},
    {SYZ, 1, VZ, +1}, {SYZ, 2, VY, +1},
};

/* Discrete energy at step n (PML off): 1/2 sum rho_stag v^{n-1/2} . v^{n+1/2}
 * + 1/2 sum sigma^n : S : sigma^n, with S the compliance (inverse of the
 * stiffness the stress update uses). */
static double energy(int nx, int ny, int nz, double *const vold[3], double *const vnew[3],
                     double *const sig[6], const double *lam, const double *mu,
                     double *const b[3], double *const mue[3])
{
    size_t ncell = (size_t)nx * ny * nz;
    double e = 0.0;
    for (size_t q = 0; q < ncell; ++q) {
        for (int c = 0; c < 3; ++c) e += 0.5 * (1.0 / b[c][q]) * vold[c][q] * vnew[c][q];
        double sxx = sig[0][q], syy = sig[1][q], szz = sig[2][q];
        if (mu[q] > 0.0) {
            double tr = sxx + syy + szz;
            e += 0.5 * ((sxx * sxx + syy * syy + szz * szz) / (2.0 * mu[q])
                        - lam[q] / (2.0 * mu[q] * (3.0 * lam[q] + 2.0 * mu[q])) * tr * tr);
        } else {
            double s = (sxx + syy + szz) / 3.0; /* fluid: the three are equal */
            e += 0.5 * s * s / lam[q];
        }
        for (int c = 0; c < 3; ++c)
            if (mue[c][q] > 0.0) e += 0.5 * sig[3 + c][q] * sig[3 + c][q] / mue[c][q];
    }
    return e;
}

/* Runs p->nt steps.  traces: [4][n_rcv][nt] (p, vx, vy, vz), may be NULL.
 * state: optional [9][ncell] totals (vx vy vz sxx syy szz sxy sxz syz): read
 * as the initial state (v at t = -1/2, stress at t = 0, all put on the x
 * split, or the first split a field has) and overwritten with the final one.
 * energy_out: optional [nt], the discrete energy at each step. */
int orc_simulate(const orc_params *p, const double *rho, const double *cp, const double *cs,
                 const orc_source *src, int nsrc, const int *rcv, int n_rcv,
                 double *traces, double *state, double *energy_out)
{
    int nx = p->nx, ny = p->ny, nz = p->nz, nt = p->nt;
    if (nx < 1 || ny < 1 || nz < 1 || nt < 0 || !(p->dt > 0)) return -1;
    size_t ncell = (size_t)nx * ny * nz;
    double dxyz[3] = {p->dx, p->dy, p->dz};
    int dims[3] = {nx, ny, nz};
    double dt = p->dt;
    int nthr = p->nthreads > 0 ? p->nthreads : 1;

    double *lam = malloc(sizeof(double) * ncell), *mu = malloc(sizeof(double) * ncell);
    double *b[3], *mue[3];
    for (int c = 0; c < 3; ++c) { b[c] = malloc(sizeof(double) * ncell); mue[c] = malloc(sizeof(double) * ncell); }
    orc_materials(rho, cp, cs, nx, ny, nz, lam, mu, b[0], b[1], b[2], mue[0], mue[1], mue[2]);

    /* PML factors per axis at centred and staggered points */
    double cref = p->pml_cref;
    if (!(cref > 0)) { cref = 0.0; for (size_t q = 0; q < ncell; ++q) if (cp[q] > cref) cref = cp[q]; }
    double *Pc[3], *Ps[3];
    for (int a = 0; a < 3; ++a) {
        Pc[a] = malloc(sizeof(double) * (size_t)dims[a]);
        Ps[a] = malloc(sizeof(double) * (size_t)dims[a]);
        orc_pml_profile(dims[a], p->pml, p->pml_alpha0, cref, dxyz[a], dt, 0, Pc[a]);
        orc_pml_profile(dims[a], p->pml, p->pml_alpha0, cref, dxyz[a], dt, 1, Ps[a]);
    }

    /* split fields: split[f][a] is the part of field f driven by derivatives
     * along axis a; NULL where Eq. (2) has no such term (sxy: no z, sxz: no y,
     * syz: no x). */
    double *split[NF][3];
    for (int f = 0; f < NF; ++f)
        for (int a = 0; a < 3; ++a) {
            int has = !((f == SXY && a == 2) || (f == SXZ && a == 1) || (f == SYZ && a == 0));
            split[f][a] = has ? calloc(ncell, sizeof(double)) : NULL;
        }
    if (state)
        for (int f = 0; f < NF; ++f) {
            int a0 = split[f][0] ? 0 : 1;
            memcpy(split[f][a0], state + (size_t)f * ncell, sizeof(double) * ncell);
        }

    double *tot[NF], *D = malloc(sizeof(double) * ncell);
    for (int f = 0; f < NF; ++f) tot[f] = malloc(sizeof(double) * ncell);
    double *vold[3] = {NULL, NULL, NULL};
    const double tau = p->tau > 0 ? p->tau : 0.0;
    double *D2 = tau > 0 ? malloc(sizeof(double) * ncell) : NULL;
    if (energy_out || tau > 0) for (int c = 0; c < 3; ++c) vold[c] = malloc(sizeof(double) * ncell);

#define TOTAL(f) do { OMP_TOTAL for (size_t q = 0; q < ncell; ++q) { double s_ = 0.0; \
        for (int a_ = 0; a_ < 3; ++a_) if (split[f][a_]) s_ += split[f][a_][q]; tot[f][q] = s_; } } while (0)

    for (int n = 0; n < nt; ++n) {
        /* ---- velocity half: v^{n-1/2} -> v^{n+1/2} from sigma^n ---- */
        for (int f = SXX; f <= SYZ; ++f) TOTAL(f);
        /* v^{n-1/2}: the energy's old velocity and the viscous terms' backward difference */
        if (energy_out || tau > 0)
            for (int c = 0; c < 3; ++c) { TOTAL(VX + c); memcpy(vold[c], tot[VX + c], sizeof(double) * ncell); }
        for (int t = 0; t < 9; ++t) {
            const term *T = &VEL_TERMS[t];
            orc_deriv(tot[T->source], nx, ny, nz, T->axis, dxyz[T->axis], T->shift, D, p->deriv_mode, p->nthreads);
            double *s = split[T->target][T->axis];
            const double *coef = b[T->target - VX];
            const double *P = stag_along(T->target, T->axis) ? Ps[T->axis] : Pc[T->axis];
            OMP_CELLS for (int k = 0; k < nz; ++k) for (int j = 0; j < ny; ++j) for (int i = 0; i < nx; ++i) {
                size_t q = IDX(i, j, k);
                int ia = T->axis == 0 ? i : (T->axis == 1 ? j : k);
                s[q] = P[ia] * (P[ia] * s[q] + dt * coef[q] * D[q]);
            }
        }
        for (int e = 0; e < nsrc; ++e) {          /* R-src, point force */
            const orc_source *S = &src[e];
            if (S->kind != 1 || n >= S->nw) continue;
            size_t q = IDX(S->ix, S->iy, S->iz);
            for (int c = 0; c < 3; ++c)
                split[VX + c][0][q] += dt * S->m[c] * S->w[n] * b[c][q] / (p->dx * p->dy * p->dz);
        }
        if (energy_out) {
            for (int c = 0; c < 3; ++c) TOTAL(VX + c);
            double *vn[3] = {tot[VX], tot[VY], tot[VZ]};
            double *sg[6] = {tot[SXX], tot[SYY], tot[SZZ], tot[SXY], tot[SXZ], tot[SYZ]};
            energy_out[n] = energy(nx, ny, nz, vold, vn, sg, lam, mu, b, mue);
        }

        /* ---- stress half: sigma^n -> sigma^{n+1} from v^{n+1/2} ---- */
        for (int f = VX; f <= VZ; ++f) TOTAL(f);
        for (int a = 0; a < 3; ++a) {
            /* normal stresses: d sigma_ii^(a) = dt (lambda + 2 mu delta_ia) dv_a/dx_a
             * + (chi + 2 eta delta_ia) (dv_a/dx_a at n+1/2 minus at n-1/2), Eq. (2) with the
             * time derivative of the strain rate as a backward difference over one step */
            orc_deriv(tot[VX + a], nx, ny, nz, a, dxyz[a], -1, D, p->deriv_mode, p->nthreads);
            if (tau > 0) orc_deriv(vold[a], nx, ny, nz, a, dxyz[a], -1, D2, p->deriv_mode, p->nthreads);
            for (int t = 0; t < 9; ++t) {
                const term *T = &STR_TERMS[t];
                if (T->axis != a) continue;
                double *s = split[T->target][a];
                int diag = (T->target - SXX) == a;
                OMP_CELLS for (int k = 0; k < nz; ++k) for (int j = 0; j < ny; ++j) for (int i = 0; i < nx; ++i) {
                    size_t q = IDX(i, j, k);
                    int ia = a == 0 ? i : (a == 1 ? j : k);
                    double c = lam[q] + (diag ? 2.0 * mu[q] : 0.0);
                    double inc = dt * c * D[q];
                    if (tau > 0) inc += tau * c * (D[q] - D2[q]);
                    s[q] = Pc[a][ia] * (Pc[a][ia] * s[q] + inc);
                }
            }
        }
        for (int t = 0; t < 6; ++t) {
            const term *T = &SHEAR_TERMS[t];
            orc_deriv(tot[T->source], nx, ny, nz, T->axis, dxyz[T->axis], T->shift, D, p->deriv_mode, p->nthreads);
            if (tau > 0)
                orc_deriv(vold[T->source - VX], nx, ny, nz, T->axis, dxyz[T->axis], T->shift, D2, p->deriv_mode,
                          p->nthreads);
            double *s = split[T->target][T->axis];
            const double *coef = mue[T->target - SXY];
            OMP_CELLS for (int k = 0; k < nz; ++k) for (int j = 0; j < ny; ++j) for (int i = 0; i < nx; ++i) {
                size_t q = IDX(i, j, k);
                int ia = T->axis == 0 ? i : (T->axis == 1 ? j : k);
                double inc = dt * coef[q] * D[q];
                if (tau > 0) inc += tau * coef[q] * (D[q] - D2[q]);
                s[q] = Ps[T->axis][ia] * (Ps[T->axis][ia] * s[q] + inc);
            }
        }
        for (int e = 0; e < nsrc; ++e) {          /* R-src, moment tensor */
            const orc_source *S = &src[e];
            if (S->kind != 0 || n >= S->nw) continue;
            if (S->g) {
                for (int c = 0; c < 6; ++c) {
                    int f = SXX + c;
                    int a0 = split[f][0] ? 0 : 1;
                    for (size_t q = 0; q < (size_t)nx * ny * nz; ++q) split[f][a0][q] += S->m[c] * S->w[n] * S->g[q];
                }
                continue;
            }
            size_t q = IDX(S->ix, S->iy, S->iz);
            for (int c = 0; c < 6; ++c) {
                int f = SXX + c;
                int a0 = split[f][0] ? 0 : 1;
                split[f][a0][q] += S->m[c] * S->w[n];
            }
        }

        /* ---- record sample n (R-rec; Eq. (3)) ---- */
        if (traces && n_rcv > 0) {
            for (int f = 0; f < NF; ++f) TOTAL(f);
            for (int r = 0; r < n_rcv; ++r) {
                size_t q = IDX(rcv[3 * r], rcv[3 * r + 1], rcv[3 * r + 2]);
                traces[((size_t)0 * n_rcv + r) * nt + n] = -(tot[SXX][q] + tot[SYY][q] + tot[SZZ][q]) / 3.0;
                traces[((size_t)1 * n_rcv + r) * nt + n] = tot[VX][q];
                traces[((size_t)2 * n_rcv + r) * nt + n] = tot[VY][q];
                traces[((size_t)3 * n_rcv + r) * nt + n] = tot[VZ][q];
            }
        }
    }
    if (state) {
        for (int f = 0; f < NF; ++f) { TOTAL(f); memcpy(state + (size_t)f * ncell, tot[f], sizeof(double) * ncell); }
    }
#undef TOTAL
    for (int f = 0; f < NF; ++f) { free(tot[f]); for (int a = 0; a < 3; ++a) free(split[f][a]); }
    for (int c = 0; c < 3; ++c) { free(b[c]); free(mue[c]); free(vold[c]); }
    for (int a = 0; a < 3; ++a) { free(Pc[a]); free(Ps[a]); }
    free(lam); free(mu); free(D); free(D2);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* 6. Seabed receivers (Sec. II-B: sensors where cs first becomes zero)       */
/* ------------------------------------------------------------------------ */

/* Receiver depth of column (ix, iy): the last index of the top run of cs == 0
 * cells (the deepest water cell; z = 0 at the sea surface).  The rx * ry grid
 * spans the non-PML interior: ix_i = L + ((2i+1)(nx-2L)) / (2 rx) in integer
 * division, likewise in y.  Returns -2 if a chosen column has no water at
 * z = 0. */
int orc_seabed_receivers(const double *cs, int nx, int ny, int nz, int L, int rx, int ry, int *rcv)
{
    if (rx < 1 || ry < 1 || nx - 2 * L < 1 || ny - 2 * L < 1) return -1;
    for (int jy = 0; jy < ry; ++jy)
        for (int jx = 0; jx < rx; ++jx) {
            int ix = L + ((2 * jx + 1) * (nx - 2 * L)) / (2 * rx);
            int iy = L + ((2 * jy + 1) * (ny - 2 * L)) / (2 * ry);
            if (cs[IDX(ix, iy, 0)] != 0.0) return -2;
            int iz = 0;
            while (iz + 1 < nz && cs[IDX(ix, iy, iz + 1)] == 0.0) ++iz;
            int r = jx + rx * jy;
            rcv[3 * r] = ix; rcv[3 * r + 1] = iy; rcv[3 * r + 2] = iz;
        }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* 7. Superposition (Sec. IV, Cases 1-3)                                      */
/* ------------------------------------------------------------------------ */

/* gather[c][r][t] = sum_e amps[e] * traces[src_of_event[e]][c][r][t - k_e],
 * k_e = floor(t0s[e] / dt + 0.5), terms with t - k_e outside [0, nt) are 0. */
int orc_superpose(const double *traces, int n_src, int n_rcv, int nt, const int *src_of_event,
                  const double *amps, const double *t0s, int n_events, double dt, int n_out,
                  double *gather)
{
    size_t plane = (size_t)4 * n_rcv;
    memset(gather, 0, sizeof(double) * plane * (size_t)n_out);
    for (int e = 0; e < n_events; ++e) {
        int s = src_of_event[e];
        if (s < 0 || s >= n_src) return -1;
        long ke = (long)floor(t0s[e] / dt + 0.5);
        for (size_t cr = 0; cr < plane; ++cr)
            for (int t = 0; t < n_out; ++t) {
                long u = (long)t - ke;
                if (u < 0 || u >= nt) continue;
                gather[cr * n_out + t] += amps[e] * traces[((size_t)s * plane + cr) * nt + (size_t)u];
            }
    }
    return 0;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
