"""Seeded synthetic inputs: velocity models, wavelets, source mechanisms,
receiver/event draws.

This module holds input generation only, none of the solver's arithmetic, so
both the CUDA path and the FP64 oracle can be fed from it.  Random numbers
come from splitmix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), written out here so that every draw is
reproducible on any machine.

The models stand in for the paper's two Marmousi2-derived marine models
(Sec. II-B, Fig. 1), which are not available: a water column over layered
sediments with lateral heterogeneity, rho / cp / cs per grid point, dx ~ 10 m.
"""
from __future__ import annotations

import math

import numpy as np

_MASK = (1 << 64) - 1


class SplitMix64:
    """splitmix64: state += golden gamma; output = mix(state)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self, n: int) -> np.ndarray:
        out = np.empty(n, dtype=np.uint64)
        s = self.state
        for i in range(n):
            s = (s + 0x9E3779B97F4A7C15) & _MASK
            z = s
            z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
            z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
            out[i] = z ^ (z >> 31)
        self.state = s
        return out

    def next_u64_fast(self, n: int) -> np.ndarray:
        """Same stream as next_u64, vectorised (for large draws)."""
        with np.errstate(over="ignore"):
            k = np.arange(1, n + 1, dtype=np.uint64)
            s = np.uint64(self.state) + k * np.uint64(0x9E3779B97F4A7C15)
            z = s
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            z = z ^ (z >> np.uint64(31))
        self.state = int(s[-1]) if n else self.state
        return z

    def uniform(self, n: int) -> np.ndarray:
        """Doubles in [0, 1) from the top 53 bits."""
        u = self.next_u64_fast(n)
        return (u >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def normal(self, n: int) -> np.ndarray:
        """Standard normals by Box-Muller."""
        m = (n + 1) // 2
        u = self.uniform(2 * m)
        u1 = 1.0 - u[:m]  # (0, 1]
        u2 = u[m:]
        r = np.sqrt(-2.0 * np.log(u1))
        z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])
        return z[:n]


# --------------------------------------------------------------------------
# velocity models ([nz][ny][nx], x fastest, z = 0 at the sea surface)
# --------------------------------------------------------------------------

def two_layer_model(n=32, water_cells=8, water=(1000.0, 1500.0, 0.0),
                    rock=(2200.0, 2500.0, 1200.0), shape=None):
    """Water over a homogeneous solid: (rho, cp, cs) float32 arrays."""
    nz, ny, nx = shape if shape is not None else (n, n, n)
    rho = np.empty((nz, ny, nx), np.float32)
    cp = np.empty_like(rho)
    cs = np.empty_like(rho)
    for arr, w, r in ((rho, water[0], rock[0]), (cp, water[1], rock[1]), (cs, water[2], rock[2])):
        arr[:water_cells] = w
        arr[water_cells:] = r
    return rho, cp, cs


def homogeneous_model(shape, rho=2200.0, cp=2500.0, cs=1200.0):
    nz, ny, nx = shape
    return (np.full((nz, ny, nx), rho, np.float32), np.full((nz, ny, nx), cp, np.float32),
            np.full((nz, ny, nx), cs, np.float32))


def gaussian_random_field(shape, corr_len, rng: SplitMix64):
    """Unit-variance field with covariance exp(-r^2 / l^2): white noise
    convolved (periodically) with exp(-2 r^2 / l^2), then renormalised."""
    nz, ny, nx = shape
    noise = rng.normal(nx * ny * nz).reshape(shape)
    spec = np.fft.rfftn(noise)
    kz = np.fft.fftfreq(nz)[:, None, None]
    ky = np.fft.fftfreq(ny)[None, :, None]
    kx = np.fft.rfftfreq(nx)[None, None, :]
    # Fourier transform of exp(-2 r^2 / l^2) is proportional to exp(-pi^2 l^2 k^2 / 2)
    filt = np.exp(-(np.pi ** 2) * corr_len ** 2 * (kx ** 2 + ky ** 2 + kz ** 2) / 2.0)
    g = np.fft.irfftn(spec * filt, s=shape, axes=(0, 1, 2))
    g -= g.mean()
    sd = g.std()
    return g / sd if sd > 0 else g


def marine_model(n=128, seed=1, dz=10.0, shape=None, water_frac=0.19, perturb=0.05,
                 corr_len=8.0, layer_tops=(1800.0, 2300.0, 2800.0, 3300.0, 3800.0),
                 gradient=0.5, cp_cap=4000.0):
    """Water column (top round(0.19 nz) cells: rho 1000, cp 1500, cs 0) over 5
    flat layers of equal thickness.  cp at each layer top from layer_tops plus
    0.5 1/s times the depth below that top, capped at 4000 m/s; then scaled by
    (1 + 0.05 g), g a Gaussian random field of correlation length 8 cells;
    cs = cp / 1.8; rho = 310 cp^0.25 (Gardner).  Water is not perturbed."""
    nz, ny, nx = shape if shape is not None else (n, n, n)
    rng = SplitMix64(seed)
    nw = int(round(water_frac * nz))
    nsolid = nz - nw
    cp1 = np.empty(nz)
    nl = len(layer_tops)
    for k in range(nw, nz):
        layer = min(nl - 1, ((k - nw) * nl) // max(1, nsolid))
        top = nw + (layer * nsolid) // nl
        cp1[k] = min(cp_cap, layer_tops[layer] + gradient * (k - top) * dz)
    g = gaussian_random_field((nz, ny, nx), corr_len, rng)
    cp = np.empty((nz, ny, nx))
    cp[nw:] = cp1[nw:, None, None] * (1.0 + perturb * g[nw:])
    cp[:nw] = 1500.0
    cs = cp / 1.8
    cs[:nw] = 0.0
    rho = 310.0 * cp ** 0.25
    rho[:nw] = 1000.0
    return rho.astype(np.float32), cp.astype(np.float32), cs.astype(np.float32)


# --------------------------------------------------------------------------
# time functions and source mechanisms (Sec. V, Eq. (6)-(7))
# --------------------------------------------------------------------------

def ricker(nt, dt, f0, amp=1.0, t0=None, delay_samples=0):
    """Ricker wavelet A (1 - 2 pi^2 f^2 tau^2) exp(-pi^2 f^2 tau^2), tau = t - t0,
    t0 = 1.5 / f, sampled at t_n = n dt (FP64), returned as float32."""
    t0 = 1.5 / f0 if t0 is None else t0
    t = (np.arange(nt) - delay_samples) * dt - t0
    a = (np.pi * f0 * t) ** 2
    w = amp * (1.0 - 2.0 * a) * np.exp(-a)
    if delay_samples > 0:
        w[:delay_samples] = 0.0
    return w.astype(np.float32)


def explosive(s=1.0):
    """Isotropic source: equal diagonal components (Sec. V-A)."""
    return np.array([s, s, s, 0.0, 0.0, 0.0])


def clvd(s=1.0):
    """CLVD diag(s, s, -2s) (Eq. (7), one amplitude)."""
    return np.array([s, s, -2.0 * s, 0.0, 0.0, 0.0])


def double_couple_xy(s=1.0):
    """DC in the x-y plane, symmetric reading of Eq. (7): only M_xy."""
    return np.array([0.0, 0.0, 0.0, s, 0.0, 0.0])


def double_couple_sdr(strike_deg, dip_deg, rake_deg, m0=1.0):
    """Moment tensor of a double couple from strike, dip and rake (Aki &
    Richards, Quantitative Seismology, Box 4.4; x = north, y = east, z = down).
    Returned as (Mxx, Myy, Mzz, Mxy, Mxz, Myz)."""
    phi, dl, lm = (math.radians(v) for v in (strike_deg, dip_deg, rake_deg))
    sd, cd, s2d, c2d = math.sin(dl), math.cos(dl), math.sin(2 * dl), math.cos(2 * dl)
    sl, cl = math.sin(lm), math.cos(lm)
    sp, cp_, s2p, c2p = math.sin(phi), math.cos(phi), math.sin(2 * phi), math.cos(2 * phi)
    mxx = -(sd * cl * s2p + s2d * sl * sp * sp)
    mxy = sd * cl * c2p + 0.5 * s2d * sl * s2p
    mxz = -(cd * cl * cp_ + c2d * sl * sp)
    myy = sd * cl * s2p - s2d * sl * cp_ * cp_
    myz = -(cd * cl * sp - c2d * sl * cp_)
    mzz = s2d * sl
    return m0 * np.array([mxx, myy, mzz, mxy, mxz, myz])


def random_dc(rng: SplitMix64, m0=1.0):
    """strike U[0,360), dip U[0,90], rake U[-180,180)."""
    u = rng.uniform(3)
    return double_couple_sdr(360.0 * u[0], 90.0 * u[1], -180.0 + 360.0 * u[2], m0)


def random_dc_batch(rng: SplitMix64, n, m0=1.0):
    """n random double couples at once ([n][6], the same draws as n calls of
    random_dc): strike U[0,360), dip U[0,90], rake U[-180,180), Aki & Richards
    Box 4.4 vectorised."""
    u = rng.uniform(3 * n).reshape(n, 3)
    phi, dl, lm = np.radians(360.0 * u[:, 0]), np.radians(90.0 * u[:, 1]), np.radians(-180.0 + 360.0 * u[:, 2])
    sd, cd, s2d, c2d = np.sin(dl), np.cos(dl), np.sin(2 * dl), np.cos(2 * dl)
    sl, cl = np.sin(lm), np.cos(lm)
    sp, cp_, s2p, c2p = np.sin(phi), np.cos(phi), np.sin(2 * phi), np.cos(2 * phi)
    out = np.empty((n, 6))
    out[:, 0] = -(sd * cl * s2p + s2d * sl * sp * sp)
    out[:, 1] = sd * cl * s2p - s2d * sl * cp_ * cp_
    out[:, 2] = s2d * sl
    out[:, 3] = sd * cl * c2p + 0.5 * s2d * sl * s2p
    out[:, 4] = -(cd * cl * cp_ + c2d * sl * sp)
    out[:, 5] = -(cd * cl * sp - c2d * sl * cp_)
    return m0 * out


def reservoir_box(shape, pml):
    """Reservoir box a third of the way down: z in [nz/3 - nz/12, nz/3 + nz/12],
    x and y in the central half; kept clear of the PML."""
    nz, ny, nx = shape
    zc = nz // 3
    z0, z1 = zc - nz // 12, zc + nz // 12
    x0, x1 = nx // 4, (3 * nx) // 4
    y0, y1 = ny // 4, (3 * ny) // 4
    lo = pml + 1
    return (max(x0, lo), min(x1, nx - lo - 1)), (max(y0, lo), min(y1, ny - lo - 1)), \
           (max(z0, lo), min(z1, nz - lo - 1))


def random_positions(rng: SplitMix64, box, n):
    (x0, x1), (y0, y1), (z0, z1) = box
    u = rng.uniform(3 * n).reshape(n, 3)
    pos = np.empty((n, 3), np.int32)
    pos[:, 0] = x0 + np.floor(u[:, 0] * (x1 - x0 + 1)).astype(np.int32)
    pos[:, 1] = y0 + np.floor(u[:, 1] * (y1 - y0 + 1)).astype(np.int32)
    pos[:, 2] = z0 + np.floor(u[:, 2] * (z1 - z0 + 1)).astype(np.int32)
    return pos


def latin_hypercube_positions(rng: SplitMix64, box, n):
    """Latin-hypercube sample of n cells in the box (Sec. III-A): each axis
    range cut into n strata, one point per stratum, strata paired by random
    permutations."""
    out = np.empty((n, 3), np.int32)
    for a, (lo, hi) in enumerate(box):
        u = rng.uniform(n)
        perm = np.argsort(rng.uniform(n), kind="stable")
        frac = (perm + u) / n
        out[:, a] = lo + np.minimum(np.floor(frac * (hi - lo + 1)).astype(np.int32), hi - lo)
    return out


def events(rng: SplitMix64, n_events, n_src, t_span=2.0, sigma=1.0):
    """Event draws for superposition (Sec. IV-C): source index uniform in
    [0, n_src) with replacement, log-normal amplitudes (mu 0, sigma), origin
    times uniform in [0, t_span)."""
    u = rng.uniform(n_events)
    src = np.minimum(np.floor(u * n_src).astype(np.int32), n_src - 1)
    amps = np.exp(sigma * rng.normal(n_events)).astype(np.float32)
    t0s = (t_span * rng.uniform(n_events)).astype(np.float32)
    return src, amps, t0s


def cluster_origin_times(rng: SplitMix64, labels, between=0.3, within_sd=0.1):
    """Origin times for clustered events (Sec. VI-A): cluster c starts at
    c * 0.3 s, events within a cluster are shifted by N(0, 0.1 s)."""
    labels = np.asarray(labels)
    return (labels * between + within_sd * rng.normal(labels.size)).astype(np.float32)
