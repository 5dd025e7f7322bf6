"""FP64 CPU oracle for the staggered-grid Fourier pseudo-spectral elastic solver
(Das, Chen & Hobson, arXiv 1705.04874, Sec. II-IV).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path (the
CUDA library and its Python binding) never imports this package and shares no
code with it.

The arithmetic lives in ``es_oracle.c`` (plain C99, FP64, OpenMP over lines);
this module compiles it on demand with gcc and marshals numpy arrays through
ctypes.  Every function cites the passage it follows; the readings of points
the paper leaves open are listed at the top of ``es_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "es_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "libes_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP) into oracle/_build/."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


class Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("pml", ctypes.c_int), ("pml_alpha0", ctypes.c_double),
                ("pml_cref", ctypes.c_double), ("dt", ctypes.c_double), ("nt", ctypes.c_int),
                ("deriv_mode", ctypes.c_int), ("nthreads", ctypes.c_int), ("tau", ctypes.c_double)]


class Source(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("ix", ctypes.c_int), ("iy", ctypes.c_int),
                ("iz", ctypes.c_int), ("m", ctypes.c_double * 6),
                ("w", ctypes.POINTER(ctypes.c_double)), ("nw", ctypes.c_int),
                ("g", ctypes.POINTER(ctypes.c_double))]


def blackman_window(n):
    """Blackman window over the n signed wavenumber bins of an axis (numpy FFT
    order), 1 at k = 0 and 0 at the Nyquist wavenumber: the classical window
    0.42 - 0.5 cos(2 pi t) + 0.08 cos(4 pi t) with t = 1/2 + m/n running over
    the spatial-frequency axis from -Nyquist to +Nyquist."""
    m = np.fft.fftfreq(n) * n
    t = 0.5 + m / n
    return 0.42 - 0.5 * np.cos(2 * np.pi * t) + 0.08 * np.cos(4 * np.pi * t)


def laplacian(f, d):
    """Spectral Laplacian (Sec. VI-A, Eq. (8)): inverse FFT of
    -(kx^2 + ky^2 + kz^2) times the 3D FFT of f [nz][ny][nx], kappa_m =
    2 pi m / (n d_axis) on the signed bins; d = (dx, dy, dz).  float64."""
    f = np.asarray(f, np.float64)
    nz, ny, nx = f.shape
    kx = 2 * np.pi * np.fft.fftfreq(nx, d[0])
    ky = 2 * np.pi * np.fft.fftfreq(ny, d[1])
    kz = 2 * np.pi * np.fft.fftfreq(nz, d[2])
    k2 = kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2
    return np.fft.ifftn(-k2 * np.fft.fftn(f)).real


def smoothed_delta(shape, pos):
    """The point source smoothed in the spatial-frequency domain (Sec. II-A):
    3D FFT of the grid-point delta at pos = (ix, iy, iz), times the product of
    the three axes' Blackman windows, inverse FFT.  [nz][ny][nx] float64."""
    nz, ny, nx = shape
    delta = np.zeros(shape)
    delta[pos[2], pos[1], pos[0]] = 1.0
    W = blackman_window(nz)[:, None, None] * blackman_window(ny)[None, :, None] * blackman_window(nx)[None, None, :]
    return np.fft.ifftn(W * np.fft.fftn(delta)).real


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            d, i = ctypes.c_double, ctypes.c_int
            pd, pi = P(d), P(i)
            lib.orc_fft.argtypes = [i, pd, pd, pd, pd, i, i]
            lib.orc_deriv.argtypes = [pd, i, i, i, i, d, i, pd, i, i]
            lib.orc_materials.argtypes = [pd, pd, pd, i, i, i] + [pd] * 8
            lib.orc_pml_profile.argtypes = [i, i, d, d, d, d, i, pd]
            lib.orc_simulate.argtypes = [P(Params), pd, pd, pd, P(Source), i, pi, i, pd, pd, pd]
            lib.orc_seabed_receivers.argtypes = [pd, i, i, i, i, i, i, pi]
            lib.orc_superpose.argtypes = [pd, i, i, i, pi, pd, pd, i, d, i, pd]
            lib.orc_num_threads.restype = i
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def default_threads() -> int:
    return int(_load().orc_num_threads())


def fft(x, inverse=False, naive=False):
    """1D DFT (forward unscaled, inverse scaled by 1/N), own FFT or the O(N^2) definition."""
    x = np.asarray(x, dtype=np.complex128).ravel()
    n = x.size
    re, im = _f64(x.real), _f64(x.imag)
    ro, io = np.empty(n), np.empty(n)
    if _load().orc_fft(n, _dp(re), _dp(im), _dp(ro), _dp(io), int(inverse), int(naive)) != 0:
        raise ValueError("orc_fft failed")
    return ro + 1j * io


def deriv(f, axis, d, shift, mode=0, nthreads=0):
    """Staggered spectral derivative D(shift)_axis f of a [nz][ny][nx] field
    (axis 0 = x).  mode 0: 1D FFT per line, 1: naive DFT, 2: 3D FFT."""
    f = _f64(f)
    nz, ny, nx = f.shape
    out = np.empty_like(f)
    rc = _load().orc_deriv(_dp(f), nx, ny, nz, int(axis), float(d), int(shift), _dp(out),
                           int(mode), int(nthreads or default_threads()))
    if rc != 0:
        raise ValueError("orc_deriv: bad arguments")
    return out


def materials(rho, cp, cs):
    """lam, mu, bx, by, bz, muxy, muxz, muyz (Eq. (4) plus the staggered averages)."""
    rho, cp, cs = _f64(rho), _f64(cp), _f64(cs)
    nz, ny, nx = rho.shape
    outs = [np.empty_like(rho) for _ in range(8)]
    _load().orc_materials(_dp(rho), _dp(cp), _dp(cs), nx, ny, nz, *[_dp(o) for o in outs])
    return dict(zip(["lam", "mu", "bx", "by", "bz", "muxy", "muxz", "muyz"], outs))


def pml_profile(n, L, alpha0, cref, d, dt, stag):
    out = np.empty(n)
    _load().orc_pml_profile(int(n), int(L), float(alpha0), float(cref), float(d), float(dt),
                            int(stag), _dp(out))
    return out


def simulate(rho, cp, cs, *, dx, dy=None, dz=None, dt, nt, pml=10, pml_alpha0=2.0,
             pml_cref=0.0, sources=(), receivers=None, state=None, energy=False,
             deriv_mode=0, nthreads=0, tau=0.0):
    """Run nt leapfrog steps (Sec. II-A) and return a dict with 'traces'
    [4][n_rcv][nt] (p, vx, vy, vz), optionally 'state' [9][nz][ny][nx] (final
    totals vx vy vz sxx syy szz sxy sxz syz) and 'energy' [nt].  tau > 0 adds
    the Kelvin-Voigt terms of Eq. (1)-(2) with chi = tau lambda, eta = tau mu,
    the time derivative of the strain rate taken as the backward difference
    of the velocity derivatives over one step (v^{n-1/2} of the given state
    counts as the previous velocity at the first step).

    sources: iterable of dicts {kind: 'moment'|'force', pos: (ix,iy,iz),
    m: 6 moment components (xx yy zz xy xz yz) or 3 force components,
    w: wavelet samples, smooth: True for a moment source smoothed with the
    Blackman window in the spatial-frequency domain (smoothed_delta)}."""
    rho, cp, cs = _f64(rho), _f64(cp), _f64(cs)
    nz, ny, nx = rho.shape
    dy = dx if dy is None else dy
    dz = dx if dz is None else dz
    p = Params(nx, ny, nz, float(dx), float(dy), float(dz), int(pml), float(pml_alpha0),
               float(pml_cref), float(dt), int(nt), int(deriv_mode),
               int(nthreads or default_threads()), float(tau))
    srcs = list(sources)
    arr = (Source * max(1, len(srcs)))()
    keep = []
    for e, s in enumerate(srcs):
        w = _f64(s["w"]).ravel()
        keep.append(w)
        m = list(s["m"]) + [0.0] * (6 - len(s["m"]))
        kind = 0 if s.get("kind", "moment") == "moment" else 1
        g = ctypes.POINTER(ctypes.c_double)()
        if kind == 0 and s.get("smooth"):
            gd = np.ascontiguousarray(smoothed_delta(rho.shape, s["pos"]))
            keep.append(gd)
            g = _dp(gd)
        arr[e] = Source(kind, int(s["pos"][0]), int(s["pos"][1]), int(s["pos"][2]),
                        (ctypes.c_double * 6)(*m), _dp(w), int(w.size), g)
    if receivers is None:
        receivers = np.zeros((0, 3), np.int32)
    rcv = np.ascontiguousarray(receivers, dtype=np.int32).reshape(-1, 3)
    n_rcv = rcv.shape[0]
    traces = np.zeros((4, n_rcv, nt)) if n_rcv else None
    st = None
    if state is not None:
        st = _f64(state).reshape(9, nz, ny, nx).copy()
    en = np.zeros(nt) if energy else None
    null = ctypes.POINTER(ctypes.c_double)()
    rc = _load().orc_simulate(ctypes.byref(p), _dp(rho), _dp(cp), _dp(cs), arr, len(srcs),
                              _ip(rcv) if n_rcv else ctypes.POINTER(ctypes.c_int)(), n_rcv,
                              _dp(traces) if traces is not None else null,
                              _dp(st) if st is not None else null,
                              _dp(en) if en is not None else null)
    if rc != 0:
        raise ValueError("orc_simulate: bad arguments")
    out = {"traces": traces if traces is not None else np.zeros((4, 0, nt))}
    if st is not None:
        out["state"] = st
    if en is not None:
        out["energy"] = en
    return out


def seabed_receivers(cs, L, rx, ry):
    """[rx*ry][3] receiver indices (ix, iy, iz) by the seabed rule (Sec. II-B)."""
    cs = _f64(cs)
    nz, ny, nx = cs.shape
    out = np.empty((rx * ry, 3), np.int32)
    rc = _load().orc_seabed_receivers(_dp(cs), nx, ny, nz, int(L), int(rx), int(ry), _ip(out))
    if rc != 0:
        raise ValueError(f"orc_seabed_receivers failed ({rc})")
    return out


def superpose(traces, src_of_event, amps, t0s, dt, n_out):
    """[4][n_rcv][n_out] gather of amplitude-scaled, time-shifted traces (Sec. IV)."""
    traces = _f64(traces)
    n_src, _, n_rcv, nt = traces.shape
    ev = np.ascontiguousarray(src_of_event, dtype=np.int32)
    a, t0 = _f64(amps), _f64(t0s)
    g = np.empty((4, n_rcv, int(n_out)))
    rc = _load().orc_superpose(_dp(traces), n_src, n_rcv, nt, _ip(ev), _dp(a), _dp(t0),
                               int(ev.size), float(dt), int(n_out), _dp(g))
    if rc != 0:
        raise ValueError("orc_superpose: bad event source index")
    return g
