"""Thin ctypes binding of libes.so (include/es.h).

Every function has the C name and only marshals arguments: numpy arrays are
passed as host pointers, torch tensors as their (host or device) data
pointers, streams as ``torch.cuda.Stream.cuda_stream`` integers.  All
computation happens in the library's CUDA kernels; there is no CPU path, and
loading fails loudly when the library cannot be built or loaded.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

ES_PREC_FP32, ES_PREC_COMPENSATED, ES_PREC_FP32_TC = 0, 1, 2
ES_NOALLOC_MAX_EVENTS = 65536  # include/es.h
ES_OK, ES_ERR_ARG, ES_ERR_SIZE, ES_ERR_CUDA, ES_ERR_OOM, ES_ERR_UNSTABLE, ES_ERR_TIMEOUT, ES_ERR_STATE = \
    0, -1, -2, -3, -4, -5, -6, -7

SUPPORTED_AXIS = (16, 32, 48, 64, 80, 96, 128, 160, 192, 256)
KERNEL_NAMES = ("vel-x", "vel-y", "vel-z", "str-x", "str-y", "str-z", "inject", "record")

_lib = None
_lock = threading.Lock()


class EsError(RuntimeError):
    def __init__(self, status, where):
        lib = _load()
        msg = lib.es_status_string(status).decode()
        detail = lib.es_last_error().decode()
        super().__init__(f"{where}: {msg} ({status})" + (f": {detail}" if detail and status == ES_ERR_CUDA else ""))
        self.status = status


def bounds_build() -> bool:
    """ES_BOUNDS=1 in the environment selects the bounds-checked debug build
    (libes_bounds.so) for this process."""
    return os.environ.get("ES_BOUNDS", "0") == "1"


def library_path() -> str:
    return _build.BOUNDS_LIB if bounds_build() else _build.LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build(bounds=bounds_build())
            lib = ctypes.CDLL(path)
            c_int, c_double, vp = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
            pi = ctypes.POINTER(ctypes.c_int)
            sig = {
                "es_model_create": ([vp, vp, vp, c_int, c_int, c_int, c_double, c_int, ctypes.POINTER(vp)], c_int),
                "es_model_set_spacing": ([vp, c_double, c_double, c_double], c_int),
                "es_model_set_pml": ([vp, c_double, c_double], c_int),
                "es_model_set_stream": ([vp, vp], c_int),
                "es_model_set_precision": ([vp, c_int], c_int),
                "es_model_set_viscosity": ([vp, c_double], c_int),
                "es_model_default_dt": ([vp, ctypes.POINTER(c_double)], c_int),
                "es_source_set": ([vp, pi, ctypes.POINTER(c_double), vp, c_int], c_int),
                "es_source_add": ([vp, pi, ctypes.POINTER(c_double), vp, c_int], c_int),
                "es_source_add_force": ([vp, pi, ctypes.POINTER(c_double), vp, c_int], c_int),
                "es_source_add_smoothed": ([vp, pi, ctypes.POINTER(c_double), vp, c_int], c_int),
                "es_source_clear": ([vp], c_int),
                "es_batch_set": ([vp, c_int, vp, vp, vp, c_int], c_int),
                "es_state_reset": ([vp], c_int),
                "es_state_get": ([vp, vp], c_int),
                "es_state_set": ([vp, vp], c_int),
                "es_run": ([vp, c_int, c_double, vp, c_int, vp], c_int),
                "es_superpose": ([vp, c_int, c_int, c_int, vp, vp, vp, c_int, c_double, c_int, vp, vp], c_int),
                "es_superpose_noalloc": ([vp, c_int, c_int, c_int, vp, vp, vp, c_int, c_double, c_int, vp, vp],
                                         c_int),
                "es_seabed_receivers": ([vp, c_int, c_int, pi], c_int),
                "es_run_group": ([c_int, ctypes.POINTER(vp), c_int, ctypes.POINTER(c_double), ctypes.POINTER(vp),
                                  pi, ctypes.POINTER(vp)], c_int),
                "es_derivative": ([vp, c_int, c_int, c_int, c_int, c_double, c_int, vp, vp], c_int),
                "es_laplacian": ([vp, c_int, c_int, c_int, c_double, c_double, c_double, vp, vp], c_int),
                "es_last_step_kernel_ms": ([vp, ctypes.POINTER(ctypes.c_float), c_int], c_int),
                "es_kernels_per_step": ([vp], c_int),
                "es_model_autotune": ([vp, c_int, ctypes.c_char_p, c_int], c_int),
                "es_fft_plan": ([c_int, c_int, pi, pi], c_int),
                "es_fft_plan_select": ([c_int, c_int, c_int, c_int], c_int),
                "es_model_destroy": ([vp], None),
                "es_status_string": ([c_int], ctypes.c_char_p),
                "es_last_error": ([], ctypes.c_char_p),
                "es_fault_inject_alloc": ([c_int], None),
                "es_debug_live_allocations": ([], ctypes.c_longlong),
                "es_debug_bounds": ([ctypes.POINTER(ctypes.c_longlong)], c_int),
            }
            for name, (args, res) in sig.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def exported_symbols():
    """Names the binding expects the library to export."""
    return ["es_model_create", "es_model_set_spacing", "es_model_set_pml", "es_model_set_stream", "es_model_set_precision", "es_model_set_viscosity",
            "es_model_default_dt", "es_source_set", "es_source_add", "es_source_add_smoothed", "es_source_add_force",
            "es_source_clear", "es_batch_set", "es_state_reset", "es_state_get", "es_state_set", "es_run",
            "es_run_group", "es_superpose", "es_superpose_noalloc", "es_seabed_receivers", "es_derivative", "es_laplacian", "es_last_step_kernel_ms",
            "es_kernels_per_step", "es_model_autotune", "es_fft_plan",
            "es_fft_plan_select", "es_sur_create", "es_sur_destroy", "es_sur_set_stream", "es_sur_num_params",
            "es_sur_get_params", "es_sur_set_params", "es_sur_set_output_scale", "es_sur_fit_output_scale",
            "es_sur_predict", "es_sur_loss_grad", "es_sur_train_step", "es_sur_combine", "es_gemm_bf16", "es_gemm_status", "es_gemm_wait_probe", "es_model_destroy", "es_status_string", "es_last_error",
            "es_fault_inject_alloc", "es_debug_live_allocations", "es_debug_bounds"]


def _check(status, where):
    if status != ES_OK:
        raise EsError(status, where)
    return status


def _ptr(a, dtype):
    """(pointer, keep-alive) for a numpy array or torch tensor of `dtype`."""
    if a is None:
        return None, None
    if hasattr(a, "data_ptr"):  # torch tensor
        import torch
        tdt = {np.float32: torch.float32, np.int32: torch.int32, np.float64: torch.float64}[dtype]
        if a.dtype != tdt or not a.is_contiguous():
            raise TypeError(f"expected a contiguous {tdt} tensor")
        return ctypes.c_void_p(a.data_ptr()), a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return ctypes.c_void_p(arr.ctypes.data), arr


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


# ---------------------------------------------------------------------------
# C-named functions
# ---------------------------------------------------------------------------

def es_model_create(rho, cp, cs, dx, pml):
    lib = _load()
    shapes = {tuple(a.shape) for a in (rho, cp, cs)}
    if len(shapes) != 1:
        raise ValueError("rho, cp, cs must have one shape [nz][ny][nx]")
    nz, ny, nx = shapes.pop()
    keep = [_ptr(a, np.float32) for a in (rho, cp, cs)]
    h = ctypes.c_void_p()
    _check(lib.es_model_create(keep[0][0], keep[1][0], keep[2][0], nx, ny, nz, float(dx), int(pml),
                               ctypes.byref(h)), "es_model_create")
    return h


def es_superpose(traces, src_of_event, amps, t0s, dt, n_out, gather=None, stream=None):
    """gather [4][n_rcv][n_out] from traces [n_src][4][n_rcv][nt] (Sec. IV)."""
    lib = _load()
    n_src, four, n_rcv, nt = traces.shape
    assert four == 4
    n_ev = len(src_of_event)
    tp, tk = _ptr(traces, np.float32)
    ep, ek = _ptr(src_of_event, np.int32)
    ap, ak = _ptr(amps, np.float32)
    t0p, t0k = _ptr(t0s, np.float32)
    if gather is None:
        gather = np.empty((4, n_rcv, int(n_out)), np.float32)
    gp, gk = _ptr(gather, np.float32)
    _check(lib.es_superpose(tp, n_src, n_rcv, nt, ep, ap, t0p, n_ev, float(dt), int(n_out), gp,
                            _stream_handle(stream)), "es_superpose")
    return gather


def es_superpose_noalloc(traces, src_of_event, amps, t0s, dt, n_out, gather, stream=None):
    """es_superpose for callers that cannot allocate: every array a torch CUDA
    tensor (gather [4][n_rcv][n_out] preallocated by the caller)."""
    lib = _load()
    n_src, four, n_rcv, nt = traces.shape
    assert four == 4
    ptrs = [_ptr(a, dt_)[0] for a, dt_ in ((traces, np.float32), (src_of_event, np.int32), (amps, np.float32),
                                           (t0s, np.float32), (gather, np.float32))]
    _check(lib.es_superpose_noalloc(ptrs[0], n_src, n_rcv, nt, ptrs[1], ptrs[2], ptrs[3], len(src_of_event),
                                    float(dt), int(n_out), ptrs[4], _stream_handle(stream)), "es_superpose_noalloc")
    return gather


def es_run_group(models, nt, dts, receivers, traces=None):
    """Advance several models together in one graph (es_run_group); returns
    the list of trace arrays (shape as Model.run)."""
    lib = _load()
    n = len(models)
    hs = (ctypes.c_void_p * n)(*[m._h for m in models])
    dd = (ctypes.c_double * n)(*[float(v) for v in dts])
    keep, rp, nr, tp = [], (ctypes.c_void_p * n)(), (ctypes.c_int * n)(), (ctypes.c_void_p * n)()
    out = []
    for i, (m, rc) in enumerate(zip(models, receivers)):
        p_, k_ = _ptr(rc, np.int32)
        keep.append(k_)
        rp[i] = p_
        nr[i] = int(np.prod(rc.shape)) // 3
        tr = traces[i] if traces is not None else np.empty(
            (4, nr[i], int(nt)) if m.nsim == 1 else (m.nsim, 4, nr[i], int(nt)), np.float32)
        t_, tk = _ptr(tr, np.float32)
        keep.append(tk)
        tp[i] = t_
        out.append(tr)
    _check(lib.es_run_group(n, hs, int(nt), dd, rp, nr, tp), "es_run_group")
    return out


def es_fft_plan(pass_kind, n):
    """(RA, RB) of the plan in use for pass kind 0 (x) / 1 (y, z) and length n."""
    ra, rb = ctypes.c_int(), ctypes.c_int()
    _check(_load().es_fft_plan(int(pass_kind), int(n), ctypes.byref(ra), ctypes.byref(rb)), "es_fft_plan")
    return ra.value, rb.value


def es_fft_plan_select(pass_kind, n, ra, rb):
    _check(_load().es_fft_plan_select(int(pass_kind), int(n), int(ra), int(rb)), "es_fft_plan_select")


# FFT plans per axis length, named (R1, n / R1); the first is the default.  (3, 25)
# and (5, 25) run as three stages (3 x 5 x 5, 5 x 5 x 5).
PLAN_CANDIDATES = {16: [(4, 4)], 32: [(8, 4), (4, 8)], 48: [(12, 4), (4, 12)], 64: [(16, 4), (8, 8), (4, 16)],
                   75: [(5, 15), (3, 25), (15, 5)], 80: [(16, 5), (5, 16)], 96: [(16, 6), (6, 16)],
                   125: [(5, 25), (25, 5)], 128: [(16, 8), (8, 16)], 160: [(16, 10), (10, 16)],
                   192: [(16, 12), (12, 16)], 256: [(16, 16)]}


def es_derivative(f, axis, d, shift, out, stream=None):
    """out = D_axis^(shift) f for [nz][ny][nx] torch CUDA tensors."""
    lib = _load()
    nz, ny, nx = f.shape
    fp, fk = _ptr(f, np.float32)
    op, ok = _ptr(out, np.float32)
    _check(lib.es_derivative(fp, nx, ny, nz, int(axis), float(d), int(shift), op, _stream_handle(stream)),
           "es_derivative")
    return out


def es_laplacian(f, d, out, stream=None):
    """out = spectral Laplacian of f (Sec. VI-A, Eq. (8)) for [nz][ny][nx] torch
    CUDA tensors; d = (dx, dy, dz)."""
    lib = _load()
    nz, ny, nx = f.shape
    fp, fk = _ptr(f, np.float32)
    op, ok = _ptr(out, np.float32)
    _check(lib.es_laplacian(fp, nx, ny, nz, float(d[0]), float(d[1]), float(d[2]), op, _stream_handle(stream)),
           "es_laplacian")
    return out


# ---------------------------------------------------------------------------
# model object
# ---------------------------------------------------------------------------

class Model:
    """A velocity model on the GPU (es_model).  rho, cp, cs: [nz][ny][nx]
    float32 numpy arrays or torch tensors; dx in metres; pml cells per face."""

    def __init__(self, rho, cp, cs, dx=10.0, pml=10, dy=None, dz=None, stream=None):
        self.shape = tuple(rho.shape)
        self.nsim = 1
        self._lib = _load()
        self._h = es_model_create(rho, cp, cs, dx, pml)
        self.pml = int(pml)
        if dy is not None or dz is not None:
            self.set_spacing(dx, dy if dy is not None else dx, dz if dz is not None else dx)
        if stream is not None:
            self.set_stream(stream)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.es_model_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_spacing(self, dx, dy, dz):
        _check(self._lib.es_model_set_spacing(self._h, dx, dy, dz), "es_model_set_spacing")

    def set_viscosity(self, tau):
        """Kelvin-Voigt relaxation time tau [s] (chi = tau lambda, eta = tau mu): es_model_set_viscosity."""
        _check(self._lib.es_model_set_viscosity(self._h, float(tau)), "es_model_set_viscosity")

    def set_precision(self, mode):
        """ES_PREC_FP32 (0), ES_PREC_COMPENSATED (1) or ES_PREC_FP32_TC (2): es_model_set_precision."""
        _check(self._lib.es_model_set_precision(self._h, int(mode)), "es_model_set_precision")

    def set_pml(self, alpha0=2.0, cref=0.0):
        _check(self._lib.es_model_set_pml(self._h, alpha0, cref), "es_model_set_pml")

    def set_stream(self, stream):
        _check(self._lib.es_model_set_stream(self._h, _stream_handle(stream)), "es_model_set_stream")

    def default_dt(self):
        v = ctypes.c_double()
        _check(self._lib.es_model_default_dt(self._h, ctypes.byref(v)), "es_model_default_dt")
        return v.value

    def _src(self, fn, pos, vals, n, wavelet):
        p = (ctypes.c_int * 3)(*[int(v) for v in pos])
        v = (ctypes.c_double * 6)(*([float(x) for x in vals] + [0.0] * (6 - len(vals))))
        wp, wk = _ptr(wavelet, np.float32)
        nw = int(wavelet.shape[0]) if wavelet is not None else 0
        _check(fn(self._h, p, v, wp, nw), fn.__name__)

    def source_set(self, pos, mt, wavelet):
        self._src(self._lib.es_source_set, pos, mt, 6, wavelet)

    def source_add(self, pos, mt, wavelet):
        self._src(self._lib.es_source_add, pos, mt, 6, wavelet)

    def source_add_force(self, pos, f, wavelet):
        self._src(self._lib.es_source_add_force, pos, f, 3, wavelet)

    def source_add_smoothed(self, pos, mt, wavelet):
        """Moment source spread over the 5 x 5 x 5 Blackman stencil
        (es_source_add_smoothed); wavelet [1.0] is an initial-value source."""
        self._src(self._lib.es_source_add_smoothed, pos, mt, 6, wavelet)

    def batch_set(self, pos, mt, wavelets):
        """nb simulations sharing this model, one moment source each:
        pos [nb][3] int, mt [nb][6] (xx yy zz xy xz yz), wavelets [nb][nw]."""
        pos = np.ascontiguousarray(pos, np.int32).reshape(-1, 3)
        nb = pos.shape[0]
        mt = np.ascontiguousarray(mt, np.float64).reshape(nb, 6)
        wp, wk = _ptr(wavelets, np.float32)
        nw = int(wavelets.shape[-1])
        _check(self._lib.es_batch_set(self._h, nb, ctypes.c_void_p(pos.ctypes.data), ctypes.c_void_p(mt.ctypes.data),
                                      wp, nw), "es_batch_set")
        self.nsim = nb

    def source_clear(self):
        _check(self._lib.es_source_clear(self._h), "es_source_clear")

    def state_reset(self):
        _check(self._lib.es_state_reset(self._h), "es_state_reset")

    def state_get(self, out=None):
        nz, ny, nx = self.shape
        if out is None:
            out = np.empty((9, nz, ny, nx) if self.nsim == 1 else (self.nsim, 9, nz, ny, nx), np.float32)
        op, ok = _ptr(out, np.float32)
        _check(self._lib.es_state_get(self._h, op), "es_state_get")
        return out

    def state_set(self, fields):
        fp, fk = _ptr(fields, np.float32)
        _check(self._lib.es_state_set(self._h, fp), "es_state_set")

    def run(self, nt, dt=0.0, receivers=None, traces=None):
        """Advance nt steps; returns traces [4][n_rcv][nt] (numpy unless a
        torch tensor `traces` is passed)."""
        if receivers is None:
            n_rcv = 0
            rp = rk = None
        else:
            rp, rk = _ptr(receivers, np.int32)
            n_rcv = int(np.prod(receivers.shape)) // 3
        if traces is None:
            shape = (4, n_rcv, int(nt)) if self.nsim == 1 else (self.nsim, 4, n_rcv, int(nt))
            traces = np.empty(shape, np.float32)
        tp, tk = _ptr(traces, np.float32)
        _check(self._lib.es_run(self._h, int(nt), float(dt), rp, n_rcv, tp if n_rcv else None), "es_run")
        return traces

    def seabed_receivers(self, rx, ry):
        out = np.empty((rx * ry, 3), np.int32)
        _check(self._lib.es_seabed_receivers(self._h, rx, ry, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int))),
               "es_seabed_receivers")
        return out

    def last_step_kernel_ms(self):
        buf = (ctypes.c_float * 16)()
        n = self._lib.es_last_step_kernel_ms(self._h, buf, 16)
        if n < 0:
            raise EsError(n, "es_last_step_kernel_ms")
        return [buf[i] for i in range(n)]

    def autotune(self, reps=5):
        """Time every FFT plan candidate on this model's passes and keep the
        fastest (es_model_autotune); returns the timing report."""
        buf = ctypes.create_string_buffer(4096)
        _check(self._lib.es_model_autotune(self._h, int(reps), buf, 4096), "es_model_autotune")
        return buf.value.decode()

    def kernels_per_step(self):
        return int(self._lib.es_kernels_per_step(self._h))


def es_debug_bounds():
    """First out-of-range index recorded by the bounds-checked build since the
    last call (0: none), as (source line, index low 40 bits, raw value)."""
    v = ctypes.c_longlong()
    _check(_load().es_debug_bounds(ctypes.byref(v)), "es_debug_bounds")
    return (v.value >> 40, v.value & ((1 << 40) - 1), v.value)
