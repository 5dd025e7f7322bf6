"""The C ABI builds, loads without a GPU, and exports every entry point that
include/es.h declares; host-side argument checks answer without touching a
device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1705_04874_gb300 import es
    return es._load()


def declared_symbols():
    import glob
    text = "".join(open(f).read() for f in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))))
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(es_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("es_model_create", "es_source_set", "es_run", "es_superpose", "es_model_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1705_04874_gb300 import es
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert set(declared_symbols()) == set(es.exported_symbols())


def test_status_strings(lib):
    for s in range(0, -8, -1):
        assert lib.es_status_string(s).decode() not in ("", "unknown status")
    assert lib.es_status_string(5).decode() == "unknown status"


def test_host_side_argument_checks(lib):
    from paper_1705_04874_gb300 import es
    h = ctypes.c_void_p()
    # null inputs / bad sizes are rejected before any device work
    assert lib.es_model_create(None, None, None, 32, 32, 32, 10.0, 6, ctypes.byref(h)) == es.ES_ERR_ARG
    a = np.ones(8, np.float32)
    p = ctypes.c_void_p(a.ctypes.data)
    # axis lengths run from 3 to 512 (FFT passes for the planned lengths, circulant passes otherwise)
    assert lib.es_model_create(p, p, p, 513, 32, 32, 10.0, 6, ctypes.byref(h)) == es.ES_ERR_SIZE
    assert lib.es_model_create(p, p, p, 2, 32, 32, 10.0, 0, ctypes.byref(h)) == es.ES_ERR_SIZE
    assert lib.es_model_create(p, p, p, 32, 32, 32, -1.0, 6, ctypes.byref(h)) == es.ES_ERR_ARG
    assert lib.es_model_create(p, p, p, 32, 32, 32, 10.0, 15, ctypes.byref(h)) == es.ES_ERR_ARG
    assert lib.es_superpose(None, 1, 1, 1, None, None, None, 0, 0.1, 1, None, None) == es.ES_ERR_ARG
    assert lib.es_derivative(p, 32, 32, 32, 3, 1.0, 1, p, None) == es.ES_ERR_ARG
    assert lib.es_derivative(p, 600, 32, 32, 0, 1.0, 1, ctypes.c_void_p(a.ctypes.data + 4), None) == es.ES_ERR_SIZE
    assert lib.es_run(None, 10, 0.0, None, 0, None) == es.ES_ERR_ARG
    assert lib.es_kernels_per_step(None) == es.ES_ERR_ARG
    lib.es_gemm_wait_probe.argtypes = [ctypes.c_double, ctypes.c_void_p]
    assert lib.es_gemm_wait_probe(0.0, None) == es.ES_ERR_ARG
    assert lib.es_gemm_wait_probe(2.5, None) == es.ES_ERR_ARG


def test_surrogate_host_side_argument_checks(lib):
    """Bad network shapes and GEMM arguments are rejected before any device work."""
    from paper_1705_04874_gb300 import es
    from paper_1705_04874_gb300.surrogate import Config
    h = ctypes.c_void_p()
    lib.es_sur_create.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(ctypes.c_void_p)]
    assert lib.es_sur_create(None, ctypes.byref(h)) == es.ES_ERR_ARG
    good = dict(nfreq=3, hidden=64, latent=16, n_rcv=4, nt=16, max_batch=32, seed=1)
    for field, bad in [("nfreq", 17), ("nfreq", -1), ("hidden", 12), ("latent", 4), ("n_rcv", 0), ("nt", 12),
                       ("max_batch", 4), ("max_batch", 20)]:
        cfg = Config(**{**good, field: bad})
        assert lib.es_sur_create(ctypes.byref(cfg), ctypes.byref(h)) == es.ES_ERR_ARG, (field, bad)
        assert not h.value
    lib.es_gemm_bf16.argtypes = [ctypes.c_int] * 3 + [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                                      ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                                      ctypes.c_float, ctypes.c_float, ctypes.c_int, ctypes.c_void_p]
    a = np.zeros(64, np.float32)
    p = ctypes.c_void_p(a.ctypes.data)
    assert lib.es_gemm_bf16(8, 8, 8, None, 8, 0, p, 8, 1, p, 8, 1.0, 0.0, 1, None) == es.ES_ERR_ARG
    assert lib.es_gemm_bf16(8, 8, 12, p, 16, 0, p, 16, 1, p, 8, 1.0, 0.0, 1, None) == es.ES_ERR_ARG  # K % 8
    assert lib.es_gemm_bf16(8, 8, 8, p, 4, 0, p, 8, 1, p, 8, 1.0, 0.0, 1, None) == es.ES_ERR_ARG  # lda < K
    assert lib.es_sur_num_params(None) == es.ES_ERR_ARG


def test_fault_injection_switch_without_a_gpu(lib):
    """The allocation fault switch and the live-allocation count are host-side
    state: they answer without a device, and a failed call leaves the count
    where it was."""
    from paper_1705_04874_gb300 import es
    live = lib.es_debug_live_allocations()
    assert live >= 0
    lib.es_fault_inject_alloc(1)
    h = ctypes.c_void_p()
    assert lib.es_model_create(None, None, None, 32, 32, 32, 10.0, 6, ctypes.byref(h)) == es.ES_ERR_ARG
    lib.es_fault_inject_alloc(0)
    assert lib.es_debug_live_allocations() == live


def test_fft_plan_table_without_a_gpu(lib):
    """The plan table is host-side: every length of the binding's candidate list
    has its first candidate as the default for both pass kinds, every other
    candidate can be selected, and a length without a plan (among them the
    paper's 301 = 7 x 43) answers ES_ERR_SIZE."""
    from paper_1705_04874_gb300 import es
    ra, rb = ctypes.c_int(), ctypes.c_int()
    for n in range(1, 513):
        for kind in (0, 1):
            rc = lib.es_fft_plan(kind, n, ctypes.byref(ra), ctypes.byref(rb))
            if n in es.PLAN_CANDIDATES:
                assert rc == es.ES_OK and (ra.value, rb.value) == es.PLAN_CANDIDATES[n][0], n
                assert ra.value * rb.value == n
            else:
                assert rc == es.ES_ERR_SIZE, n
    for n, cands in es.PLAN_CANDIDATES.items():
        for kind in (0, 1):
            for c in cands[::-1]:
                assert lib.es_fft_plan_select(kind, n, *c) == es.ES_OK
                assert lib.es_fft_plan(kind, n, ctypes.byref(ra), ctypes.byref(rb)) == es.ES_OK
                assert (ra.value, rb.value) == c
            assert lib.es_fft_plan_select(kind, n, n, 1) == es.ES_ERR_SIZE
    assert lib.es_fft_plan_select(2, 64, 8, 8) == es.ES_ERR_ARG


def test_derivative_entry_points_check_alignment_without_a_gpu(lib):
    """es_derivative and es_laplacian refuse input or output arrays off a
    16-byte boundary (the passes move 8- and 16-byte vectors) before touching
    a device."""
    from paper_1705_04874_gb300 import es
    p, q = ctypes.c_void_p(0x10000), ctypes.c_void_p(0x20004)
    assert lib.es_derivative(p, 32, 32, 32, 0, ctypes.c_double(10.0), 1, q, None) == es.ES_ERR_ARG
    assert lib.es_derivative(q, 32, 32, 32, 0, ctypes.c_double(10.0), 1, p, None) == es.ES_ERR_ARG
    assert lib.es_laplacian(p, 32, 32, 32, ctypes.c_double(10.0), ctypes.c_double(10.0), ctypes.c_double(10.0),
                            q, None) == es.ES_ERR_ARG


def test_bounds_query_in_the_release_build(lib):
    """The release library checks no indexes: es_debug_bounds answers
    ES_ERR_STATE (ES_ERR_ARG for a null pointer) without touching a device."""
    from paper_1705_04874_gb300 import es
    v = ctypes.c_longlong(7)
    assert lib.es_debug_bounds(None) == es.ES_ERR_ARG
    assert lib.es_debug_bounds(ctypes.byref(v)) == es.ES_ERR_STATE
    assert v.value == 0


def test_traffic_record_matches_the_pass_kernels():
    """profiles/traffic.json (ncu DRAM bytes per pass launch, which bench.py
    reports as roofline.traffic) is keyed by the pass kernels' code; the
    committed record is that of the committed kernels."""
    import importlib.util
    import json
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    assert bench.kernel_code_hash().startswith(rec["kernel_code_sha256_prefix"])
    assert all(rec[f"256:{k}"] > 0 for k in ("vel-x", "vel-y", "vel-z", "str-x", "str-y", "str-z"))
