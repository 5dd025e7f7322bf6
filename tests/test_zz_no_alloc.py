"""es_superpose_noalloc: the superposition entry point for callers that cannot
allocate device memory (their memory is owned by their own pool allocator, or
cudaMalloc / cudaFree would synchronise a streaming pipeline).  Called
through the C ABI and checked against es_superpose on the same inputs, on two
calls in a row (the fixed scratch array carries the first call's contents
into the second).  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_1705_04874_gb300 import synth

pytestmark = pytest.mark.gpu



@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_04874_gb300 import es
    return es, es._load(), torch


def _call(lib, torch, tr, src, amps, t0s, dt, n_out, gather=None):
    n_src, _, n_rcv, nt = tr.shape
    if gather is None:
        gather = torch.full((4, n_rcv, n_out), 7.0, device="cuda")
    vp = ctypes.c_void_p
    rc = lib.es_superpose_noalloc(vp(tr.data_ptr()), n_src, n_rcv, nt, vp(src.data_ptr()), vp(amps.data_ptr()),
                                  vp(t0s.data_ptr()), src.numel(), float(dt), int(n_out), vp(gather.data_ptr()),
                                  vp(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return rc, gather


def _inputs(torch, seed, n_src, n_rcv, nt, n_ev, span):
    rng = synth.SplitMix64(seed)
    tr = rng.normal(n_src * 4 * n_rcv * nt).reshape(n_src, 4, n_rcv, nt).astype(np.float32)
    src, amps, t0s = synth.events(rng, n_ev, n_src, t_span=span)
    cu = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return cu(tr), cu(src), cu(amps), cu(t0s)


def test_noalloc_matches_es_superpose_twice(env):
    es, lib, torch = env
    dt = 1e-3
    for seed, (n_src, n_rcv, nt, n_ev, n_out) in ((5, (6, 9, 400, 300, 1100)), (6, (3, 4, 250, 17, 520))):
        tr, src, amps, t0s = _inputs(torch, seed, n_src, n_rcv, nt, n_ev, span=0.6)
        rc, got = _call(lib, torch, tr, src, amps, t0s, dt, n_out)
        assert rc == es.ES_OK
        ref = torch.empty((4, n_rcv, n_out), device="cuda")
        es.es_superpose(tr, src, amps, t0s, dt, n_out, gather=ref)
        # the same kernel and the same event shifts as es_superpose: equal bit for bit
        assert np.array_equal(got.cpu().numpy(), ref.cpu().numpy())


def test_noalloc_at_the_event_limit(env):
    """ES_NOALLOC_MAX_EVENTS events, more than fit in shared memory at once:
    equal to es_superpose bit for bit, on two calls in a row."""
    es, lib, torch = env
    n_ev = es.ES_NOALLOC_MAX_EVENTS
    tr, src, amps, t0s = _inputs(torch, 11, 8, 2, 300, n_ev, span=0.5)
    ref = torch.empty((4, 2, 900), device="cuda")
    es.es_superpose(tr, src, amps, t0s, 1e-3, 900, gather=ref)
    for _ in range(2):
        rc, got = _call(lib, torch, tr, src, amps, t0s, 1e-3, 900)
        assert rc == es.ES_OK
        assert np.array_equal(got.cpu().numpy(), ref.cpu().numpy())


def test_noalloc_rejects_bad_input_without_writing(env):
    es, lib, torch = env
    tr, src, amps, t0s = _inputs(torch, 7, 2, 3, 50, 10, span=0.05)
    bad = src.clone()
    bad[4] = 5  # only 2 sources
    rc, g = _call(lib, torch, tr, bad, amps, t0s, 1e-3, 80)
    assert rc == es.ES_ERR_ARG
    assert torch.all(g == 7.0)
    # host arrays are refused: this entry point takes device memory only
    host = np.zeros((4, 3, 80), np.float32)
    vp = ctypes.c_void_p
    rc = lib.es_superpose_noalloc(vp(tr.data_ptr()), 2, 3, 50, vp(src.data_ptr()), vp(amps.data_ptr()),
                                  vp(t0s.data_ptr()), 10, 1e-3, 80, vp(host.ctypes.data), None)
    assert rc == es.ES_ERR_ARG
    # beyond the fixed scratch size
    rc = lib.es_superpose_noalloc(vp(tr.data_ptr()), 2, 3, 50, vp(src.data_ptr()), vp(amps.data_ptr()),
                                  vp(t0s.data_ptr()), 65537, 1e-3, 80, vp(g.data_ptr()), None)
    assert rc == es.ES_ERR_ARG
