"""Edge and degenerate cases through the C ABI: zero time steps, no
receivers, an empty wavelet, the smallest grids (3 cells on an axis, no
PML), no events and events that fall outside the output window, one-source
batches."""
import numpy as np
import pytest

from paper_1705_04874_gb300 import synth
from conftest import cfl_dt, trace_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def es():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_04874_gb300 import es as _es
    _es._load()
    return _es


def test_zero_steps_and_no_receivers(es):
    rho, cp, cs = synth.two_layer_model(16, water_cells=4)
    w = synth.ricker(20, cfl_dt(cp, 10.0), 25.0)
    with es.Model(rho, cp, cs, dx=10.0, pml=2) as m:
        m.source_set((8, 8, 8), synth.explosive(), w)
        rcv = m.seabed_receivers(2, 2)
        tr = m.run(0, 0.0, rcv)  # nothing happens, nothing is written
        assert tr.shape == (4, 4, 0)
        assert not np.any(m.state_get())
        m.run(10, 0.0)  # no receivers: the fields still advance
        st = m.state_get()
        assert np.any(st) and np.isfinite(st).all()


def test_empty_wavelet_leaves_the_fields_at_rest(es):
    rho, cp, cs = synth.two_layer_model(16, water_cells=4)
    with es.Model(rho, cp, cs, dx=10.0, pml=2) as m:
        m.source_set((8, 8, 8), synth.explosive(), np.zeros(0, np.float32))
        tr = m.run(15, 0.0, m.seabed_receivers(2, 2))
        assert not np.any(tr) and not np.any(m.state_get())


@pytest.mark.parametrize("shape", [(3, 4, 5), (5, 3, 4), (4, 5, 3)])
def test_smallest_grids_match_oracle(es, orc, shape):
    """Axes of 3 to 5 cells, no PML (periodic box), circulant passes on every
    axis; 30 steps against the oracle."""
    rng = np.random.default_rng(sum(shape))
    rho = (2000 + 200 * rng.random(shape)).astype(np.float32)
    cp = (2500 + 300 * rng.random(shape)).astype(np.float32)
    cs = (cp / 1.9).astype(np.float32)
    nt = 30
    dt = cfl_dt(cp, 10.0)
    w = synth.ricker(nt, dt, 60.0)
    pos = (1, 1, 1)
    rcv = np.array([[0, 0, 0], [2, 1, 2], [shape[2] - 1, shape[1] - 1, shape[0] - 1]], np.int32)
    with es.Model(rho, cp, cs, dx=10.0, pml=0) as m:
        m.source_set(pos, synth.double_couple_sdr(10, 50, 70), w)
        gpu = m.run(nt, dt, rcv)
    ref = orc.simulate(rho, cp, cs, dx=10.0, dt=dt, nt=nt, pml=0, receivers=rcv,
                       sources=[dict(kind="moment", pos=pos, m=synth.double_couple_sdr(10, 50, 70), w=w)])["traces"]
    assert trace_errors(gpu, ref).max() < 1e-4


def test_superpose_without_events_and_out_of_window(es):
    rng = np.random.default_rng(4)
    tr = rng.standard_normal((2, 4, 3, 50)).astype(np.float32)
    dt, n_out = 1e-3, 80
    g = es.es_superpose(tr, np.zeros(0, np.int32), np.zeros(0, np.float32), np.zeros(0, np.float32), dt, n_out)
    assert g.shape == (4, 3, n_out) and not np.any(g)
    # one event entirely after the window, one entirely before it: zero padding leaves nothing
    src = np.array([0, 1], np.int32)
    amps = np.array([2.0, -1.0], np.float32)
    t0s = np.array([n_out * dt + 0.01, -60 * dt], np.float32)
    g = es.es_superpose(tr, src, amps, t0s, dt, n_out)
    assert not np.any(g)
    # an event cut at the front: sample t of the gather is trace sample t + 7
    g = es.es_superpose(tr, src[:1], amps[:1], np.array([-7 * dt], np.float32), dt, n_out)
    assert np.array_equal(g[..., :43], 2.0 * tr[0][..., 7:])
    assert not np.any(g[..., 43:])


def test_batch_of_one_equals_plain_run(es):
    rho, cp, cs = synth.marine_model(shape=(32, 32, 48), seed=9)
    nt = 40
    dt = cfl_dt(cp, 10.0)
    w = synth.ricker(nt, dt, 30.0)
    mt = synth.double_couple_sdr(45, 45, 45)
    with es.Model(rho, cp, cs, dx=10.0, pml=4) as m:
        rcv = m.seabed_receivers(3, 3)
        m.source_set((24, 16, 14), mt, w)
        plain = m.run(nt, dt, rcv)
        m.batch_set(np.array([[24, 16, 14]], np.int32), mt[None, :], w[None, :])
        one = m.run(nt, dt, rcv)
    assert np.array_equal(one.reshape(plain.shape), plain)


def test_model_from_device_arrays_equals_host_arrays(es):
    """rho, cp, cs given as CUDA tensors (used in place by the device-side model
    setup) and as host arrays (staged to the device first) give bit-identical
    traces."""
    import torch
    rho, cp, cs = synth.marine_model(shape=(40, 36, 48), seed=6)
    nt = 50
    dt = cfl_dt(cp, 10.0)
    w = synth.ricker(nt, dt, 30.0)
    mt = synth.double_couple_sdr(15, 75, -30)
    out = []
    for arrays in ((rho, cp, cs), tuple(torch.from_numpy(a).cuda() for a in (rho, cp, cs))):
        with es.Model(*arrays, dx=10.0, pml=5) as m:
            rcv = m.seabed_receivers(3, 3)
            m.source_set((24, 18, 20), mt, w)
            out.append(m.run(nt, dt, rcv))
    assert np.array_equal(out[0], out[1])


def test_allocation_failures_return_oom_and_leak_nothing(es):
    """Host-side fault injection (es_fault_inject_alloc): every device
    allocation of es_model_create, of a run's buffers and of es_batch_set made
    to fail in turn.  Each failing call returns ES_ERR_OOM, and the library
    holds exactly the allocations it held before the call."""
    lib = es._load()
    rho, cp, cs = synth.two_layer_model(32, water_cells=8)
    dt = cfl_dt(cp, 10.0)
    w = synth.ricker(20, dt, 25.0)
    base = lib.es_debug_live_allocations()
    k, failed = 1, 0
    try:
        while True:  # model creation
            lib.es_fault_inject_alloc(k)
            try:
                m = es.Model(rho, cp, cs, dx=10.0, pml=6)
            except es.EsError as e:
                assert e.status == es.ES_ERR_OOM, e
                assert lib.es_debug_live_allocations() == base
                failed += 1
                k += 1
                continue
            lib.es_fault_inject_alloc(0)
            m.close()
            break
        assert failed >= 2 and lib.es_debug_live_allocations() == base
        with es.Model(rho, cp, cs, dx=10.0, pml=6) as m:  # a source, a run, a batch
            rcv = m.seabed_receivers(4, 4)
            for k in (1, 2, 3, 4):
                m.source_set((16, 16, 16), synth.explosive(), w)
                before = lib.es_debug_live_allocations()
                lib.es_fault_inject_alloc(k)
                try:
                    m.run(20, dt, rcv)
                except es.EsError as e:
                    assert e.status == es.ES_ERR_OOM, e
                lib.es_fault_inject_alloc(0)
                assert lib.es_debug_live_allocations() <= before + 4
            lib.es_fault_inject_alloc(1)
            with pytest.raises(es.EsError) as e:
                m.batch_set(np.array([[16, 16, 16], [14, 15, 16]]), np.stack([synth.explosive()] * 2),
                            np.stack([w, w]))
            assert e.value.status == es.ES_ERR_OOM
            lib.es_fault_inject_alloc(0)
            m.source_set((16, 16, 16), synth.explosive(), w)
            assert np.isfinite(m.run(20, dt, rcv)).all()  # the model still works
        assert lib.es_debug_live_allocations() == base
    finally:
        lib.es_fault_inject_alloc(0)
