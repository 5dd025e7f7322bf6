"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same
seeded inputs.  Floating point: per-trace relative L2 <= 1e-4 with a floor
of 1e-3 of the largest trace of the component for near-zero traces;
integer maps bit-exact; linearity identities bit-exact."""
import numpy as np
import pytest

from paper_1705_04874_gb300 import synth
from conftest import cfl_dt, rel_l2, trace_errors

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def es():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_04874_gb300 import es as _es
    _es._load()
    return _es


# --------------------------------------------------------------------------
# one derivative pass (Sec. II-A spectral derivative, staggered)
# --------------------------------------------------------------------------
SHAPES = [(32, 32, 32), (48, 64, 96), (16, 80, 48), (96, 16, 160), (64, 48, 16), (32, 192, 256),
          (256, 32, 128)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("shift", [+1, -1])
def test_derivative_matches_oracle(es, orc, shape, axis, shift):
    import torch
    rng = np.random.default_rng(hash((shape, axis, shift)) % 2 ** 32)
    f = rng.standard_normal(shape).astype(np.float32)
    d = [10.0, 12.5, 7.5][axis]
    ref = orc.deriv(f.astype(np.float64), axis, d, shift)
    ft = torch.from_numpy(f).cuda()
    out = torch.empty_like(ft)
    es.es_derivative(ft, axis, d, shift, out)
    got = out.cpu().numpy().astype(np.float64)
    assert rel_l2(got, ref) < 2e-6
    assert np.abs(got - ref).max() < 2e-5 * np.abs(ref).max()


def test_derivative_of_nyquist_and_smooth_modes(es):
    import torch
    n, d = 64, 10.0
    x = np.arange(n)
    shape = (16, 32, n)
    for m in (1, 7, 31, 32):
        f = np.broadcast_to(np.cos(2 * np.pi * m * x / n + 0.3), shape).astype(np.float32).copy()
        out = torch.empty(shape, device="cuda")
        es.es_derivative(torch.from_numpy(f).cuda(), 0, d, +1, out)
        k = 2 * np.pi * m / (n * d)
        if 2 * m == n:
            ex = -(np.pi / d) * np.cos(np.pi * x + 0.3)
        else:
            ex = -k * np.sin(k * (x + 0.5) * d + 0.3)
        got = out.cpu().numpy()[3, 5]
        assert np.abs(got - ex).max() < 3e-6 * max(k, np.pi / d)


# --------------------------------------------------------------------------
# full runs: materials, PML, sources, recording
# --------------------------------------------------------------------------

def _run_both(es, orc, rho, cp, cs, *, pml, nt, sources, rcv, d=(10.0, 10.0, 10.0), dt=None, alpha0=2.0,
              prec=0):
    dt = cfl_dt(cp, min(d)) if dt is None else dt
    with es.Model(rho, cp, cs, dx=d[0], pml=pml) as m:
        if prec:
            m.set_precision(prec)
        if d[1] != d[0] or d[2] != d[0]:
            m.set_spacing(*d)
        m.set_pml(alpha0, 0.0)
        for s in sources:
            if s["kind"] == "moment":
                m.source_add(s["pos"], s["m"], s["w"])
            else:
                m.source_add_force(s["pos"], s["m"], s["w"])
        gpu = m.run(nt, dt, rcv)
    ref = orc.simulate(rho, cp, cs, dx=d[0], dy=d[1], dz=d[2], dt=dt, nt=nt, pml=pml,
                       pml_alpha0=alpha0, sources=sources, receivers=rcv)["traces"]
    return gpu, ref


def test_config1_two_layer_explosive(es, orc):
    """32^3 incl. 6-cell PML, water over rock, explosive at the centre, Ricker
    25 Hz, CFL 0.3, 300 steps, 16 seabed receivers."""
    rho, cp, cs = synth.two_layer_model(32, water_cells=8)
    dt = cfl_dt(cp, 10.0)
    nt = 300
    w = synth.ricker(nt, dt, 25.0)
    with es.Model(rho, cp, cs, dx=10.0, pml=6) as m:
        rcv = m.seabed_receivers(4, 4)
    assert np.array_equal(rcv, orc.seabed_receivers(cs, 6, 4, 4))
    src = [dict(kind="moment", pos=(16, 16, 16), m=synth.explosive(), w=w)]
    gpu, ref = _run_both(es, orc, rho, cp, cs, pml=6, nt=nt, sources=src, rcv=rcv)
    err = trace_errors(gpu, ref)
    assert err.max() < TOL, err.max()


def test_marine_dc_and_force_uneven_grid(es, orc):
    _marine_dc_and_force(es, orc, 0)


def _marine_dc_and_force(es, orc, prec):
    shape = (48, 64, 96)
    rho, cp, cs = synth.marine_model(shape=shape, seed=1)
    nt = 220
    dt = cfl_dt(cp, 10.0)
    w = synth.ricker(nt, dt, 30.0)
    with es.Model(rho, cp, cs, dx=10.0, pml=8) as m:
        rcv = m.seabed_receivers(6, 5)
    assert np.array_equal(rcv, orc.seabed_receivers(cs, 8, 6, 5))
    src = [dict(kind="moment", pos=(40, 30, 25), m=synth.double_couple_sdr(30, 60, 90), w=w),
           dict(kind="force", pos=(55, 33, 28), m=(0.2, -1.0, 0.4), w=w * 1e7)]
    gpu, ref = _run_both(es, orc, rho, cp, cs, pml=8, nt=nt, sources=src, rcv=rcv, prec=prec)
    err = trace_errors(gpu, ref)
    assert err.max() < TOL, err.max()
    return err


# The two long heterogeneous runs again with compensated derivative arithmetic
# (es_model_set_precision, every axis through the error-free circulant pass).
def test_compensated_marine_dc_and_force_meets_1e4(es, orc):
    _marine_dc_and_force(es, orc, es.ES_PREC_COMPENSATED)


def test_compensated_anisotropic_meets_1e4(es, orc):
    _anisotropic(es, orc, es.ES_PREC_COMPENSATED)


def test_precision_mode_checked(es):
    rho, cp, cs = synth.two_layer_model(16, water_cells=4)
    with es.Model(rho, cp, cs, dx=10.0, pml=2) as m:
        with pytest.raises(es.EsError) as e:
            m.set_precision(3)
        assert e.value.status == es.ES_ERR_ARG


def test_anisotropic_spacing_and_pml_strength(es, orc):
    _anisotropic(es, orc, 0)


def _anisotropic(es, orc, prec):
    shape = (80, 32, 64)
    rho, cp, cs = synth.marine_model(shape=shape, seed=3)
    nt = 160
    d = (12.5, 12.5, 10.0)
    dt = cfl_dt(cp, 10.0)
    w = synth.ricker(nt, dt, 20.0)
    rcv = orc.seabed_receivers(cs, 5, 4, 4)
    src = [dict(kind="moment", pos=(30, 15, 40), m=synth.clvd(), w=w)]
    gpu, ref = _run_both(es, orc, rho, cp, cs, pml=5, nt=nt, sources=src, rcv=rcv, d=d, alpha0=3.0, prec=prec)
    err = trace_errors(gpu, ref)
    assert err.max() < TOL, err.max()
    return err


def test_no_pml_and_thin_pml(es, orc):
    rho, cp, cs = synth.two_layer_model(shape=(32, 48, 32), water_cells=6)
    nt = 120
    dt = cfl_dt(cp, 10.0)
    w = synth.ricker(nt, dt, 30.0)
    rcv = orc.seabed_receivers(cs, 0, 3, 3)
    for pml in (0, 1):
        src = [dict(kind="moment", pos=(12, 20, 14), m=synth.double_couple_xy(), w=w)]
        gpu, ref = _run_both(es, orc, rho, cp, cs, pml=pml, nt=nt, sources=src, rcv=rcv)
        assert trace_errors(gpu, ref).max() < TOL, pml


def test_state_roundtrip_and_continuation(es):
    rho, cp, cs = synth.two_layer_model(shape=(32, 32, 48), water_cells=6)
    nt = 50
    dt = cfl_dt(cp, 10.0)
    w = synth.ricker(2 * nt, dt, 30.0)
    with es.Model(rho, cp, cs, dx=10.0, pml=4) as m:
        rcv = m.seabed_receivers(2, 2)
        m.source_set((20, 16, 16), synth.explosive(), w)
        whole = m.run(2 * nt, dt, rcv)
        m.state_reset()
        a = m.run(nt, dt, rcv)
        b = m.run(nt, dt, rcv)
        assert np.array_equal(np.concatenate([a, b], axis=-1), whole)
        st = m.state_get()
        m.state_set(st)
        assert np.array_equal(m.state_get(), st)


def test_plane_wave_closed_form_on_gpu(es):
    """P plane wave along x with PML off: sigma^n = sigma^0 (cos n th - tan(th/2) sin n th),
    sin(th/2) = cp kappa dt / 2."""
    shape = (16, 16, 32)
    RHO, CP, CS = 2000.0, 3000.0, 1700.0
    rho, cp, cs = synth.homogeneous_model(shape, RHO, CP, CS)
    lam, mu = RHO * (CP ** 2 - 2 * CS ** 2), RHO * CS ** 2
    k = 2 * np.pi * 3 / (32 * 10.0)
    x = np.arange(32) * 10.0
    st = np.zeros((9,) + shape, np.float32)
    st[3] = (lam + 2 * mu) * 1e-6 * np.cos(k * x)
    st[4] = lam * 1e-6 * np.cos(k * x)
    st[5] = st[4]
    dt = 0.3 * 10.0 / CP
    nt = 101
    with es.Model(rho, cp, cs, dx=10.0, pml=0) as m:
        m.state_set(st)
        m.run(nt, dt)
        out = m.state_get()
    th = 2 * np.arcsin(CP * k * dt / 2)
    fac = np.cos(nt * th) - np.tan(th / 2) * np.sin(nt * th)
    for f in (3, 4, 5):
        assert np.abs(out[f] - fac * st[f]).max() < 1e-5 * np.abs(st[3]).max()


def test_linearity_exact_on_gpu(es):
    rho, cp, cs = synth.marine_model(shape=(32, 32, 64), seed=7)
    nt = 80
    dt = cfl_dt(cp, 10.0)
    w = synth.ricker(nt, dt, 30.0)
    mt = synth.double_couple_sdr(10, 80, 30)
    k = 13
    with es.Model(rho, cp, cs, dx=10.0, pml=5) as m:
        rcv = m.seabed_receivers(3, 3)
        m.source_set((30, 16, 16), mt, w)
        base = m.run(nt, dt, rcv)
        m.state_reset()
        m.source_set((30, 16, 16), mt, (2.0 * w).astype(np.float32))
        twice = m.run(nt, dt, rcv)
        m.state_reset()
        wd = np.concatenate([np.zeros(k, np.float32), w])[:nt]
        m.source_set((30, 16, 16), mt, wd)
        late = m.run(nt, dt, rcv)
    assert np.array_equal(twice, 2.0 * base)
    assert np.array_equal(late[..., k:], base[..., :nt - k])
    assert np.all(late[..., :k] == 0)


def test_errors_are_reported(es):
    rho, cp, cs = synth.two_layer_model(32, water_cells=8)
    w = synth.ricker(10, 1e-3, 25.0)
    with es.Model(rho, cp, cs, dx=10.0, pml=6) as m:
        with pytest.raises(es.EsError) as e:
            m.source_set((3, 16, 16), synth.explosive(), w)  # inside the PML
        assert e.value.status == es.ES_ERR_ARG
        with pytest.raises(es.EsError) as e:
            m.run(5, 0.01)  # far beyond the stability limit
        assert e.value.status == es.ES_ERR_UNSTABLE
        with pytest.raises(es.EsError) as e:
            m.run(5, 0.0, np.array([[40, 1, 1]], np.int32))
        assert e.value.status == es.ES_ERR_ARG
        bad = w.copy()
        bad[3] = np.nan
        m.source_set((16, 16, 16), synth.explosive(), bad)
        with pytest.raises(es.EsError) as e:
            m.run(10, 0.0)
        assert e.value.status == es.ES_ERR_UNSTABLE
    with pytest.raises(es.EsError) as e:
        es.Model(*synth.two_layer_model(shape=(32, 32, 520)), dx=10.0, pml=4)
    assert e.value.status == es.ES_ERR_SIZE


# --------------------------------------------------------------------------
# superposition (Sec. IV)
# --------------------------------------------------------------------------

def test_superpose_golden_and_random(es, orc):
    import json, os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "superpose_small.json")))
    tr = np.array(g["traces"], np.float32)
    got = es.es_superpose(tr, np.array(g["src_of_event"], np.int32), np.array(g["amps"], np.float32),
                          np.array(g["t0s"], np.float32), g["dt"], g["n_out"])
    assert np.array_equal(got, np.array(g["expected"], np.float32))
    rng = synth.SplitMix64(3)
    tr = rng.normal(5 * 4 * 7 * 300).reshape(5, 4, 7, 300).astype(np.float32)
    src, amps, t0s = synth.events(rng, 60, 5, t_span=0.6)
    dt = 1e-3
    got = es.es_superpose(tr, src, amps, t0s, dt, 900)
    ref = orc.superpose(tr.astype(np.float64), src, amps.astype(np.float64),
                        t0s.astype(np.float64), dt, 900)
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()


def test_superpose_device_buffers(es):
    import torch
    rng = np.random.default_rng(0)
    tr = rng.standard_normal((3, 4, 2, 50)).astype(np.float32)
    src = np.array([0, 2, 1, 2], np.int32)
    amps = np.array([1.0, -0.5, 2.0, 0.25], np.float32)
    t0 = np.array([0.0, 0.01, -0.005, 0.049], np.float32)
    host = es.es_superpose(tr, src, amps, t0, 1e-3, 120)
    out = torch.empty((4, 2, 120), device="cuda")
    es.es_superpose(torch.from_numpy(tr).cuda(), torch.from_numpy(src).cuda(), torch.from_numpy(amps).cuda(),
                    torch.from_numpy(t0).cuda(), 1e-3, 120, gather=out)
    assert np.array_equal(out.cpu().numpy(), host)


# --------------------------------------------------------------------------
# smoothed point sources (Sec. II-A: Blackman window in the spatial-frequency domain)
# --------------------------------------------------------------------------

def _run_smoothed(es, orc, rho, cp, cs, *, pml, nt, src, rcv):
    dt = cfl_dt(cp, 10.0)
    with es.Model(rho, cp, cs, dx=10.0, pml=pml) as m:
        for s in src:
            if s.get("smooth"):
                m.source_add_smoothed(s["pos"], s["m"], s["w"])
            else:
                m.source_add(s["pos"], s["m"], s["w"])
        gpu = m.run(nt, dt, rcv)
        st = m.state_get()
    ref = orc.simulate(rho, cp, cs, dx=10.0, dt=dt, nt=nt, pml=pml, sources=src, receivers=rcv,
                       state=np.zeros((9,) + rho.shape))
    return gpu, st, ref


def test_smoothed_source_matches_oracle(es, orc):
    """Double couple smoothed over the 5 x 5 x 5 Blackman stencil plus a
    point explosion, 32^3 water over rock, 150 steps."""
    rho, cp, cs = synth.two_layer_model(32, water_cells=8)
    nt = 150
    w = synth.ricker(nt, cfl_dt(cp, 10.0), 25.0)
    rcv = orc.seabed_receivers(cs, 6, 4, 4)
    src = [dict(kind="moment", pos=(15, 17, 18), m=synth.double_couple_sdr(30, 60, 90), w=w, smooth=True),
           dict(kind="moment", pos=(20, 12, 22), m=synth.explosive(0.5), w=w)]
    gpu, st, ref = _run_smoothed(es, orc, rho, cp, cs, pml=6, nt=nt, src=src, rcv=rcv)
    err = trace_errors(gpu, ref["traces"])
    assert err.max() < TOL, err.max()
    for f in range(9):
        assert rel_l2(st[f], ref["state"][f]) < TOL, f


def test_initial_value_source_matches_oracle(es, orc):
    """The paper's initial-value form: a smoothed stress distribution set at
    the first step (wavelet = [1]) on an odd 27 x 30 x 33 grid."""
    rho, cp, cs = synth.two_layer_model(shape=(27, 30, 33), water_cells=6)
    rcv = orc.seabed_receivers(cs, 4, 3, 3)
    src = [dict(kind="moment", pos=(16, 15, 15), m=synth.explosive(), w=np.ones(1, np.float32), smooth=True)]
    gpu, st, ref = _run_smoothed(es, orc, rho, cp, cs, pml=4, nt=80, src=src, rcv=rcv)
    err = trace_errors(gpu, ref["traces"])
    assert err.max() < TOL, err.max()
    for f in range(9):
        assert rel_l2(st[f], ref["state"][f]) < TOL, f


def test_smoothed_source_must_clear_the_pml(es):
    rho, cp, cs = synth.two_layer_model(32, water_cells=8)
    w = np.ones(4, np.float32)
    with es.Model(rho, cp, cs, dx=10.0, pml=6) as m:
        m.source_add((8, 16, 16), synth.explosive(), w)            # a point source fits at pml + 2
        with pytest.raises(es.EsError) as e:
            m.source_add_smoothed((7, 16, 16), synth.explosive(), w)  # its stencil would reach x = 5
        assert e.value.status == es.ES_ERR_ARG
        m.source_add_smoothed((8, 16, 16), synth.explosive(), w)


def test_fused_sources_and_receivers_equal_the_separate_kernels(es, orc):
    """With every axis on the FFT passes, point sources are injected and the
    receivers recorded inside the passes (6 launches per step).  A smoothed
    source of zero moment adds nothing but sends the run through the separate
    injection and recording kernels (8 + 1 launches): traces and final state
    agree bit for bit.  Two moment sources share a cell (their order matters),
    a receiver sits on a source cell, and a point force is present; the fused
    run also matches the oracle."""
    shape = (32, 48, 64)
    rho, cp, cs = synth.marine_model(shape=shape, seed=7)
    dt = cfl_dt(cp, 10.0)
    nt = 90
    w = synth.ricker(nt, dt, 30.0)
    srcs = [dict(kind="moment", pos=(30, 20, 15), m=synth.double_couple_sdr(30, 60, 90), w=w),
            dict(kind="moment", pos=(30, 20, 15), m=synth.clvd(), w=0.5 * w),
            dict(kind="force", pos=(40, 28, 17), m=(0.2, -1.0, 0.4), w=w * 1e7)]
    with es.Model(rho, cp, cs, dx=10.0, pml=5) as m:
        rcv = np.concatenate([m.seabed_receivers(4, 3), np.array([[30, 20, 15]], np.int32)])
        out = []
        for extra in (False, True):
            m.state_reset()
            m.source_clear()
            for s in srcs:
                if s["kind"] == "moment":
                    m.source_add(s["pos"], s["m"], s["w"])
                else:
                    m.source_add_force(s["pos"], s["m"], s["w"])
            if extra:
                m.source_add_smoothed((32, 24, 16), np.zeros(6), w)
            assert m.kernels_per_step() == (9 if extra else 6)
            out.append((m.run(nt, dt, rcv), m.state_get()))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    ref = orc.simulate(rho, cp, cs, dx=10.0, dt=dt, nt=nt, pml=5, sources=srcs, receivers=rcv)["traces"]
    assert trace_errors(out[0][0], ref).max() < TOL


def test_fused_batch_equals_separate_kernels(es):
    """A batch of moment sources on FFT axes (fused) against the same batch
    run one source at a time with a zero smoothed source beside it (the
    separate kernels): equal bit for bit."""
    shape = (32, 32, 48)
    rho, cp, cs = synth.marine_model(shape=shape, seed=8)
    dt, nt = cfl_dt(cp, 10.0), 60
    rng = synth.SplitMix64(5)
    box = synth.reservoir_box(shape, 4)
    pos = synth.random_positions(rng, box, 3)
    mts = np.array([synth.random_dc(rng) for _ in range(3)])
    wav = np.stack([synth.ricker(nt, dt, 30.0)] * 3)
    with es.Model(rho, cp, cs, dx=10.0, pml=4) as m:
        rcv = m.seabed_receivers(3, 3)
        m.batch_set(pos, mts, wav)
        assert m.kernels_per_step() == 6
        batched = m.run(nt, dt, rcv)
    for b in range(3):
        with es.Model(rho, cp, cs, dx=10.0, pml=4) as m1:
            m1.source_set(pos[b], mts[b], wav[b])
            m1.source_add_smoothed((24, 16, 10), np.zeros(6), wav[b])
            assert m1.kernels_per_step() == 8
            assert np.array_equal(m1.run(nt, dt, rcv), batched[b]), b
