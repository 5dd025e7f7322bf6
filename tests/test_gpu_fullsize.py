"""Parity at the benchmark's full grid sizes, in the launch configuration the
benchmark times (es_run and es_run_group through the C ABI): 128^3 and 256^3
marine models, and the batched group of 64 + 16 + 8 sources on 128^3, 96^3
and 160^3.
Every trace of the 128^3 configuration over its full 2000 steps and of the
256^3 configuration over its first 400 steps against the oracle; whole field
states after a few steps; and properties that hold at any length (exact
linearity and delay, receiver maps, energy conservation with the PML off) over
longer runs on the GPU alone."""
import numpy as np
import pytest

from paper_1705_04874_gb300 import synth
from conftest import cfl_dt, rel_l2, trace_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def es():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_04874_gb300 import es as _es
    _es._load()
    return _es


def _field_parity(es, orc, n, pml, mt, nt, seed, rx):
    rho, cp, cs = synth.marine_model(n, seed=seed)
    dt = cfl_dt(cp, 10.0)
    box = synth.reservoir_box((n, n, n), pml)
    pos = tuple((lo + hi) // 2 for lo, hi in box)
    w = synth.ricker(nt, dt, 30.0, t0=4 * dt)
    with es.Model(rho, cp, cs, dx=10.0, pml=pml) as m:
        rcv = m.seabed_receivers(rx, rx)
        m.source_set(pos, mt, w)
        traces = m.run(nt, dt, rcv)
        st = m.state_get()
    assert np.array_equal(rcv, orc.seabed_receivers(cs, pml, rx, rx))
    ref = orc.simulate(rho, cp, cs, dx=10.0, dt=dt, nt=nt, pml=pml,
                       sources=[dict(kind="moment", pos=pos, m=mt, w=w)], receivers=rcv,
                       state=np.zeros((9, n, n, n)))
    for f in range(9):
        assert rel_l2(st[f], ref["state"][f]) < 1e-4, f
    assert np.isfinite(traces).all()


def test_marine_128_field_parity(es, orc):
    """128^3 marine model, PML 10, double couple (strike 30, dip 60, rake 90)
    at the reservoir-box centre, 32 x 32 seabed receivers."""
    _field_parity(es, orc, 128, 10, synth.double_couple_sdr(30, 60, 90), 60, 1, 32)


def test_marine_256_field_parity(es, orc):
    """256^3 marine model, PML 12, random strike/dip/rake double couple,
    64 x 64 seabed receivers: the benchmark's grid and launch configuration."""
    mt = synth.random_dc(synth.SplitMix64(2))
    _field_parity(es, orc, 256, 12, mt, 10, 1, 64)


def _bench_trace_parity(es, orc, name, nt):
    """Every trace of a benchmarked configuration (bench.py's own inputs and
    receivers, es_run as the benchmark calls it) against the oracle, per
    trace within 1e-4 (floor 1e-3 of the component's largest trace)."""
    import bench
    w = bench.workload(name)
    inp = bench.build_inputs(w)
    with es.Model(inp["rho"], inp["cp"], inp["cs"], dx=10.0, pml=w["pml"]) as m:
        rcv = m.seabed_receivers(w["rx"], w["rx"])
        m.source_set(inp["pos"], inp["mt"], inp["wav"][:nt])
        gpu = m.run(nt, inp["dt"], rcv)
    ref = orc.simulate(inp["rho"], inp["cp"], inp["cs"], dx=10.0, dt=inp["dt"], nt=nt, pml=w["pml"],
                       sources=[dict(kind="moment", pos=inp["pos"], m=inp["mt"], w=inp["wav"][:nt])],
                       receivers=rcv)["traces"]
    err = trace_errors(gpu, ref)
    assert err.max() < 1e-4, (np.median(err), err.max())
    return err


def test_c2_traces_full_length(es, orc):
    """The 128^3 benchmark configuration (marine model, PML 10, DC strike 30
    dip 60 rake 90, Ricker 30 Hz, 32 x 32 seabed receivers) for all 2000
    steps: all 1024 4C traces (about 200 s of oracle time on 16 cores)."""
    _bench_trace_parity(es, orc, "128", 2000)


def test_c3_traces_first_400_steps(es, orc):
    """The 256^3 benchmark configuration (PML 12, random double couple in the
    reservoir box, 64 x 64 seabed receivers) for its first 400 steps, by which
    the P and S arrivals have crossed the seabed: all 4096 4C traces (about
    360 s of oracle time on 16 cores)."""
    _bench_trace_parity(es, orc, "256", 400)


def test_marine_256_linearity_over_many_steps(es):
    n, pml, nt = 256, 12, 400
    rho, cp, cs = synth.marine_model(n, seed=1)
    dt = cfl_dt(cp, 10.0)
    mt = synth.random_dc(synth.SplitMix64(2))
    box = synth.reservoir_box((n, n, n), pml)
    pos = tuple((lo + hi) // 2 for lo, hi in box)
    w = synth.ricker(nt, dt, 30.0)
    k = 37
    with es.Model(rho, cp, cs, dx=10.0, pml=pml) as m:
        rcv = m.seabed_receivers(64, 64)
        m.source_set(pos, mt, w)
        a = m.run(nt, dt, rcv)
        m.state_reset()
        m.source_set(pos, mt, (2 * w).astype(np.float32))
        b = m.run(nt, dt, rcv)
        m.state_reset()
        m.source_set(pos, mt, np.concatenate([np.zeros(k, np.float32), w])[:nt])
        c = m.run(nt, dt, rcv)
    assert np.abs(a).max() > 0
    # Doubling the source doubles every operation's result exactly in binary
    # floating point, except where an intermediate falls below FP32's normal
    # range (2^-126), where rounding is absolute: the spectral derivative
    # reaches every cell after the first step, so the earliest samples far
    # from the source pass through such values.  Bit-exact wherever the trace
    # is above 2^-90; below it, equal to within 2^-100.
    big = np.abs(a) >= 2.0 ** -90
    assert big.sum() > 0.9 * a.size
    assert np.array_equal(b[big], 2 * a[big])
    assert np.abs(b.astype(np.float64) - 2 * a.astype(np.float64)).max() <= 2.0 ** -100
    # a delayed source repeats the same operations on the same values: exact
    assert np.array_equal(c[..., k:], a[..., :nt - k])


def _energy(orc_mats, prev, cur):
    """Discrete energy at step n from the states at n and n+1 (v^{n-1/2},
    sigma^n and v^{n+1/2}), PML off."""
    lam, mu = orc_mats["lam"], orc_mats["mu"]
    e = 0.0
    for c, b in enumerate(("bx", "by", "bz")):
        e += 0.5 * np.sum(prev[c].astype(np.float64) * cur[c] / orc_mats[b])
    s = prev[3:].astype(np.float64)
    tr = s[0] + s[1] + s[2]
    solid = mu > 0
    with np.errstate(divide="ignore", invalid="ignore"):
        en = np.where(solid, (s[0] ** 2 + s[1] ** 2 + s[2] ** 2) / (2 * mu)
                      - lam / (2 * mu * (3 * lam + 2 * mu)) * tr ** 2, (tr / 3) ** 2 / lam)
    e += 0.5 * np.sum(en)
    for c, name in enumerate(("muxy", "muxz", "muyz")):
        me = orc_mats[name]
        with np.errstate(divide="ignore", invalid="ignore"):
            e += 0.5 * np.sum(np.where(me > 0, s[3 + c] ** 2 / me, 0.0))
    return e


def test_energy_conserved_without_pml_128(es, orc):
    n = 128
    rho, cp, cs = synth.marine_model(n, seed=4)
    dt = cfl_dt(cp, 10.0)
    nw = 120
    w = synth.ricker(nw, dt, 30.0)
    mats = orc.materials(rho, cp, cs)
    with es.Model(rho, cp, cs, dx=10.0, pml=0) as m:
        m.source_set((64, 64, 60), synth.double_couple_sdr(45, 50, 10), w)
        m.run(nw + 10, dt)
        es_ = []
        for _ in range(3):
            s0 = m.state_get()
            m.run(1, dt)
            s1 = m.state_get()
            es_.append(_energy(mats, s0, s1))
            m.run(300, dt)
    es_ = np.array(es_)
    assert es_.min() > 0
    assert (es_.max() - es_.min()) / es_.max() < 2e-4, es_


def test_batched_group_full_size(es, orc):
    """The batched workload as the benchmark runs it: 64 sources on the 128^3
    marine model, 16 on 96^3 and 8 on 160^3 (random double couples in the
    reservoir boxes, Ricker 30 Hz), 32 x 32 seabed receivers each, all in one
    graph through es_run_group, 200 steps.  Sampled simulations of every model
    equal single-source runs bit for bit (same kernels, same arithmetic), and
    the first simulation on 96^3 matches the oracle over all 200 samples."""
    nt = 200
    specs = [(128, 10, 64), (96, 8, 16), (160, 10, 8)]
    models, rcvs, dts, inputs = [], [], [], []
    try:
        for i, (n, pml, nb) in enumerate(specs):
            rho, cp, cs = synth.marine_model(n, seed=1)
            dt = 0.3 * 10.0 / float(cp.max())
            rng = synth.SplitMix64(40 + i)
            box = synth.reservoir_box((n, n, n), pml)
            pos = synth.random_positions(rng, box, nb)
            mts = np.array([synth.random_dc(rng) for _ in range(nb)])
            wav = np.stack([synth.ricker(nt, dt, 30.0)] * nb)
            m = es.Model(rho, cp, cs, dx=10.0, pml=pml)
            rcv = m.seabed_receivers(32, 32)
            m.batch_set(pos, mts, wav)
            models.append(m)
            rcvs.append(rcv)
            dts.append(dt)
            inputs.append((rho, cp, cs, pml, pos, mts, wav))
        got = es.es_run_group(models, nt, dts, rcvs)
    finally:
        for m in models:
            m.close()
    for i, b in [(0, 0), (0, 63), (1, 15), (2, 7)]:
        rho, cp, cs, pml, pos, mts, wav = inputs[i]
        with es.Model(rho, cp, cs, dx=10.0, pml=pml) as m1:
            m1.source_set(pos[b], mts[b], wav[b])
            single = m1.run(nt, dts[i], rcvs[i])
        assert np.array_equal(got[i][b], single), (i, b)
    rho, cp, cs, pml, pos, mts, wav = inputs[1]
    ref = orc.simulate(rho, cp, cs, dx=10.0, dt=dts[1], nt=nt, pml=pml,
                       sources=[dict(kind="moment", pos=pos[0], m=mts[0], w=wav[0])], receivers=rcvs[1])["traces"]
    err = trace_errors(got[1][0], ref)
    assert err.max() < 1e-4, (np.median(err), err.max())
