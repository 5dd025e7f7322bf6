"""Batched sources on one model (es_batch_set) and several models in one
graph (es_run_group) compute exactly what separate single-source runs
compute: every simulation goes through the same kernels with the same
arithmetic, so the traces agree bit for bit."""
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


def _sources(rng, shape, pml, nb, nt, dt):
    box = synth.reservoir_box(shape, pml)
    pos = synth.random_positions(rng, box, nb)
    mts = np.array([synth.random_dc(rng) for _ in range(nb)])
    wav = np.stack([synth.ricker(nt, dt, 25.0 + 5.0 * b) for b in range(nb)])
    return pos, mts, wav


def test_batch_equals_single_runs(es, orc):
    shape = (48, 64, 96)
    rho, cp, cs = synth.marine_model(shape=shape, seed=11)
    dt, nt, pml, nb = cfl_dt(cp, 10.0), 140, 6, 5
    pos, mts, wav = _sources(synth.SplitMix64(12), shape, pml, nb, nt, dt)
    with es.Model(rho, cp, cs, dx=10.0, pml=pml) as m:
        rcv = m.seabed_receivers(5, 4)
        m.batch_set(pos, mts, wav)
        batched = m.run(nt, dt, rcv)
        st = m.state_get()
        assert batched.shape == (nb, 4, len(rcv), nt) and st.shape == (nb, 9) + shape
    for b in range(nb):
        with es.Model(rho, cp, cs, dx=10.0, pml=pml) as m1:
            m1.source_set(pos[b], mts[b], wav[b])
            single = m1.run(nt, dt, rcv)
            assert np.array_equal(m1.state_get(), st[b])
        assert np.array_equal(batched[b], single), b
    # and the first simulation against the oracle
    ref = orc.simulate(rho, cp, cs, dx=10.0, dt=dt, nt=nt, pml=pml,
                       sources=[dict(kind="moment", pos=pos[0], m=mts[0], w=wav[0])], receivers=rcv)["traces"]
    assert trace_errors(batched[0], ref).max() < 1e-4


def test_batch_back_to_single_and_resize(es):
    shape = (32, 32, 48)
    rho, cp, cs = synth.two_layer_model(shape=shape, water_cells=6)
    dt, nt = cfl_dt(cp, 10.0), 40
    pos, mts, wav = _sources(synth.SplitMix64(3), shape, 4, 3, nt, dt)
    with es.Model(rho, cp, cs, dx=10.0, pml=4) as m:
        rcv = m.seabed_receivers(2, 2)
        m.batch_set(pos, mts, wav)
        a = m.run(nt, dt, rcv)
        m.batch_set(pos[:2], mts[:2], wav[:2])
        b = m.run(nt, dt, rcv)
        assert np.array_equal(a[:2], b)
        m.batch_set(pos[:1], mts[:1], wav[:1])
        m.nsim = 1
        c = m.run(nt, dt, rcv)
        assert np.array_equal(c, a[0])


def test_group_of_uneven_grids_equals_separate_runs(es):
    specs = [((48, 48, 48), 4, 1), ((32, 64, 32), 4, 3), ((64, 32, 80), 5, 2)]
    models, rcvs, dts, want = [], [], [], []
    nt = 90
    try:
        for i, (shape, pml, nb) in enumerate(specs):
            rho, cp, cs = synth.marine_model(shape=shape, seed=20 + i)
            dt = cfl_dt(cp, 10.0)
            pos, mts, wav = _sources(synth.SplitMix64(30 + i), shape, pml, nb, nt, dt)
            m = es.Model(rho, cp, cs, dx=10.0, pml=pml)
            rcv = m.seabed_receivers(3, 3)
            m.batch_set(pos, mts, wav)
            want.append(m.run(nt, dt, rcv))
            m.state_reset()
            models.append(m)
            rcvs.append(rcv)
            dts.append(dt)
        got = es.es_run_group(models, nt, dts, rcvs)
        for g, w_ in zip(got, want):
            assert np.array_equal(g, w_)
    finally:
        for m in models:
            m.close()
