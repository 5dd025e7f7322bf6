"""Kelvin-Voigt viscosity (Eq. (1)-(2), chi = tau lambda, eta = tau mu)
through the C ABI against the FP64 oracle: a heterogeneous run on a grid that
mixes FFT and circulant axes, tau = 0 equal to the elastic path, the
stability bound q_max (1 + 2 tau / dt) <= 4, and batching."""
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


def _setup(shape=(32, 40, 48), seed=3, nt=120):
    rho, cp, cs = synth.marine_model(shape=shape, seed=seed)
    dt = cfl_dt(cp, 10.0)
    w = synth.ricker(nt, dt, 30.0)
    return rho, cp, cs, dt, w


@pytest.mark.parametrize("r,prec", [(0.1, 0), (0.2, 0), (0.1, 1)])
def test_viscous_run_matches_oracle(es, orc, r, prec):
    """FP32 and compensated derivatives (es_model_set_precision): every trace
    and every field within 1e-4."""
    rho, cp, cs, dt, w = _setup()
    nt, pml = len(w), 4
    src = [dict(kind="moment", pos=(24, 20, 14), m=synth.double_couple_sdr(20, 70, 110), w=w)]
    rcv = orc.seabed_receivers(cs, pml, 4, 4)
    with es.Model(rho, cp, cs, dx=10.0, pml=pml) as m:
        m.set_viscosity(r * dt)
        if prec:
            m.set_precision(es.ES_PREC_COMPENSATED)
        m.source_set(src[0]["pos"], src[0]["m"], w)
        gpu = m.run(nt, dt, rcv)
        st = m.state_get()
        assert m.kernels_per_step() == 9
    ref = orc.simulate(rho, cp, cs, dx=10.0, dt=dt, nt=nt, pml=pml, sources=src, receivers=rcv,
                       state=np.zeros((9,) + rho.shape), tau=r * dt)
    err = trace_errors(gpu, ref["traces"])
    assert err.max() < TOL, (np.median(err), err.max())
    for f in range(9):
        assert rel_l2(st[f], ref["state"][f]) < TOL, f
    # and it differs from the elastic run by far more than the tolerance
    elastic = orc.simulate(rho, cp, cs, dx=10.0, dt=dt, nt=nt, pml=pml, sources=src, receivers=rcv)["traces"]
    assert trace_errors(gpu, elastic).max() > 100 * TOL


def test_zero_viscosity_is_the_elastic_path(es):
    rho, cp, cs, dt, w = _setup(nt=60)
    outs = []
    for tau in (None, 0.0):
        with es.Model(rho, cp, cs, dx=10.0, pml=4) as m:
            if tau is not None:
                m.set_viscosity(tau)
            m.source_set((24, 20, 14), synth.explosive(), w)
            outs.append(m.run(len(w), dt, m.seabed_receivers(3, 3)))
    assert np.array_equal(outs[0], outs[1])


def test_viscous_stability_bound_is_enforced(es):
    rho, cp, cs, dt, w = _setup(nt=10)
    qmax = (float(cp.max()) * dt * np.pi * np.sqrt(3) / 10.0) ** 2
    r_lim = (4 / qmax - 1) / 2
    with es.Model(rho, cp, cs, dx=10.0, pml=4) as m:
        m.source_set((24, 20, 14), synth.explosive(), w)
        m.set_viscosity(1.02 * r_lim * dt)
        with pytest.raises(es.EsError) as e:
            m.run(10, dt)
        assert e.value.status == es.ES_ERR_UNSTABLE
        m.set_viscosity(0.98 * r_lim * dt)
        m.run(10, dt)
        with pytest.raises(es.EsError) as e:
            m.set_viscosity(-1.0)
        assert e.value.status == es.ES_ERR_ARG


def test_viscous_batch_equals_single_runs(es):
    rho, cp, cs, dt, w = _setup(nt=50)
    nb, pml = 3, 4
    rng = synth.SplitMix64(13)
    pos = synth.random_positions(rng, synth.reservoir_box(rho.shape, pml), nb)
    mts = np.array([synth.random_dc(rng) for _ in range(nb)])
    wav = np.stack([w] * nb)
    with es.Model(rho, cp, cs, dx=10.0, pml=pml) as m:
        rcv = m.seabed_receivers(3, 3)
        m.set_viscosity(0.15 * dt)
        m.batch_set(pos, mts, wav)
        batched = m.run(len(w), dt, rcv)
    for b in range(nb):
        with es.Model(rho, cp, cs, dx=10.0, pml=pml) as m1:
            m1.set_viscosity(0.15 * dt)
            m1.source_set(pos[b], mts[b], wav[b])
            assert np.array_equal(m1.run(len(w), dt, rcv), batched[b]), b
