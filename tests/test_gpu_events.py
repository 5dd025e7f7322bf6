"""Clustered events (Sec. VI-A): the density Laplacian (Eq. (8)) on the GPU
against the oracle's spectral definition, the threshold selection of event
locations, and a clustered superposition of solver traces."""
import numpy as np
import pytest

from paper_1705_04874_gb300 import synth
from conftest import cfl_dt

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_04874_gb300 import es, events
    es._load()
    return es, events


@pytest.mark.parametrize("shape,d", [((64, 64, 64), (10.0, 10.0, 10.0)), ((30, 48, 40), (12.5, 12.5, 10.0)),
                                     ((301, 75, 125), (12.5, 12.5, 10.0))])
def test_density_laplacian_matches_oracle(ev, orc, shape, d):
    es, events = ev
    rho, _, _ = synth.marine_model(shape=shape, seed=2)
    got = events.density_laplacian(rho, d).cpu().numpy()
    ref = orc.laplacian(rho.astype(np.float64), d)
    assert np.linalg.norm(got - ref) <= 5e-5 * np.linalg.norm(ref)


def test_event_selection_and_clustered_superposition(ev, orc):
    es, events = ev
    shape = (48, 48, 48)
    rho, cp, cs = synth.marine_model(shape=shape, seed=3)
    lap = events.density_laplacian(rho)
    box = synth.reservoir_box(shape, 6)
    locs = synth.latin_hypercube_positions(synth.SplitMix64(5), box, 60)
    ref = orc.laplacian(rho.astype(np.float64), (10.0, 10.0, 10.0))
    ref_vals = np.array([ref[z, y, x] for x, y, z in locs])
    thr = float(np.median(np.abs(ref_vals)))
    sel, vals = events.select_event_locations(lap, locs, thr)
    # the same decision as the oracle's wherever |L| is not within rounding of the threshold
    clear = np.abs(np.abs(ref_vals) - thr) > 1e-4 * np.abs(ref_vals).max()
    want = np.abs(ref_vals) > thr
    assert np.array_equal((np.isin(np.arange(len(locs)), sel))[clear], want[clear])
    assert 10 <= len(sel) <= 50
    # three clusters by depth, close origin times within each, one record of all events
    depth = locs[sel, 2]
    labels = np.digitize(depth, np.quantile(depth, [1 / 3, 2 / 3]))
    src, amps, t0s = events.clustered_events(synth.SplitMix64(6), labels)
    nt = 60
    dt = cfl_dt(cp, 10.0)
    wav = np.stack([synth.ricker(nt, dt, 30.0)] * len(sel))
    mts = np.array([synth.random_dc(synth.SplitMix64(100 + i)) for i in range(len(sel))])
    with es.Model(rho, cp, cs, dx=10.0, pml=6) as m:
        rcv = m.seabed_receivers(4, 4)
        m.batch_set(locs[sel], mts, wav)
        traces = m.run(nt, dt, rcv)
    n_out = nt + int(np.ceil((t0s.max() + 0.1) / dt))
    got = es.es_superpose(traces, src, amps, t0s, dt, n_out)
    want = orc.superpose(traces.astype(np.float64), src, amps.astype(np.float64), t0s.astype(np.float64), dt, n_out)
    assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max()
    # the clusters follow each other in time (means 0.3 s apart, spread 0.1 s)
    mean_t0 = [float(np.mean(t0s[labels == c])) for c in range(3)]
    assert mean_t0[0] < mean_t0[1] < mean_t0[2]
