"""FFT passes on odd lengths: the 5-smooth plans of the paper's x and y axes
(125 = 5 x 5 x 5, 75 = 5 x 15 or 3 x 5 x 5, Sec. III), the x pass on a length that is not
a multiple of 16, and the y / z passes with an odd nx (pencil pairs moved as
two floats).  Single derivatives, full runs against the FP64 oracle (with the
point sources and receivers fused into the passes), and the fused kernels and
batches against their separate / single-source counterparts bit for bit."""
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


# [nz][ny][nx]: x 75 / 125 through the any-length x pass, y and z with odd nx;
# the last two end on a partial tile of 13 and 3 lines (cells past its last
# 16-byte chunk)
SHAPES = [(48, 32, 75), (32, 75, 125), (125, 16, 17), (75, 48, 33), (16, 16, 125), (5, 9, 75), (7, 5, 125)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("shift", [+1, -1])
def test_odd_length_derivative_matches_oracle(es, orc, shape, axis, shift):
    import torch
    rng = np.random.default_rng(sum(shape) * 11 + axis * 2 + (shift > 0))
    f = rng.standard_normal(shape).astype(np.float32)
    d = [12.5, 12.5, 10.0][axis]
    ref = orc.deriv(f.astype(np.float64), axis, d, shift)
    out = torch.empty(shape, device="cuda")
    es.es_derivative(torch.from_numpy(f).cuda(), axis, d, shift, out)
    got = out.cpu().numpy().astype(np.float64)
    assert rel_l2(got, ref) < 2e-6
    assert np.abs(got - ref).max() < 2e-5 * np.abs(ref).max()


def test_paper_xy_axes_take_fft_plans(es):
    assert es.es_fft_plan(0, 125) == (5, 25)  # three stages of radix 5
    assert es.es_fft_plan(1, 75) == (5, 15)   # (3, 25): radices 3, 5, 5, the other candidate
    with pytest.raises(es.EsError):
        es.es_fft_plan(1, 301)


def test_paper_xy_section_run_matches_oracle(es, orc):
    """125 x 75 cells in x and y as in the paper (12.5 m), 48 cells of 10 m in
    z: every axis through the FFT passes (x 125 any-length, y 75 with odd nx,
    z 48 with odd nx), sources and receivers fused; 6-cell PML, 9 water
    cells, an explosive source and a point force below the seabed, 100 steps,
    5 x 4 seabed 4C receivers."""
    shape = (48, 75, 125)
    rho, cp, cs = synth.marine_model(shape=shape, seed=3)
    d = (12.5, 12.5, 10.0)
    nt = 100
    dt = cfl_dt(cp, min(d))
    w = synth.ricker(nt, dt, 30.0)
    rcv = orc.seabed_receivers(cs, 6, 5, 4)
    srcs = [dict(kind="moment", pos=(62, 37, 26), m=synth.explosive(), w=w),
            dict(kind="force", pos=(40, 30, 30), m=(0.2, -1.0, 0.4), w=w * 1e7)]
    with es.Model(rho, cp, cs, dx=d[0], pml=6) as m:
        m.set_spacing(*d)
        m.source_add(srcs[0]["pos"], srcs[0]["m"], w)
        m.source_add_force(srcs[1]["pos"], srcs[1]["m"], srcs[1]["w"])
        assert m.kernels_per_step() == 6
        gpu = m.run(nt, dt, rcv)
        state = m.state_get()
    ref = orc.simulate(rho, cp, cs, dx=d[0], dy=d[1], dz=d[2], dt=dt, nt=nt, pml=6, sources=srcs, receivers=rcv,
                       state=np.zeros((9,) + rho.shape))
    err = trace_errors(gpu, ref["traces"])
    assert err.max() < TOL, (np.median(err), err.max())
    for f in range(9):
        assert rel_l2(state[f], ref["state"][f]) < TOL, f


def test_odd_nx_fused_equals_separate_kernels(es):
    """On a 75 x 32 x 48 grid (odd nx, all FFT axes) the fused sources and
    receivers against the separate injection / recording kernels (forced by a
    zero smoothed source beside them): traces and fields equal bit for bit."""
    shape = (48, 32, 75)
    rho, cp, cs = synth.marine_model(shape=shape, seed=4)
    nt = 80
    dt = cfl_dt(cp, 10.0)
    w = synth.ricker(nt, dt, 30.0)
    out = []
    with es.Model(rho, cp, cs, dx=10.0, pml=5) as m:
        rcv = m.seabed_receivers(4, 3)
        for extra in (False, True):
            m.state_reset()
            m.source_clear()
            m.source_add((37, 16, 30), synth.double_couple_sdr(30, 60, 90), w)
            m.source_add_force((20, 10, 28), np.array([1e-3, 0.0, 2e-3]), w)
            if extra:
                m.source_add_smoothed((37, 16, 24), np.zeros(6), w)
            assert m.kernels_per_step() == (9 if extra else 6)
            out.append((m.run(nt, dt, rcv), m.state_get()))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])


def test_odd_nx_batch_equals_single_runs(es):
    shape = (32, 48, 75)
    rho, cp, cs = synth.marine_model(shape=shape, seed=6)
    nt, pml, nb = 60, 4, 3
    dt = cfl_dt(cp, 10.0)
    rng = synth.SplitMix64(12)
    box = synth.reservoir_box(shape, pml)
    pos = synth.random_positions(rng, box, nb)
    mts = np.array([synth.random_dc(rng) for _ in range(nb)])
    wav = np.stack([synth.ricker(nt, dt, 30.0)] * nb)
    with es.Model(rho, cp, cs, dx=10.0, pml=pml) as m:
        rcv = m.seabed_receivers(3, 3)
        m.batch_set(pos, mts, wav)
        assert m.kernels_per_step() == 6
        batched = m.run(nt, dt, rcv)
    for b in range(nb):
        with es.Model(rho, cp, cs, dx=10.0, pml=pml) as m1:
            m1.source_set(pos[b], mts[b], wav[b])
            assert np.array_equal(m1.run(nt, dt, rcv), batched[b]), b


def test_odd_cell_count_batch_equals_single_runs(es):
    """75 x 75 x 125 cells, an odd count, so every other simulation of a batch
    starts off a 16-byte boundary and its x passes update cell by cell instead
    of four at a time: a batch of three equals single runs bit for bit."""
    shape = (125, 75, 75)
    rho, cp, cs = synth.marine_model(shape=shape, seed=7)
    nt, pml, nb = 40, 5, 3
    dt = cfl_dt(cp, 10.0)
    rng = synth.SplitMix64(21)
    box = synth.reservoir_box(shape, pml)
    pos = synth.random_positions(rng, box, nb)
    mts = np.array([synth.random_dc(rng) for _ in range(nb)])
    wav = np.stack([synth.ricker(nt, dt, 30.0)] * nb)
    with es.Model(rho, cp, cs, dx=10.0, pml=pml) as m:
        rcv = m.seabed_receivers(4, 4)
        m.batch_set(pos, mts, wav)
        assert m.kernels_per_step() == 6
        batched = m.run(nt, dt, rcv)
        st = m.state_get()
    for b in range(nb):
        with es.Model(rho, cp, cs, dx=10.0, pml=pml) as m1:
            m1.source_set(pos[b], mts[b], wav[b])
            assert np.array_equal(m1.run(nt, dt, rcv), batched[b]), b
            assert np.array_equal(m1.state_get(), st[b]), b
