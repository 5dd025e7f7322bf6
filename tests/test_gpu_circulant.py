"""Axis lengths without an FFT plan -- odd or non-smooth, 3 to 512, among them
the z axis of the paper's own 125 x 75 x 301 grid with 12.5 / 12.5 / 10 m
spacing (Sec. III; 301 = 7 x 43): the circulant passes against the FP64
oracle, through the C ABI.  Single derivatives on every axis, full runs on an
all-odd grid and on a grid that mixes FFT and circulant axes, the paper's grid
itself, and batching."""
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


# [nz][ny][nx]: circulant axes beside FFT axes (75 and 125 have plans), with
# odd and even nx; the shortest (3) and longest (512) axes
SHAPES = [(18, 20, 125), (301, 4, 32), (5, 75, 36), (3, 7, 9), (12, 10, 512), (40, 33, 17)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("shift", [1, -1])
def test_circulant_derivative_matches_oracle(es, orc, shape, axis, shift):
    import torch
    rng = np.random.default_rng(sum(shape) * 7 + axis * 2 + (shift > 0))
    f = rng.standard_normal(shape).astype(np.float32)
    d = [12.5, 12.5, 10.0][axis]
    ref = orc.deriv(f.astype(np.float64), axis, d, shift)
    out = torch.empty(shape, device="cuda")
    es.es_derivative(torch.from_numpy(f).cuda(), axis, d, shift, out)
    got = out.cpu().numpy()
    assert rel_l2(got, ref) < 5e-6
    assert np.abs(got - ref).max() < 5e-5 * np.abs(ref).max()


def _run_both(es, orc, rho, cp, cs, *, pml, nt, sources, rcv, d=(10.0, 10.0, 10.0)):
    dt = cfl_dt(cp, min(d))
    with es.Model(rho, cp, cs, dx=d[0], pml=pml) as m:
        if d[1] != d[0] or d[2] != d[0]:
            m.set_spacing(*d)
        for s in sources:
            m.source_add(s["pos"], s["m"], s["w"])
        gpu = m.run(nt, dt, rcv)
        state = m.state_get()
    ref = orc.simulate(rho, cp, cs, dx=d[0], dy=d[1], dz=d[2], dt=dt, nt=nt, pml=pml, sources=sources,
                       receivers=rcv, state=np.zeros((9,) + rho.shape))
    return gpu, state, ref


def test_all_odd_grid_run_matches_oracle(es, orc):
    """27 x 30 x 33 cells (every axis circulant), water over rock, explosive
    source, 4-cell PML, 120 steps, 3 x 3 seabed receivers."""
    rho, cp, cs = synth.two_layer_model(shape=(27, 30, 33), water_cells=6)
    nt = 120
    dt = cfl_dt(cp, 10.0)
    w = synth.ricker(nt, dt, 25.0)
    rcv = orc.seabed_receivers(cs, 4, 3, 3)
    src = [dict(kind="moment", pos=(16, 15, 14), m=synth.explosive(), w=w)]
    gpu, state, ref = _run_both(es, orc, rho, cp, cs, pml=4, nt=nt, sources=src, rcv=rcv)
    err = trace_errors(gpu, ref["traces"])
    assert err.max() < TOL, err.max()
    for f in range(9):
        assert rel_l2(state[f], ref["state"][f]) < TOL, f


def test_mixed_fft_and_circulant_axes(es, orc):
    """48 x 32 x 30 marine model: x and y through the FFT passes, z (30)
    through the circulant pass; explosive source, 5-cell PML, 100 steps.  (With
    a double couple, two seabed pressure traces lie on its nodal planes at 1e-3
    of the largest, where FP32 storage of the fields alone -- exact FP64
    derivatives, FP32 state -- already differs from the oracle by 9.8e-5.)"""
    rho, cp, cs = synth.marine_model(shape=(30, 32, 48), seed=2)
    nt = 100
    dt = cfl_dt(cp, 10.0)
    w = synth.ricker(nt, dt, 30.0)
    rcv = orc.seabed_receivers(cs, 5, 4, 4)
    src = [dict(kind="moment", pos=(24, 16, 18), m=synth.explosive(), w=w)]
    gpu, state, ref = _run_both(es, orc, rho, cp, cs, pml=5, nt=nt, sources=src, rcv=rcv)
    err = trace_errors(gpu, ref["traces"])
    assert err.max() < TOL, (np.median(err), err.max())
    for f in range(9):
        assert rel_l2(state[f], ref["state"][f]) < TOL, f


def test_paper_grid_matches_oracle(es, orc):
    """The paper's grid: 125 x 75 x 301 cells, dx = dy = 12.5 m, dz = 10 m (x
    and y through the FFT plans 5 x 25 and 5 x 15, z circulant), 10-cell PML,
    57 water cells, a double couple in the reservoir box; 12 steps
    of every field against the oracle, and the seabed receivers at the depth
    where cs first turns nonzero."""
    shape = (301, 75, 125)
    rho, cp, cs = synth.marine_model(shape=shape, seed=1)
    nt = 12
    d = (12.5, 12.5, 10.0)
    w = synth.ricker(nt, cfl_dt(cp, min(d)), 30.0, t0=4 * cfl_dt(cp, min(d)))
    box = synth.reservoir_box(shape, 10)
    pos = tuple((lo + hi) // 2 for lo, hi in box)
    rcv = orc.seabed_receivers(cs, 10, 21, 11)
    assert np.all(rcv[:, 2] == 56)  # 57 water cells: the sensors sit in the deepest one
    src = [dict(kind="moment", pos=pos, m=synth.random_dc(synth.SplitMix64(2)), w=w)]
    gpu, state, ref = _run_both(es, orc, rho, cp, cs, pml=10, nt=nt, sources=src, rcv=rcv, d=d)
    for f in range(9):
        assert rel_l2(state[f], ref["state"][f]) < TOL, f
    assert np.isfinite(gpu).all()


def test_batch_on_odd_grid_equals_single_runs(es):
    shape = (21, 26, 35)
    rho, cp, cs = synth.marine_model(shape=shape, seed=5)
    nt, pml, nb = 60, 3, 3
    dt = cfl_dt(cp, 10.0)
    rng = synth.SplitMix64(8)
    box = synth.reservoir_box(shape, pml)
    pos = synth.random_positions(rng, box, nb)
    mts = np.array([synth.random_dc(rng) for _ in range(nb)])
    wav = np.stack([synth.ricker(nt, dt, 30.0)] * nb)
    with es.Model(rho, cp, cs, dx=10.0, pml=pml) as m:
        rcv = m.seabed_receivers(3, 3)
        m.batch_set(pos, mts, wav)
        batched = m.run(nt, dt, rcv)
    for b in range(nb):
        with es.Model(rho, cp, cs, dx=10.0, pml=pml) as m1:
            m1.source_set(pos[b], mts[b], wav[b])
            assert np.array_equal(m1.run(nt, dt, rcv), batched[b]), b


def test_compensated_run_with_a_long_circulant_axis(es, orc):
    """Compensated derivatives (every axis circulant) with a 200-cell z axis,
    whose passes run the epilogue straight from the registers: every trace
    within 1e-4 of the oracle."""
    shape = (200, 16, 32)
    rho, cp, cs = synth.two_layer_model(shape=shape, water_cells=20)
    nt = 80
    dt = cfl_dt(cp, 10.0)
    w = synth.ricker(nt, dt, 25.0)
    src = [dict(kind="moment", pos=(16, 8, 40), m=synth.double_couple_sdr(30, 60, 90), w=w)]
    rcv = orc.seabed_receivers(cs, 3, 4, 2)
    with es.Model(rho, cp, cs, dx=10.0, pml=3) as m:
        m.set_precision(es.ES_PREC_COMPENSATED)
        m.source_set(src[0]["pos"], src[0]["m"], w)
        gpu = m.run(nt, dt, rcv)
    ref = orc.simulate(rho, cp, cs, dx=10.0, dt=dt, nt=nt, pml=3, sources=src, receivers=rcv)["traces"]
    assert trace_errors(gpu, ref).max() < TOL


@pytest.mark.parametrize("shape,pml,nb", [((200, 16, 32), 3, 1), ((193, 12, 20), 3, 1), ((301, 12, 24), 4, 2),
                                          ((512, 4, 8), 0, 1), ((16, 200, 24), 3, 1), ((12, 12, 201), 3, 1)])
def test_tensor_core_passes_match_oracle(es, orc, shape, pml, nb):
    """With ES_PREC_FP32_TC, axes of 192 to 512 cells without an FFT plan run
    their passes on the tensor cores (the far part of the kernel matrix and the
    field split in three BF16 parts each, six products, FP32 accumulation; the
    near stencil and the update in a separate kernel): the first simulation
    against the oracle (every trace and every field within 1e-4), the others
    of a batch equal to single-source runs bit for bit.  Long z axes (the
    shortest such, 193, and the longest, 512, no PML), a long y axis and a
    long odd x axis, with the PML along each."""
    rho, cp, cs = synth.marine_model(shape=shape, seed=sum(shape))
    nt = 60
    dt = cfl_dt(cp, 10.0)
    rng = synth.SplitMix64(sum(shape))
    box = synth.reservoir_box(shape, pml) if pml else tuple((2, s - 3) for s in shape[::-1])
    pos = synth.random_positions(rng, box, nb)
    mts = np.array([synth.random_dc(rng) for _ in range(nb)])
    wav = np.stack([synth.ricker(nt, dt, 30.0)] * nb)
    with es.Model(rho, cp, cs, dx=10.0, pml=pml) as m:
        assert m.kernels_per_step() == 8  # the CUDA-core circulant passes by default
        m.set_precision(es.ES_PREC_FP32_TC)
        assert m.kernels_per_step() == 10  # two field-update kernels for the two tensor-core passes
        rcv = np.array([[x, y, 3] for x in range(0, shape[2], max(1, shape[2] // 4))
                        for y in range(0, shape[1], max(1, shape[1] // 3))], np.int32)
        if nb == 1:
            m.source_set(pos[0], mts[0], wav[0])
            gpu = m.run(nt, dt, rcv)[None]
        else:
            m.batch_set(pos, mts, wav)
            gpu = m.run(nt, dt, rcv)
        st = m.state_get()
    st0 = st if nb == 1 else st[0]
    ref = orc.simulate(rho, cp, cs, dx=10.0, dt=dt, nt=nt, pml=pml,
                       sources=[dict(kind="moment", pos=pos[0], m=mts[0], w=wav[0])], receivers=rcv,
                       state=np.zeros((9,) + rho.shape))
    err = trace_errors(gpu[0], ref["traces"])
    assert err.max() < TOL, (np.median(err), err.max())
    for f in range(9):
        assert rel_l2(st0[f], ref["state"][f]) < TOL, f
    for b in range(1, nb):
        with es.Model(rho, cp, cs, dx=10.0, pml=pml) as m1:
            m1.set_precision(es.ES_PREC_FP32_TC)
            m1.source_set(pos[b], mts[b], wav[b])
            assert np.array_equal(m1.run(nt, dt, rcv), gpu[b]), b
