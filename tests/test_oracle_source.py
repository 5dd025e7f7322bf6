"""Pins of the oracle's smoothed point source (Sec. II-A: a grid-point delta
smoothed with a Blackman window in the spatial-frequency domain).  The oracle
builds it with a 3D FFT; these tests hold it to closed forms: the window's
values, its inverse transform (a 5-point stencil per axis, wrapping at the
edges), and the linearity of the solver (one smoothed source = 125 weighted
point sources)."""
import numpy as np
import pytest

import oracle
from paper_1705_04874_gb300 import synth

S5 = np.array([0.04, 0.25, 0.42, 0.25, 0.04])


def test_blackman_window_values():
    for n in (8, 13, 16, 75):
        w = oracle.blackman_window(n)
        assert abs(w[0] - 1.0) < 1e-15                  # zero wavenumber passes
        assert np.allclose(w, w[(-np.arange(n)) % n])   # even in k
        if n % 2 == 0:
            assert abs(w[n // 2]) < 1e-15               # Nyquist removed
        assert np.all(w >= -1e-15) and np.all(w <= 1 + 1e-15)


@pytest.mark.parametrize("shape,pos", [((12, 11, 13), (6, 5, 4)), ((9, 16, 7), (0, 1, 8)), ((20, 5, 5), (4, 2, 19))])
def test_smoothed_delta_is_the_separable_stencil(shape, pos):
    g = oracle.smoothed_delta(shape, pos)
    ref = np.zeros(shape)
    for dz in range(-2, 3):
        for dy in range(-2, 3):
            for dx in range(-2, 3):
                ref[(pos[2] + dz) % shape[0], (pos[1] + dy) % shape[1], (pos[0] + dx) % shape[2]] += \
                    S5[dz + 2] * S5[dy + 2] * S5[dx + 2]
    assert np.abs(g - ref).max() < 1e-14
    assert abs(g.sum() - 1.0) < 1e-13


def test_smoothed_source_equals_weighted_point_sources():
    rho, cp, cs = synth.two_layer_model(shape=(16, 14, 18), water_cells=4)
    nt, dt = 40, 0.3 * 10.0 / float(cp.max())
    w = synth.ricker(nt, dt, 30.0)
    mt = synth.double_couple_sdr(30, 60, 90)
    pos = (9, 7, 9)
    rcv = oracle.seabed_receivers(cs, 3, 3, 3)
    a = oracle.simulate(rho, cp, cs, dx=10.0, dt=dt, nt=nt, pml=3, receivers=rcv, state=np.zeros((9,) + rho.shape),
                        sources=[dict(kind="moment", pos=pos, m=mt, w=w, smooth=True)])
    pts = []
    for dz in range(-2, 3):
        for dy in range(-2, 3):
            for dx in range(-2, 3):
                s = S5[dz + 2] * S5[dy + 2] * S5[dx + 2]
                pts.append(dict(kind="moment", pos=(pos[0] + dx, pos[1] + dy, pos[2] + dz), m=mt * s, w=w))
    b = oracle.simulate(rho, cp, cs, dx=10.0, dt=dt, nt=nt, pml=3, receivers=rcv, state=np.zeros((9,) + rho.shape),
                        sources=pts)
    scale = np.abs(b["state"]).max()
    assert np.abs(a["state"] - b["state"]).max() < 1e-12 * scale
    assert np.abs(a["traces"] - b["traces"]).max() < 1e-12 * np.abs(b["traces"]).max()
