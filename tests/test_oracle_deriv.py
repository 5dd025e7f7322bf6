"""Pins for the staggered Fourier pseudo-spectral derivative (Sec. II-A).

D(+/-) f(x) = f'(x +/- d/2) is exact for every sampled sinusoid up to and
including the Nyquist mode, along each axis and in each of the oracle's three
modes (1D FFT per line, naive DFT, full 3D FFT).  The + and - operators are
minus each other's adjoints, which is what makes the leapfrog scheme conserve
energy."""
import numpy as np
import pytest


def _mode_field(shape, axis, m, d, phase):
    n = shape[2 - axis]
    x = np.arange(n) * d
    L = n * d
    f = np.cos(2 * np.pi * m * x / L + phase)
    bshape = [1, 1, 1]
    bshape[2 - axis] = n
    return np.broadcast_to(f.reshape(bshape), shape).copy(), x, L


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("shift", [+1, -1])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_derivative_of_sinusoids_is_exact(orc, axis, shift, mode):
    shape = (12, 10, 16)  # nz, ny, nx: even and odd-free mixed sizes
    n = shape[2 - axis]
    d = [10.0, 12.5, 7.0][axis]
    for m in range(0, n // 2 + 1):
        phase = 0.37 * (m + 1)
        f, x, L = _mode_field(shape, axis, m, d, phase)
        D = orc.deriv(f, axis, d, shift, mode=mode)
        k = 2 * np.pi * m / L
        if 2 * m == n:
            # Nyquist: the samples are cos(phase) (-1)^j; the staggered
            # derivative of that sampled mode is -/+ (pi/d) cos(phase) (-1)^j
            ex1 = -shift * (np.pi / d) * np.cos(np.pi * np.arange(n) + phase)
        else:
            ex1 = -k * np.sin(k * (x + shift * d / 2) + phase)
        bshape = [1, 1, 1]
        bshape[2 - axis] = n
        ex = np.broadcast_to(ex1.reshape(bshape), shape)
        scale = max(k, 1e-30)
        assert np.abs(D - ex).max() <= 1e-12 * max(scale, np.pi / d), (m, shift)


def test_odd_length_axis(orc):
    n, d = 15, 5.0
    x = np.arange(n) * d
    L = n * d
    for m in range(0, 8):
        f = np.sin(2 * np.pi * m * x / L)
        F = np.broadcast_to(f, (2, 3, n)).copy()
        D = orc.deriv(F, 0, d, +1)
        ex = (2 * np.pi * m / L) * np.cos(2 * np.pi * m * (x + d / 2) / L)
        assert np.abs(D[1, 2] - ex).max() < 1e-12 * (1 + 2 * np.pi * m / L)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_modes_agree_on_random_fields(orc, axis):
    rng = np.random.default_rng(7)
    f = rng.standard_normal((6, 10, 8))
    d = 3.0
    a = orc.deriv(f, axis, d, +1, mode=0)
    b = orc.deriv(f, axis, d, +1, mode=1)
    c = orc.deriv(f, axis, d, +1, mode=2)
    s = np.abs(a).max()
    assert np.abs(a - b).max() < 1e-12 * s
    assert np.abs(a - c).max() < 1e-12 * s


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_plus_and_minus_are_negative_adjoints(orc, axis):
    rng = np.random.default_rng(11 + axis)
    f = rng.standard_normal((8, 6, 10))
    g = rng.standard_normal((8, 6, 10))
    lhs = np.sum(orc.deriv(f, axis, 2.0, +1) * g)
    rhs = -np.sum(f * orc.deriv(g, axis, 2.0, -1))
    assert abs(lhs - rhs) < 1e-12 * (abs(lhs) + 1)


def test_derivative_of_constant_is_zero(orc):
    f = np.full((4, 5, 6), 3.25)
    for axis in range(3):
        assert np.abs(orc.deriv(f, axis, 1.0, +1)).max() < 1e-13
