"""Pins for the oracle's own transforms (Sec. II-A: FFT / IFFT of the
pseudo-spectral method).  The naive DFT is the definition; the mixed-radix
FFT must agree with it, with numpy's independent FFT, with Parseval and with
transforms known in closed form."""
import numpy as np
import pytest

SIZES = list(range(1, 41)) + [45, 96, 125, 128, 160, 256, 301]


@pytest.mark.parametrize("n", SIZES)
def test_fft_matches_naive_dft_and_numpy(orc, n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    y = orc.fft(x)
    ref = np.fft.fft(x)
    assert np.abs(y - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())
    if n <= 160:
        yn = orc.fft(x, naive=True)
        assert np.abs(yn - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())
    # inverse scaled by 1/n returns the input
    assert np.abs(orc.fft(y, inverse=True) - x).max() <= 1e-13 * max(1.0, np.abs(x).max())
    # Parseval: sum |x|^2 = sum |X|^2 / n
    assert np.isclose(np.sum(np.abs(x) ** 2), np.sum(np.abs(y) ** 2) / n, rtol=1e-12)


@pytest.mark.parametrize("n", [8, 12, 30, 96, 160])
def test_fft_closed_forms(orc, n):
    delta = np.zeros(n, complex)
    delta[0] = 1.0
    assert np.abs(orc.fft(delta) - 1.0).max() < 1e-14
    for m in (1, n // 3, n - 1):
        tone = np.exp(2j * np.pi * m * np.arange(n) / n)
        expect = np.zeros(n, complex)
        expect[m] = n
        assert np.abs(orc.fft(tone) - expect).max() < 1e-11
        assert np.abs(orc.fft(tone, naive=True) - expect).max() < 1e-11
