"""Pins of the oracle's Laplacian (Sec. VI-A, Eq. (8)): closed forms on
products of cosines, Nyquist modes included, and agreement with the oracle's
own staggered derivatives composed as D(+) D(-) along each axis."""
import numpy as np

import oracle


def test_laplacian_of_cosine_products():
    nz, ny, nx = 12, 10, 16
    d = (12.5, 10.0, 7.5)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    for mx, my, mz in [(1, 2, 3), (8, 0, 0), (3, 5, 6), (0, 0, 0)]:  # 8 = Nyquist of x, 5 of y, 6 of z
        f = np.cos(2 * np.pi * mx * x / nx + 0.2) * np.cos(2 * np.pi * my * y / ny) * np.cos(2 * np.pi * mz * z / nz)
        if mx == nx // 2:
            f = np.cos(np.pi * x) * np.cos(2 * np.pi * my * y / ny) * np.cos(2 * np.pi * mz * z / nz)
        k2 = (2 * np.pi * mx / (nx * d[0])) ** 2 + (2 * np.pi * my / (ny * d[1])) ** 2 + (2 * np.pi * mz / (nz * d[2])) ** 2
        assert np.abs(oracle.laplacian(f, d) + k2 * f).max() < 1e-12 * max(1.0, k2)


def test_laplacian_equals_composed_staggered_derivatives():
    oracle.build()
    rng = np.random.default_rng(3)
    f = rng.standard_normal((9, 12, 10))
    d = (10.0, 12.5, 7.5)
    comp = sum(oracle.deriv(oracle.deriv(f, a, d[a], -1), a, d[a], +1) for a in range(3))
    ref = oracle.laplacian(f, d)
    assert np.abs(comp - ref).max() < 1e-11 * np.abs(ref).max()
