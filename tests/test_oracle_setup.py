"""Pins for the oracle's set-up and post-processing steps: Lame parameters
(Eq. (4)), staggered material averages, the PML profile (Sec. II-B), the
seabed receiver rule (Sec. II-B, Fig. 2) and superposition (Sec. IV), each
against values worked out by hand or closed forms."""
import json
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_lame_parameters_closed_form(orc):
    shape = (3, 4, 5)
    rho = np.full(shape, 2000.0)
    cp = np.full(shape, 3000.0)
    cs = np.full(shape, 1700.0)
    m = orc.materials(rho, cp, cs)
    assert np.allclose(m["mu"], 2000.0 * 1700.0 ** 2, rtol=1e-15)       # 5.78e9
    assert np.allclose(m["lam"], 6.44e9, rtol=1e-14)                     # rho (cp^2 - 2 cs^2)
    for b in ("bx", "by", "bz"):
        assert np.allclose(m[b], 1 / 2000.0, rtol=1e-15)
    for e in ("muxy", "muxz", "muyz"):
        assert np.allclose(m[e], 5.78e9, rtol=1e-14)


def test_buoyancy_at_interfaces_and_wrap(orc):
    shape = (2, 3, 6)
    rho = np.full(shape, 3000.0)
    rho[..., :3] = 1000.0
    one = np.ones(shape)
    m = orc.materials(rho, one * 2000.0, one * 1000.0)
    bx = m["bx"][0, 0]
    assert np.allclose(bx, [1e-3, 1e-3, 5e-4, 1 / 3000.0, 1 / 3000.0, 5e-4], rtol=1e-15)
    assert np.allclose(m["by"], 1 / rho, rtol=1e-15)


def test_edge_shear_modulus_is_harmonic_mean_or_zero(orc):
    # mu = 1, 2, 3, 4 at (i,j) = (0,0), (1,0), (0,1), (1,1): every xy edge sees all four
    mu = np.array([[1.0, 2.0], [3.0, 4.0]]).reshape(1, 2, 2)
    rho = np.ones((1, 2, 2))
    cp = np.full((1, 2, 2), 10.0)
    m = orc.materials(rho, cp, np.sqrt(mu))
    assert np.allclose(m["muxy"], 48.0 / 25.0, rtol=1e-14)  # 4 / (1 + 1/2 + 1/3 + 1/4)
    mu2 = mu.copy()
    mu2[0, 1, 1] = 0.0  # one water neighbour
    m2 = orc.materials(rho, cp, np.sqrt(mu2))
    assert np.all(m2["muxy"] == 0.0)
    # along z with nz = 1 the z-neighbour is the cell itself: mean of (a, b, a, b)
    assert np.allclose(m["muxz"][0, 0, 0], 4.0 / (2 / 1.0 + 2 / 2.0), rtol=1e-14)


def test_pml_profile_values(orc):
    n, L, a0, cref, d, dt = 40, 6, 2.0, 3000.0, 10.0, 1e-3
    Pc = orc.pml_profile(n, L, a0, cref, d, dt, 0)
    Ps = orc.pml_profile(n, L, a0, cref, d, dt, 1)
    outer = np.exp(-a0 * cref / d * dt / 2)
    assert Pc[0] == pytest.approx(outer, rel=1e-15) and Pc[-1] == pytest.approx(outer, rel=1e-15)
    assert np.all(Pc[L:n - L] == 1.0)
    assert np.all(Ps[L:n - L - 1] == 1.0)
    assert Ps[L - 1] == pytest.approx(np.exp(-a0 * cref / d * (0.5 / L) ** 4 * dt / 2), rel=1e-15)
    assert Pc[L - 1] == pytest.approx(np.exp(-a0 * cref / d * (1.0 / L) ** 4 * dt / 2), rel=1e-15)
    assert Ps[-1] == pytest.approx(outer, rel=1e-15)  # clamped at the outermost point
    assert np.allclose(Pc, Pc[::-1], rtol=0, atol=0)
    assert np.allclose(Ps[:-1], Ps[:-1][::-1], rtol=1e-15)
    assert np.all(np.diff(Pc[:L + 1]) > 0)
    assert np.all(orc.pml_profile(n, 0, a0, cref, d, dt, 0) == 1.0)


def test_seabed_receivers_golden(orc):
    g = json.load(open(os.path.join(GOLD, "seabed_receivers.json")))
    c = g["cases"][0]
    nx, ny, nz = c["nx"], c["ny"], c["nz"]
    cs = np.full((nz, ny, nx), 1000.0)
    for iy in range(ny):
        for ix in range(nx):
            cs[: 2 + (ix + iy) % 3, iy, ix] = 0.0
    px, py = c["pocket"]["column"]
    cs[:, py, px] = 1000.0
    cs[:2, py, px] = 0.0
    cs[c["pocket"]["water_z"], py, px] = 0.0
    got = orc.seabed_receivers(cs, c["L"], c["rx"], c["ry"])
    assert got.tolist() == c["expected"]
    c2 = g["cases"][1]
    cs2 = np.full((c2["nz"], c2["ny"], c2["nx"]), 1500.0)
    cs2[:57] = 0.0
    got2 = orc.seabed_receivers(cs2, c2["L"], c2["rx"], c2["ry"])
    assert np.all(got2[:, 2] == c2["expected_iz"])
    assert sorted(set(got2[:, 0].tolist())) == list(range(5))


def test_seabed_receivers_rejects_dry_column(orc):
    cs = np.full((6, 4, 4), 1000.0)
    with pytest.raises(ValueError):
        orc.seabed_receivers(cs, 0, 2, 2)


def test_superpose_golden(orc):
    g = json.load(open(os.path.join(GOLD, "superpose_small.json")))
    tr = np.array(g["traces"], np.float64)
    t0s = np.array(g["t0s"], np.float32).astype(np.float64)
    got = orc.superpose(tr, g["src_of_event"], g["amps"], t0s, g["dt"], g["n_out"])
    assert np.array_equal(got, np.array(g["expected"]))


def test_superpose_is_linear_and_shift_invariant(orc):
    rng = np.random.default_rng(3)
    tr = rng.standard_normal((3, 4, 5, 20))
    a = orc.superpose(tr, [0, 2], [1.0, 1.0], [0.0, 0.0], 0.1, 40)
    b = orc.superpose(tr, [0], [1.0], [0.0], 0.1, 40) + orc.superpose(tr, [2], [1.0], [0.0], 0.1, 40)
    assert np.allclose(a, b, rtol=0, atol=1e-14)
    s = orc.superpose(tr, [1], [1.0], [0.7], 0.1, 40)  # 7 samples later
    assert np.array_equal(s[..., 7:27], tr[1])
    assert np.all(s[..., :7] == 0) and np.all(s[..., 27:] == 0)
