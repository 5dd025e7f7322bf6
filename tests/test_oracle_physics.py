"""Pins for the oracle's time stepping against what the mathematics fixes.

* single plane-wave modes follow the leapfrog recurrence in closed form
  (sin(theta/2) = c |kappa| dt / 2, Sec. II-A leapfrog + pseudo-spectral);
* the discrete energy is conserved exactly once sources stop (PML off);
* source-receiver reciprocity holds exactly for point forces (PML off);
* the system is linear: superposed runs, scaling and delays (Sec. IV);
* the PML absorbs (Sec. II-B).

A dropped term, a wrong sign, a transposed operand or a wrong staggering in
Eq. (2) breaks at least one of these."""
import numpy as np
import pytest

from paper_1705_04874_gb300 import synth
from conftest import cfl_dt

RHO, CP, CS = 2000.0, 3000.0, 1700.0
LAM = RHO * (CP ** 2 - 2 * CS ** 2)
MU = RHO * CS ** 2


def _positions(shape, d):
    """Coordinates of each of the 9 fields (vx vy vz sxx syy szz sxy sxz syz)
    at their staggered points, as (X, Y, Z) arrays."""
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    half = {0: (0.5, 0, 0), 1: (0, 0.5, 0), 2: (0, 0, 0.5), 3: (0, 0, 0), 4: (0, 0, 0),
            5: (0, 0, 0), 6: (0.5, 0.5, 0), 7: (0.5, 0, 0.5), 8: (0, 0.5, 0.5)}
    return {f: ((x + h[0]) * d[0], (y + h[1]) * d[1], (z + h[2]) * d[2]) for f, h in half.items()}


@pytest.mark.parametrize("mvec", [(3, 0, 0), (0, 2, 0), (0, 0, 5), (2, 3, 0), (1, 2, 2), (8, 0, 0)])
def test_p_plane_wave_follows_closed_form(orc, mvec):
    shape = (10, 12, 16)
    d = (10.0, 12.0, 8.0)
    rho, cp, cs = synth.homogeneous_model(shape, RHO, CP, CS)
    kap = np.array([2 * np.pi * mvec[a] / (shape[2 - a] * d[a]) for a in range(3)])
    kn = np.linalg.norm(kap)
    nvec = kap / kn
    A = 1e-3
    S = LAM * A * np.eye(3) + 2 * MU * A * np.outer(nvec, nvec)
    pos = _positions(shape, d)
    state = np.zeros((9,) + shape)
    comp = {3: (0, 0), 4: (1, 1), 5: (2, 2), 6: (0, 1), 7: (0, 2), 8: (1, 2)}
    for f, (i, j) in comp.items():
        X, Y, Z = pos[f]
        state[f] = S[i, j] * np.cos(kap[0] * X + kap[1] * Y + kap[2] * Z)
    dt = 0.3 * min(d) / CP
    nt = 37
    out = orc.simulate(rho, cp, cs, dx=d[0], dy=d[1], dz=d[2], dt=dt, nt=nt, pml=0, state=state)
    theta = 2 * np.arcsin(CP * kn * dt / 2)
    factor = np.cos(nt * theta) - np.tan(theta / 2) * np.sin(nt * theta)
    for f in comp:
        np.testing.assert_allclose(out["state"][f], factor * state[f], atol=1e-12 * np.abs(S).max())


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_s_plane_wave_follows_closed_form(orc, axis):
    shape = (12, 12, 12)
    d = (10.0, 10.0, 10.0)
    rho, cp, cs = synth.homogeneous_model(shape, RHO, CP, CS)
    m = 3
    k = 2 * np.pi * m / (12 * 10.0)
    pos = _positions(shape, d)
    # shear stress varying along `axis`, in the plane of `axis` and the next axis
    f = {0: 6, 1: 8, 2: 7}[axis]  # sxy along x, syz along y, sxz along z
    state = np.zeros((9,) + shape)
    state[f] = MU * 1e-3 * np.cos(k * pos[f][axis])
    dt = 0.3 * 10.0 / CP
    nt = 41
    out = orc.simulate(rho, cp, cs, dx=10.0, dt=dt, nt=nt, pml=0, state=state)
    theta = 2 * np.arcsin(CS * k * dt / 2)
    factor = np.cos(nt * theta) - np.tan(theta / 2) * np.sin(nt * theta)
    np.testing.assert_allclose(out["state"][f], factor * state[f], atol=1e-12 * MU * 1e-3)
    others = [g for g in range(3, 9) if g != f]
    assert np.abs(out["state"][others]).max() < 1e-12 * MU * 1e-3


def _water_rock(shape):
    return synth.two_layer_model(shape=shape, water_cells=5)


@pytest.mark.parametrize("model", ["homogeneous", "water_rock", "random"])
def test_energy_is_conserved_without_pml(orc, model):
    shape = (16, 12, 14)
    if model == "homogeneous":
        rho, cp, cs = synth.homogeneous_model(shape)
    elif model == "water_rock":
        rho, cp, cs = _water_rock(shape)
    else:
        rho, cp, cs = synth.marine_model(shape=shape, seed=5, corr_len=2.0, perturb=0.1)
    dt = cfl_dt(cp, 10.0)
    nt, nw = 160, 50
    w = synth.ricker(nw, dt, 40.0)
    srcs = [dict(kind="moment", pos=(7, 6, 10), m=synth.double_couple_sdr(30, 60, 90), w=w),
            dict(kind="force", pos=(4, 5, 12), m=(0.3, -1.0, 0.5), w=w * 1e6)]
    out = orc.simulate(rho, cp, cs, dx=10.0, dt=dt, nt=nt, pml=0, sources=srcs, energy=True)
    e = out["energy"][nw:]
    assert e.max() > 0
    assert (e.max() - e.min()) / e.max() < 1e-11


def test_energy_decays_with_pml(orc):
    shape = (24, 24, 24)
    rho, cp, cs = synth.homogeneous_model(shape)
    dt = cfl_dt(cp, 10.0)
    nw = 60
    w = synth.ricker(nw, dt, 40.0).astype(np.float64)
    w -= w.mean()  # zero net stress injection: nothing static is left behind
    out = orc.simulate(rho, cp, cs, dx=10.0, dt=dt, nt=400, pml=6,
                       sources=[dict(kind="moment", pos=(12, 12, 12), m=synth.explosive(), w=w)],
                       energy=True)
    e = out["energy"]
    assert e[-1] < 1e-3 * e[nw:].max()
    assert np.all(np.diff(e[nw:]) <= 1e-12 * e[nw:].max())


@pytest.mark.parametrize("ci,cj", [(0, 1), (2, 0), (1, 1)])
def test_reciprocity_of_point_forces(orc, ci, cj):
    shape = (16, 14, 18)
    rho, cp, cs = synth.marine_model(shape=shape, seed=9, corr_len=2.0, perturb=0.1)
    dt = cfl_dt(cp, 10.0)
    nt = 90
    w = synth.ricker(nt, dt, 35.0) * 1e6
    A, B = (5, 4, 9), (11, 9, 6)
    fj = np.zeros(3); fj[cj] = 1.0
    fi = np.zeros(3); fi[ci] = 1.0
    ab = orc.simulate(rho, cp, cs, dx=10.0, dt=dt, nt=nt, pml=0,
                      sources=[dict(kind="force", pos=A, m=fj, w=w)], receivers=[B])["traces"]
    ba = orc.simulate(rho, cp, cs, dx=10.0, dt=dt, nt=nt, pml=0,
                      sources=[dict(kind="force", pos=B, m=fi, w=w)], receivers=[A])["traces"]
    g_ab = ab[1 + ci, 0]  # v_ci at B from force cj at A
    g_ba = ba[1 + cj, 0]  # v_cj at A from force ci at B
    assert np.abs(g_ab).max() > 0
    assert np.abs(g_ab - g_ba).max() < 1e-10 * np.abs(g_ab).max()


def test_linearity_superposition_scaling_and_delay(orc):
    rho, cp, cs = synth.two_layer_model(shape=(20, 16, 24), water_cells=5)
    dt = cfl_dt(cp, 10.0)
    nt = 120
    w = synth.ricker(nt, dt, 30.0)
    rcv = orc.seabed_receivers(cs, 3, 3, 2)
    a = dict(kind="moment", pos=(8, 7, 12), m=synth.explosive(), w=w)
    b = dict(kind="moment", pos=(14, 9, 10), m=synth.double_couple_sdr(10, 70, -40), w=w)
    run = lambda s: orc.simulate(rho, cp, cs, dx=10.0, dt=dt, nt=nt, pml=3, sources=s,
                                 receivers=rcv)["traces"]
    ta, tb, tab = run([a]), run([b]), run([a, b])
    assert np.abs(tab - (ta + tb)).max() < 1e-12 * np.abs(tab).max()
    a2 = dict(a, w=(2.0 * w.astype(np.float64)))
    assert np.array_equal(run([a2]), 2.0 * ta)  # exact: scaling by 2 commutes with every step
    k = 17
    wd = np.concatenate([np.zeros(k), w.astype(np.float64)])[:nt]
    td = run([dict(a, w=wd)])
    assert np.array_equal(td[..., k:], ta[..., :nt - k])
    assert np.all(td[..., :k] == 0.0)
