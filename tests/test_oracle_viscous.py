"""Pins of the oracle's Kelvin-Voigt terms (Eq. (1)-(2): chi, eta; read with
chi = tau lambda, eta = tau mu and the time derivative of the strain rate as
the backward difference of the velocity derivatives over one step).

For one Fourier mode the scheme's amplification per step z satisfies
    z^2 + (q (1 + r) - 2) z + (1 - q r) = 0,   q = c^2 |kappa|^2 dt^2,  r = tau / dt,
so with v^{-1/2} = 0 a plane wave's stress is exactly
    sigma^n = sigma^0 rho^n (cos n th + (cos th - 1/rho) / sin th sin n th),
    rho^2 = 1 - q r,  2 rho cos th = 2 - q (1 + r),
whose envelope decays as (1 - q r)^(n/2) -> exp(-tau c^2 kappa^2 t / 2), the
Kelvin-Voigt rate; r = 0 gives back the elastic closed form.  Both roots stay
inside the unit circle (Schur-Cohn) iff q (1 + 2 r) <= 4 for every mode: the
explicit viscous term tightens the elastic bound q <= 4."""
import numpy as np
import pytest

import oracle
from paper_1705_04874_gb300 import synth
from conftest import cfl_dt

RHO, CP, CS = 2000.0, 3000.0, 1600.0
MU = RHO * CS ** 2
LAM = RHO * CP ** 2 - 2 * MU


@pytest.fixture(scope="module")
def orc():
    oracle.build()
    return oracle


def _positions(shape, d):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    X, Y, Z = x * d[0], y * d[1], z * d[2]
    h = (0.5 * d[0], 0.5 * d[1], 0.5 * d[2])
    return {3: (X, Y, Z), 4: (X, Y, Z), 5: (X, Y, Z), 6: (X + h[0], Y + h[1], Z), 7: (X + h[0], Y, Z + h[2]),
            8: (X, Y + h[1], Z + h[2])}


def _factor(q, r, n):
    rho = np.sqrt(1 - q * r)
    th = np.arccos((2 - q * (1 + r)) / (2 * rho))
    return rho ** n * (np.cos(n * th) + (np.cos(th) - 1 / rho) / np.sin(th) * np.sin(n * th))


@pytest.mark.parametrize("r", [0.0, 0.25, 0.5])  # q_max (1 + 2 r) <= 4 on this grid up to r = 0.578
def test_viscous_p_plane_wave_follows_the_discrete_closed_form(orc, r):
    shape = (10, 12, 16)
    d = (10.0, 12.0, 8.0)
    mvec = (2, 1, 1)
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
    out = orc.simulate(rho, cp, cs, dx=d[0], dy=d[1], dz=d[2], dt=dt, nt=nt, pml=0, state=state, tau=r * dt)
    fac = _factor((CP * kn * dt) ** 2, r, nt)
    for f in comp:
        np.testing.assert_allclose(out["state"][f], fac * state[f], atol=1e-12 * np.abs(S).max())
    if r > 0:
        assert abs(fac) < 1.0


def test_viscous_s_plane_wave_follows_the_discrete_closed_form(orc):
    shape = (12, 12, 12)
    rho, cp, cs = synth.homogeneous_model(shape, RHO, CP, CS)
    k = 2 * np.pi * 3 / (12 * 10.0)
    pos = _positions(shape, (10.0, 10.0, 10.0))
    state = np.zeros((9,) + shape)
    state[6] = MU * 1e-3 * np.cos(k * pos[6][0])  # sxy varying along x
    dt = 0.3 * 10.0 / CP
    nt, r = 41, 0.2  # q_max (1 + 2 r) = 2.66 x 1.4 <= 4
    out = orc.simulate(rho, cp, cs, dx=10.0, dt=dt, nt=nt, pml=0, state=state, tau=r * dt)
    fac = _factor((CS * k * dt) ** 2, r, nt)
    np.testing.assert_allclose(out["state"][6], fac * state[6], atol=1e-12 * MU * 1e-3)


def test_decay_rate_tends_to_kelvin_voigt():
    """(1 - q r)^(n/2) over a fixed time -> exp(-tau c^2 kappa^2 t / 2) as dt -> 0."""
    c, kap, tau, t = 3000.0, 2 * np.pi / 200.0, 2e-4, 0.05
    exact = np.exp(-tau * c ** 2 * kap ** 2 * t / 2)
    errs = []
    for dt in (1e-4, 5e-5, 2.5e-5):
        q, r, n = (c * kap * dt) ** 2, tau / dt, t / dt
        errs.append(abs((1 - q * r) ** (n / 2) - exact))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-3 * exact


def test_zero_tau_is_the_elastic_scheme_and_viscosity_dissipates(orc):
    shape = (16, 12, 14)
    rho, cp, cs = synth.marine_model(shape=shape, seed=5, corr_len=2.0, perturb=0.1)
    dt = cfl_dt(cp, 10.0)
    nt, nw = 140, 40
    w = synth.ricker(nw, dt, 40.0)
    srcs = [dict(kind="moment", pos=(7, 6, 10), m=synth.double_couple_sdr(30, 60, 90), w=w)]
    base = orc.simulate(rho, cp, cs, dx=10.0, dt=dt, nt=nt, pml=0, sources=srcs, energy=True,
                        state=np.zeros((9,) + shape))
    zero = orc.simulate(rho, cp, cs, dx=10.0, dt=dt, nt=nt, pml=0, sources=srcs, energy=True,
                        state=np.zeros((9,) + shape), tau=0.0)
    assert np.array_equal(base["state"], zero["state"])
    visc = orc.simulate(rho, cp, cs, dx=10.0, dt=dt, nt=nt, pml=0, sources=srcs, energy=True,
                        state=np.zeros((9,) + shape), tau=0.2 * dt)
    e = visc["energy"][nw:]
    assert np.all(np.diff(e) <= 1e-12 * e.max())  # never gains energy once the source stopped
    assert e[-1] < 0.9 * base["energy"][-1]


def test_stability_bound_of_the_viscous_scheme(orc):
    """Just inside q_max (1 + 2 r) <= 4 the discrete energy never rises above
    its start and decays; just outside, the Nyquist-corner mode grows without
    bound (homogeneous box, PML off, a random initial state)."""
    shape = (8, 8, 8)
    rho, cp, cs = synth.homogeneous_model(shape, RHO, CP, CS)
    dt = 0.3 * 10.0 / CP
    qmax = (CP * dt * np.pi * np.sqrt(3) / 10.0) ** 2
    r_lim = (4 / qmax - 1) / 2
    state = np.random.default_rng(1).standard_normal((9,) + shape)
    inside = orc.simulate(rho, cp, cs, dx=10.0, dt=dt, nt=300, pml=0, state=state, tau=0.95 * r_lim * dt,
                          energy=True)["energy"]
    outside = orc.simulate(rho, cp, cs, dx=10.0, dt=dt, nt=300, pml=0, state=state, tau=1.05 * r_lim * dt,
                           energy=True)["energy"]
    assert inside.max() <= inside[0] * (1 + 1e-12) and inside[-1] < 0.1 * inside[0]
    assert outside[-1] > 1e6 * outside[0]
