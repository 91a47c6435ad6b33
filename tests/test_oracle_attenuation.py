"""Pins for the attenuation oracle (oracle/attenuation.py, Eq. 10 with y = 0, 2).

  reduction     alpha0 = 0 is the C oracle's leapfrog: traces and gradient
  power law     the decay of a narrowband wave between two receivers, over
                the same run without attenuation, is alpha0 w^y (y = 0, 2)
  gradient      Taylor remainder O(h^2); central differences in m for both
                y, with and without density, in the interior and the sponge
"""
import numpy as np
import pytest

import oracle
from oracle import attenuation as att
from paper_2110_03345_gb300 import inputs


def problem(shape=(36, 40), dx=0.5e-3, nt=120, nb=6, vd=True, seed=0):
    vp, rho = inputs.random_smooth_model(shape, dx, seed)
    dt = 0.4 * dx / vp.max()
    g = oracle.Grid(shape, dx, dt=dt, nt=nt, order=8, nb=nb, c_ref=1500.0)
    src = inputs.random_points(1, shape, dx, seed + 1, margin=8)
    rec = inputs.random_points(5, shape, dx, seed + 2, margin=8)
    w = inputs.ricker(5e5, dt, nt)[None, :]
    return g, vp, (rho if vd else None), src, w, rec


@pytest.mark.parametrize("y", [0, 2])
def test_zero_attenuation_is_the_leapfrog(y):
    g, vp, rho, src, w, rec = problem()
    ref = oracle.forward(g, vp, rho, src[None], w[None], rec)[0]
    d = att.forward(g, vp, rho, 0.0, y, src, w, rec)
    np.testing.assert_allclose(d, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    obs = oracle.forward(g, vp * 1.03, rho, src[None], w[None], rec)[0]
    J0, g0, _ = oracle.gradient(g, vp, rho, src[None], w[None], rec, obs[None])
    J1, g1, _ = att.gradient(g, vp, rho, 0.0, y, src, w, rec, obs)
    assert J1 == pytest.approx(J0, rel=1e-11)
    np.testing.assert_allclose(g1, g0, rtol=0, atol=1e-10 * np.abs(g0).max())


@pytest.mark.parametrize("y", [0, 2])
def test_power_law_attenuation(y):
    """Homogeneous water, a 10-cycle burst at f0; receivers 8 and 18 mm from
    the source; reflections arrive after the record.  The spectral ratio at f0
    of the attenuated to the lossless run decays as exp(-alpha0 w0^y r)."""
    n, dx, c, f0 = 200, 0.5e-3, 1500.0, 3e5
    w0 = 2 * np.pi * f0
    target = 20.0                                    # nepers per metre at f0
    alpha0 = target / w0 ** y
    dt = 0.4 * dx / c
    nt = 420
    g = oracle.Grid((n, n), dx, dt=dt, nt=nt, order=8, nb=0, c_ref=c)
    w = inputs.tone_burst(f0, dt, nt, cycles=10)[None, :]
    ctr = (n // 2) * dx
    src = np.array([[ctr, ctr]])
    r1, r2 = 8e-3, 18e-3
    rec = np.array([[ctr, ctr + r1], [ctr, ctr + r2]])
    vp = np.full((n, n), c)
    d0 = att.forward(g, vp, None, 0.0, y, src, w, rec)
    da = att.forward(g, vp, None, alpha0, y, src, w, rec)
    nf = 1 << 14
    k = int(round(f0 * nf * dt))
    ratio = np.abs(np.fft.rfft(da, nf)[:, k]) / np.abs(np.fft.rfft(d0, nf)[:, k])
    measured = -np.log(ratio[1] / ratio[0]) / (r2 - r1)
    assert measured == pytest.approx(target, rel=0.03), measured   # 19.8 (y=0), 19.6 (y=2)


def _misfit(g, vp, rho, alpha0, y, src, w, rec, obs):
    d = att.forward(g, vp, rho, alpha0, y, src, w, rec)
    return 0.5 * float(np.sum((d - obs) ** 2))


ALPHA = {0: 200.0, 2: 2e-11}      # strong enough to matter in 120 steps


def _setup(y, vd=True):
    g, vp, rho, src, w, rec = problem(vd=vd)
    idx = np.indices(g.shape).astype(float)
    ctr = (np.array(g.shape, dtype=float) / 2).reshape(-1, 1, 1)
    true = vp * (1.0 + 0.03 * np.exp(-((idx - ctr) ** 2).sum(0) / 30.0))
    obs = att.forward(g, true, rho, ALPHA[y], y, src, w, rec)
    return g, vp, rho, src, w, rec, obs


@pytest.mark.parametrize("y", [0, 2])
def test_attenuation_changes_the_data(y):
    g, vp, rho, src, w, rec = problem()
    d0 = att.forward(g, vp, rho, 0.0, y, src, w, rec)
    d1 = att.forward(g, vp, rho, ALPHA[y], y, src, w, rec)
    assert np.linalg.norm(d1 - d0) > 0.05 * np.linalg.norm(d0)
    assert np.linalg.norm(d1) < np.linalg.norm(d0)


@pytest.mark.parametrize("y", [0, 2])
def test_gradient_taylor_remainder_is_second_order(y):
    g, vp, rho, src, w, rec, obs = _setup(y)
    J0, grad, _ = att.gradient(g, vp, rho, ALPHA[y], y, src, w, rec, obs)
    m = 1.0 / vp ** 2
    dm = m * np.random.default_rng(4).standard_normal(m.shape) * 0.1
    hs = np.array([1e-1, 5e-2, 2.5e-2, 1.25e-2])
    rem = [abs(_misfit(g, 1.0 / np.sqrt(m + h * dm), rho, ALPHA[y], y, src, w, rec, obs) - J0
               - h * np.vdot(grad, dm)) for h in hs]
    slopes = np.diff(np.log(rem)) / np.diff(np.log(hs))
    assert np.all(np.abs(slopes - 2.0) < 0.1), slopes


@pytest.mark.parametrize("y,vd", [(0, False), (0, True), (2, False), (2, True)])
def test_gradient_central_differences(y, vd):
    g, vp, rho, src, w, rec, obs = _setup(y, vd)
    J0, grad, _ = att.gradient(g, vp, rho, ALPHA[y], y, src, w, rec, obs)
    assert J0 == pytest.approx(_misfit(g, vp, rho, ALPHA[y], y, src, w, rec, obs), rel=1e-13)
    m = 1.0 / vp ** 2
    for p in [(18, 20), (12, 27), (2, 3)]:                     # (2, 3) lies in the sponge
        h = 1e-4 * m[p]
        mp, mm = m.copy(), m.copy()
        mp[p] += h
        mm[p] -= h
        fd = (_misfit(g, 1 / np.sqrt(mp), rho, ALPHA[y], y, src, w, rec, obs)
              - _misfit(g, 1 / np.sqrt(mm), rho, ALPHA[y], y, src, w, rec, obs)) / (2 * h)
        assert fd == pytest.approx(grad[p], rel=1e-6, abs=1e-9 * np.abs(grad).max())
