"""Pins for the fourth-order-in-time oracle (oracle/time4.py).

  reduction        without the correction it is the C oracle's leapfrog:
                   traces and gradient
  time order       self-convergence in dt: error ratio ~16 per halving (the
                   leapfrog's ~4 on the same problem)
  stability        stable just below sqrt(3) x the leapfrog limit, blows up
                   just above
  adjoint          dot-product test of the step operator G and its transpose
  gradient         Taylor remainder O(h^2); central differences, in the
                   interior and in the sponge, constant and variable density
  physics          at twice the leapfrog's step it follows the closed-form 2D
                   Green's function 20x more closely (0.12% against 2.3%)
"""
import numpy as np
import pytest

import oracle
from oracle import time4
from paper_2110_03345_gb300 import inputs


def problem(shape=(36, 40), dx=0.5e-3, nt=120, nb=6, vd=True, seed=0, order=8, cfl=0.4):
    vp, rho = inputs.random_smooth_model(shape, dx, seed)
    dt = cfl * dx / vp.max()
    g = oracle.Grid(shape, dx, dt=dt, nt=nt, order=order, nb=nb, c_ref=1500.0)
    src = inputs.random_points(1, shape, dx, seed + 1, margin=8)
    rec = inputs.random_points(5, shape, dx, seed + 2, margin=8)
    w = inputs.ricker(5e5, dt, nt)[None, :]
    return g, vp, (rho if vd else None), src, w, rec


@pytest.mark.parametrize("vd", [False, True])
def test_without_correction_it_is_the_leapfrog(vd):
    g, vp, rho, src, w, rec = problem(vd=vd)
    ref = oracle.forward(g, vp, rho, src[None], w[None], rec)[0]
    d = time4.forward(g, vp, rho, src, w, rec, correction=False)
    np.testing.assert_allclose(d, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    true = vp * 1.03
    obs = oracle.forward(g, true, rho, src[None], w[None], rec)[0]
    J0, g0, _ = oracle.gradient(g, vp, rho, src[None], w[None], rec, obs[None])
    J1, g1, _ = time4.gradient(g, vp, rho, src, w, rec, obs, correction=False)
    assert J1 == pytest.approx(J0, rel=1e-11)
    np.testing.assert_allclose(g1, g0, rtol=0, atol=1e-10 * np.abs(g0).max())


def _run(scheme_correction, refine, base_nt=60, dx=0.5e-3, n=56):
    """Traces of a smooth source in a smooth medium without sponge, at time
    step dt0 / refine; returned on the coarse time samples."""
    vp, _ = inputs.random_smooth_model((n, n), dx, 4, c_range=(1450.0, 1550.0), sigma=3e-3)
    dt0 = 0.45 * dx / 1550.0
    dt = dt0 / refine
    nt = base_nt * refine + 1
    g = oracle.Grid((n, n), dx, dt=dt, nt=nt, order=8, nb=0, c_ref=1500.0)
    q = inputs.ricker_fn(2.5e5, t0=6e-6)
    w = q(np.arange(nt) * dt)[None, :]
    src = np.array([[14.2e-3, 13.1e-3]])
    rec = np.array([[18.0e-3, 15.5e-3], [9.5e-3, 20.25e-3]])
    d = time4.forward(g, vp, None, src, w, rec, correction=scheme_correction)
    return d[:, ::refine]


@pytest.mark.parametrize("correction,ratio", [(True, 16.0), (False, 4.0)])
def test_order_of_accuracy_in_time(correction, ratio):
    d1, d2, d4 = (_run(correction, r) for r in (1, 2, 4))
    e1 = np.linalg.norm(d1 - d2)
    e2 = np.linalg.norm(d2 - d4)
    assert e2 > 0
    assert e1 / e2 == pytest.approx(ratio, rel=0.25), e1 / e2


@pytest.mark.parametrize("order", [8, 10])
def test_stability_limit(order):
    w2, _ = oracle.fd_weights(order)
    limit = time4.stability_limit(2, w2)
    lam = abs(w2[0] + 2 * sum((-1) ** j * w2[j] for j in range(1, len(w2))))
    assert limit == pytest.approx(np.sqrt(3.0) * 2.0 / np.sqrt(2 * lam), rel=1e-14)
    n, dx, c = 24, 1e-3, 1500.0
    rng = np.random.default_rng(3)
    out = {}
    for fac in (0.98, 1.04):
        dt = fac * limit * dx / c
        g = oracle.Grid((n, n), dx, dt=dt, nt=500, order=order, nb=0)
        w = rng.standard_normal((1, g.nt))
        with np.errstate(over="ignore", invalid="ignore"):
            tr = time4.forward(g, np.full((n, n), c), None, np.array([[10.3e-3, 11.7e-3]]), w,
                               np.array([[12e-3, 12e-3]]))
        out[fac] = np.abs(tr).max()
    assert np.isfinite(out[0.98]) and out[0.98] < 1e3
    assert not np.isfinite(out[1.04]) or out[1.04] > 1e12


@pytest.mark.parametrize("vd", [False, True])
def test_step_operator_dot_product(vd):
    g, vp, rho, *_ = problem(vd=vd, shape=(30, 34))
    rng = np.random.default_rng(7)
    x = rng.standard_normal(g.npoints)
    y = rng.standard_normal(g.npoints)
    lhs = np.dot(time4.apply_G(g, vp, rho, x), y)
    rhs = np.dot(x, time4.apply_GT(g, vp, rho, y))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def _misfit(g, vp, rho, src, w, rec, obs):
    d = time4.forward(g, vp, rho, src, w, rec)
    return 0.5 * float(np.sum((d - obs) ** 2))


def _setup(vd=True):
    g, vp, rho, src, w, rec = problem(vd=vd)
    idx = np.indices(g.shape).astype(float)
    ctr = (np.array(g.shape, dtype=float) / 2).reshape(-1, 1, 1)
    true = vp * (1.0 + 0.03 * np.exp(-((idx - ctr) ** 2).sum(0) / 30.0))
    obs = time4.forward(g, true, rho, src, w, rec)
    return g, vp, rho, src, w, rec, obs


def test_gradient_taylor_remainder_is_second_order():
    g, vp, rho, src, w, rec, obs = _setup()
    J0, grad, _ = time4.gradient(g, vp, rho, src, w, rec, obs)
    m = 1.0 / vp ** 2
    dm = m * np.random.default_rng(4).standard_normal(m.shape) * 0.1
    hs = np.array([1e-1, 5e-2, 2.5e-2, 1.25e-2])
    rem = [abs(_misfit(g, 1.0 / np.sqrt(m + h * dm), rho, src, w, rec, obs) - J0
               - h * np.vdot(grad, dm)) for h in hs]
    slopes = np.diff(np.log(rem)) / np.diff(np.log(hs))
    assert np.all(np.abs(slopes - 2.0) < 0.1), slopes


@pytest.mark.parametrize("vd", [False, True])
def test_gradient_central_differences(vd):
    g, vp, rho, src, w, rec, obs = _setup(vd=vd)
    J0, grad, _ = time4.gradient(g, vp, rho, src, w, rec, obs)
    assert J0 == pytest.approx(_misfit(g, vp, rho, src, w, rec, obs), rel=1e-13)
    m = 1.0 / vp ** 2
    for p in [(18, 20), (12, 27), (2, 3)]:                     # (2, 3) lies in the sponge
        h = 1e-4 * m[p]
        mp, mm = m.copy(), m.copy()
        mp[p] += h
        mm[p] -= h
        fd = (_misfit(g, 1 / np.sqrt(mp), rho, src, w, rec, obs)
              - _misfit(g, 1 / np.sqrt(mm), rho, src, w, rec, obs)) / (2 * h)
        assert fd == pytest.approx(grad[p], rel=1e-6, abs=1e-9 * np.abs(grad).max())


def test_gradient_3d_central_differences():
    shape, dx = (16, 18, 20), 0.5e-3
    vp, rho = inputs.random_smooth_model(shape, dx, 2)
    dt = 0.4 * dx / vp.max()
    g = oracle.Grid(shape, dx, dt=dt, nt=60, order=10, nb=3, c_ref=1500.0)
    src = np.array([[4.1e-3, 4.3e-3, 4.6e-3]])
    rec = np.array([[3.2e-3, 5.1e-3, 6.4e-3], [5.0e-3, 3.3e-3, 2.9e-3]])
    w = inputs.ricker(6e5, dt, g.nt)[None, :]
    obs = time4.forward(g, vp * 1.02, rho, src, w, rec)
    J0, grad, _ = time4.gradient(g, vp, rho, src, w, rec, obs)
    m = 1.0 / vp ** 2
    p = (8, 9, 7)
    h = 1e-4 * m[p]
    mp, mm = m.copy(), m.copy()
    mp[p] += h
    mm[p] -= h
    fd = (_misfit(g, 1 / np.sqrt(mp), rho, src, w, rec, obs)
          - _misfit(g, 1 / np.sqrt(mm), rho, src, w, rec, obs)) / (2 * h)
    assert fd == pytest.approx(grad[p], rel=1e-6)


def test_accuracy_against_the_analytic_solution_at_twice_the_step():
    """Homogeneous 2D medium, order 10, 6 points per wavelength at 2.5 x the
    Ricker peak, off-grid source and receivers with sinc weights (small
    interpolation error), record ending before boundary echoes: at CFL 0.8
    (half the steps) the fourth-order scheme follows the closed-form Green's
    function (Sec. 3.1) far more closely than the leapfrog at CFL 0.4."""
    from oracle import sinc
    c, f0 = 1500.0, 3e5
    dx = c / (2.5 * f0) / 6
    n = int(60e-3 / dx)
    q = inputs.ricker_fn(f0, t0=1.5 / f0)
    ctr = (n // 2 + 0.5) * dx
    src = np.array([[ctr, ctr - 0.3 * dx]])
    R = 9e-3
    ang = np.linspace(0, 2 * np.pi, 8, endpoint=False)
    rec = np.stack([ctr + R * np.sin(ang), ctr - 0.3 * dx + R * np.cos(ang)], 1)
    vp = np.full((n, n), c)
    err = {}
    for corr, cfl in ((False, 0.4), (True, 0.8)):
        dt = cfl * dx / c
        nt = int(20e-6 / dt)
        g = oracle.Grid((n, n), dx, dt=dt, nt=nt, order=10, nb=10, c_ref=c)
        w = q(np.arange(nt) * dt)[None, :]
        ana = oracle.analytic_2d(q, R, np.arange(nt) * dt, c)
        d = time4.forward(g, vp, None, src, w, rec, correction=corr, interp=sinc.hicks())
        err[corr] = np.sqrt(np.mean((d - ana[None]) ** 2)) / np.sqrt(np.mean(ana ** 2))
    assert err[True] < 3e-3 and err[True] < err[False] / 5, err   # measured 0.0012, 0.023
