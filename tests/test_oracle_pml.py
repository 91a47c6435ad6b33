"""Pins for the PML oracle (oracle/pml.py, 2D and 3D, constant density).

  reduction     without a layer it is the C oracle's leapfrog (2D, 3D)
  stencil       the first-derivative stencil is antisymmetric (zero extension)
  absorption    the reflection off a PML is far below that off a sponge of
                the same width and profile (2D 10 points, 3D 8 points); no
                growth at late times
  gradient      Taylor remainder O(h^2); central differences, inside the
                layer too (2D, 3D)
"""
import numpy as np
import pytest

import oracle
from oracle import pml
from paper_2110_03345_gb300 import inputs


def test_without_a_layer_it_is_the_leapfrog():
    shape, dx = (40, 44), 0.5e-3
    vp, _ = inputs.random_smooth_model(shape, dx, 1)
    dt = 0.4 * dx / vp.max()
    g = oracle.Grid(shape, dx, dt=dt, nt=150, order=8, nb=0, c_ref=1500.0)
    src = inputs.random_points(1, shape, dx, 2, margin=8)
    rec = inputs.random_points(4, shape, dx, 3, margin=8)
    w = inputs.ricker(5e5, dt, g.nt)[None, :]
    ref = oracle.forward(g, vp, None, src[None], w[None], rec)[0]
    d = pml.forward(g, vp, src, w, rec)
    np.testing.assert_allclose(d, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("order", [8, 10])
def test_first_derivative_is_antisymmetric(order):
    g = oracle.Grid((30, 34), (0.5e-3, 0.4e-3), dt=1e-7, nt=2, order=order)
    rng = np.random.default_rng(1)
    f, h = rng.standard_normal(g.shape), rng.standard_normal(g.shape)
    for ax in (0, 1):
        assert np.vdot(pml.d1(g, f, ax), h) == pytest.approx(-np.vdot(f, pml.d1(g, h, ax)), rel=1e-12)
    x = np.arange(34) * 0.4e-3
    lin = np.broadcast_to(3.0 * x[None, :], g.shape)
    assert np.allclose(pml.d1(g, lin, 1)[:, order:-order], 3.0, rtol=1e-12)   # exact on lines


def _reflection(kind, nb=10):
    """Energy, at a receiver 4 mm from a face, of what the small domain's
    boundary sends back: trace(small) - trace(large), the large domain
    reflecting nothing within the record."""
    c, dx, f0 = 1500.0, 0.25e-3, 4e5
    dt = 0.4 * dx / c
    nt = 700
    q = inputs.ricker_fn(f0, t0=1.5 / f0)
    w = q(np.arange(nt) * dt)[None, :]
    out = {}
    for n, lay in ((100, nb), (400, 0)):
        g = oracle.Grid((n, n), dx, dt=dt, nt=nt, order=8, nb=lay, c_ref=c)
        ctr = (n // 2) * dx
        src = np.array([[ctr, ctr]])
        rec = np.array([[ctr, ctr + (50 - nb) * dx - 4e-3]])       # 4 mm from the small layer
        vp = np.full((n, n), c)
        if kind == "pml" and lay:
            out[n] = pml.forward(g, vp, src, w, rec)[0]
        else:
            out[n] = oracle.forward(g, vp, None, src[None], w[None], rec)[0, 0]
    direct = out[400]
    return np.sum((out[100] - direct) ** 2) / np.sum(direct ** 2)


def test_pml_reflects_far_less_than_the_sponge():
    r_pml = _reflection("pml")
    r_sponge = _reflection("sponge")
    assert r_pml < 0.01 * r_sponge, (r_pml, r_sponge)     # measured 6.0e-5 against 5.0e-2
    assert r_pml < 2e-4


def test_no_late_time_growth():
    n, dx, c = 60, 0.5e-3, 1500.0
    dt = 0.4 * dx / c
    g = oracle.Grid((n, n), dx, dt=dt, nt=6000, order=8, nb=10, c_ref=c)
    w = inputs.ricker(3e5, dt, g.nt)[None, :]
    d = pml.forward(g, np.full((n, n), c), np.array([[15e-3, 14e-3]]), w,
                    np.array([[20e-3, 20e-3], [6e-3, 6e-3]]))
    early = np.abs(d[:, :1000]).max()
    late = np.abs(d[:, -1000:]).max()
    assert np.isfinite(late) and late < 1e-3 * early


def _gsetup():
    shape, dx = (40, 44), 0.5e-3
    vp, _ = inputs.random_smooth_model(shape, dx, 0)
    dt = 0.4 * dx / vp.max()
    g = oracle.Grid(shape, dx, dt=dt, nt=140, order=8, nb=8, c_ref=1500.0)
    src = np.array([[10.3e-3, 11.1e-3]])
    rec = np.array([[4.2e-3, 15.0e-3], [16.0e-3, 3.1e-3], [12.0e-3, 18.4e-3]])   # two in the layer
    w = inputs.ricker(5e5, dt, g.nt)[None, :]
    idx = np.indices(shape).astype(float)
    ctr = (np.array(shape, dtype=float) / 2).reshape(-1, 1, 1)
    true = vp * (1.0 + 0.03 * np.exp(-((idx - ctr) ** 2).sum(0) / 30.0))
    obs = pml.forward(g, true, src, w, rec)
    return g, vp, src, w, rec, obs


def _misfit(g, vp, src, w, rec, obs):
    return 0.5 * float(np.sum((pml.forward(g, vp, src, w, rec) - obs) ** 2))


def test_gradient_taylor_remainder_is_second_order():
    g, vp, src, w, rec, obs = _gsetup()
    J0, grad, _ = pml.gradient(g, vp, src, w, rec, obs)
    m = 1.0 / vp ** 2
    dm = m * np.random.default_rng(4).standard_normal(m.shape) * 0.1
    hs = np.array([1e-1, 5e-2, 2.5e-2, 1.25e-2])
    rem = [abs(_misfit(g, 1.0 / np.sqrt(m + h * dm), src, w, rec, obs) - J0 - h * np.vdot(grad, dm))
           for h in hs]
    slopes = np.diff(np.log(rem)) / np.diff(np.log(hs))
    assert np.all(np.abs(slopes - 2.0) < 0.1), slopes


def test_gradient_central_differences():
    g, vp, src, w, rec, obs = _gsetup()
    J0, grad, _ = pml.gradient(g, vp, src, w, rec, obs)
    assert J0 == pytest.approx(_misfit(g, vp, src, w, rec, obs), rel=1e-13)
    m = 1.0 / vp ** 2
    for p in [(20, 22), (14, 30), (3, 20), (25, 2)]:          # the last two lie in the layer
        h = 1e-4 * m[p]
        mp, mm = m.copy(), m.copy()
        mp[p] += h
        mm[p] -= h
        fd = (_misfit(g, 1 / np.sqrt(mp), src, w, rec, obs)
              - _misfit(g, 1 / np.sqrt(mm), src, w, rec, obs)) / (2 * h)
        assert fd == pytest.approx(grad[p], rel=1e-6, abs=1e-9 * np.abs(grad).max())


def test_3d_without_a_layer_it_is_the_leapfrog():
    shape, dx = (18, 20, 22), 0.5e-3
    vp, _ = inputs.random_smooth_model(shape, dx, 4)
    dt = 0.35 * dx / vp.max()
    g = oracle.Grid(shape, dx, dt=dt, nt=60, order=10, nb=0, c_ref=1500.0)
    src = np.array([[4.3e-3, 5.1e-3, 5.6e-3]])
    rec = np.array([[3.1e-3, 6.2e-3, 7.7e-3], [6.0e-3, 3.4e-3, 3.3e-3]])
    w = inputs.ricker(6e5, dt, g.nt)[None, :]
    ref = oracle.forward(g, vp, None, src[None], w[None], rec)[0]
    np.testing.assert_allclose(pml.forward(g, vp, src, w, rec), ref, rtol=0,
                               atol=1e-12 * np.abs(ref).max())


def test_3d_pml_reflects_far_less_than_the_sponge():
    """8-point layers on a 40^3 grid against a 120^3 reference; receiver 3 mm
    from the layer."""
    c, dx, f0 = 1500.0, 0.5e-3, 2.5e5
    dt = 0.35 * dx / c
    nt = 220
    q = inputs.ricker_fn(f0, t0=1.5 / f0)
    w = q(np.arange(nt) * dt)[None, :]
    out = {}
    for n, lay, kind in ((40, 8, "pml"), (40, 8, "sponge"), (120, 0, "ref")):
        g = oracle.Grid((n, n, n), dx, dt=dt, nt=nt, order=8, nb=lay, c_ref=c)
        ctr = (n // 2) * dx
        src = np.array([[ctr, ctr, ctr]])
        rec = np.array([[ctr, ctr, ctr + (20 - 8) * dx - 3e-3]])
        vp = np.full((n, n, n), c)
        if kind == "pml":
            out[kind] = pml.forward(g, vp, src, w, rec)[0]
        else:
            out[kind] = oracle.forward(g, vp, None, src[None], w[None], rec)[0, 0]
    ref = out["ref"]
    r = {k: np.sum((out[k] - ref) ** 2) / np.sum(ref ** 2) for k in ("pml", "sponge")}
    assert r["pml"] < 0.01 * r["sponge"] and r["pml"] < 2e-4, r   # measured 1.1e-5, 1.2e-2


def test_3d_gradient_central_differences():
    shape, dx = (16, 18, 20), 0.5e-3
    vp, _ = inputs.random_smooth_model(shape, dx, 2)
    dt = 0.35 * dx / vp.max()
    g = oracle.Grid(shape, dx, dt=dt, nt=70, order=8, nb=3, c_ref=1500.0)
    src = np.array([[4.1e-3, 4.3e-3, 4.6e-3]])
    rec = np.array([[3.2e-3, 5.1e-3, 6.4e-3], [0.6e-3, 3.3e-3, 2.9e-3]])   # one in the layer
    w = inputs.ricker(6e5, dt, g.nt)[None, :]
    obs = pml.forward(g, vp * 1.02, src, w, rec)
    J0, grad, _ = pml.gradient(g, vp, src, w, rec, obs)
    m = 1.0 / vp ** 2
    for p in [(8, 9, 7), (1, 8, 9)]:                          # the second lies in the layer
        h = 1e-4 * m[p]
        mp, mm = m.copy(), m.copy()
        mp[p] += h
        mm[p] -= h
        fd = (_misfit(g, 1 / np.sqrt(mp), src, w, rec, obs)
              - _misfit(g, 1 / np.sqrt(mm), src, w, rec, obs)) / (2 * h)
        assert fd == pytest.approx(grad[p], rel=1e-6, abs=1e-9 * np.abs(grad).max())


def _density_with_constant_rim(shape, dx, reach, seed=6):
    """Smooth random density in the interior, 1000 kg/m^3 over the outer
    `reach` points (the layer and the stencil reach next to it)."""
    _, rho = inputs.random_smooth_model(shape, dx, seed)
    idx = np.indices(shape)
    dist = np.min([np.minimum(i, n - 1 - i) for i, n in zip(idx, shape)], axis=0)
    ramp = np.clip((dist - reach) / 4.0, 0.0, 1.0)
    return 1000.0 + ramp * (rho - 1000.0)


def test_variable_density_without_a_layer_is_the_leapfrog_and_is_checked():
    shape, dx = (40, 44), 0.5e-3
    vp, rho = inputs.random_smooth_model(shape, dx, 1)
    dt = 0.4 * dx / vp.max()
    g = oracle.Grid(shape, dx, dt=dt, nt=150, order=8, nb=0, c_ref=1500.0)
    src = inputs.random_points(1, shape, dx, 2, margin=8)
    rec = inputs.random_points(4, shape, dx, 3, margin=8)
    w = inputs.ricker(5e5, dt, g.nt)[None, :]
    ref = oracle.forward(g, vp, rho, src[None], w[None], rec)[0]
    np.testing.assert_allclose(pml.forward(g, vp, src, w, rec, rho=rho), ref, rtol=0,
                               atol=1e-12 * np.abs(ref).max())
    g8 = oracle.Grid(shape, dx, dt=dt, nt=10, order=8, nb=8, c_ref=1500.0)
    with pytest.raises(ValueError):
        pml.forward(g8, vp, src, w[:, :10], rec, rho=rho)         # density varies in the layer


def test_variable_density_gradient_central_differences():
    g, vp, src, w, rec, _ = _gsetup()
    rho = _density_with_constant_rim(g.shape, 0.5e-3, g.nb + 4)
    obs = pml.forward(g, vp * 1.02, src, w, rec, rho=rho)
    J0, grad, _ = pml.gradient(g, vp, src, w, rec, obs, rho=rho)
    m = 1.0 / vp ** 2
    for p in [(20, 22), (14, 30), (3, 20)]:
        h = 1e-4 * m[p]
        mp, mm = m.copy(), m.copy()
        mp[p] += h
        mm[p] -= h
        Jp = 0.5 * np.sum((pml.forward(g, 1 / np.sqrt(mp), src, w, rec, rho=rho) - obs) ** 2)
        Jm = 0.5 * np.sum((pml.forward(g, 1 / np.sqrt(mm), src, w, rec, rho=rho) - obs) ** 2)
        assert (Jp - Jm) / (2 * h) == pytest.approx(grad[p], rel=1e-6, abs=1e-9 * np.abs(grad).max())
