"""Pins for the oracle of the inversion loop (oracle/inversion.py).

  low-pass            frequency response (unit gain at 0, half gain at the
                      cut-off, flat pass band, small stop band), zero phase,
                      brute force and numpy.convolve, commutes with the solver
  dJ/dvp              central finite differences of the misfit in vp
  gradient descent    descent, step normalisation, clipping, mask, zero gradient
  inversion loop      zero step keeps the model and gives the per-shot-subset
                      misfits; the error to the true model falls; the
                      filtered data agree at the true model
"""
import numpy as np
import pytest

import oracle
from oracle import inversion as inv
from paper_2110_03345_gb300 import inputs


def response(h, f, dt):
    """|H(f)| of taps h_j, j = -M..M (zero-phase: H is real)."""
    M = (len(h) - 1) // 2
    j = np.arange(-M, M + 1)
    return np.abs(np.exp(-2j * np.pi * np.outer(f, j) * dt) @ h)


@pytest.mark.parametrize("dt,f_max", [(0.08e-6, 300e3), (0.08e-6, 600e3), (25e-9, 300e3),
                                      (0.32e-6, 75e3)])
def test_lowpass_frequency_response(dt, f_max):
    M = int(np.ceil(3.0 / (f_max * dt)))
    h = inv.lowpass_taps(dt, f_max, M)
    assert len(h) == 2 * M + 1
    np.testing.assert_allclose(h, h[::-1], rtol=0, atol=1e-15)      # zero phase
    assert h.sum() == pytest.approx(1.0, abs=1e-13)                  # unit DC gain
    assert response(h, [f_max], dt)[0] == pytest.approx(0.5, abs=0.01)
    fp = np.linspace(0.0, 0.7 * f_max, 64)
    assert np.max(np.abs(response(h, fp, dt) - 1.0)) < 0.01
    fs = np.linspace(1.5 * f_max, min(6 * f_max, 0.5 / dt), 256)
    assert np.max(response(h, fs, dt)) < 2.5e-3


def test_lowpass_is_the_stated_convolution():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((3, 257))
    dt, f, M = 0.1e-6, 400e3, 40
    h = inv.lowpass_taps(dt, f, M)
    y = inv.lowpass(x, dt, f, M)
    for r in range(3):
        np.testing.assert_allclose(y[r], np.convolve(x[r], h, mode="same"), rtol=0, atol=1e-13)
    # filter longer than the record: brute force with zero extension
    xs = rng.standard_normal(7)
    hs = inv.lowpass_taps(dt, 2e6, 9)
    ys = inv.lowpass(xs, dt, 2e6, 9)
    ref = [sum(hs[j + 9] * xs[n - j] for j in range(-9, 10) if 0 <= n - j < 7) for n in range(7)]
    np.testing.assert_allclose(ys, ref, rtol=0, atol=1e-14)
    np.testing.assert_array_equal(inv.lowpass(x, dt, f, 0), x)     # M = 0: identity


def test_lowpass_keeps_low_and_removes_high_frequencies():
    dt, f = 0.08e-6, 300e3
    M = int(np.ceil(3.0 / (f * dt)))
    t = np.arange(4000) * dt
    lo = np.cos(2 * np.pi * 0.3 * f * t + 0.4)
    hi = np.cos(2 * np.pi * 3.0 * f * t)
    y = inv.lowpass(lo + hi, dt, f, M)
    core = slice(M, 4000 - M)
    assert np.max(np.abs(y[core] - lo[core])) < 1e-2                # no phase shift


def test_lowpass_commutes_with_the_solver():
    """The solver is linear and time invariant in the source: low-passing the
    wavelet low-passes the traces, exactly for n < nt - M (beyond, the
    traces' low-pass would need samples after the record)."""
    p = inputs.config_homogeneous_2d(n=64, dx=0.5e-3, nt=300, nrec=6, radius=10e-3, f0=300e3)
    g = oracle.Grid(p.shape, p.spacing, p.dt, p.nt, p.order, p.nb, p.c_ref)
    f, M = 400e3, 40
    w = inputs.tone_burst(300e3, p.dt, p.nt, t0=(M + 5) * p.dt)[None, None, :]
    d = oracle.forward(g, p.vp, None, p.src_xyz, w, p.rec_xyz)
    d_f = oracle.forward(g, p.vp, None, p.src_xyz, inv.lowpass(w, p.dt, f, M), p.rec_xyz)
    ref = inv.lowpass(d, p.dt, f, M)
    n = p.nt - M
    scale = np.max(np.abs(ref))
    assert scale > 0
    np.testing.assert_allclose(d_f[..., :n], ref[..., :n], rtol=0, atol=1e-11 * scale)
    assert np.max(np.abs(d_f[..., n:] - ref[..., n:])) > 1e-6 * scale   # the stated edge


def small_cd_problem(seed=1):
    shape, dx = (40, 44), 0.5e-3
    vp, _ = inputs.random_smooth_model(shape, dx, seed)
    dt = 0.4 * dx / vp.max()
    g = oracle.Grid(shape, dx, dt=dt, nt=140, order=8, nb=8, c_ref=1500.0)
    src = inputs.random_points(2, shape, dx, seed + 1, margin=10)[:, None, :]
    rec = inputs.random_points(6, shape, dx, seed + 2, margin=10)
    wav = np.stack([inputs.ricker(500e3, dt, g.nt)[None], inputs.ricker(600e3, dt, g.nt)[None]])
    true = vp * (1.0 + 0.04 * np.exp(-0.5 * ((np.indices(shape) - 21.0) ** 2).sum(0) / 36.0))
    obs = oracle.forward(g, true, None, src, wav, rec)
    return g, vp, src, wav, rec, obs


def test_vp_gradient_matches_finite_differences():
    g, vp, src, wav, rec, obs = small_cd_problem()
    J, gm, _ = oracle.gradient(g, vp, None, src, wav, rec, obs)
    gv = inv.vp_gradient(gm, vp)
    for idx in [(20, 22), (15, 30), (25, 12)]:
        h = 1e-4 * vp[idx]
        vpp, vpm = vp.copy(), vp.copy()
        vpp[idx] += h
        vpm[idx] -= h
        Jp = oracle.gradient(g, vpp, None, src, wav, rec, obs)[0]
        Jm = oracle.gradient(g, vpm, None, src, wav, rec, obs)[0]
        fd = (Jp - Jm) / (2 * h)
        assert gv[idx] == pytest.approx(fd, rel=1e-4, abs=1e-7 * np.abs(gv).max())


def test_vp_update_descends_and_normalises():
    g, vp, src, wav, rec, obs = small_cd_problem()
    J, gm, _ = oracle.gradient(g, vp, None, src, wav, rec, obs)
    step = 2.0
    new = inv.vp_update(vp, gm, step, 1000.0, 2000.0)
    d = inv.vp_gradient(gm, vp)
    k = np.unravel_index(np.argmax(np.abs(d)), d.shape)
    assert np.max(np.abs(new - vp)) == pytest.approx(step, rel=1e-12)
    assert new[k] - vp[k] == pytest.approx(-step * np.sign(d[k]), rel=1e-12)
    J1 = oracle.gradient(g, new, None, src, wav, rec, obs)[0]
    assert J1 < J


def test_vp_update_clips_masks_and_ignores_zero_gradient():
    rng = np.random.default_rng(5)
    vp = rng.uniform(1450.0, 1550.0, (30, 31))
    gm = rng.standard_normal((30, 31)) * 1e-9
    new = inv.vp_update(vp, gm, 80.0, 1480.0, 1520.0)
    assert new.min() >= 1480.0 and new.max() <= 1520.0
    raw = vp - 80.0 * inv.vp_gradient(gm, vp) / np.max(np.abs(inv.vp_gradient(gm, vp)))
    np.testing.assert_array_equal(new[raw >= 1520.0], 1520.0)
    np.testing.assert_array_equal(new[raw <= 1480.0], 1480.0)
    mask = (rng.uniform(size=vp.shape) > 0.5).astype(float)
    m_new = inv.vp_update(vp, gm, 5.0, 0.0, 1e4, mask)
    np.testing.assert_array_equal(m_new[mask == 0], vp[mask == 0])
    assert np.max(np.abs(m_new - vp)) == pytest.approx(5.0, rel=1e-12)
    np.testing.assert_array_equal(inv.vp_update(vp, np.zeros_like(vp), 5.0, 0.0, 1e4), vp)


def tiny_inversion(scale=8.0):
    p = inputs.config_inversion_2d(scale=scale)
    g = oracle.Grid(p.shape, p.spacing, p.dt, p.nt, p.order, p.nb, p.c_ref)
    obs = oracle.forward(g, p.vp_true, None, p.src_xyz, p.wavelet, p.rec_xyz)
    M = [int(np.ceil(p.extra["filter_cycles"] / (f * p.dt))) for f in p.extra["freqs"]]
    return p, g, obs, M


def test_invert_with_zero_step_reports_the_subset_misfits():
    p, g, obs, M = tiny_inversion()
    sched = [[s[0], s[1]] for s in p.extra["schedule"][:2]]      # two blocks, two iterations
    freqs = p.extra["freqs"][:2]
    vp, Js = inv.invert(g, p.vp, None, p.src_xyz, p.wavelet, p.rec_xyz, obs, freqs, sched,
                        0.0, 1400.0, 1600.0, p.extra["mask"], M[:2])
    np.testing.assert_array_equal(vp, p.vp)
    for b in range(2):
        for i in range(2):
            ids = sched[b][i]
            wf = inv.lowpass(p.wavelet[ids], p.dt, freqs[b], M[b])
            of = inv.lowpass(obs[ids], p.dt, freqs[b], M[b])
            J = oracle.gradient(g, p.vp, None, p.src_xyz[ids], wf, p.rec_xyz, of)[0]
            assert Js[b][i] == pytest.approx(J, rel=1e-12)
            assert J > 0


def test_invert_reduces_the_model_error():
    """The first four iterations (64 shots) of the Sec. 3.2 experiment at 1/4
    scale (at 1/8 scale the filter's record-end edge dominates the misfit)."""
    p = inputs.config_inversion_2d(scale=4.0)
    g = oracle.Grid(p.shape, p.spacing, p.dt, p.nt, p.order, p.nb, p.c_ref)
    sched = [p.extra["schedule"][0][:4]]
    used = np.concatenate(sched[0])
    obs = np.zeros((p.nshots, p.rec_xyz.shape[0], p.nt))
    obs[used] = oracle.forward(g, p.vp_true, None, p.src_xyz[used], p.wavelet[used], p.rec_xyz)
    M = [int(np.ceil(p.extra["filter_cycles"] / (p.extra["freqs"][0] * p.dt)))]
    mask = p.extra["mask"]
    vp, Js = inv.invert(g, p.vp, None, p.src_xyz, p.wavelet, p.rec_xyz, obs,
                        p.extra["freqs"][:1], sched, 5.0, 1400.0, 1600.0, mask, M)
    e0 = inv.model_error(p.vp, p.vp_true, mask)
    e1 = inv.model_error(vp, p.vp_true, mask)
    assert e1 < 0.9 * e0, (e0, e1)                         # measured 23.8 -> 20.7 m/s
    np.testing.assert_array_equal(vp[mask == 0], p.vp[mask == 0])


def test_filtered_data_agree_at_the_true_model():
    """Low-passing the wavelet stands for low-passing the modelled traces; the
    two differ only where the traces' low-pass would need samples after the
    record.  At half scale (and at full scale, 1e-4) that leaves the misfit of
    the true model negligible against the starting model's."""
    p = inputs.config_inversion_2d(scale=2.0)
    g = oracle.Grid(p.shape, p.spacing, p.dt, p.nt, p.order, p.nb, p.c_ref)
    s = [5]
    f = p.extra["freqs"][0]
    M = int(np.ceil(p.extra["filter_cycles"] / (f * p.dt)))
    obs = oracle.forward(g, p.vp_true, None, p.src_xyz[s], p.wavelet[s], p.rec_xyz)
    wf = inv.lowpass(p.wavelet[s], p.dt, f, M)
    of = inv.lowpass(obs, p.dt, f, M)
    J_true = oracle.gradient(g, p.vp_true, None, p.src_xyz[s], wf, p.rec_xyz, of)[0]
    J_start = oracle.gradient(g, p.vp, None, p.src_xyz[s], wf, p.rec_xyz, of)[0]
    assert J_true < 2e-3 * J_start, (J_true, J_start)      # measured 5e-4
