"""The inversion loop on the GPU against the FP64 oracle (oracle/inversion.py):
the low-pass kernel, the gradient-descent update and whole iterations of the
Sec. 3.2 experiment at 1/8 scale (the same observed data on both sides, from
the oracle)."""
import numpy as np
import pytest

import oracle
from oracle import inversion as oinv
from paper_2110_03345_gb300 import binding, inputs, invert
from _helpers import rel_l2, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n_in,rows,nt,ids,dt,f,M", [
    (5, 3, 2085, [4, 0, 2, 2], 0.08e-6, 300e3, 125),     # several segments, ragged tail
    (2, 4, 700, [1], 25e-9, 300e3, 400),                  # M > 1024-sample segment / 2
    (3, 2, 100, [0, 2], 0.32e-6, 600e3, 150),              # filter longer than the record
    (1, 1, 5000, [0], 0.1e-6, 1e6, 2048),                  # largest half-width
    (700, 1, 64, list(range(699, -1, -1)), 1e-7, 1e6, 8),  # more ids than one launch takes
])
def test_lowpass_matches_oracle(n_in, rows, nt, ids, dt, f, M):
    rng = np.random.default_rng(n_in * 7 + M)
    x = rng.standard_normal((n_in, rows, nt))
    ref = oinv.lowpass(x[ids], dt, f, M)
    out = binding.lowpass(to_dev(x), ids, dt, f, M).cpu().numpy()
    assert rel_l2(out, ref) < 1e-5
    assert np.max(np.abs(out - ref)) < 1e-5 * max(np.max(np.abs(ref)), 1e-30) * 10


def test_lowpass_zero_width_copies_and_empty_is_a_no_op():
    rng = np.random.default_rng(1)
    x = to_dev(rng.standard_normal((3, 2, 333)))
    y = binding.lowpass(x, [2, 0], 1e-7, 1e6, 0)
    assert np.array_equal(y.cpu().numpy(), x[[2, 0]].cpu().numpy())
    e = binding.lowpass(x, [], 1e-7, 1e6, 8)
    assert tuple(e.shape) == (0, 2, 333)


def test_lowpass_rejects_bad_arguments():
    x = to_dev(np.zeros((2, 1, 50)))
    for args in [([2], 1e-7, 1e6, 8), ([-1], 1e-7, 1e6, 8), ([0], 0.0, 1e6, 8),
                 ([0], 1e-7, -1.0, 8), ([0], 1e-7, 1e6, 2049), ([0], 1e-7, 1e6, -1)]:
        with pytest.raises(binding.FwiError) as ei:
            binding.lowpass(x, *args)
        assert ei.value.status == 1
    with pytest.raises(binding.FwiError):
        binding.lowpass(x, [0, 1], 1e-7, 1e6, 8, out=x)          # overlaps its input


@pytest.mark.parametrize("masked", [False, True])
def test_vp_update_matches_oracle(masked):
    rng = np.random.default_rng(11 + masked)
    shape = (97, 131)                                            # ragged against 256 threads
    vp = rng.uniform(1450.0, 1550.0, shape)
    gm = rng.standard_normal(shape) * 1e-8
    mask = (rng.uniform(size=shape) > 0.3).astype(float) if masked else None
    ref = oinv.vp_update(vp.astype(np.float32), gm.astype(np.float32), 20.0, 1460.0, 1540.0, mask)
    v = to_dev(vp)
    binding.vp_update(v, to_dev(gm), 20.0, 1460.0, 1540.0, mask=None if mask is None else to_dev(mask))
    out = v.cpu().numpy()
    assert np.max(np.abs(out - ref)) < 2e-3
    assert out.min() >= 1460.0 and out.max() <= 1540.0
    if masked:                                                   # frozen points are only clipped
        frozen = np.clip(vp.astype(np.float32), 1460.0, 1540.0)[mask == 0]
        np.testing.assert_array_equal(out[mask == 0], frozen)


def test_vp_update_edge_cases():
    v = to_dev(np.full((5, 7), 1500.0))
    binding.vp_update(v, to_dev(np.zeros((5, 7))), 10.0, 1400.0, 1600.0)
    assert np.all(v.cpu().numpy() == 1500.0)                      # zero gradient: unchanged
    g = np.zeros((5, 7))
    g[2, 3] = np.nan
    binding.vp_update(v, to_dev(g), 10.0, 1400.0, 1600.0)
    assert np.all(np.isnan(v.cpu().numpy()))                      # non-finite: poisoned
    with pytest.raises(binding.FwiError):
        binding.vp_update(v, to_dev(g), -1.0, 1400.0, 1600.0)
    with pytest.raises(binding.FwiError):
        binding.vp_update(v, to_dev(g), 1.0, 1600.0, 1400.0)


def _setup(scale=8.0):
    p = inputs.config_inversion_2d(scale=scale)
    g = oracle.Grid(p.shape, p.spacing, p.dt, p.nt, p.order, p.nb, p.c_ref)
    obs = oracle.forward(g, p.vp_true, None, p.src_xyz, p.wavelet, p.rec_xyz)
    return p, g, obs


def _gpu_inversion(p, obs):
    plan = binding.Plan(p.shape, p.spacing, p.nt, p.dt, order=p.order, sponge=p.nb, c_ref=p.c_ref)
    run = invert.Inversion(plan, p.src_xyz, p.rec_xyz, to_dev(p.wavelet), to_dev(obs),
                           mask=to_dev(p.extra["mask"]), bounds=(1400.0, 1600.0),
                           filter_cycles=p.extra["filter_cycles"])
    return plan, run


def test_inversion_iterations_match_oracle():
    """Two blocks x two iterations of 16 shots: misfits and model updates."""
    p, g, obs = _setup()
    sched = [b[:2] for b in p.extra["schedule"][:2]]
    freqs = p.extra["freqs"][:2]
    M = [invert.half_width(f, p.dt, p.extra["filter_cycles"]) for f in freqs]
    vp_o, J_o = oinv.invert(g, p.vp, None, p.src_xyz, p.wavelet, p.rec_xyz, obs, freqs, sched,
                            10.0, 1400.0, 1600.0, p.extra["mask"], M)
    _, run = _gpu_inversion(p, obs)
    vp = to_dev(p.vp)
    rec = run.run(vp, freqs, sched, 10.0)
    vp_g = vp.cpu().numpy()
    for b in range(2):
        for i in range(2):
            assert rec.misfits[b][i] == pytest.approx(J_o[b][i], rel=1e-3)
    assert rel_l2(vp_g - p.vp, vp_o - p.vp) < 1e-2
    assert np.max(np.abs(vp_g - vp_o)) < 0.25
    assert np.array_equal(vp_g[p.extra["mask"] == 0], p.vp[p.extra["mask"] == 0])
    assert rec.shot_gradients == 64


def test_inversion_reduces_the_model_error():
    """All four blocks of the Sec. 3.2 schedule at 1/4 scale."""
    p, g, obs = _setup(scale=4.0)
    _, run = _gpu_inversion(p, obs)
    vp = to_dev(p.vp)
    rec = run.run(vp, p.extra["freqs"], p.extra["schedule"], 5.0)
    mask = p.extra["mask"]
    e0 = oinv.model_error(p.vp, p.vp_true, mask)
    e1 = oinv.model_error(vp.cpu().numpy(), p.vp_true, mask)
    assert e1 < 0.5 * e0, (e0, e1)           # the oracle run of this schedule: 23.8 -> 6.1 m/s
    assert rec.shot_gradients == 4 * 128
