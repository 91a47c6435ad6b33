"""Host-side logic that needs no GPU: the seeded workload generators (sizes,
determinism, the time step at CFL 0.4), the serving latency statistics and
the autotuner's problem classes."""
import types

import numpy as np
import pytest

from paper_2110_03345_gb300 import autotune, inputs, serve


def test_breast_workload_matches_its_description():
    p = inputs.config_breast_2d(n=128, dx=0.8e-3, nt=40)   # same recipe, scaled down
    assert p.shape == (128, 128) and p.nshots == 128 and p.rec_xyz.shape == (256, 2)
    # sources are the even ring elements, every element receives
    np.testing.assert_allclose(p.src_xyz[:, 0, :], p.rec_xyz[::2])
    assert 1400.0 <= p.vp.min() and p.vp.max() <= 1600.0
    assert 950.0 <= p.rho.min() and p.rho.max() <= 1100.0
    assert p.dt == pytest.approx(0.4 * 0.8e-3 / 1600.0)
    assert not np.array_equal(p.vp, p.vp_true)             # observed data from a perturbed model


def test_full_size_breast_time_step():
    """The 1024^2 benchmark workload: 0.1 mm, CFL 0.4 at c_max = 1600 m/s gives 25 ns."""
    assert inputs.cfl_dt(0.1e-3, 1600.0, 0.4) == pytest.approx(25e-9)


def test_generators_are_seeded():
    a = inputs.config_breast_2d(n=96, dx=1e-3, nt=20)
    b = inputs.config_breast_2d(n=96, dx=1e-3, nt=20)
    assert np.array_equal(a.vp, b.vp) and np.array_equal(a.rho, b.rho)
    assert np.array_equal(a.wavelet, b.wavelet)
    s1 = inputs.config_skull_3d(n=40, dx=1.6e-3, nt=20)
    s2 = inputs.config_skull_3d(n=40, dx=1.6e-3, nt=20)
    assert np.array_equal(s1.vp, s2.vp) and np.array_equal(s1.rec_xyz, s2.rec_xyz)
    assert s1.nshots == 32 and s1.rec_xyz.shape == (512, 3)
    assert set(np.unique(s1.vp)) >= {1500.0, 2800.0}


def test_uneven_batch_recipe():
    ps = inputs.config_uneven_batch(nprob=12, seed=4, side=(64, 128), nt=(50, 80), shots=(1, 16))
    assert len(ps) == 12
    for p in ps:
        assert p.shape[0] == p.shape[1] and p.shape[0] % 4 == 0 and 64 <= p.shape[0] <= 128
        assert 50 <= p.nt <= 80 and 1 <= p.nshots <= 16
    ps2 = inputs.config_uneven_batch(nprob=12, seed=4, side=(64, 128), nt=(50, 80), shots=(1, 16))
    assert [p.shape for p in ps] == [p.shape for p in ps2]


def test_serving_stream_recipe():
    st = inputs.config_serving(nreq=200, seed=5, rate=20.0, side2d=(64, 96), side3d=(24, 32),
                               nt=(30, 40))
    t = np.array([a for a, _, _ in st])
    assert np.all(np.diff(t) > 0)
    assert 200 / t[-1] == pytest.approx(20.0, rel=0.25)     # Poisson at 20 per second
    frac2d = np.mean([len(p.shape) == 2 for _, _, p in st])
    fracfwd = np.mean([k == "forward" for _, k, _ in st])
    assert 0.65 < frac2d < 0.85 and 0.4 < fracfwd < 0.6
    assert all(p.nshots == 1 for _, _, p in st)


def test_latency_statistics():
    reqs = [types.SimpleNamespace(t_submit=float(i), t_done=float(i) + 1.0 + (i == 99) * 9.0,
                                  shots=1) for i in range(100)]
    st = serve.latency_stats(reqs)
    assert st["p50_s"] == pytest.approx(1.0)
    assert st["p99_s"] > 1.0 and st["requests"] == 100
    assert st["shots_per_s"] == pytest.approx(100 / (109.0 - 0.0))


def test_autotune_problem_classes():
    k1 = autotune.problem_key((1024, 1024), 8, True, True, 15)
    k2 = autotune.problem_key((1000, 1020), 8, True, True, 15)   # same tile-rounded class
    k3 = autotune.problem_key((1024, 1024), 8, True, True, 8)
    assert k1 == k2 and k1 != k3
    assert autotune.problem_key((256, 256, 256), 10, True, True, 1).startswith("3d-o10-vd-grad")
    assert all(5 <= c["tile"] <= 12 for c in autotune.CANDIDATES_3D)   # TMA-staged 3D variants


def test_shot_schedule_uses_every_shot_once_per_block():
    s = inputs.shot_schedule(128, 16, 4, seed=7)
    assert len(s) == 4 and all(len(b) == 8 for b in s)
    for b in s:
        ids = np.concatenate(b)
        assert sorted(ids.tolist()) == list(range(128))
    assert not np.array_equal(np.concatenate(s[0]), np.concatenate(s[1]))
    again = inputs.shot_schedule(128, 16, 4, seed=7)
    assert all(np.array_equal(x, y) for bx, by in zip(s, again) for x, y in zip(bx, by))
    ragged = inputs.shot_schedule(10, 4, 1, seed=1)[0]
    assert [len(x) for x in ragged] == [4, 4, 2]


def _golden(name):
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    return {r[0]: [float(v) for v in r[1:]] for r in rows}


def test_inversion_workload_matches_the_paper_setup():
    """The Sec. 3.2 values in tests/golden/paper_sec32_setup.txt."""
    ref = _golden("paper_sec32_setup.txt")
    p = inputs.config_inversion_2d()
    assert list(p.shape) == [int(v) for v in ref["grid"]] and p.spacing == ref["dx_m"][0]
    assert p.dt == pytest.approx(ref["dt_s"][0]) and p.rho is None
    assert p.nt * p.dt == pytest.approx(ref["duration_s"][0])
    assert p.nshots == ref["transducers"][0] and p.rec_xyz.shape == (ref["transducers"][0], 2)
    np.testing.assert_allclose(p.src_xyz[:, 0, :], p.rec_xyz)        # every transducer fires
    assert np.all(p.vp == ref["start_vp"][0]) and p.vp_true.min() >= 1400.0
    cfl = p.vp_true.max() * p.dt / p.spacing
    assert cfl <= ref["cfl_max"][0] + 5e-3 and cfl > ref["cfl_max"][0] - 0.02
    f = p.extra["freqs"]
    assert f[0] == ref["f_first_hz"][0] and f[-1] == ref["f_last_hz"][0]
    assert all(len(b) == ref["iterations"][0] for b in p.extra["schedule"])
    assert all(len(i) == ref["shots_per_iter"][0] for b in p.extra["schedule"] for i in b)
    w = p.wavelet[0, 0]
    on = np.nonzero(w)[0]
    assert on[0] * p.dt >= 3.0 / f[0] - p.dt                          # burst after the filter reach
    T = ref["burst_cycles"][0] / ref["burst_hz"][0]
    assert (on[-1] - on[0]) * p.dt == pytest.approx(T, abs=3 * p.dt)
    spec = np.abs(np.fft.rfft(w, 1 << 16))
    fr = np.fft.rfftfreq(1 << 16, p.dt)
    assert fr[np.argmax(spec)] == pytest.approx(ref["burst_hz"][0], rel=0.05)   # centred at 500 kHz
    small = inputs.config_inversion_2d(scale=4)
    assert small.shape == (114, 121) and small.dt == pytest.approx(0.32e-6)
    assert small.extra["mask"].max() == 1.0 and small.extra["mask"][0, 0] == 0.0


def test_inversion_filter_half_width():
    from paper_2110_03345_gb300 import invert
    assert invert.half_width(300e3, 0.08e-6) == 125                 # 3 periods of 300 kHz
    assert invert.half_width(600e3, 0.08e-6) == 63
    assert invert.half_width(300e3, 0.08e-6, cycles=1.0) == 42
    with pytest.raises(ValueError):
        invert.half_width(1e3, 0.08e-6)                            # beyond the kernel's 2048


def test_inversion_driver_checks_its_arguments_on_the_host():
    """invert.Inversion and binding.lowpass reject inconsistent arrays before
    any device work (CPU tensors stand in for the device arrays here)."""
    torch = pytest.importorskip("torch")
    from paper_2110_03345_gb300 import binding, invert
    plan = types.SimpleNamespace(nt=50, dt=1e-7, shape=(16, 16), stream=None)
    src = np.zeros((4, 1, 2))
    rec = np.zeros((6, 2))
    wav = torch.zeros((4, 1, 50))
    obs = torch.zeros((4, 6, 50))
    invert.Inversion(plan, src, rec, wav, obs)                          # consistent: accepted
    with pytest.raises(ValueError):
        invert.Inversion(plan, src, rec, wav, torch.zeros((3, 6, 50)))  # shot count
    with pytest.raises(ValueError):
        invert.Inversion(plan, src, rec, torch.zeros((4, 1, 40)), torch.zeros((4, 6, 40)))  # nt
    with pytest.raises(ValueError):
        invert.Inversion(plan, src, np.zeros((5, 2)), wav, obs)         # receiver count
    run = invert.Inversion(plan, src, rec, wav, obs, max_shots=2)
    with pytest.raises(ValueError):
        run.iterate(torch.zeros((16, 16)), [0, 1, 2], 1e6, 1.0)         # more than max_shots
    assert run.iterate(torch.zeros((16, 16)), [], 1e6, 1.0) == 0.0     # nothing to do
    with pytest.raises(ValueError):
        binding.lowpass(torch.zeros((4, 50)), [0], 1e-7, 1e6, 8)        # not [n][rows][nt]


def test_binding_checks_array_sizes_and_devices():
    """The C ABI takes bare pointers; the binding checks element counts and
    devices before any call, so a short array cannot be read past its end."""
    torch = pytest.importorskip("torch")
    from paper_2110_03345_gb300 import binding
    t = torch.zeros((3, 4, 5))
    binding.check_array(t, 60, "t")                                    # exact count: accepted
    binding.check_array(None, 60, "t", optional=True)
    with pytest.raises(ValueError, match="expected 64"):
        binding.check_array(t, 64, "t")
    with pytest.raises(ValueError, match="required"):
        binding.check_array(None, 60, "t")
    with pytest.raises(ValueError, match="plan runs on"):
        binding.check_array(t, 60, "t", device=torch.device("cuda", 0))
