"""Error handling of the C ABI on a GPU: every failure is a status code and a
message; the CUDA context stays usable afterwards.  No test faults the GPU:
the failures are bad arguments caught on the host, values flagged by the
model-validation kernel, and a bounded device wait made to give up on an
mbarrier that nothing completes (no copy in flight)."""
import numpy as np
import pytest

from paper_2110_03345_gb300 import binding, inputs
from _helpers import gpu_forward, to_dev

pytestmark = pytest.mark.gpu


def _problem():
    return inputs.breast_problem((64, 80), 0.5e-3, 60, nelem=16, shots=[0, 8], nb=8,
                                 radius=0.3 * 64 * 0.5e-3)


def _expect(status, fn):
    with pytest.raises(binding.FwiError) as ei:
        fn()
    assert ei.value.status == status, str(ei.value)
    assert len(str(ei.value)) > 20


def test_invalid_grid():
    _expect(1, lambda: binding.Plan((64, 80), 0.5e-3, 60, 1e-7, order=6))
    _expect(1, lambda: binding.Plan((64, 80), 0.5e-3, 60, 1e-7, sponge=40))
    _expect(1, lambda: binding.Plan((64, 80), 0.5e-3, 0, 1e-7))
    _expect(1, lambda: binding.Plan((64, 80), 0.5e-3, 60, -1.0))


def test_point_outside_grid():
    p = _problem()
    plan = binding.Plan(p.shape, p.spacing, p.nt, p.dt, sponge=p.nb, c_ref=1500.0)
    bad = p.src_xyz.copy()
    bad[0, 0, 1] = 1.0   # 1 m: far outside
    geo = binding.Geometry(bad, p.rec_xyz)
    _expect(1, lambda: plan.forward(to_dev(p.vp), None, geo, to_dev(p.wavelet)))


def test_unstable_cfl_rejected():
    p = _problem()
    plan = binding.Plan(p.shape, p.spacing, p.nt, p.dt * 1.5, sponge=p.nb, c_ref=1500.0)
    geo = binding.Geometry(p.src_xyz, p.rec_xyz)
    _expect(2, lambda: plan.forward(to_dev(p.vp), None, geo, to_dev(p.wavelet)))


def test_budget_exceeded():
    p = _problem()
    plan = binding.Plan(p.shape, p.spacing, p.nt, p.dt, sponge=p.nb, c_ref=1500.0, budget=1 << 16)
    geo = binding.Geometry(p.src_xyz, p.rec_xyz)
    _expect(3, lambda: plan.forward(to_dev(p.vp), None, geo, to_dev(p.wavelet)))


def test_nonfinite_and_nonpositive_model():
    p = _problem()
    plan = binding.Plan(p.shape, p.spacing, p.nt, p.dt, sponge=p.nb, c_ref=1500.0)
    geo = binding.Geometry(p.src_xyz, p.rec_xyz)
    vp = p.vp.copy()
    vp[10, 10] = np.nan
    _expect(5, lambda: plan.forward(to_dev(vp), None, geo, to_dev(p.wavelet)))
    rho = p.rho.copy()
    rho[3, 4] = 0.0
    _expect(5, lambda: plan.forward(to_dev(p.vp), to_dev(rho), geo, to_dev(p.wavelet)))
    # the plan and the context still work
    tr = plan.forward(to_dev(p.vp), to_dev(p.rho), geo, to_dev(p.wavelet))
    assert np.isfinite(tr.cpu().numpy()).all()


def test_estimate_and_stats():
    p = _problem()
    plan = binding.Plan(p.shape, p.spacing, p.nt, p.dt, sponge=p.nb, c_ref=1500.0)
    geo = binding.Geometry(p.src_xyz, p.rec_xyz)
    est_f = plan.estimate(geo, gradient=False)
    est_g = plan.estimate(geo, gradient=True)
    assert 0 < est_f < est_g
    _, plan = gpu_forward(p, plan=plan)
    s = plan.stats()
    assert s["fwd_launches"] == p.nt - 1 and s["batch"] == 2
    assert s["updates"] == 2 * 64 * 80 * (p.nt - 1)


def test_reserved_option_and_tile_range():
    p = _problem()
    plan = binding.Plan(p.shape, p.spacing, p.nt, p.dt, sponge=p.nb, c_ref=1500.0)
    lib = binding.load()
    import ctypes
    opts = binding.COptions(0, 0, 0, 0, 1, 0)   # use_graphs = 1
    assert lib.fwi_plan_set_options(plan._h, ctypes.byref(opts)) == 7   # FWI_ERR_UNSUPPORTED
    plan.set_options(tile=13)   # out of range: reported by the next call
    _expect(1, lambda: plan.forward(to_dev(p.vp), None, binding.Geometry(p.src_xyz, p.rec_xyz),
                                    to_dev(p.wavelet)))


def test_mem_available_counts_the_pool_reserve():
    """A destroyed plan's workspace stays reserved in the stream-ordered pool;
    fwi_mem_available still counts it, so a new plan's default budget does."""
    import torch
    free0, _ = torch.cuda.mem_get_info()
    a0 = binding.mem_available()
    assert a0 >= free0 * 0.99
    p = inputs.breast_problem((512, 512), 0.1e-3, 400, nelem=32, shots=list(range(8)), nb=20,
                              radius=0.4 * 512 * 0.1e-3)
    plan = binding.Plan(p.shape, p.spacing, p.nt, p.dt, sponge=p.nb, c_ref=1600.0)
    plan.forward(to_dev(p.vp), None, binding.Geometry(p.src_xyz, p.rec_xyz), to_dev(p.wavelet))
    held = plan.stats()["workspace_bytes"]
    plan.close()
    torch.cuda.synchronize()
    assert binding.mem_available() >= a0 - 0.05 * held - (64 << 20)


def test_sampled_launch_timing():
    """profile = n puts CUDA events around every n-th stencil launch."""
    p = _problem()
    plan = binding.Plan(p.shape, p.spacing, p.nt, p.dt, sponge=p.nb, c_ref=1500.0)
    geo = binding.Geometry(p.src_xyz, p.rec_xyz)
    for every, want in ((1, p.nt - 1), (4, (p.nt - 1 + 3) // 4), (0, 0)):
        plan.set_options(profile=every)
        plan.forward(to_dev(p.vp), None, geo, to_dev(p.wavelet))
        s = plan.stats()
        assert s["fwd_launches"] == p.nt - 1
        assert s["fwd_timed"] == want
        assert (s["fwd_ms"] > 0) == (want > 0)
    with pytest.raises(binding.FwiError):
        plan.set_options(profile=-1)


def test_equal_batches():
    """16 shots with at most 15 per launch run as two batches of 8."""
    p = inputs.breast_problem((64, 80), 0.5e-3, 40, nelem=32, shots=list(range(0, 32, 2)), nb=8,
                              radius=0.3 * 64 * 0.5e-3)
    plan = binding.Plan(p.shape, p.spacing, p.nt, p.dt, sponge=p.nb, c_ref=1500.0)
    plan.set_options(batch=15)
    plan.forward(to_dev(p.vp), None, binding.Geometry(p.src_xyz, p.rec_xyz), to_dev(p.wavelet))
    s = plan.stats()
    assert s["batch"] == 8 and s["fwd_launches"] == 2 * (p.nt - 1)


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    """The guard of every TMA pipeline wait: a wait that cannot complete gives
    up after its poll limit, the flag reaches the host as FWI_ERR_TIMEOUT,
    and the next call runs normally."""
    assert binding.check_bounded_wait(1000) == 6   # FWI_ERR_TIMEOUT
    assert "gave up after 1000 polls" in binding.load().fwi_last_error().decode()
    assert binding.check_bounded_wait(0) == 1      # FWI_ERR_INVALID_ARG
    p = _problem()
    ref, _ = gpu_forward(p)
    assert np.isfinite(ref).all() and np.abs(ref).max() > 0
