"""Extended schemes of Sec. 2.4 on the GPU against their FP64 oracles.

* The fourth-order-in-time scheme (options.time_order = 4; oracle/time4.py):
  traces and gradient in 2D (8th order, constant and variable density) and
  3D (10th order, variable density), at time steps beyond the leapfrog's
  stability limit, with full history and with checkpoints.
* The power-law attenuation term of Eq. 10 with y = 0 and y = 2
  (fwi_model.alpha0, oracle/attenuation.py): traces and gradient with a
  spatially varying alpha0, in 2D and 3D, with and without density, with
  full history and with checkpoints.

Tolerances as for the leapfrog: relative L2 of 1e-4 on traces, 1e-3 on
gradients; misfits within 1e-3.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import attenuation as oatt
from oracle import time4 as ot4
from paper_2110_03345_gb300 import binding, inputs
from _helpers import TOL_GRAD, TOL_TRACES, rel_l2, to_dev

pytestmark = pytest.mark.gpu


def problem(shape, dx, nt, order, cfl, nb, nshots=2, nsrc=1, nrec=12, seed=0, f0=None):
    vp, rho = inputs.random_smooth_model(shape, dx, seed)
    dt = cfl * dx / vp.max()
    src = inputs.random_points(nshots * nsrc, shape, dx, seed + 1, margin=nb + 2)
    src = src.reshape(nshots, nsrc, len(shape))
    rec = inputs.random_points(nrec, shape, dx, seed + 2, margin=nb + 2)
    f0 = f0 or 0.25 * 1500.0 / dx / 4.0      # ~16 points per wavelength at the peak
    w = inputs.ricker(f0, dt, nt)
    wav = np.broadcast_to(w, (nshots, nsrc, nt)).copy()
    p = inputs.Problem("ext", shape, dx, dt, nt, order, nb, vp, rho, src, rec, wav,
                       c_ref=float(vp.max()))
    idx = np.indices(shape).astype(float)
    ctr = (np.array(shape, dtype=float) / 2).reshape((-1,) + (1,) * len(shape))
    p.vp_true = vp * (1.0 + 0.04 * np.exp(-((idx - ctr) ** 2).sum(0) / (0.2 * min(shape)) ** 2))
    return p


def ogrid(p):
    return oracle.Grid(p.shape, p.spacing, dt=p.dt, nt=p.nt, order=p.order, nb=p.nb, c_ref=p.c_ref)


def run_gpu(p, vd, time_order=0, alpha0=None, y=0, ckpt=-1, observed=None, vp=None):
    plan = binding.Plan(p.shape, p.spacing, p.nt, p.dt, order=p.order, sponge=p.nb, c_ref=p.c_ref)
    plan.set_options(time_order=time_order, ckpt_every=ckpt)
    a0 = to_dev(alpha0) if alpha0 is not None else None
    plan.set_attenuation(a0, y)
    geo = binding.Geometry(p.src_xyz, p.rec_xyz)
    v = to_dev(p.vp if vp is None else vp)
    rho = to_dev(p.rho) if vd else None
    wav = to_dev(p.wavelet)
    if observed is None:
        out = plan.forward(v, rho, geo, wav).cpu().numpy().astype(np.float64)
        plan.close()
        return out
    J, g, d = plan.gradient(v, rho, geo, wav, to_dev(observed), traces=True)
    st = plan.stats()
    plan.close()
    return J, g.cpu().numpy().astype(np.float64), d.cpu().numpy().astype(np.float64), st


# ----------------------------------------------------------------- fourth order

T4_CASES = {
    "2d-o8-cd": dict(shape=(70, 83), dx=0.4e-3, nt=220, order=8, cfl=0.8, nb=8, vd=False),
    "2d-o8-vd": dict(shape=(70, 83), dx=0.4e-3, nt=220, order=8, cfl=0.8, nb=8, vd=True),
    "3d-o10-vd": dict(shape=(30, 34, 37), dx=0.5e-3, nt=110, order=10, cfl=0.65, nb=6, vd=True),
}


@pytest.mark.parametrize("case", list(T4_CASES))
def test_time4_forward(case):
    c = dict(T4_CASES[case])
    vd = c.pop("vd")
    p = problem(**c)
    got = run_gpu(p, vd, time_order=4)
    rho = p.rho if vd else None
    for s in range(p.nshots):
        ref = ot4.forward(ogrid(p), p.vp, rho, p.src_xyz[s], p.wavelet[s], p.rec_xyz)
        assert rel_l2(got[s], ref) <= TOL_TRACES


def test_time4_rejects_steps_beyond_its_limit():
    c = dict(T4_CASES["2d-o8-cd"])
    c.pop("vd")
    c["cfl"] = 1.0       # above sqrt(3) x the leapfrog limit (0.96 for order 8 in 2D)
    p = problem(**c)
    with pytest.raises(binding.FwiError) as ei:
        run_gpu(p, False, time_order=4)
    assert ei.value.status == 2


@pytest.mark.parametrize("case,ckpt", [("2d-o8-cd", -1), ("2d-o8-vd", 17), ("3d-o10-vd", -1)])
def test_time4_gradient(case, ckpt):
    c = dict(T4_CASES[case])
    vd = c.pop("vd")
    p = problem(**c)
    rho = p.rho if vd else None
    g = ogrid(p)
    obs = np.stack([ot4.forward(g, p.vp_true, rho, p.src_xyz[s], p.wavelet[s], p.rec_xyz)
                    for s in range(p.nshots)])
    J_ref, g_ref, d_ref = 0.0, np.zeros(p.shape), []
    for s in range(p.nshots):
        J_s, g_s, d_s = ot4.gradient(g, p.vp, rho, p.src_xyz[s], p.wavelet[s], p.rec_xyz, obs[s])
        J_ref += J_s
        g_ref += g_s
        d_ref.append(d_s)
    J, gg, d, st = run_gpu(p, vd, time_order=4, ckpt=ckpt, observed=obs)
    assert st["ckpt_every"] == (0 if ckpt < 0 else ckpt)
    assert rel_l2(d, np.stack(d_ref)) <= TOL_TRACES
    assert abs(J - J_ref) <= 1e-3 * abs(J_ref)
    assert rel_l2(gg, g_ref) <= TOL_GRAD


# ----------------------------------------------------------------- attenuation

# nepers/m (y = 0), nepers/m/(rad/s)^2 (y = 2): 100 times typical soft tissue,
# so that the term matters within a few hundred steps.  The y = 2 term is
# explicit (a backward difference in time): with r = k lambda_max and
# s = r (2 alpha0 vp / dt) the step is stable for r + 2 s <= 4, which 4e-12
# keeps (s < 0.5 here) and 2e-11 would break in 3D.
ALPHA = {0: 200.0, 2: 4e-12}

ATT_CASES = {
    "2d-y0-vd": dict(ndim=2, y=0, vd=True),
    "2d-y0-cd": dict(ndim=2, y=0, vd=False),
    "2d-y2-vd": dict(ndim=2, y=2, vd=True),
    "2d-y2-cd": dict(ndim=2, y=2, vd=False),
    "3d-y0-vd": dict(ndim=3, y=0, vd=True),
    "3d-y2-vd": dict(ndim=3, y=2, vd=True),
}


def att_problem(ndim):
    if ndim == 2:
        p = problem((62, 71), 0.5e-3, 200, 8, 0.4, 8)
    else:
        p = problem((28, 30, 33), 0.5e-3, 110, 10, 0.35, 6)
    return p


def alpha_field(p, y, seed=7):
    a, _ = inputs.random_smooth_model(p.shape, p.spacing, seed, c_range=(0.5, 1.5))
    return ALPHA[y] * a


@pytest.mark.parametrize("case", list(ATT_CASES))
def test_attenuation_forward(case):
    c = ATT_CASES[case]
    p = att_problem(c["ndim"])
    a0 = alpha_field(p, c["y"])
    got = run_gpu(p, c["vd"], alpha0=a0, y=c["y"])
    rho = p.rho if c["vd"] else None
    lossless = run_gpu(p, c["vd"])
    for s in range(p.nshots):
        ref = oatt.forward(ogrid(p), p.vp, rho, a0.reshape(-1), c["y"], p.src_xyz[s], p.wavelet[s],
                           p.rec_xyz)
        assert rel_l2(got[s], ref) <= TOL_TRACES
    # the attenuation is not negligible at this strength
    assert rel_l2(got, lossless) > 1e-2


@pytest.mark.parametrize("case,ckpt", [("2d-y0-vd", -1), ("2d-y2-cd", -1), ("2d-y2-vd", 13),
                                       ("2d-y0-cd", 13), ("3d-y0-vd", -1), ("3d-y2-vd", 11)])
def test_attenuation_gradient(case, ckpt):
    c = ATT_CASES[case]
    y = c["y"]
    p = att_problem(c["ndim"])
    a0 = alpha_field(p, y)
    rho = p.rho if c["vd"] else None
    g = ogrid(p)
    a0f = a0.reshape(-1)      # the oracle takes a field flattened
    obs = np.stack([oatt.forward(g, p.vp_true, rho, a0f, y, p.src_xyz[s], p.wavelet[s], p.rec_xyz)
                    for s in range(p.nshots)])
    J_ref, g_ref, d_ref = 0.0, np.zeros(p.shape), []
    for s in range(p.nshots):
        J_s, g_s, d_s = oatt.gradient(g, p.vp, rho, a0f, y, p.src_xyz[s], p.wavelet[s], p.rec_xyz,
                                      obs[s])
        J_ref += J_s
        g_ref += g_s
        d_ref.append(d_s)
    J, gg, d, st = run_gpu(p, c["vd"], alpha0=a0, y=y, ckpt=ckpt, observed=obs)
    assert st["ckpt_every"] == (0 if ckpt < 0 else ckpt)
    assert rel_l2(d, np.stack(d_ref)) <= TOL_TRACES
    assert abs(J - J_ref) <= 1e-3 * abs(J_ref)
    assert rel_l2(gg, g_ref) <= TOL_GRAD


def test_attenuation_y2_refuses_unstable_strength():
    """alpha0 beyond the y = 2 term's stability bound is refused before any step."""
    p = att_problem(3)
    with pytest.raises(binding.FwiError) as ei:
        run_gpu(p, True, alpha0=np.full(p.shape, 5e-11), y=2)
    assert ei.value.status == 2


def test_attenuation_zero_alpha_is_the_leapfrog():
    """alpha0 = 0 through the attenuation kernels gives the default kernels'
    traces to rounding (different kernel family and summation order)."""
    p = att_problem(2)
    ref = run_gpu(p, True)
    for y in (0, 2):
        got = run_gpu(p, True, alpha0=np.zeros(p.shape), y=y)
        assert rel_l2(got, ref) <= 1e-6
