"""Differentiation pattern: the split gradient (fwi_misfit_forward /
fwi_misfit_backward) and the torch.autograd.Function built on it, against
the fused fwi_gradient, the FP64 oracle and finite differences."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2110_03345_gb300 import autograd, binding, inputs
from _helpers import (TOL_GRAD, TOL_TRACES, gpu_gradient, gpu_plan, observed_from_oracle,
                      oracle_grid, rel_l2, strong_perturbation, to_dev)

pytestmark = pytest.mark.gpu


def breast(n=(140, 157), nt=300, shots=(0, 30, 64, 90)):
    p = inputs.breast_problem(n, 0.25e-3, nt, nelem=128, shots=list(shots), order=8, nb=20,
                              radius=0.35 * min(n) * 0.25e-3)
    p.vp_true = strong_perturbation(p)
    return p


def skull(n=(40, 44, 48), nt=180):
    p = inputs.skull_problem(n, 0.5e-3, nt, nrec=64, every=32, order=10, nb=8,
                             radius=0.33 * min(n) * 0.5e-3)
    p.vp_true = strong_perturbation(p)
    return p


def _args(p):
    geo = binding.Geometry(p.src_xyz, p.rec_xyz)
    return geo, to_dev(p.rho), to_dev(p.wavelet)


@pytest.mark.parametrize("ckpt", [-1, 7])
def test_split_equals_fused(ckpt):
    p = breast()
    obs = observed_from_oracle(p)
    J0, g0, d0, _ = gpu_gradient(p, obs, batch=2, ckpt_every=ckpt)
    plan = gpu_plan(p, batch=2, ckpt_every=ckpt)
    geo, rho, wav = _args(p)
    J1, d1 = plan.misfit_forward(to_dev(p.vp), rho, geo, wav, to_dev(obs), traces=True)
    g1 = plan.misfit_backward().cpu().numpy()
    assert plan.stats()["ckpt_every"] == (0 if ckpt < 0 else ckpt)
    assert abs(J1 - J0) <= 1e-12 * abs(J0)
    assert np.array_equal(d1.cpu().numpy(), d0)
    assert np.array_equal(g1, g0)
    with pytest.raises(binding.FwiError):   # the kept state is used once
        plan.misfit_backward()


def test_autograd_2d_against_oracle():
    p = breast()
    obs = observed_from_oracle(p)
    J_ref, g_ref, _ = oracle.gradient(oracle_grid(p), p.vp, p.rho, p.src_xyz, p.wavelet,
                                      p.rec_xyz, obs)
    plan = gpu_plan(p)
    geo, rho, wav = _args(p)
    m = to_dev(1.0 / p.vp ** 2).requires_grad_(True)
    J = autograd.misfit(m, plan, rho, geo, wav, to_dev(obs))
    J.backward()
    assert abs(J.item() - J_ref) <= 1e-3 * abs(J_ref)
    assert rel_l2(m.grad.cpu().numpy(), g_ref) <= TOL_GRAD
    # a scaled loss scales the gradient
    m2 = m.detach().clone().requires_grad_(True)
    (3.0 * autograd.misfit(m2, plan, rho, geo, wav, to_dev(obs))).backward()
    assert rel_l2(m2.grad.cpu().numpy(), 3.0 * m.grad.cpu().numpy()) < 1e-6


def test_autograd_vp_chain_rule():
    """d J / d vp = -2 g_m / vp^3 through torch's chain rule."""
    p = breast(nt=200)
    obs = observed_from_oracle(p)
    _, g_ref, _ = oracle.gradient(oracle_grid(p), p.vp, p.rho, p.src_xyz, p.wavelet, p.rec_xyz, obs)
    plan = gpu_plan(p)
    geo, rho, wav = _args(p)
    vp = to_dev(p.vp).requires_grad_(True)
    autograd.misfit_vp(vp, plan, rho, geo, wav, to_dev(obs)).backward()
    assert rel_l2(vp.grad.cpu().numpy(), -2.0 * g_ref / p.vp ** 3) <= TOL_GRAD


def test_autograd_3d_checkpointed_against_oracle():
    """3D, 10th order, variable density, sqrt(nt) checkpoints with recompute."""
    p = skull()
    obs = observed_from_oracle(p)
    J_ref, g_ref, _ = oracle.gradient(oracle_grid(p), p.vp, p.rho, p.src_xyz, p.wavelet,
                                      p.rec_xyz, obs)
    K = math.ceil(math.sqrt(2 * p.nt))
    plan = gpu_plan(p, ckpt_every=K)
    geo, rho, wav = _args(p)
    m = to_dev(1.0 / p.vp ** 2).requires_grad_(True)
    J = autograd.misfit(m, plan, rho, geo, wav, to_dev(obs))
    J.backward()
    assert plan.stats()["ckpt_every"] == K
    assert abs(J.item() - J_ref) <= 1e-3 * abs(J_ref)
    assert rel_l2(m.grad.cpu().numpy(), g_ref) <= TOL_GRAD


def test_autograd_directional_finite_difference():
    """Central difference of J along a smooth direction against <grad, dm>."""
    p = breast(nt=300)
    obs = to_dev(observed_from_oracle(p))
    plan = gpu_plan(p)
    geo, rho, wav = _args(p)
    m0 = 1.0 / p.vp ** 2
    m = to_dev(m0).requires_grad_(True)
    autograd.misfit(m, plan, rho, geo, wav, obs).backward()
    rng = np.random.default_rng(5)
    from scipy.ndimage import gaussian_filter
    dm = gaussian_filter(rng.standard_normal(p.shape), 4.0)
    dm *= 0.01 * m0 / np.abs(dm).max()
    h = 1.0
    with torch.no_grad():
        Jp = autograd.misfit(to_dev(m0 + h * dm), plan, rho, geo, wav, obs).item()
        Jm = autograd.misfit(to_dev(m0 - h * dm), plan, rho, geo, wav, obs).item()
    fd = (Jp - Jm) / (2 * h)
    an = float(np.vdot(m.grad.cpu().numpy().astype(np.float64), dm))
    assert fd == pytest.approx(an, rel=1e-2)
