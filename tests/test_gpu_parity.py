"""GPU (FP32, CUDA library through the C ABI) vs FP64 oracle parity.

Tolerances (relative L2 over the whole array): traces 1e-4, gradients 1e-3.
Sizes span several tiles with ragged edges (non-multiples of the 128-wide
2D tile and of the 32 x 16 3D column), both stencil orders, constant and
variable density, several shots per launch and off-grid transducers.
"""
import numpy as np
import pytest

import oracle
from paper_2110_03345_gb300 import inputs
from _helpers import (TOL_GRAD, TOL_TRACES, gpu_forward, gpu_gradient, observed_from_oracle,
                      oracle_forward, oracle_grid, rel_l2, strong_perturbation)

pytestmark = pytest.mark.gpu


def small_breast(n=(200, 333), nt=600, shots=(0, 50, 101), order=8, dx=0.25e-3):
    """Breast-like 2D problem on a ragged grid (3 shots, 128-element ring)."""
    p = inputs.breast_problem(n, dx, nt, nelem=128, shots=list(shots), order=order, nb=20,
                              radius=0.35 * min(n) * dx)
    p.vp_true = strong_perturbation(p)
    return p


def small_skull(n=(40, 45, 50), nt=200, order=10, nshots=2, dx=0.5e-3):
    """Head-like 3D problem on a ragged grid (2 shots, 64 receivers)."""
    p = inputs.skull_problem(n, dx, nt, nrec=64, every=64 // nshots, order=order, nb=8,
                             radius=0.33 * min(n) * dx)
    p.vp_true = strong_perturbation(p)
    return p


# ------------------------------------------------------------------ forward

def test_config1_homogeneous_forward():
    """256^2, 0.2 mm, c = 1500, 8th order, CFL 0.4, 1000 steps, 64-receiver ring."""
    p = inputs.config_homogeneous_2d()
    ref = oracle_forward(p, variable_density=False)
    got, _ = gpu_forward(p, variable_density=False)
    assert rel_l2(got, ref) <= TOL_TRACES
    # variable-density path with constant rho reduces exactly to constant density
    p_vd = inputs.config_homogeneous_2d(variable_density=True)
    got_vd, _ = gpu_forward(p_vd, variable_density=True)
    assert np.array_equal(got_vd, got)


def test_config1_against_analytic():
    """GPU traces of the homogeneous case against the 2D Green's function,
    receivers 20 mm from the source, window before the first sponge echo.
    At CFL 0.4 the leapfrog's own time dispersion gives an NRMSE of ~8% at
    this distance (second order in dt, pinned in the oracle tests); the GPU
    must reproduce the oracle's error, not beat physics."""
    p = inputs.config_homogeneous_2d()
    got, _ = gpu_forward(p, variable_density=False)
    ref = oracle_forward(p, variable_density=False)
    t = np.arange(p.nt) * p.dt
    an = oracle.analytic_2d(inputs.ricker_fn(500e3), 20e-3, t, 1500.0)
    t_echo = (2 * (128 - p.nb) * p.spacing - 20e-3) / 1500.0
    m = t < t_echo

    def nrmse(x):
        return np.sqrt(np.mean((x[m] - an[m]) ** 2)) / np.sqrt(np.mean(an[m] ** 2))
    for k in (0, 16, 32, 48):
        assert nrmse(got[0, k]) < 0.1
        assert abs(nrmse(got[0, k]) - nrmse(ref[0, k])) < 1e-3


@pytest.mark.parametrize("order", [8, 10])
@pytest.mark.parametrize("vd", [False, True])
def test_forward_2d_ragged(order, vd):
    p = small_breast(order=order)
    ref = oracle_forward(p, variable_density=vd)
    got, _ = gpu_forward(p, variable_density=vd)
    assert rel_l2(got, ref) <= TOL_TRACES
    for s in range(got.shape[0]):
        assert rel_l2(got[s], ref[s]) <= TOL_TRACES


@pytest.mark.parametrize("order", [8, 10])
@pytest.mark.parametrize("vd", [False, True])
def test_forward_3d_ragged(order, vd):
    p = small_skull(order=order)
    ref = oracle_forward(p, variable_density=vd)
    got, _ = gpu_forward(p, variable_density=vd)
    assert rel_l2(got, ref) <= TOL_TRACES


@pytest.mark.parametrize("tile", [1, 2, 3, 4, 5, 6, 7, 8])
def test_tile_variants_2d(tile):
    """Shared-memory-staged variants (1-4) agree bit for bit among themselves,
    TMA-staged shot-loop variants (5-8) likewise; the two families differ only
    in the order of the variable-density adjoint terms (rounding)."""
    p = small_breast(nt=300)
    fam = 1 if tile <= 4 else 5
    base, _ = gpu_forward(p, tile=fam)
    got, plan = gpu_forward(p, tile=tile)
    assert plan.stats()["tile"] == tile
    assert np.array_equal(got, base)
    other, _ = gpu_forward(p, tile=6 - fam if fam == 1 else 1)
    assert rel_l2(got, other) < 1e-6


@pytest.mark.parametrize("spc", [1, 2, 3])
def test_shots_per_cta_2d(spc):
    """Looping 1, 2 or 3 shots inside a CTA changes nothing in the traces and
    only the summation order of the gradient."""
    p = small_breast(n=(130, 140), nt=150, shots=(0, 30, 64, 90))
    obs = observed_from_oracle(p)
    J0, g0, d0, _ = gpu_gradient(p, obs, tile=5, shots_per_cta=4)
    J1, g1, d1, _ = gpu_gradient(p, obs, tile=5, shots_per_cta=spc)
    assert np.array_equal(d1, d0)
    assert rel_l2(g1, g0) < 1e-6
    assert abs(J1 - J0) <= 1e-12 * abs(J0)


@pytest.mark.parametrize("vd", [False, True])
def test_gradient_2d_smem_family(vd):
    """The shared-memory-staged kernels (one shot per CTA) against the oracle."""
    p = small_breast(n=(150, 171), nt=400, shots=(0, 64), order=10)
    obs = observed_from_oracle(p, variable_density=vd)
    J_ref, g_ref, d_ref = oracle.gradient(oracle_grid(p), p.vp, p.rho if vd else None, p.src_xyz,
                                          p.wavelet, p.rec_xyz, obs)
    J, g, d, _ = gpu_gradient(p, obs, variable_density=vd, tile=2)
    assert rel_l2(d, d_ref) <= TOL_TRACES
    assert rel_l2(g, g_ref) <= TOL_GRAD


@pytest.mark.parametrize("tile", [1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12])
@pytest.mark.parametrize("vd", [False, True])
def test_tile_variants_3d(tile, vd):
    """3D: shared-memory-staged variants (1-4) agree bit for bit among
    themselves, TMA plane-ring variants with one (5-8) and two (9-12) x points
    per thread likewise (one family: the same rounding order), and the two
    families to rounding."""
    p = small_skull(nt=120)
    fam = 1 if tile <= 4 else 5
    base, _ = gpu_forward(p, tile=fam, variable_density=vd)
    got, plan = gpu_forward(p, tile=tile, variable_density=vd)
    assert plan.stats()["tile"] == tile
    assert np.array_equal(got, base)
    other, _ = gpu_forward(p, tile=6 - fam if fam == 1 else 1, variable_density=vd)
    assert rel_l2(got, other) < 1e-6


@pytest.mark.parametrize("tile", [1, 5, 10])
def test_gradient_3d_both_families(tile):
    p = small_skull(n=(36, 38, 41), nt=160, order=10)
    obs = observed_from_oracle(p)
    J_ref, g_ref, d_ref = oracle.gradient(oracle_grid(p), p.vp, p.rho, p.src_xyz, p.wavelet,
                                          p.rec_xyz, obs)
    J, g, d, _ = gpu_gradient(p, obs, tile=tile)
    assert rel_l2(d, d_ref) <= TOL_TRACES
    assert rel_l2(g, g_ref) <= TOL_GRAD


def test_batch_invariance_and_determinism():
    p = small_breast(nt=300)
    a, _ = gpu_forward(p, batch=1)
    b, _ = gpu_forward(p, batch=0)
    c, _ = gpu_forward(p, batch=2)
    assert np.array_equal(a, b) and np.array_equal(a, c)
    d, _ = gpu_forward(p, batch=0)
    assert np.array_equal(b, d)


# ------------------------------------------------------------------ gradient

@pytest.mark.parametrize("order", [8, 10])
@pytest.mark.parametrize("vd", [False, True])
def test_gradient_2d(order, vd):
    p = small_breast(n=(150, 171), nt=400, shots=(0, 64), order=order)
    obs = observed_from_oracle(p, variable_density=vd)
    J_ref, g_ref, d_ref = oracle.gradient(oracle_grid(p), p.vp, p.rho if vd else None, p.src_xyz,
                                          p.wavelet, p.rec_xyz, obs)
    J, g, d, _ = gpu_gradient(p, obs, variable_density=vd)
    assert rel_l2(d, d_ref) <= TOL_TRACES
    assert abs(J - J_ref) <= 1e-3 * abs(J_ref)
    assert rel_l2(g, g_ref) <= TOL_GRAD


@pytest.mark.parametrize("vd", [False, True])
def test_gradient_3d(vd):
    p = small_skull(n=(36, 38, 41), nt=160, order=10)
    obs = observed_from_oracle(p, variable_density=vd)
    J_ref, g_ref, d_ref = oracle.gradient(oracle_grid(p), p.vp, p.rho if vd else None, p.src_xyz,
                                          p.wavelet, p.rec_xyz, obs)
    J, g, d, _ = gpu_gradient(p, obs, variable_density=vd)
    assert rel_l2(d, d_ref) <= TOL_TRACES
    assert abs(J - J_ref) <= 1e-3 * abs(J_ref)
    assert rel_l2(g, g_ref) <= TOL_GRAD


@pytest.mark.parametrize("ndim", [2, 3])
def test_checkpointing_matches_full_history(ndim):
    """Recomputation from checkpoints repeats the forward bit for bit."""
    p = small_breast(n=(130, 140), nt=150, shots=(0, 64)) if ndim == 2 else small_skull(nt=100)
    obs = observed_from_oracle(p)
    J0, g0, d0, _ = gpu_gradient(p, obs, ckpt_every=-1)
    for K in (7, 32):
        J1, g1, d1, plan = gpu_gradient(p, obs, ckpt_every=K)
        assert plan.stats()["ckpt_every"] == K
        assert J1 == J0 and np.array_equal(g1, g0) and np.array_equal(d1, d0)


def test_gradient_batching():
    """Shots batched differently give the same traces exactly and the same
    gradient up to the order of the per-slot sums."""
    p = small_breast(n=(130, 140), nt=150, shots=(0, 30, 64, 90))
    obs = observed_from_oracle(p)
    J1, g1, d1, _ = gpu_gradient(p, obs, batch=1)
    J4, g4, d4, _ = gpu_gradient(p, obs, batch=4)
    J2, g2, d2, _ = gpu_gradient(p, obs, batch=3)
    assert np.array_equal(d1, d4) and np.array_equal(d1, d2)
    assert rel_l2(g4, g1) < 1e-6 and rel_l2(g2, g1) < 1e-6
    assert abs(J4 - J1) < 1e-12 * abs(J1)


@pytest.mark.parametrize("tile", [5, 8, 9, 12])
def test_gradient_batching_3d(tile):
    """3D: four shots in one batch (shots per CTA requested > 1, which the 3D
    kernels ignore) give the gradient of four one-shot batches and of the
    oracle."""
    p = small_skull(n=(36, 38, 41), nt=140, nshots=4)
    obs = observed_from_oracle(p)
    J1, g1, d1, _ = gpu_gradient(p, obs, batch=1, tile=tile)
    J4, g4, d4, plan = gpu_gradient(p, obs, batch=4, tile=tile, shots_per_cta=4)
    assert plan.stats()["batch"] == 4
    assert np.array_equal(d1, d4)
    assert rel_l2(g4, g1) < 1e-6
    assert abs(J4 - J1) < 1e-12 * abs(J1)
    _, g_ref, _ = oracle.gradient(oracle_grid(p), p.vp, p.rho, p.src_xyz, p.wavelet, p.rec_xyz, obs)
    assert rel_l2(g4, g_ref) <= TOL_GRAD


@pytest.mark.parametrize("dim", [2, 3])
def test_overlapped_steps_match_serialised_steps(dim):
    """Consecutive steps overlap through programmatic dependent launch unless
    events separate them (profile = 1 records events around every launch):
    both give the same bits, so no step reads a wavefield before the previous
    step has finished writing it."""
    p = small_breast(nt=300) if dim == 2 else small_skull(nt=140)
    obs = observed_from_oracle(p)
    J0, g0, d0, _ = gpu_gradient(p, obs, profile=0)
    J1, g1, d1, _ = gpu_gradient(p, obs, profile=1)
    assert J0 == J1
    assert np.array_equal(g0, g1) and np.array_equal(d0, d1)
