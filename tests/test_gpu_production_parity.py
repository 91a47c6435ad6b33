"""Oracle parity in the launch configurations the benchmark uses.

* 3D grids wide enough that the default two-point kernel (64 x points per CTA
  row) runs three CTAs along x, so the x halo crosses CTA seams, for every
  tile variant (bit for bit within a family) and against the FP64 oracle.
* The 256^3 skull workload (10th order, variable density) at full grid size
  with the time axis cut to 150 steps, one shot, against the oracle gradient.
* 2D gradients with the shot groups of the benchmark (6 shots per CTA, 15
  shots per launch) and a multi-problem batch at 16 shots per CTA, against
  the oracle.

Tolerances as everywhere: relative L2 of 1e-4 on traces, 1e-3 on gradients.
"""
import numpy as np
import pytest

import oracle
from paper_2110_03345_gb300 import binding, inputs
from _helpers import (TOL_GRAD, TOL_TRACES, gpu_forward, gpu_gradient, oracle_forward, oracle_grid,
                      rel_l2, strong_perturbation, to_dev)

pytestmark = pytest.mark.gpu


def wide_3d(nt=120, order=10, nshots=2, shape=(26, 30, 150), dx=0.4e-3, seed=13):
    """Smooth random 3D model on a grid 150 points wide in x (three CTAs of
    the two-point kernels, five of the one-point kernels), sources and
    receivers spread along x so that waves cross every CTA seam."""
    vp, rho = inputs.random_smooth_model(shape, dx, seed, c_range=(1450.0, 1650.0),
                                         sigma=1.2e-3)
    nb = 6
    rec = inputs.random_points(40, shape, dx, seed + 1, margin=nb + 2)
    src = inputs.random_points(nshots, shape, dx, seed + 2, margin=nb + 2)[:, None, :]
    dt = inputs.cfl_dt(dx, 1650.0)
    w = inputs.ricker(0.5e6, dt, nt)
    wav = np.broadcast_to(w, (nshots, 1, nt)).copy()
    p = inputs.Problem("wide_3d", shape, dx, dt, nt, order, nb, vp, rho, src, rec, wav,
                       c_ref=1650.0)
    p.vp_true = strong_perturbation(p)
    return p


@pytest.fixture(scope="module")
def wide():
    return wide_3d()


@pytest.mark.parametrize("vd", [False, True])
def test_wide_3d_forward_all_variants(wide, vd):
    """Every 3D variant on the wide grid: bit for bit within its family, the
    families to rounding, and the default variant against the oracle."""
    p = wide
    ref = oracle_forward(p, variable_density=vd)
    base = {}
    for tile in range(1, 13):
        got, plan = gpu_forward(p, tile=tile, variable_density=vd)
        assert plan.stats()["tile"] == tile
        fam = 1 if tile <= 4 else 5
        if fam in base:
            assert np.array_equal(got, base[fam]), f"variant {tile} differs from its family"
        else:
            base[fam] = got
        assert rel_l2(got, ref) <= TOL_TRACES, f"variant {tile}"
    assert rel_l2(base[1], base[5]) < 1e-6


@pytest.mark.parametrize("tile", [8, 12])
def test_wide_3d_gradient(wide, tile):
    p = wide
    obs = oracle_forward(p, vp=p.vp_true)
    J_ref, g_ref, d_ref = oracle.gradient(oracle_grid(p), p.vp, p.rho, p.src_xyz, p.wavelet,
                                          p.rec_xyz, obs)
    J, g, d, plan = gpu_gradient(p, obs, tile=tile)
    assert plan.stats()["tile"] == tile
    assert rel_l2(d, d_ref) <= TOL_TRACES
    assert abs(J - J_ref) <= 1e-3 * abs(J_ref)
    assert rel_l2(g, g_ref) <= TOL_GRAD


def test_skull_256_cropped_time_gradient():
    """The benchmark's 3D workload at full grid size (256^3, 0.25 mm, 10th
    order, variable density, 512 receivers), one shot, the time axis cut to
    150 steps: gradient, misfit and traces against the FP64 oracle, in the
    default variant and the batch the plan chooses.  Observed data are zero,
    so the residual is the modelled traces themselves."""
    p = inputs.config_skull_3d(nt=150, shots=[0])
    obs = np.zeros((1, p.rec_xyz.shape[0], p.nt))
    J_ref, g_ref, d_ref = oracle.gradient(oracle_grid(p), p.vp, p.rho, p.src_xyz, p.wavelet,
                                          p.rec_xyz, obs, ckpt_every=13)
    J, g, d, plan = gpu_gradient(p, obs)
    assert plan.stats()["tile"] == 12
    assert rel_l2(d, d_ref) <= TOL_TRACES
    assert abs(J - J_ref) <= 1e-3 * abs(J_ref)
    assert rel_l2(g, g_ref) <= TOL_GRAD


@pytest.mark.parametrize("vd", [False, True])
def test_gradient_2d_six_shots_per_cta(vd):
    """15 shots in one launch, 6 shots per CTA (groups of 6, 6 and 3): the
    benchmark's shot grouping and tile variant, against the oracle."""
    p = inputs.breast_problem((150, 171), 0.25e-3, 400, nelem=64, shots=list(range(0, 60, 4)),
                              order=8, nb=20, radius=0.35 * 150 * 0.25e-3)
    p.vp_true = strong_perturbation(p)
    assert p.nshots == 15
    obs = oracle_forward(p, vp=p.vp_true, variable_density=vd)
    J_ref, g_ref, d_ref = oracle.gradient(oracle_grid(p), p.vp, p.rho if vd else None, p.src_xyz,
                                          p.wavelet, p.rec_xyz, obs)
    J, g, d, plan = gpu_gradient(p, obs, variable_density=vd, tile=6, batch=15, shots_per_cta=6)
    st = plan.stats()
    assert st["batch"] == 15 and st["tile"] == 6
    assert rel_l2(d, d_ref) <= TOL_TRACES
    assert abs(J - J_ref) <= 1e-3 * abs(J_ref)
    assert rel_l2(g, g_ref) <= TOL_GRAD


def test_batch_sixteen_shots_per_cta_against_oracle():
    """A multi-problem batch run as the batch autotuner chose for the uneven
    workload (variant 8, 16 shots per CTA): an 18-shot problem (groups of 16
    and 2) and a 3-shot problem, against the oracle."""
    ps = [inputs.breast_problem((120, 136), 0.4e-3, 220, nelem=36, shots=list(range(0, 36, 2)),
                                order=8, nb=12, seed=41, radius=0.42 * 120 * 0.4e-3),
          inputs.breast_problem((100, 100), 0.4e-3, 160, nelem=12, shots=[0, 4, 8], order=8,
                                nb=12, seed=42, radius=0.42 * 100 * 0.4e-3)]
    entries = [dict(shape=p.shape, spacing=p.spacing, nt=p.nt, dt=p.dt, order=p.order,
                    sponge=p.nb, c_ref=p.c_ref, vp=to_dev(p.vp), rho=to_dev(p.rho),
                    geometry=binding.Geometry(p.src_xyz, p.rec_xyz), wavelet=to_dev(p.wavelet))
               for p in ps]
    b = binding.Batch(entries, use_graph=True, tile=8, shots_per_cta=16)
    got = [t.cpu().numpy().astype(np.float64) for t in b.run()]
    b.close()
    assert ps[0].nshots == 18
    for p, gtr in zip(ps, got):
        ref = oracle_forward(p)
        assert rel_l2(gtr, ref) <= TOL_TRACES
        for s in range(p.nshots):
            assert rel_l2(gtr[s], ref[s]) <= TOL_TRACES
