"""GPU versions of the oracle's invariant pins, at FP32 tolerances.

* Adjoint exactness: the dot-product test <F q, y> = <q, F* y> of the linear
  map F: wavelets -> traces, with F* y the wavelet gradient of the misfit
  (fwi_misfit_backward_ex) for zero wavelets and observed data -y, whose
  residual is then exactly y; relative difference <= 1e-5.  F* y is also
  compared with the oracle's adjoint sweep sampled at the sources.
* Symmetry: homogeneous medium, on-node centred source on an odd grid
  (257^2, otherwise the homogeneous 2D setup; the 256^2 grid has no centre
  node, so its sponge is one node closer on one side): receivers related by
  the mirror y -> -y record the same traces within 1e-6 of the largest
  sample (the y taps are summed symmetrically).  A quarter turn or the
  diagonal mirror swaps the x and y taps, which the kernels sum in different
  orders: those traces agree to the FP32 rounding accumulated over the 1000
  steps (measured 1.0e-6 of the largest sample; bound 1e-5).
* Linearity: doubling the wavelet doubles the traces.  Scaling by two is
  exact in FP32 except where a subnormal result is rounded, and the fields
  start from zero, so the stencil's precursor ahead of every wavefront passes
  through the subnormal range: the rounding differences that enter there
  grow with the precursor and spread over the record at the level of one
  unit in the last place (measured: 3D run bit for bit, 2D run with density
  31% of the samples bit for bit, relative L2 5e-7).  The test requires
  relative L2 <= 1e-6 and zero traces for a zero wavelet.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2110_03345_gb300 import binding, inputs
from _helpers import TOL_TRACES, gpu_forward, oracle_grid, rel_l2, to_dev

pytestmark = pytest.mark.gpu


def band_limited(rng, rows, nt, dt, f0, count=3):
    """rows x nt signals, each a sum of `count` Ricker pulses of peak
    frequency f0 with random delays and amplitudes (random data inside the
    band the grid resolves, so that FP32 rounding of the wavefields does not
    dominate the inner products)."""
    out = np.zeros((rows, nt))
    T = nt * dt
    for r in range(rows):
        for _ in range(count):
            t0 = rng.uniform(0.1, 0.8) * T
            out[r] += rng.standard_normal() * inputs.ricker(f0, dt, nt, t0=t0)
    return out


def small_2d(seed=5, nsrc=2, nshots=2, nt=300):
    shape, dx = (90, 117), 0.3e-3
    vp, rho = inputs.random_smooth_model(shape, dx, seed)
    src = inputs.random_points(nshots * nsrc, shape, dx, seed + 1, margin=10).reshape(nshots, nsrc, 2)
    rec = inputs.random_points(24, shape, dx, seed + 2, margin=10)
    dt = inputs.cfl_dt(dx, 1600.0)
    wav = np.zeros((nshots, nsrc, nt))
    return inputs.Problem("dot_2d", shape, dx, dt, nt, 8, 8, vp, rho, src, rec, wav, c_ref=1600.0)


def small_3d(seed=6, nsrc=2, nshots=2, nt=140):
    shape, dx = (36, 40, 44), 0.4e-3
    vp, rho = inputs.random_smooth_model(shape, dx, seed)
    src = inputs.random_points(nshots * nsrc, shape, dx, seed + 1, margin=8).reshape(nshots, nsrc, 3)
    rec = inputs.random_points(30, shape, dx, seed + 2, margin=8)
    dt = inputs.cfl_dt(dx, 1600.0)
    wav = np.zeros((nshots, nsrc, nt))
    return inputs.Problem("dot_3d", shape, dx, dt, nt, 10, 6, vp, rho, src, rec, wav, c_ref=1600.0)


@pytest.mark.parametrize("case", ["2d-cd", "2d-vd", "3d-vd"])
def test_dot_product_wavelet_adjoint(case):
    p = small_2d() if case.startswith("2d") else small_3d()
    vd = case.endswith("vd")
    rho = to_dev(p.rho) if vd else None
    rng = np.random.default_rng(17)
    f0 = 0.25 * 1500.0 / (4 * p.spacing)          # ~16 points per wavelength at the peak
    ns, nsrc, nrec = p.nshots, p.src_xyz.shape[1], p.rec_xyz.shape[0]
    q = band_limited(rng, ns * nsrc, p.nt, p.dt, f0).reshape(ns, nsrc, p.nt)
    y = band_limited(rng, ns * nrec, p.nt, p.dt, f0).reshape(ns, nrec, p.nt)
    q32, y32 = q.astype(np.float32), y.astype(np.float32)
    plan = binding.Plan(p.shape, p.spacing, p.nt, p.dt, order=p.order, sponge=p.nb, c_ref=p.c_ref)
    geo = binding.Geometry(p.src_xyz, p.rec_xyz)
    vp = to_dev(p.vp)
    Fq = plan.forward(vp, rho, geo, to_dev(q32)).cpu().numpy().astype(np.float64)
    zero = torch.zeros((ns, nsrc, p.nt), device="cuda", dtype=torch.float32)
    J, _ = plan.misfit_forward(vp, rho, geo, zero, to_dev(-y32))
    _, Fty = plan.misfit_backward_ex(grad=None, grad_wavelet=True)
    Fty = Fty.cpu().numpy().astype(np.float64)
    plan.close()
    assert J == pytest.approx(0.5 * float(np.sum(y32.astype(np.float64) ** 2)), rel=1e-12)
    lhs = float(np.vdot(Fq, y32.astype(np.float64)))
    rhs = float(np.vdot(q32.astype(np.float64), Fty))
    assert abs(lhs - rhs) <= 1e-5 * max(abs(lhs), abs(rhs))
    assert np.all(Fty[:, :, -1] == 0.0)
    # F* y of the first shot against the oracle's adjoint sweep at the sources
    ref = oracle.adjoint_sources(oracle_grid(p), p.vp, p.rho if vd else None, p.rec_xyz,
                                 y32[0].astype(np.float64), p.src_xyz[0])
    assert rel_l2(Fty[0], ref) <= TOL_TRACES


def test_wavelet_gradient_with_model_gradient():
    """Both outputs of one backward: the model gradient is the one
    fwi_misfit_backward gives, and dJ/dq matches the oracle's adjoint of the
    residual (nonzero wavelets, observed data from another model)."""
    p = small_2d(nt=260)
    p.wavelet[:] = inputs.ricker(0.25 * 1500.0 / (4 * p.spacing), p.dt, p.nt)
    vt = p.vp * 1.03
    obs = oracle.forward(oracle_grid(p), vt, p.rho, p.src_xyz, p.wavelet, p.rec_xyz)
    plan = binding.Plan(p.shape, p.spacing, p.nt, p.dt, order=p.order, sponge=p.nb, c_ref=p.c_ref)
    geo = binding.Geometry(p.src_xyz, p.rec_xyz)
    vp, rho, wav, ob = to_dev(p.vp), to_dev(p.rho), to_dev(p.wavelet), to_dev(obs)
    plan.misfit_forward(vp, rho, geo, wav, ob)
    g_m = plan.misfit_backward().cpu().numpy()
    _, d = plan.misfit_forward(vp, rho, geo, wav, ob, traces=True)
    g_m2, g_q = plan.misfit_backward_ex(grad=True, grad_wavelet=True)
    plan.close()
    assert np.array_equal(g_m2.cpu().numpy(), g_m)
    resid = d.cpu().numpy().astype(np.float64) - obs.astype(np.float32).astype(np.float64)
    for s in range(p.nshots):
        ref = oracle.adjoint_sources(oracle_grid(p), p.vp, p.rho, p.rec_xyz, resid[s],
                                     p.src_xyz[s])
        assert rel_l2(g_q[s].cpu().numpy(), ref) <= 1e-3


def test_symmetry_centred_source_odd_grid():
    p = inputs.config_homogeneous_2d(n=257)
    tr, _ = gpu_forward(p, variable_density=False)
    tr = tr[0]
    nrec = tr.shape[0]
    scale = np.abs(tr).max()
    ks = np.arange(1, nrec // 4)
    for k in ks:
        assert np.abs(tr[k] - tr[nrec - k]).max() <= 1e-6 * scale          # mirror y -> -y
        assert np.abs(tr[k] - tr[k + nrec // 4]).max() <= 1e-5 * scale     # quarter turn
        assert np.abs(tr[k] - tr[nrec // 4 - k]).max() <= 1e-5 * scale     # mirror about the diagonal
    print("symmetry: quarter turn %.2e, diagonal %.2e of the largest sample" % (
        np.abs(tr[ks + nrec // 4] - tr[ks]).max() / scale,
        np.abs(tr[nrec // 4 - ks] - tr[ks]).max() / scale))


@pytest.mark.parametrize("case", ["2d-vd", "3d-cd"])
def test_linearity(case):
    if case == "2d-vd":
        p = inputs.breast_problem((150, 203), 0.3e-3, 400, nelem=64, shots=[0, 21, 42], order=8,
                                  nb=16, radius=0.35 * 150 * 0.3e-3)
        vd = True
    else:
        p = inputs.skull_problem((40, 45, 50), 0.5e-3, 200, nrec=64, every=32, order=10, nb=8,
                                 radius=0.33 * 40 * 0.5e-3)
        vd = False
    t1, _ = gpu_forward(p, variable_density=vd)
    p2 = inputs.Problem(p.name, p.shape, p.spacing, p.dt, p.nt, p.order, p.nb, p.vp, p.rho,
                        p.src_xyz, p.rec_xyz, 2.0 * p.wavelet, c_ref=p.c_ref)
    t2, _ = gpu_forward(p2, variable_density=vd)
    assert rel_l2(t2, 2.0 * t1) <= 1e-6
    same = t2 == 2.0 * t1
    print(f"linearity: {same.mean():.4f} of the samples bit for bit, relative L2 "
          f"{rel_l2(t2, 2.0 * t1):.2e}")
    p0 = inputs.Problem(p.name, p.shape, p.spacing, p.dt, p.nt, p.order, p.nb, p.vp, p.rho,
                        p.src_xyz, p.rec_xyz, 0.0 * p.wavelet, c_ref=p.c_ref)
    t0, _ = gpu_forward(p0, variable_density=vd)
    assert np.all(t0 == 0.0)
