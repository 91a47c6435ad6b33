"""Kaiser-windowed sinc (Hicks) off-grid sources and receivers in the solve
(options.interp = FWI_INTERP_SINC; Sec. 2.4), against the oracle's sinc
weights (oracle/sinc.py) driving its leapfrog (oracle/attenuation.py with
alpha0 = 0 is the plain leapfrog and takes the interpolation weights):

* traces and gradients in 2D (8th order, constant and variable density,
  the default TMA kernels and the shared-memory kernels) and 3D (10th
  order, variable density), several sources per shot;
* sinc points with the y = 0 attenuation kernels;
* the accuracy pin of the oracle repeated on the GPU: source and receivers
  off the grid at 4 points per wavelength, against the closed-form 2D
  Green's function (Sec. 3.1): NRMSE below 0.5% with sinc weights, above 5%
  with bilinear ones.
"""
import numpy as np
import pytest

import oracle
from oracle import attenuation as oatt
from oracle import sinc as osinc
from paper_2110_03345_gb300 import binding, inputs
from _helpers import TOL_GRAD, TOL_TRACES, rel_l2, to_dev

pytestmark = pytest.mark.gpu


def problem(shape, dx, nt, order, nb, nshots=2, nsrc=2, nrec=10, seed=4):
    vp, rho = inputs.random_smooth_model(shape, dx, seed)
    dt = 0.4 * dx / vp.max()
    m = nb + 4           # sinc points lie at least r - 1 = 3 nodes inside every face
    src = inputs.random_points(nshots * nsrc, shape, dx, seed + 1, margin=m).reshape(nshots, nsrc, -1)
    rec = inputs.random_points(nrec, shape, dx, seed + 2, margin=m)
    w = inputs.ricker(0.25 * 1500.0 / dx / 4.0, dt, nt)
    wav = np.broadcast_to(w, (nshots, nsrc, nt)).copy()
    p = inputs.Problem("sinc", shape, dx, dt, nt, order, nb, vp, rho, src, rec, wav,
                       c_ref=float(vp.max()))
    p.vp_true = vp * 1.02
    return p


def ogrid(p):
    return oracle.Grid(p.shape, p.spacing, dt=p.dt, nt=p.nt, order=p.order, nb=p.nb, c_ref=p.c_ref)


def gpu(p, vd, observed=None, tile=0, alpha0=None, interp=binding.INTERP_SINC):
    plan = binding.Plan(p.shape, p.spacing, p.nt, p.dt, order=p.order, sponge=p.nb, c_ref=p.c_ref)
    plan.set_options(interp=interp, tile=tile)
    if alpha0 is not None:
        plan.set_attenuation(to_dev(alpha0), 0)
    geo = binding.Geometry(p.src_xyz, p.rec_xyz)
    vp, rho, wav = to_dev(p.vp), (to_dev(p.rho) if vd else None), to_dev(p.wavelet)
    if observed is None:
        out = plan.forward(vp, rho, geo, wav).cpu().numpy().astype(np.float64)
        plan.close()
        return out
    J, g, d = plan.gradient(vp, rho, geo, wav, to_dev(observed), traces=True)
    plan.close()
    return J, g.cpu().numpy().astype(np.float64), d.cpu().numpy().astype(np.float64)


CASES = {
    "2d-cd": dict(shape=(70, 79), dx=0.4e-3, nt=240, order=8, nb=8, vd=False, tile=0),
    "2d-vd": dict(shape=(70, 79), dx=0.4e-3, nt=240, order=8, nb=8, vd=True, tile=0),
    "2d-vd-smem": dict(shape=(70, 79), dx=0.4e-3, nt=240, order=8, nb=8, vd=True, tile=2),
    "3d-vd": dict(shape=(30, 33, 36), dx=0.5e-3, nt=110, order=10, nb=6, vd=True, tile=0),
}


@pytest.mark.parametrize("case", list(CASES))
def test_sinc_forward_and_gradient(case):
    c = dict(CASES[case])
    vd, tile = c.pop("vd"), c.pop("tile")
    p = problem(**c)
    rho = p.rho if vd else None
    g = ogrid(p)
    interp = osinc.hicks()
    obs = np.stack([oatt.forward(g, p.vp_true, rho, 0.0, 0, p.src_xyz[s], p.wavelet[s], p.rec_xyz,
                                 interp=interp) for s in range(p.nshots)])
    J_ref, g_ref, d_ref = 0.0, np.zeros(p.shape), []
    for s in range(p.nshots):
        J_s, g_s, d_s = oatt.gradient(g, p.vp, rho, 0.0, 0, p.src_xyz[s], p.wavelet[s], p.rec_xyz,
                                      obs[s], interp=interp)
        J_ref += J_s
        g_ref += g_s
        d_ref.append(d_s)
    J, gg, d = gpu(p, vd, observed=obs, tile=tile)
    assert rel_l2(d, np.stack(d_ref)) <= TOL_TRACES
    assert abs(J - J_ref) <= 1e-3 * abs(J_ref)
    assert rel_l2(gg, g_ref) <= TOL_GRAD
    # the sinc points are not the bilinear ones
    lin = gpu(p, vd, interp=binding.INTERP_LINEAR, tile=tile)
    assert rel_l2(lin, d) > 1e-3


def test_sinc_with_attenuation():
    p = problem((62, 70), 0.5e-3, 200, 8, 8)
    a0, _ = inputs.random_smooth_model(p.shape, p.spacing, 9, c_range=(100.0, 300.0))
    got = gpu(p, True, alpha0=a0)
    for s in range(p.nshots):
        ref = oatt.forward(ogrid(p), p.vp, p.rho, a0.reshape(-1), 0, p.src_xyz[s], p.wavelet[s],
                           p.rec_xyz, interp=osinc.hicks())
        assert rel_l2(got[s], ref) <= TOL_TRACES


def test_sinc_points_too_close_to_a_face_are_refused():
    p = problem((60, 64), 0.5e-3, 50, 8, 2)
    p.rec_xyz[0] = [1.5 * p.spacing, 30 * p.spacing]
    with pytest.raises(binding.FwiError) as ei:
        gpu(p, False)
    assert ei.value.status == 1


def test_sinc_accuracy_against_the_analytic_solution():
    c, f0 = 1500.0, 3e5
    dx = c / (2.5 * f0) / 4
    n = int(60e-3 / dx)
    dt = 0.1 * dx / c
    nt = int(20e-6 / dt)
    q = inputs.ricker_fn(f0, t0=1.5 / f0)
    w = q(np.arange(nt) * dt)[None, None, :]
    ctr = (n // 2 + 0.5) * dx
    src = np.array([[[ctr, ctr - 0.3 * dx]]])
    R = 9e-3
    ang = np.linspace(0, 2 * np.pi, 8, endpoint=False)
    rec = np.stack([ctr + R * np.sin(ang), ctr - 0.3 * dx + R * np.cos(ang)], 1)
    ana = oracle.analytic_2d(q, R, np.arange(nt) * dt, c)
    p = inputs.Problem("sinc_analytic", (n, n), dx, dt, nt, 10, 10, np.full((n, n), c), None,
                       src, rec, w, c_ref=c)

    def nrmse(d):
        return np.sqrt(np.mean((d - ana[None]) ** 2)) / np.sqrt(np.mean(ana ** 2))

    e_sinc = nrmse(gpu(p, False)[0])
    e_lin = nrmse(gpu(p, False, interp=binding.INTERP_LINEAR)[0])
    print(f"NRMSE against the analytic solution: sinc {e_sinc:.4f}, bilinear {e_lin:.4f}")
    assert e_sinc < 5e-3 and e_lin > 5e-2
