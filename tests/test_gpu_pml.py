"""Perfectly matched layer (options.boundary = PML; Sec. 2.4) on the GPU
against the FP64 oracle (oracle/pml.py):

* traces and the gradient with respect to m = 1/vp^2 in 2D (8th order) and
  3D (10th order), constant density and variable density (constant over the
  layer and the stencil reach next to it), receivers inside the layer, with
  full history and with checkpoints (the PML state q, phi checkpointed with
  u^n, u^{n-1});
* absorption: the energy the boundary of a small domain sends back to a
  receiver 4 mm from a 10-point layer, against a large domain that reflects
  nothing within the record: the PML's is below 1% of the sponge's of the
  same width and profile, and below 2e-4 of the direct wave (the oracle
  measures 6.0e-5 against 5.0e-2).

Tolerances: relative L2 1e-4 on traces, 1e-3 on gradients.
"""
import numpy as np
import pytest

import oracle
from oracle import pml as opml
from paper_2110_03345_gb300 import binding, inputs
from _helpers import TOL_GRAD, TOL_TRACES, rel_l2, to_dev

pytestmark = pytest.mark.gpu


def density_with_constant_rim(shape, dx, reach, seed=6):
    _, rho = inputs.random_smooth_model(shape, dx, seed)
    idx = np.indices(shape)
    dist = np.min([np.minimum(i, n - 1 - i) for i, n in zip(idx, shape)], axis=0)
    ramp = np.clip((dist - reach) / 4.0, 0.0, 1.0)
    return 1000.0 + ramp * (rho - 1000.0)


def problem(ndim, vd, nshots=2, seed=0):
    if ndim == 2:
        shape, dx, nt, order, nb = (60, 67), 0.5e-3, 200, 8, 10
    else:
        shape, dx, nt, order, nb = (30, 32, 34), 0.5e-3, 110, 10, 6
    vp, _ = inputs.random_smooth_model(shape, dx, seed)
    rho = density_with_constant_rim(shape, dx, nb + order // 2 + 1) if vd else None
    dt = 0.4 * dx / vp.max()
    src = inputs.random_points(nshots, shape, dx, seed + 1, margin=nb + 3)[:, None, :]
    rec_in = inputs.random_points(8, shape, dx, seed + 2, margin=nb + 3)
    rec_layer = inputs.random_points(4, shape, dx, seed + 3, margin=1)   # some inside the layer
    rec = np.concatenate([rec_in, rec_layer])
    w = inputs.ricker(0.25 * 1500.0 / dx / 4.0, dt, nt)
    wav = np.broadcast_to(w, (nshots, 1, nt)).copy()
    p = inputs.Problem("pml", shape, dx, dt, nt, order, nb, vp, rho, src, rec, wav, c_ref=1500.0)
    idx = np.indices(shape).astype(float)
    ctr = (np.array(shape, dtype=float) / 2).reshape((-1,) + (1,) * ndim)
    p.vp_true = vp * (1.0 + 0.03 * np.exp(-((idx - ctr) ** 2).sum(0) / (0.2 * min(shape)) ** 2))
    return p


def ogrid(p):
    return oracle.Grid(p.shape, p.spacing, dt=p.dt, nt=p.nt, order=p.order, nb=p.nb, c_ref=p.c_ref)


def gpu(p, observed=None, ckpt=-1, boundary=binding.BOUNDARY_PML):
    plan = binding.Plan(p.shape, p.spacing, p.nt, p.dt, order=p.order, sponge=p.nb, c_ref=p.c_ref)
    plan.set_options(boundary=boundary, ckpt_every=ckpt)
    geo = binding.Geometry(p.src_xyz, p.rec_xyz)
    vp, wav = to_dev(p.vp), to_dev(p.wavelet)
    rho = to_dev(p.rho) if p.rho is not None else None
    if observed is None:
        out = plan.forward(vp, rho, geo, wav).cpu().numpy().astype(np.float64)
        plan.close()
        return out
    J, g, d = plan.gradient(vp, rho, geo, wav, to_dev(observed), traces=True)
    st = plan.stats()
    plan.close()
    return J, g.cpu().numpy().astype(np.float64), d.cpu().numpy().astype(np.float64), st


@pytest.mark.parametrize("case,ckpt", [("2d-cd", -1), ("2d-vd", 23), ("3d-cd", -1), ("3d-vd", 13)])
def test_pml_forward_and_gradient(case, ckpt):
    ndim, vd = int(case[0]), case.endswith("vd")
    p = problem(ndim, vd)
    g = ogrid(p)
    obs = np.stack([opml.forward(g, p.vp_true, p.src_xyz[s], p.wavelet[s], p.rec_xyz, rho=p.rho)
                    for s in range(p.nshots)])
    J_ref, g_ref, d_ref = 0.0, np.zeros(p.shape), []
    for s in range(p.nshots):
        J_s, g_s, d_s = opml.gradient(g, p.vp, p.src_xyz[s], p.wavelet[s], p.rec_xyz, obs[s],
                                      rho=p.rho)
        J_ref += J_s
        g_ref += g_s
        d_ref.append(d_s)
    fwd = gpu(p)
    assert rel_l2(fwd, np.stack(d_ref)) <= TOL_TRACES
    J, gg, d, st = gpu(p, observed=obs, ckpt=ckpt)
    assert st["ckpt_every"] == (0 if ckpt < 0 else ckpt)
    assert np.array_equal(d, fwd)
    assert abs(J - J_ref) <= 1e-3 * abs(J_ref)
    assert rel_l2(gg, g_ref) <= TOL_GRAD


def reflection(boundary, nb=10):
    c, dx, f0 = 1500.0, 0.25e-3, 4e5
    dt = 0.4 * dx / c
    nt = 700
    q = inputs.ricker_fn(f0, t0=1.5 / f0)
    w = q(np.arange(nt) * dt)[None, None, :]
    out = {}
    for n, lay in ((100, nb), (400, 0)):
        ctr = (n // 2) * dx
        src = np.array([[[ctr, ctr]]])
        rec = np.array([[ctr, ctr + (50 - nb) * dx - 4e-3]])
        p = inputs.Problem("refl", (n, n), dx, dt, nt, 8, lay, np.full((n, n), c), None, src, rec,
                           w, c_ref=c)
        out[n] = gpu(p, boundary=boundary if lay else binding.BOUNDARY_SPONGE)[0, 0]
    direct = out[400]
    return float(np.sum((out[100] - direct) ** 2) / np.sum(direct ** 2))


def test_pml_reflects_far_less_than_the_sponge():
    r_pml = reflection(binding.BOUNDARY_PML)
    r_sponge = reflection(binding.BOUNDARY_SPONGE)
    print(f"reflected energy: PML {r_pml:.2e}, sponge {r_sponge:.2e}")
    assert r_pml < 0.01 * r_sponge and r_pml < 2e-4
