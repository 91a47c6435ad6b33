"""Shared helpers for the tests: run a synthetic problem through the CUDA
library (C ABI via the ctypes binding) and through the FP64 oracle."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2110_03345_gb300 import inputs

TOL_TRACES = 1e-4     # relative L2, FP32 GPU vs FP64 oracle (traces)
TOL_GRAD = 1e-3       # relative L2, FP32 GPU vs FP64 oracle (gradient)


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def oracle_grid(p: inputs.Problem) -> oracle.Grid:
    return oracle.Grid(p.shape, p.spacing, dt=p.dt, nt=p.nt, order=p.order, nb=p.nb, c_ref=p.c_ref)


def oracle_forward(p: inputs.Problem, vp=None, variable_density=True):
    vp = p.vp if vp is None else vp
    rho = p.rho if variable_density else None
    return oracle.forward(oracle_grid(p), vp, rho, p.src_xyz, p.wavelet, p.rec_xyz)


def strong_perturbation(p: inputs.Problem, amp=0.04, width=0.2):
    """Model for observed data in the small parity tests: vp x (1 + amp g),
    g a centred Gaussian of width `width` x the smallest side.  It keeps the
    residual a sizeable fraction of the data (tiny perturbations make the
    residual a difference of nearly equal traces, which magnifies FP32
    rounding of the traces in the misfit and gradient)."""
    idx = np.indices(p.shape).astype(float)
    ctr = (np.array(p.shape, dtype=float) / 2).reshape((-1,) + (1,) * len(p.shape))
    sig = width * min(p.shape)
    g = np.exp(-0.5 * ((idx - ctr) ** 2).sum(0) / sig ** 2)
    return p.vp * (1.0 + amp * g)


def observed_from_oracle(p: inputs.Problem, variable_density=True):
    """Observed data: oracle traces of the perturbed model (an input to both sides)."""
    vt = p.vp_true if p.vp_true is not None else p.vp * 1.01
    return oracle_forward(p, vp=vt, variable_density=variable_density)


def gpu_plan(p: inputs.Problem, **opts):
    from paper_2110_03345_gb300 import binding
    plan = binding.Plan(p.shape, p.spacing, p.nt, p.dt, order=p.order, sponge=p.nb, c_ref=p.c_ref)
    if opts:
        plan.set_options(**opts)
    return plan


def to_dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


def gpu_forward(p: inputs.Problem, variable_density=True, plan=None, **opts):
    from paper_2110_03345_gb300 import binding
    plan = plan or gpu_plan(p, **opts)
    geo = binding.Geometry(p.src_xyz, p.rec_xyz)
    vp = to_dev(p.vp)
    rho = to_dev(p.rho) if (variable_density and p.rho is not None) else None
    tr = plan.forward(vp, rho, geo, to_dev(p.wavelet))
    return tr.cpu().numpy().astype(np.float64), plan


def gpu_gradient(p: inputs.Problem, observed, variable_density=True, plan=None, **opts):
    from paper_2110_03345_gb300 import binding
    plan = plan or gpu_plan(p, **opts)
    geo = binding.Geometry(p.src_xyz, p.rec_xyz)
    vp = to_dev(p.vp)
    rho = to_dev(p.rho) if (variable_density and p.rho is not None) else None
    J, g, tr = plan.gradient(vp, rho, geo, to_dev(p.wavelet), to_dev(observed), traces=True)
    return J, g.cpu().numpy().astype(np.float64), tr.cpu().numpy().astype(np.float64), plan
