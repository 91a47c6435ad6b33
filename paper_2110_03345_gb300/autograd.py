"""torch.autograd binding of the misfit: J(m) with its adjoint-state gradient.

The paper composes operators whose adjoints give gradients by reverse-mode
differentiation (Sec. 2.2, Eqs. 1-4 and Listings 1-2) and applies it to the
PDE-constrained misfit (Eqs. 5-9).  Here that pair is one
``torch.autograd.Function``:

* forward: ``fwi_misfit_forward`` — every shot's forward propagation through
  the CUDA kernels, the L2 misfit (FP64), and in the plan whatever the
  adjoint needs: the wavefield history when it fits the HBM budget, otherwise
  sqrt(nt)-spaced checkpoints;
* backward: ``fwi_misfit_backward`` — the adjoint propagations with the fused
  imaging condition (recomputing each checkpoint segment first), i.e. the
  hand-written adjoint kernel returns dJ/dm.

The variable is the squared slowness m = 1/vp^2, the library's own model
parameter, so no arithmetic of the path runs in torch; ``misfit_vp`` maps a
sound-speed tensor to m with torch ops for users who differentiate with
respect to vp (the paper's ``vp.grad``).
"""
from __future__ import annotations

import torch

from . import binding


class FwiMisfit(torch.autograd.Function):
    """J(m) = 1/2 sum_shots sum_rec sum_n (d(m) - d_obs)^2 (FP64 scalar).

    Arguments: m (CUDA float32, the grid's shape), a binding.Plan, rho (CUDA
    float32 or None), a binding.Geometry, wavelets [shots][src][nt] and
    observed data [shots][rec][nt] (CUDA float32).  The inputs other than m
    are not differentiated.  One backward per forward."""

    @staticmethod
    def forward(ctx, m, plan, rho, geometry, wavelet, observed):
        J, _ = plan.misfit_forward(m.detach(), rho, geometry, wavelet, observed,
                                   param=binding.PARAM_M)
        ctx.plan = plan
        return torch.tensor(J, dtype=torch.float64, device=m.device)

    @staticmethod
    def backward(ctx, grad_J):
        g = ctx.plan.misfit_backward()
        # chain rule with the incoming gradient, on the device (no host
        # synchronisation; multiplying by 1 leaves the bits unchanged)
        g.mul_(grad_J.to(g.dtype))
        return g, None, None, None, None, None


def misfit(m, plan, rho, geometry, wavelet, observed):
    """Differentiable misfit of the squared slowness m."""
    return FwiMisfit.apply(m, plan, rho, geometry, wavelet, observed)


def misfit_vp(vp, plan, rho, geometry, wavelet, observed):
    """Differentiable misfit of the sound speed vp (m = vp^-2 through torch)."""
    return FwiMisfit.apply(vp.pow(-2), plan, rho, geometry, wavelet, observed)
