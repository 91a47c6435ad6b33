"""FP64 oracle of high-order sinc interpolation of off-grid sources and
receivers (Sec. 2.4 names it next to bi-/tri-linear interpolation, citing
Hicks' Kaiser-windowed sinc functions).

TEST INFRASTRUCTURE ONLY, like the rest of this package: the tests,
``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may use it; the
product never imports it.

Per axis, a point at x (in grid units) takes the 2r nodes i with
floor(x) - r < i <= floor(x) + r and the weights

    w_i = K(i - x) sinc(i - x),   K(d) = I0(b sqrt(1 - (d/r)^2)) / I0(b), |d| <= r,

with sinc(d) = sin(pi d) / (pi d); in 2D and 3D the weights are the
products of the per-axis weights ((2r)^ndim nodes).  Sources are spread with
these weights over the cell volume and receivers sample with them, exactly as
the bi-/tri-linear weights are used by the rest of the oracle, so
``interp=hicks()`` plugs into ``oracle.attenuation`` (alpha0 = 0 is the plain
leapfrog) and ``oracle.time4``-style drivers.

Readings: r = 4 and b = 6.31 (the window that minimises the largest error of
interpolating cos(k x + phi) for k up to pi/2, i.e. down to 4 points per
wavelength: 1.3e-3); points must lie at least r - 1 nodes inside every face
(the weights are not folded at a boundary: the sponge keeps sources away
from it).

Parity status: pinned (on-node points reduce to the bi-/tri-linear result;
the interpolation error of band-limited functions; b is the minimiser of that
error; exact gradients through the reverse sweep, central differences).
"""
from __future__ import annotations

import numpy as np
from scipy.special import i0


def weights_1d(x: float, r: int = 4, b: float = 6.31):
    """(nodes, weights) of one axis for a point at x grid units."""
    f = int(np.floor(x))
    idx = np.arange(f - r + 1, f + r + 1)
    d = idx - x
    arg = np.clip(1.0 - (d / r) ** 2, 0.0, None)
    win = np.where(np.abs(d) <= r, i0(b * np.sqrt(arg)) / i0(b), 0.0)
    return idx, win * np.sinc(d)


def hicks(r: int = 4, b: float = 6.31):
    """interp(grid, point) -> (flat node indices, weights) for the oracles."""

    def interp(grid, xyz):
        xyz = np.asarray(xyz, dtype=np.float64).reshape(grid.ndim)
        axes = []
        for d in range(grid.ndim):
            x = xyz[d] / grid.spacing[d]
            idx, w = weights_1d(x, r, b)
            if idx[0] < 0 or idx[-1] > grid.shape[d] - 1:
                raise ValueError(f"point {xyz} is closer than {r - 1} nodes to a face")
            axes.append((idx, w))
        grids = np.meshgrid(*[a[0] for a in axes], indexing="ij")
        wts = np.ones(grids[0].shape)
        for d in range(grid.ndim):
            wts = wts * axes[d][1].reshape([-1 if e == d else 1 for e in range(grid.ndim)])
        flat = np.ravel_multi_index([g.ravel() for g in grids], grid.shape)
        return flat, wts.ravel()

    return interp
