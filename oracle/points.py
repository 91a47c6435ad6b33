"""Point sources and receivers for the numpy-stepped oracles (time4,
attenuation, pml): per-point node weights and the source fields s^n.

TEST INFRASTRUCTURE ONLY, like the rest of this package.  The bi-/tri-linear
weights are the C oracle's (pinned in tests/test_oracle_pins.py); any other
weights come in through `interp` (see oracle.sinc)."""
from __future__ import annotations

import numpy as np

from . import Grid, point_weights


def point_list(grid: Grid, xyz, interp=None):
    """Per point: flat node indices and interpolation weights (bi-/tri-linear
    from the C oracle, or interp(grid, point) -> (indices, weights))."""
    xyz = np.asarray(xyz, dtype=np.float64).reshape(-1, grid.ndim)
    f = point_weights if interp is None else interp
    return [f(grid, p) for p in xyz]


def source_fields(grid: Grid, src_xyz, wavelet, interp=None):
    """s^n for n = -1 .. nt (zero outside the record), [nt + 2][N]: the
    wavelet samples spread onto the nodes with weight / cell volume;
    S[n + 1] = s^n."""
    N = grid.npoints
    dV = float(np.prod(grid.spacing))
    wav = np.asarray(wavelet, dtype=np.float64).reshape(-1, grid.nt)
    S = np.zeros((grid.nt + 2, N))
    for (idx, w), q in zip(point_list(grid, src_xyz, interp), wav):
        for i, wi in zip(idx, w):
            S[1:grid.nt + 1, i] += (wi / dV) * q
    return S
