"""FP64 oracle of the full-waveform inversion loop (Sec. 2.3 Listings 3-4,
Sec. 3.2 Listings 13-14): frequency blocks, random shot subsets, trace and
wavelet low-pass, gradient descent on the sound speed.

TEST INFRASTRUCTURE ONLY, like the rest of this package: the tests,
``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may use it; the
product never imports it, and it imports nothing from the product.  The
gradient itself comes from the C oracle (``oracle.gradient``); the steps below
are numpy written out from their definitions.

The paper names these steps but not their formulas; the readings taken here:
  * the per-block processing of wavelets and traces is a zero-phase low-pass
    with cut-off f_max: a Hann-windowed sinc of half-width M samples,
    normalised to unit gain at zero frequency, applied to the wavelet and the
    observed traces (the modelled traces follow from the filtered wavelet);
  * the gradient-descent step (Sec. 2.3: one optimiser step per computed
    gradient) is taken on vp with dJ/dvp = -2 (dJ/dm) / vp^3, scaled so
    that the largest change of any point is `step` m/s, restricted to a mask
    and clipped to [vp_min, vp_max];
  * each block draws a permutation of the shots and every iteration takes the
    next `per_iter` of them (each shot used once per block, Sec. 3.2); the
    permutation is an input.

Parity status: lowpass_taps / lowpass pinned (frequency response at 0,
f_max, pass and stop band; brute force against numpy.convolve; the solver
commutes with the filter); vp_gradient pinned (finite differences of J in
vp); vp_update pinned (descent, step normalisation, clipping, mask);
invert pinned by invariants (zero step keeps the model and reproduces the
oracle misfit of each shot subset; the error to the true model falls; at the
true model the filtered data agree, up to the record-end edge of the trace
filter).  The paper prints no reconstruction values in its text (the error
of its 2D breast reconstruction is a figure label on a dataset that is not
available): parity with them is unpinned.
"""
from __future__ import annotations

import numpy as np

from . import Grid, gradient


def lowpass_taps(dt: float, f_max: float, half_width: int) -> np.ndarray:
    """Taps h_j, j = -M..M, of the zero-phase low-pass with cut-off f_max:
    h_j proportional to sinc(2 f_max dt j) times the Hann window
    0.5 (1 + cos(pi j / (M + 1))), scaled so that sum_j h_j = 1."""
    M = int(half_width)
    h = np.empty(2 * M + 1)
    for k in range(2 * M + 1):
        j = k - M
        a = 2.0 * f_max * dt * j
        s = 1.0 if j == 0 else np.sin(np.pi * a) / (np.pi * a)
        w = 0.5 * (1.0 + np.cos(np.pi * j / (M + 1)))
        h[k] = s * w
    return h / h.sum()


def lowpass(x, dt: float, f_max: float, half_width: int) -> np.ndarray:
    """y[..., n] = sum_{j=-M}^{M} h_j x[..., n - j], with x = 0 outside the
    record 0 <= n < nt (the filter is applied along the last axis)."""
    x = np.asarray(x, dtype=np.float64)
    h = lowpass_taps(dt, f_max, half_width)
    M = int(half_width)
    nt = x.shape[-1]
    y = np.zeros_like(x)
    for k in range(2 * M + 1):
        j = k - M                    # y[n] += h_j x[n - j]
        if j >= 0:
            if j < nt:
                y[..., j:] += h[k] * x[..., :nt - j]
        else:
            if -j < nt:
                y[..., :nt + j] += h[k] * x[..., -j:]
    return y


def vp_gradient(grad_m, vp) -> np.ndarray:
    """dJ/dvp from dJ/dm with m = 1/vp^2: dm/dvp = -2 / vp^3."""
    vp = np.asarray(vp, dtype=np.float64)
    return -2.0 * np.asarray(grad_m, dtype=np.float64) / vp ** 3


def vp_update(vp, grad_m, step: float, vp_min: float, vp_max: float, mask=None) -> np.ndarray:
    """One gradient-descent step on vp: d = mask * dJ/dvp, s = max |d|,
    vp - step * d / s clipped to [vp_min, vp_max] (vp unchanged when s = 0)."""
    vp = np.asarray(vp, dtype=np.float64)
    d = vp_gradient(grad_m, vp)
    if mask is not None:
        d = d * np.asarray(mask, dtype=np.float64)
    s = np.max(np.abs(d)) if d.size else 0.0
    if not s > 0.0:
        return vp.copy()
    return np.clip(vp - step * d / s, vp_min, vp_max)


def invert(grid: Grid, vp0, rho, src_xyz, wavelet, rec_xyz, observed, freqs, schedule,
           step: float, vp_min: float, vp_max: float, mask=None, half_widths=None):
    """Frequency-continuation gradient descent (Sec. 3.2, Listings 13-14).

    For block b (cut-off freqs[b], half-width half_widths[b]) and each id set
    of schedule[b]: low-pass the wavelets and observed traces of those shots,
    compute the misfit and dJ/dm of those shots at the current vp, take one
    vp_update step.  Returns (vp, misfits): misfits[b][i] is the misfit of
    iteration i of block b, evaluated before its update."""
    vp = np.array(vp0, dtype=np.float64)
    src_xyz = np.asarray(src_xyz, dtype=np.float64)
    wavelet = np.asarray(wavelet, dtype=np.float64)
    observed = np.asarray(observed, dtype=np.float64)
    misfits = []
    for b, f_max in enumerate(freqs):
        M = int(half_widths[b])
        Jb = []
        for ids in schedule[b]:
            ids = np.asarray(ids, dtype=np.int64)
            wav_f = lowpass(wavelet[ids], grid.dt, f_max, M)
            obs_f = lowpass(observed[ids], grid.dt, f_max, M)
            J, g, _ = gradient(grid, vp, rho, src_xyz[ids], wav_f, rec_xyz, obs_f)
            Jb.append(J)
            vp = vp_update(vp, g, step, vp_min, vp_max, mask)
        misfits.append(Jb)
    return vp, misfits


def model_error(vp, vp_true, region=None) -> float:
    """epsilon of Sec. 3.2: the mean absolute difference to the true model
    (over `region`, a 0/1 array, when given)."""
    d = np.abs(np.asarray(vp, dtype=np.float64) - np.asarray(vp_true, dtype=np.float64))
    if region is None:
        return float(d.mean())
    r = np.asarray(region) > 0
    return float(d[r].mean())
