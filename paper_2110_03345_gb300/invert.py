"""The full-waveform inversion loop (Sec. 2.3 Listings 3-4, Sec. 3.2 Listings
13-14) on top of the gradient path: blocks of increasing upper frequency,
each iteration on a subset of the shots, gradient descent on the sound speed.

Host orchestration only.  Per iteration it enqueues, on the plan's stream,
the low-pass of the selected shots' wavelets and observed traces
(``fwi_lowpass``), the misfit gradient of those shots (``fwi_gradient``) and
the model update (``fwi_vp_update``); every step runs in the CUDA library.
The shot subsets are an input (``inputs.shot_schedule`` draws them as in
Sec. 3.2: random subsets, each shot once per block).
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import binding


def half_width(f_max: float, dt: float, cycles: float = 3.0) -> int:
    """Filter half-width for a block: `cycles` periods of f_max (3 keeps the
    pass band below 0.7 f_max within 1% and the stop band above 1.5 f_max
    below 0.25%)."""
    M = int(math.ceil(cycles / (f_max * dt)))
    if M > binding.LOWPASS_MAX_HALF_WIDTH:
        raise ValueError(f"f_max {f_max:g} Hz needs a half-width of {M} samples "
                         f"(at most {binding.LOWPASS_MAX_HALF_WIDTH})")
    return M


@dataclass
class Record:
    """What one run of the loop measured."""
    misfits: list = field(default_factory=list)   # [block][iteration] misfit before the update
    seconds: float = 0.0                            # host wall time of the whole loop
    shot_gradients: int = 0
    point_updates: int = 0                          # forward + adjoint grid-point updates


class Inversion:
    """Gradient descent on vp over frequency blocks.

    plan: a binding.Plan for the grid and time axis.  src_xyz [nshots][nsrc]
    [ndim] and rec_xyz [nrec][ndim] are host arrays; wavelet [nshots][nsrc]
    [nt] and observed [nshots][nrec][nt] CUDA float32 tensors for every shot;
    rho a CUDA tensor or None; mask a CUDA tensor (0 freezes a point) or
    None; bounds (vp_min, vp_max)."""

    def __init__(self, plan: binding.Plan, src_xyz, rec_xyz, wavelet, observed, rho=None,
                 mask=None, bounds=(1400.0, 1600.0), filter_cycles=3.0, max_shots=None):
        import torch
        self.plan = plan
        self.src = np.ascontiguousarray(src_xyz, dtype=np.float64)
        self.rec = np.ascontiguousarray(rec_xyz, dtype=np.float64)
        self.wavelet, self.observed, self.rho, self.mask = wavelet, observed, rho, mask
        self.bounds = (float(bounds[0]), float(bounds[1]))
        self.cycles = float(filter_cycles)
        ns, nsrc, nt = (int(v) for v in wavelet.shape)
        nrec = int(observed.shape[1])
        if observed.shape[0] != ns or observed.shape[2] != nt or nt != plan.nt:
            raise ValueError("wavelet and observed must cover the same shots and the plan's nt")
        if self.src.shape[:2] != (ns, nsrc) or self.rec.shape[0] != nrec:
            raise ValueError("geometry does not match the wavelet / observed arrays")
        cap = ns if max_shots is None else int(max_shots)
        dev = wavelet.device
        self._wav = torch.empty((cap, nsrc, nt), device=dev, dtype=torch.float32)
        self._obs = torch.empty((cap, nrec, nt), device=dev, dtype=torch.float32)
        self.grad = torch.empty(plan.shape, device=dev, dtype=torch.float32)   # last dJ/dm
        self._work = torch.empty(1, device=dev, dtype=torch.float32)

    def iterate(self, vp, ids, f_max: float, step: float) -> float:
        """One iteration: low-pass the shots `ids` at f_max, misfit and
        gradient at vp, one update of vp (in place).  Returns the misfit."""
        ids = np.asarray(ids, dtype=np.int64).reshape(-1)
        k = len(ids)
        if k == 0:
            return 0.0
        if k > self._wav.shape[0]:
            raise ValueError("more shots in one iteration than max_shots")
        st = self.plan.stream
        M = half_width(f_max, self.plan.dt, self.cycles)
        wav = self._wav[:k]
        obs = self._obs[:k]
        binding.lowpass(self.wavelet, ids, self.plan.dt, f_max, M, out=wav, stream=st)
        binding.lowpass(self.observed, ids, self.plan.dt, f_max, M, out=obs, stream=st)
        geo = binding.Geometry(self.src[ids], self.rec)
        J, _, _ = self.plan.gradient(vp, self.rho, geo, wav, obs, grad=self.grad)
        binding.vp_update(vp, self.grad, step, self.bounds[0], self.bounds[1], mask=self.mask,
                          work=self._work, stream=st)
        return J

    def run(self, vp, freqs, schedule, step: float, callback=None) -> Record:
        """All blocks: schedule[b] lists the id sets of block b (upper
        frequency freqs[b]).  vp is updated in place."""
        import torch
        rec = Record()
        npts = int(np.prod(self.plan.shape))
        torch.cuda.synchronize(vp.device)
        t0 = time.perf_counter()
        for b, f_max in enumerate(freqs):
            Jb = []
            for i, ids in enumerate(schedule[b]):
                Jb.append(self.iterate(vp, ids, f_max, step))
                rec.shot_gradients += len(ids)
                rec.point_updates += 2 * len(ids) * npts * (self.plan.nt - 1)
                if callback is not None:
                    callback(b, i, Jb[-1])
            rec.misfits.append(Jb)
        torch.cuda.synchronize(vp.device)
        rec.seconds = time.perf_counter() - t0
        return rec
