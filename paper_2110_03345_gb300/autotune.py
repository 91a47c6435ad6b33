"""Autotuner for the kernel variant (tile shape, staging) and the number of
shots looped inside a CTA.

For a problem it runs a short slice of the real workload (same grid, model,
geometry and shot batch, a few dozen time steps) once per candidate, reads the
device time of every stencil launch from the plan's CUDA events, and keeps the
variant with the lowest time per step (forward + adjoint for gradients).
Results are cached in a JSON file keyed by the problem class (dimension,
order, density mode, grid rounded to the tile sizes, shots per batch), so a
class is tuned once per machine.
"""
from __future__ import annotations

import json
import os
import threading

import numpy as np

from . import binding

_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_autotune_cache.json")
_lock = threading.Lock()

CANDIDATES_2D = [dict(tile=t, shots_per_cta=s) for t in (5, 6, 7, 8) for s in (2, 3, 4, 5, 6, 8)] + \
                [dict(tile=t) for t in (1, 2, 3, 4)]
CANDIDATES_3D = [dict(tile=t) for t in (5, 6, 7, 8, 9, 10, 11, 12)]


def problem_key(shape, order, variable_density, gradient, shots):
    rounded = tuple(int(np.ceil(s / 64.0)) * 64 for s in shape)
    return f"{len(shape)}d-o{order}-{'vd' if variable_density else 'cd'}-" \
           f"{'grad' if gradient else 'fwd'}-{'x'.join(map(str, rounded))}-b{shots}"


def _load_cache(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store_cache(path, cache):
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(shape, spacing, dt, order, sponge, c_ref, vp, rho, geometry, wavelet, observed=None,
         steps=60, candidates=None, cache_path=_CACHE, refresh=False, verbose=False, batch=0):
    """Best options (dict for Plan.set_options) for this problem class.

    vp, rho, wavelet[, observed] are CUDA tensors of the full problem; only the
    first `steps` time samples are used.  With observed given the gradient
    (forward + adjoint kernels) is timed, else the forward.  batch: shots per
    launch of the real run (0: all shots), kept fixed while tuning."""
    gradient = observed is not None
    nb = batch or geometry.nshots
    key = problem_key(shape, order, rho is not None, gradient, nb)
    with _lock:
        cache = _load_cache(cache_path)
        if not refresh and key in cache:
            return dict(cache[key]["options"])
    if candidates is None:
        candidates = CANDIDATES_2D if len(shape) == 2 else CANDIDATES_3D
    nt = int(min(steps, wavelet.shape[-1]))
    wav = wavelet[..., :nt].contiguous()
    obs = observed[..., :nt].contiguous() if gradient else None
    plan = binding.Plan(shape, spacing, nt, dt, order=order, sponge=sponge, c_ref=c_ref)
    results = []
    try:
        for cand in candidates:
            plan.set_options(profile=True, batch=nb, **cand)
            try:
                for _ in range(2):   # the second run is timed (first pays for set-up)
                    if gradient:
                        plan.gradient(vp, rho, geometry, wav, obs)
                    else:
                        plan.forward(vp, rho, geometry, wav)
            except binding.FwiError:
                continue
            s = plan.stats()
            # time per step of one batch of nb shots
            batches = -(-geometry.nshots // max(s["batch"], 1))
            per_step = (s["fwd_ms"] + s["adj_ms"]) / max(nt - 1, 1) / batches
            results.append((per_step, cand))
            if verbose:
                print(f"autotune {key} {cand}: {per_step * 1e3:.1f} us/step")
    finally:
        plan.close()
    if not results:
        return {}
    best = min(results, key=lambda r: r[0])
    with _lock:
        cache = _load_cache(cache_path)
        cache[key] = {"options": best[1], "ms_per_step": best[0],
                      "tried": [[r[0], r[1]] for r in results]}
        _store_cache(cache_path, cache)
    return dict(best[1])


BATCH_CANDIDATES = [dict(tile=t, shots_per_cta=s) for t in (5, 6, 7, 8) for s in (0, 2, 4, 6)] + \
                   [dict(tile=t, shots_per_cta=s) for t in (6, 8) for s in (8, 12, 16)]


def batch_key(problems):
    """Problem class of an uneven batch: order, density mode, problem count,
    total shots and the grid-point volume (rounded)."""
    pts = sum(int(np.prod(pr["shape"])) * pr["geometry"].nshots for pr in problems)
    first = problems[0]
    return f"batch-o{first.get('order', 8)}-{'vd' if first.get('rho') is not None else 'cd'}-" \
           f"p{len(problems)}-s{sum(pr['geometry'].nshots for pr in problems)}-" \
           f"v{int(round(np.log2(max(pts, 1)) * 4))}"


def tune_batch(problems, steps=80, candidates=None, cache_path=_CACHE, refresh=False,
               verbose=False):
    """Tile variant and shots per CTA of an uneven batch (binding.Batch
    problems).  Every problem is cut to its first `steps` time samples, so the
    candidates are timed with every problem running (graph replays, device
    time from the batch's events)."""
    key = batch_key(problems)
    with _lock:
        cache = _load_cache(cache_path)
        if not refresh and key in cache:
            return dict(cache[key]["options"])
    cut = []
    for pr in problems:
        q = dict(pr)
        q["nt"] = int(min(steps, pr["nt"]))
        q["wavelet"] = pr["wavelet"][..., :q["nt"]].contiguous()
        cut.append(q)
    results = []
    for cand in candidates or BATCH_CANDIDATES:
        try:
            b = binding.Batch(cut, use_graph=True, **cand)
        except binding.FwiError:
            continue
        try:
            b.run()
            b.run()
            ms = b.stats()["run_ms"]
        finally:
            b.close()
        results.append((ms, cand))
        if verbose:
            print(f"autotune {key} {cand}: {ms:.2f} ms")
    if not results:
        return {}
    best = min(results, key=lambda r: r[0])
    with _lock:
        cache = _load_cache(cache_path)
        cache[key] = {"options": best[1], "ms_per_run": best[0],
                      "tried": [[r[0], r[1]] for r in results]}
        _store_cache(cache_path, cache)
    return dict(best[1])
