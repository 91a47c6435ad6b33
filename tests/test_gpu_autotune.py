"""The autotuner: it times every candidate on a short slice of the problem,
returns the fastest one it timed, caches it per problem class, and its pick
gives the default variant's traces (bit for bit within the TMA-staged
family, to FP32 rounding across families)."""
import json

import numpy as np
import pytest

from paper_2110_03345_gb300 import autotune, binding, inputs
from _helpers import rel_l2, to_dev

pytestmark = pytest.mark.gpu


def small_problem():
    return inputs.breast_problem((320, 384), 0.25e-3, 200, nelem=64, shots=np.arange(0, 64, 8),
                                 order=8, nb=16)


def test_tune_returns_the_fastest_candidate_and_caches_it(tmp_path):
    p = small_problem()
    geo = binding.Geometry(p.src_xyz, p.rec_xyz)
    vp, rho, wav = to_dev(p.vp), to_dev(p.rho), to_dev(p.wavelet)
    cands = [dict(tile=6, shots_per_cta=2), dict(tile=6, shots_per_cta=4), dict(tile=8, shots_per_cta=4),
             dict(tile=1)]
    cache = str(tmp_path / "cache.json")
    args = (p.shape, p.spacing, p.dt, p.order, p.nb, p.c_ref, vp, rho, geo, wav)
    best = autotune.tune(*args, steps=40, candidates=cands, cache_path=cache)
    rec = json.load(open(cache))
    assert len(rec) == 1
    entry = next(iter(rec.values()))
    tried = entry["tried"]
    assert len(tried) == len(cands)                       # every candidate was timed
    assert all(t[0] > 0 for t in tried)
    fastest = min(tried, key=lambda t: t[0])
    assert best == fastest[1] and entry["ms_per_step"] == fastest[0]
    # a second call of the same class comes from the cache (no candidate runs:
    # an empty candidate list would otherwise return {})
    assert autotune.tune(*args, steps=40, candidates=[], cache_path=cache) == best
    # the pick computes what the default variant computes
    ref_plan = binding.Plan(p.shape, p.spacing, p.nt, p.dt, order=p.order, sponge=p.nb,
                            c_ref=p.c_ref)
    ref = ref_plan.forward(vp, rho, geo, wav).cpu().numpy()
    ref_plan.close()
    plan = binding.Plan(p.shape, p.spacing, p.nt, p.dt, order=p.order, sponge=p.nb, c_ref=p.c_ref)
    plan.set_options(**best)
    got = plan.forward(vp, rho, geo, wav).cpu().numpy()
    plan.close()
    if best.get("tile", 0) >= 5:
        assert np.array_equal(got, ref)
    else:
        assert rel_l2(got, ref) < 1e-6
