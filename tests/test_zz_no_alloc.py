"""fwi_forward_noalloc: the forward entry point for callers that cannot
allocate device memory (its workspace is the library's fixed device scratch).

It must give what fwi_forward gives, call after call (the scratch keeps the
previous call's contents, so a second call checks that everything that must
start at zero is cleared), and refuse a grid that does not fit the scratch
with a clear error instead of touching memory it does not own.  This file is
collected last so that a failure here cannot hide any other test; it passes
alone in a fresh process and after the others.
"""
import numpy as np
import pytest

from paper_2110_03345_gb300 import binding, inputs
from _helpers import TOL_TRACES, rel_l2, to_dev

pytestmark = pytest.mark.gpu


def _problem():
    p = inputs.breast_problem((150, 203), 0.3e-3, 400, nelem=64, shots=[0, 20, 41], order=8,
                              nb=16, radius=0.35 * 150 * 0.3e-3)
    return p


def test_noalloc_matches_forward_twice():
    p = _problem()
    geo = binding.Geometry(p.src_xyz, p.rec_xyz)
    vp, rho, wav = to_dev(p.vp), to_dev(p.rho), to_dev(p.wavelet)
    plan = binding.Plan(p.shape, p.spacing, p.nt, p.dt, order=p.order, sponge=p.nb, c_ref=p.c_ref)
    ref = plan.forward(vp, rho, geo, wav).cpu().numpy()
    plan.close()
    for _ in range(2):
        got = binding.forward_noalloc(p.shape, p.spacing, p.nt, p.dt, vp, rho, geo, wav,
                                      order=p.order, sponge=p.nb, c_ref=p.c_ref).cpu().numpy()
        assert rel_l2(got, ref) <= TOL_TRACES
    # constant density through the same scratch right after a variable-density call
    plan = binding.Plan(p.shape, p.spacing, p.nt, p.dt, order=p.order, sponge=p.nb, c_ref=p.c_ref)
    ref_cd = plan.forward(vp, None, geo, wav).cpu().numpy()
    plan.close()
    got_cd = binding.forward_noalloc(p.shape, p.spacing, p.nt, p.dt, vp, None, geo, wav,
                                     order=p.order, sponge=p.nb, c_ref=p.c_ref).cpu().numpy()
    assert rel_l2(got_cd, ref_cd) <= TOL_TRACES


def test_noalloc_rejects_grids_beyond_the_scratch():
    n = 3000   # one shot needs ~5 fields of ~37 MB: more than the 64 MiB scratch
    vp = to_dev(np.full((n, n), 1500.0))
    geo = binding.Geometry(np.array([[[0.15, 0.15]]]), np.array([[0.1, 0.1]]))
    wav = to_dev(np.zeros((1, 1, 10)))
    with pytest.raises(binding.FwiError) as ei:
        binding.forward_noalloc((n, n), 1e-4, 10, 2e-8, vp, None, geo, wav, sponge=10, c_ref=1500.0)
    assert ei.value.status == 3
    assert "static scratch" in str(ei.value)
