"""fwi_forward_noalloc: the forward entry point for callers that cannot
allocate device memory (its workspace is the library's fixed device scratch).

It must give what fwi_forward gives, bit for bit (the same kernels on the same
tile and batch choices), call after call: the scratch keeps the previous
call's contents, so the repeated calls check that everything that must start
at zero is cleared.  A grid that does not fit the scratch is refused with a
clear error instead of touching memory the library does not own.  This file
is collected last so that a failure here cannot hide any other test; it
passes alone in a fresh process and after the others.
"""
import numpy as np
import pytest

from paper_2110_03345_gb300 import binding, inputs
from _helpers import to_dev

pytestmark = pytest.mark.gpu


def _problem_2d():
    return inputs.breast_problem((150, 203), 0.3e-3, 400, nelem=64, shots=[0, 20, 41], order=8,
                                 nb=16, radius=0.35 * 150 * 0.3e-3)


def _problem_3d():
    return inputs.skull_problem((40, 40, 40), 0.5e-3, 160, nrec=64, every=32, order=10, nb=8,
                                radius=0.33 * 40 * 0.5e-3)


def _plan_forward(p, vp, rho, geo, wav):
    plan = binding.Plan(p.shape, p.spacing, p.nt, p.dt, order=p.order, sponge=p.nb, c_ref=p.c_ref)
    out = plan.forward(vp, rho, geo, wav).cpu().numpy()
    plan.close()
    return out


@pytest.mark.parametrize("make", [_problem_2d, _problem_3d], ids=["2d", "3d"])
def test_noalloc_matches_forward_twice(make):
    p = make()
    geo = binding.Geometry(p.src_xyz, p.rec_xyz)
    vp, rho, wav = to_dev(p.vp), to_dev(p.rho), to_dev(p.wavelet)
    ref = _plan_forward(p, vp, rho, geo, wav)
    for _ in range(2):
        got = binding.forward_noalloc(p.shape, p.spacing, p.nt, p.dt, vp, rho, geo, wav,
                                      order=p.order, sponge=p.nb, c_ref=p.c_ref).cpu().numpy()
        assert np.array_equal(got, ref)
    # constant density through the same scratch right after a variable-density call
    ref_cd = _plan_forward(p, vp, None, geo, wav)
    got_cd = binding.forward_noalloc(p.shape, p.spacing, p.nt, p.dt, vp, None, geo, wav,
                                     order=p.order, sponge=p.nb, c_ref=p.c_ref).cpu().numpy()
    assert np.array_equal(got_cd, ref_cd)


def test_noalloc_rejects_grids_beyond_the_scratch():
    n = 3000   # one shot needs ~5 fields of ~37 MB: more than the 64 MiB scratch
    vp = to_dev(np.full((n, n), 1500.0))
    geo = binding.Geometry(np.array([[[0.15, 0.15]]]), np.array([[0.1, 0.1]]))
    wav = to_dev(np.zeros((1, 1, 10)))
    with pytest.raises(binding.FwiError) as ei:
        binding.forward_noalloc((n, n), 1e-4, 10, 2e-8, vp, None, geo, wav, sponge=10, c_ref=1500.0)
    assert ei.value.status == 3
    assert "static scratch" in str(ei.value)
