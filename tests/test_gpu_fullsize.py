"""Parity at the full size of the benchmark workload (1024^2 breast-like
phantom, 0.1 mm, variable density, 8th order, 4000 steps, 256 receivers).

The oracle cannot run 128 shots, so the checks sample: the traces of shots
taken from a 13-shot batch launched as the benchmark launches it, and the
gradient of one full shot.  Batch invariance (traces bit for bit, gradients to
summation order) is tested separately on small grids, which ties the two.
"""
import numpy as np
import pytest

import oracle
from paper_2110_03345_gb300 import inputs
from _helpers import TOL_GRAD, TOL_TRACES, gpu_forward, gpu_gradient, oracle_grid, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def breast():
    return inputs.config_breast_2d()


def test_fullsize_traces_sampled_from_a_batch(breast):
    p = breast
    p13 = inputs.config_breast_2d(shots=np.arange(0, 26, 2))   # 13 shots, one batch
    got, plan = gpu_forward(p13, batch=13)
    assert plan.stats()["batch"] == 13
    for k in (0, 12):
        ref = oracle.forward(oracle_grid(p13), p13.vp, p13.rho, p13.src_xyz[k:k + 1],
                             p13.wavelet[k:k + 1], p13.rec_xyz)[0]
        assert rel_l2(got[k], ref) <= TOL_TRACES


def test_fullsize_gradient_one_shot(breast):
    p = inputs.config_breast_2d(shots=[40])
    g = oracle_grid(p)
    obs = oracle.forward(g, p.vp_true, p.rho, p.src_xyz, p.wavelet, p.rec_xyz)
    J_ref, g_ref, d_ref = oracle.gradient(g, p.vp, p.rho, p.src_xyz, p.wavelet, p.rec_xyz, obs,
                                          ckpt_every=64)
    J, gg, d, plan = gpu_gradient(p, obs)
    assert rel_l2(d, d_ref) <= TOL_TRACES
    assert abs(J - J_ref) <= 1e-3 * abs(J_ref)
    assert rel_l2(gg, g_ref) <= TOL_GRAD
