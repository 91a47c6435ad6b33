"""Uneven batches: many independent 2D problems advanced by one multi-problem
launch per step, captured in one CUDA graph, against one plan per problem
(bit for bit: the same kernel body and tile shape) and the FP64 oracle."""
import numpy as np
import pytest

from paper_2110_03345_gb300 import binding, inputs
from _helpers import TOL_TRACES, gpu_forward, oracle_forward, rel_l2, to_dev

pytestmark = pytest.mark.gpu


def problems(nprob=5):
    return inputs.config_uneven_batch(nprob=nprob, seed=7, side=(96, 200), nt=(60, 260),
                                      shots=(1, 4), dx=0.4e-3, nelem=16, nb=12)


def as_batch_entries(ps):
    out = []
    for p in ps:
        out.append(dict(shape=p.shape, spacing=p.spacing, nt=p.nt, dt=p.dt, order=p.order,
                        sponge=p.nb, c_ref=p.c_ref, vp=to_dev(p.vp), rho=to_dev(p.rho),
                        geometry=binding.Geometry(p.src_xyz, p.rec_xyz),
                        wavelet=to_dev(p.wavelet)))
    return out


@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_matches_single_problem_runs(use_graph):
    ps = problems()
    assert len({p.nt for p in ps}) > 1 and len({p.shape for p in ps}) > 1
    b = binding.Batch(as_batch_entries(ps), use_graph=use_graph)
    got = [t.cpu().numpy().astype(np.float64) for t in b.run()]
    for p, g in zip(ps, got):
        ref, _ = gpu_forward(p)   # the default (TMA-staged) variant, as in the batch
        assert np.array_equal(g, ref)
    # a second run (graph replay) gives the same traces
    again = [t.cpu().numpy().astype(np.float64) for t in b.run()]
    assert all(np.array_equal(a, g) for a, g in zip(again, got))
    st = b.stats()
    assert st["problems"] == len(ps) and st["launches"] == max(p.nt for p in ps) - 1 + 2 * len(ps)
    b.close()


def test_batch_against_oracle():
    ps = problems(3)
    b = binding.Batch(as_batch_entries(ps))
    got = b.run()
    k = int(np.argmax([p.nshots for p in ps]))
    ref = oracle_forward(ps[k])
    assert rel_l2(got[k].cpu().numpy(), ref) <= TOL_TRACES
    b.close()
