"""Uneven batches: many independent 2D problems in one CUDA graph (forward
modelling: one multi-problem launch per step; gradients: one branch per
problem), against one plan per problem (bit for bit: the same kernel body,
tile shape and shot groups) and the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2110_03345_gb300 import binding, inputs
from _helpers import (TOL_GRAD, TOL_TRACES, gpu_forward, gpu_gradient, gpu_plan, oracle_forward,
                      oracle_grid, rel_l2, strong_perturbation, to_dev)

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


def gradient_entries(ps):
    """Batch entries of gradient problems: observed data from a perturbed model
    (one plan per problem, the default variant)."""
    import torch
    entries = as_batch_entries(ps)
    obs = []
    for p, e in zip(ps, entries):
        plan = gpu_plan(p)
        o = plan.forward(to_dev(strong_perturbation(p)), to_dev(p.rho),
                         binding.Geometry(p.src_xyz, p.rec_xyz), to_dev(p.wavelet))
        plan.close()
        torch.cuda.synchronize()
        e["observed"] = o
        obs.append(o.cpu().numpy().astype(np.float64))
    return entries, obs


@pytest.mark.parametrize("use_graph,spc", [(True, 0), (False, 0), (True, 4)])
def test_gradient_batch_matches_single_problem_runs(use_graph, spc):
    """A gradient batch (each problem's forward with the history, misfit,
    adjoint with imaging and finalisation on a branch of its own) gives each
    problem's misfit and gradient bit for bit as one plan per problem with its
    full history and the batch's shot groups (same kernels, tile shape and
    summation order)."""
    ps = problems()
    entries, obs = gradient_entries(ps)
    b = binding.Batch(entries, use_graph=use_graph, gradient=True, shots_per_cta=spc)
    J, grads = b.run()
    S = b.stats()["shots_per_cta"]   # spc, or sized for the whole batch
    assert 1 <= S <= (spc or 6)
    for p, o, Jb, gb in zip(ps, obs, J, grads):
        plan = gpu_plan(p, batch=p.nshots, ckpt_every=-1, shots_per_cta=spc or S)
        Jr, gr, _, _ = gpu_gradient(p, o, plan=plan)
        plan.close()
        assert Jb == Jr
        assert np.array_equal(gb.cpu().numpy().astype(np.float64), gr)
    J2, grads2 = b.run()   # a second run (graph replay) gives the same results
    assert J2 == J and all(torch_equal(a, g) for a, g in zip(grads2, grads))
    b.close()


def test_gradient_batch_with_checkpointed_problems():
    """A budget that leaves the last problem too little room for its full
    history: it runs with sqrt(nt) checkpoints inside the batch, and every
    gradient still equals, bit for bit, one plan per problem with its full
    history (the recomputed segments repeat the forward exactly)."""
    ps = problems()
    entries, obs = gradient_entries(ps)
    S = 2

    def est(p, ckpt):
        plan = gpu_plan(p, batch=p.nshots, ckpt_every=ckpt, shots_per_cta=S)
        n = plan.estimate(binding.Geometry(p.src_xyz, p.rec_xyz), True)
        plan.close()
        return n

    full = [est(p, -1) for p in ps]
    last = ps[-1]
    K = max(2, int(np.ceil(np.sqrt(2.0 * max(last.nt, 2)))))
    ck = est(last, K)
    assert ck < full[-1]
    budget = sum(full[:-1]) + ck + (full[-1] - ck) // 2
    b = binding.Batch(entries, budget=budget, gradient=True, shots_per_cta=S)
    assert b.stats()["checkpointed"] >= 1
    J, grads = b.run()
    for p, o, Jb, gb in zip(ps, obs, J, grads):
        plan = gpu_plan(p, batch=p.nshots, ckpt_every=-1, shots_per_cta=S)
        Jr, gr, _, _ = gpu_gradient(p, o, plan=plan)
        plan.close()
        assert Jb == Jr
        assert np.array_equal(gb.cpu().numpy().astype(np.float64), gr)
    b.close()


def torch_equal(a, b):
    return bool((a == b).all())


def test_gradient_batch_against_oracle():
    ps = problems(3)
    entries, obs = gradient_entries(ps)
    b = binding.Batch(entries, gradient=True)
    J, grads = b.run()
    k = int(np.argmax([p.nshots for p in ps]))
    p = ps[k]
    J_ref, g_ref, _ = oracle.gradient(oracle_grid(p), p.vp, p.rho, p.src_xyz, p.wavelet,
                                      p.rec_xyz, obs[k])
    assert abs(J[k] - J_ref) <= 1e-3 * abs(J_ref)
    assert rel_l2(grads[k].cpu().numpy(), g_ref) <= TOL_GRAD
    b.close()
