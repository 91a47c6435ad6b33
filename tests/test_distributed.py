"""Shot sharding and the gradient sum across ranks (world size 2, gloo, CPU).

Each rank computes the FP64 oracle gradient of its shard of shots; the sum
over ranks must equal the gradient of all shots computed in one process."""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2110_03345_gb300 import distributed as fd


def test_shard_covers_every_shot_once():
    for n in (1, 5, 128, 129):
        for w in (1, 2, 3, 8):
            got = [s for r in range(w) for s in fd.shard(n, r, w)]
            assert got == list(range(n))
            sizes = [len(fd.shard(n, r, w)) for r in range(w)]
            assert max(sizes) - min(sizes) <= 1


def _problem():
    from paper_2110_03345_gb300 import inputs
    p = inputs.breast_problem((60, 64), 0.5e-3, 90, nelem=16, shots=[0, 4, 8, 12], nb=8,
                              radius=0.3 * 60 * 0.5e-3)
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    p = _problem()
    g = oracle.Grid(p.shape, p.spacing, dt=p.dt, nt=p.nt, order=p.order, nb=p.nb, c_ref=p.c_ref)
    obs = oracle.forward(g, p.vp * 1.01, p.rho, p.src_xyz, p.wavelet, p.rec_xyz)
    shots = list(fd.shard(p.nshots, rank, world))
    J, grad, _ = oracle.gradient(g, p.vp, p.rho, p.src_xyz, p.wavelet, p.rec_xyz, obs, shots=shots)
    t = torch.from_numpy(grad)
    J = fd.sum_over_ranks(t, J)
    if rank == 0:
        np.save(out, np.concatenate([[J], t.numpy().ravel()]))
    dist.destroy_process_group()


def test_gradient_sum_over_two_ranks(tmp_path):
    import oracle
    out = str(tmp_path / "g.npy")
    port = 29500 + (os.getpid() % 1000)
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn")
    res = np.load(out)
    p = _problem()
    g = oracle.Grid(p.shape, p.spacing, dt=p.dt, nt=p.nt, order=p.order, nb=p.nb, c_ref=p.c_ref)
    obs = oracle.forward(g, p.vp * 1.01, p.rho, p.src_xyz, p.wavelet, p.rec_xyz)
    J, grad, _ = oracle.gradient(g, p.vp, p.rho, p.src_xyz, p.wavelet, p.rec_xyz, obs)
    assert res[0] == pytest.approx(J, rel=1e-12)
    np.testing.assert_allclose(res[1:].reshape(p.shape), grad, rtol=1e-10, atol=1e-12 * abs(grad).max())


@pytest.mark.parametrize("workload", ["breast2d", "skull3d"])
def test_bench_ranks_fire_distinct_shots(workload):
    """The benchmark's ranks together fire world x (128 | 32) distinct shots
    (no rank repeats another rank's source positions)."""
    import argparse
    import bench
    for world in (1, 2, 8):
        seen = set()
        for r in range(world):
            a = argparse.Namespace(workload=workload, n=64 if workload == "breast2d" else 32,
                                   nt=8, shots=0)
            p = bench.make_problem(a, r, world)
            pts = {tuple(np.round(s, 15)) for s in p.src_xyz[:, 0, :]}
            assert len(pts) == p.nshots
            seen |= pts
        assert len(seen) == world * (128 if workload == "breast2d" else 32)
