"""Serving pattern: requests admitted by HBM budget onto concurrent lanes;
each result equals the result of the same request run alone."""
import time

import numpy as np
import pytest
import torch

from paper_2110_03345_gb300 import binding, inputs, serve
from _helpers import to_dev

pytestmark = pytest.mark.gpu


def make_requests(n=20, seed=11):
    stream = inputs.config_serving(nreq=n, seed=seed, rate=200.0, side2d=(96, 160),
                                   side3d=(36, 48), nt=(120, 260))
    reqs = []
    for t, kind, p in stream:
        obs = None
        if kind == "gradient":
            obs = to_dev(np.zeros((p.nshots, p.rec_xyz.shape[0], p.nt)) + 1e-6)
        nb = min(p.nb, min(p.shape) // 4)
        reqs.append((t, serve.Request(p.shape, p.spacing, p.nt, p.dt, to_dev(p.vp), to_dev(p.rho),
                                      binding.Geometry(p.src_xyz, p.rec_xyz), to_dev(p.wavelet),
                                      obs, order=p.order, sponge=nb, c_ref=p.c_ref)))
    return reqs


def results_equal(a, b):
    if isinstance(a, tuple):
        return a[0] == b[0] and torch.equal(a[1], b[1])
    return torch.equal(a, b)


def test_mixed_stream_equals_alone():
    reqs = make_requests()
    assert {r.kind for _, r in reqs} == {"forward", "gradient"}
    assert {len(r.shape) for _, r in reqs} == {2, 3}
    server = serve.Server(budget_bytes=24 << 30, lanes=4)
    futs = []
    t0 = time.perf_counter()
    for t, r in reqs:
        while time.perf_counter() - t0 < t:
            time.sleep(0.0005)
        futs.append(server.submit(r))
    done = [f.result(timeout=300) for f in futs]
    server.drain()
    server.close()
    assert server.peak_running >= 2          # requests overlapped on the device
    st = serve.latency_stats(done)
    assert st["p99_s"] >= st["p50_s"] > 0
    alone = torch.cuda.Stream()
    for _, r in reqs:
        ref = serve.run_request(r, alone)
        torch.cuda.synchronize()
        assert results_equal(r.result, ref)


def test_budget_limits_concurrency():
    reqs = make_requests(n=5, seed=12)
    big = max(serve.estimate_bytes(r) for _, r in reqs)
    server = serve.Server(budget_bytes=big, lanes=4, request_cap=big)
    futs = [server.submit(r) for _, r in reqs]
    for f in futs:
        f.result(timeout=300)
    server.drain()
    server.close()
    assert server.peak_bytes <= big
    assert len(server.completed) == 5


def test_oversized_request_is_refused():
    (t, r), = make_requests(n=1, seed=13)
    server = serve.Server(budget_bytes=1 << 20, lanes=2, request_cap=1 << 40)
    fut = server.submit(r)
    with pytest.raises(binding.FwiError) as ei:
        fut.result(timeout=60)
    assert ei.value.status == 3
    server.close()


def test_fill_weights_serialise_large_requests():
    """With fill_points below every request's size each request weighs 1, so
    requests run one at a time; results are those of the requests alone."""
    reqs = make_requests(n=6, seed=14)
    server = serve.Server(budget_bytes=24 << 30, lanes=4, fill_points=1)
    futs = [server.submit(r) for _, r in reqs]
    done = [f.result(timeout=300) for f in futs]
    server.drain()
    server.close()
    assert server.peak_running == 1
    alone = torch.cuda.Stream()
    for r in done:
        ref = serve.run_request(r, alone)
        torch.cuda.synchronize()
        assert results_equal(r.result, ref)


def test_fixed_shot_groups_equal_alone():
    """With a fixed shot group (Server(shots_per_cta=4)), multi-shot gradient
    requests give in the mix what they give alone with that shot group."""
    ps = inputs.config_uneven_batch(nprob=4, seed=7, side=(96, 200), nt=(60, 200), shots=(2, 5),
                                    dx=0.4e-3, nelem=16, nb=12)
    reqs = [serve.Request(p.shape, p.spacing, p.nt, p.dt, to_dev(p.vp), to_dev(p.rho),
                          binding.Geometry(p.src_xyz, p.rec_xyz), to_dev(p.wavelet),
                          to_dev(np.zeros((p.nshots, p.rec_xyz.shape[0], p.nt)) + 1e-6),
                          order=p.order, sponge=p.nb, c_ref=p.c_ref) for p in ps]
    assert max(r.shots for r in reqs) >= 3
    server = serve.Server(budget_bytes=24 << 30, lanes=4, shots_per_cta=4)
    futs = [server.submit(r) for r in reqs]
    for f in futs:
        f.result(timeout=300)
    server.drain()
    server.close()
    alone = torch.cuda.Stream()
    for r in reqs:
        ref = serve.run_request(r, alone, shots_per_cta=4)
        torch.cuda.synchronize()
        assert results_equal(r.result, ref)
