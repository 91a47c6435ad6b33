"""Serving loop: forward and gradient solves admitted by HBM budget.

Requests (one problem each: a grid, a model already resident on the device,
a geometry and wavelets; gradient requests also carry observed data) arrive
over time.  The server keeps a FIFO queue and a set of lanes; a lane is a
worker thread with its own CUDA stream.  A queued request is admitted as soon
as a lane is free AND its device footprint (fwi_plan_estimate of its plan)
fits in the budget left by the requests already running, so requests that
arrive while others are on the GPU start as slots and memory free up, and the
kernels of all admitted requests run concurrently on the device.  Plan
workspaces come from the stream-ordered allocator, so admitting or
retiring a request never synchronises the other lanes.

This is the request-level counterpart of the paper's task farm (Sec. 2.5,
Mosaic runs independent shot gradients on whatever worker is free) on one
GPU: lanes play the role of workers, the HBM budget the role of node memory.

Each result is computed by the same kernels with the same launch shapes
whether the request runs alone or in the mix, so results are identical.
"""
from __future__ import annotations

import collections
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field

import torch

from . import binding


@dataclass
class Request:
    """A forward (observed is None) or gradient solve of one problem."""
    shape: tuple
    spacing: float
    nt: int
    dt: float
    vp: torch.Tensor                 # device-resident model (float32)
    rho: torch.Tensor | None
    geometry: binding.Geometry
    wavelet: torch.Tensor            # device [shots][src][nt]
    observed: torch.Tensor | None = None
    order: int = 8
    sponge: int = 20
    c_ref: float = 0.0
    tag: object = None
    # filled by the server
    t_submit: float = 0.0
    t_start: float = 0.0
    t_done: float = 0.0
    bytes: int = 0
    result: object = None

    @property
    def kind(self):
        return "forward" if self.observed is None else "gradient"

    @property
    def shots(self):
        return self.geometry.nshots


def _make_plan(req: Request, stream, budget=0):
    return binding.Plan(req.shape, req.spacing, req.nt, req.dt, order=req.order,
                        sponge=req.sponge, c_ref=req.c_ref, stream=stream, budget=budget)


def estimate_bytes(req: Request, cap: int = 0, stream=None) -> int:
    """Device bytes the request will hold (workspace of its plan) when its plan
    may use at most `cap` bytes (0: the free memory); a gradient whose
    wavefield history does not fit switches to checkpointing."""
    stream = stream or torch.cuda.current_stream()
    plan = _make_plan(req, stream, budget=cap)
    try:
        return plan.estimate(req.geometry, gradient=req.observed is not None)
    finally:
        plan.close()


def run_request(req: Request, stream, budget=0, shots_per_cta=0):
    """Solve one request on `stream` (used by the lanes and for 'alone' runs);
    shots_per_cta > 0 fixes the shot group of the 2D kernels (0: the plan's
    own choice)."""
    with torch.cuda.stream(stream):
        plan = _make_plan(req, stream, budget=budget)
        if shots_per_cta:
            plan.set_options(shots_per_cta=shots_per_cta)
        try:
            if req.observed is None:
                out = plan.forward(req.vp, req.rho, req.geometry, req.wavelet)
                return out
            J, g, _ = plan.gradient(req.vp, req.rho, req.geometry, req.wavelet, req.observed)
            return (J, g)
        finally:
            plan.close()


class Server:
    """Continuous admission of requests onto `lanes` concurrent CUDA streams
    within `budget_bytes` of device memory.

    fill_points (optional): grid points x shots that fill the GPU.  A request
    then weighs min(1, its points x shots / fill_points) and requests run
    together only while their weights sum to at most 1 (one always runs), so
    requests that each fill the GPU do not contend for it.

    shots_per_cta (optional): the shot group of every request's 2D launches.
    Concurrent requests fill the GPU together, so each may take larger groups
    than its plan alone would (which lowers S until its own launch fills the
    GPU); a fixed value keeps each result the same alone and in the mix."""

    def __init__(self, budget_bytes: int, lanes: int = 4, device=None, request_cap: int = 0,
                 fill_points: int = 0, shots_per_cta: int = 0):
        self.budget = int(budget_bytes)
        self.shots_per_cta = int(shots_per_cta)
        self.lanes = lanes
        self.fill_points = int(fill_points)
        self._load = 0.0
        # one request may hold at most this much (default: an equal share per lane)
        self.request_cap = int(request_cap) or self.budget // lanes
        self.device = device if device is not None else torch.cuda.current_device()
        self._cv = threading.Condition()
        self._queue: collections.deque = collections.deque()
        self._free_lanes = list(range(lanes))
        self._used = 0
        self._streams = [torch.cuda.Stream(device=self.device) for _ in range(lanes)]
        self._stop = False
        self.completed: list[Request] = []
        self.peak_bytes = 0
        self.peak_running = 0
        self._running = 0
        self._sched = threading.Thread(target=self._schedule, daemon=True)
        self._sched.start()

    # -- public ------------------------------------------------------------
    def submit(self, req: Request) -> Future:
        fut: Future = Future()
        if not req.bytes:
            req.bytes = estimate_bytes(req, cap=self.request_cap)
        if req.bytes > self.budget:
            fut.set_exception(binding.FwiError(3, f"request needs {req.bytes} bytes, "
                                                  f"the budget is {self.budget}"))
            return fut
        req.t_submit = time.perf_counter()
        with self._cv:
            self._queue.append((req, fut))
            self._cv.notify_all()
        return fut

    def close(self):
        with self._cv:
            self._stop = True
            self._cv.notify_all()
        self._sched.join()

    def drain(self):
        """Wait until the queue is empty and every lane is idle."""
        with self._cv:
            self._cv.wait_for(lambda: not self._queue and self._running == 0)

    # -- internals ---------------------------------------------------------
    def _schedule(self):
        torch.cuda.set_device(self.device)
        while True:
            with self._cv:
                self._cv.wait_for(lambda: self._stop or self._admissible())
                if self._stop and not self._queue:
                    return
                if not self._admissible():
                    continue
                req, fut = self._queue.popleft()   # FIFO: the head goes first
                lane = self._free_lanes.pop()
                self._used += req.bytes
                self._load += self._weight(req)
                self._running += 1
                self.peak_bytes = max(self.peak_bytes, self._used)
                self.peak_running = max(self.peak_running, self._running)
            threading.Thread(target=self._work, args=(req, fut, lane), daemon=True).start()

    def _weight(self, req: Request) -> float:
        if not self.fill_points:
            return 0.0
        pts = 1
        for n in req.shape:
            pts *= int(n)
        return min(1.0, pts * req.shots / self.fill_points)

    def _admissible(self):
        if not (self._queue and self._free_lanes):
            return False
        head = self._queue[0][0]
        if self._used + head.bytes > self.budget:
            return False
        return self._running == 0 or self._load + self._weight(head) <= 1.0 + 1e-9

    def _work(self, req: Request, fut: Future, lane: int):
        torch.cuda.set_device(self.device)
        stream = self._streams[lane]
        req.t_start = time.perf_counter()
        try:
            req.result = run_request(req, stream, budget=req.bytes,
                                     shots_per_cta=self.shots_per_cta)
            req.t_done = time.perf_counter()
            fut.set_result(req)
        except Exception as e:   # noqa: BLE001 - handed to the caller's future
            req.t_done = time.perf_counter()
            fut.set_exception(e)
        finally:
            with self._cv:
                self._used -= req.bytes
                self._load -= self._weight(req)
                self._running -= 1
                self._free_lanes.append(lane)
                self.completed.append(req)
                self._cv.notify_all()


def latency_stats(reqs) -> dict:
    """p50 / p99 of completion - arrival (seconds) and shots per second."""
    import numpy as np
    lat = np.array([r.t_done - r.t_submit for r in reqs])
    span = max(r.t_done for r in reqs) - min(r.t_submit for r in reqs)
    shots = sum(r.shots for r in reqs)
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "shots_per_s": shots / span, "requests": len(reqs),
            "span_s": span}
