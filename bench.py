#!/usr/bin/env python
"""Benchmark of the acoustic FWI hot path on GB300.

One step = one full misfit gradient (Sec. 2.2 Eqs. 5-9; one forward and one
adjoint propagation per shot, imaging fused into the adjoint) of the 2D
breast-like workload: 1024 x 1024 grid at 0.1 mm, variable density, 8th
order, 128 shots of 4000 steps, 256 receivers (synthetic inputs, seed 2).

Prints one JSON line: grid-point updates per second (Gpts/s, counting one
update per grid point per time step per propagation: 2 propagations per
shot), the HBM roofline of the dominant kernel (CUDA events on the plan's
stream), the FP64 oracle timed on a bounded sample on the host cores, and an
end-to-end figure through the public API with host buffers.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Algorithmic HBM bytes per grid-point update (FP32 fields, no halo re-reads):
# forward step with history store, adjoint step with fused imaging.
BYTES_PER_UPDATE = {("fwd", True): 24, ("fwd", False): 20, ("adj", True): 32, ("adj", False): 28}

WORKLOADS = {
    "breast2d": "2D breast-like phantom 1024x1024, dx=0.1 mm, vd, o8, 128 shots x 4000 steps, 256 receivers",
    "skull3d": "3D skull phantom 256^3, dx=0.25 mm, vd, o10, 32 shots x 2000 steps, 512 receivers",
    "uneven": "64 independent 2D problems, side U{256..1024}, 500-4000 steps, 1-16 shots, vd, o8 (forward)",
    "serving": "Poisson stream (20 req/s) of forward/gradient requests, 75% 2D 512^2-1024^2, 25% 3D 128^3-192^3, 1000-3000 steps",
    "invert": "Sec. 3.2 2D breast imaging: 456x485 at 0.5 mm, 128 ring transducers, 3-cycle 500 kHz tone burst, "
              "2500 steps of 0.08 us, cd, o8; 4 frequency blocks 300-600 kHz x 8 iterations x 16 random shots",
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--workload", default="breast2d", choices=sorted(WORKLOADS))
    ap.add_argument("--shots", type=int, default=0, help="override shot count (testing only)")
    ap.add_argument("--nt", type=int, default=0, help="override time steps (testing only)")
    ap.add_argument("--n", type=int, default=0, help="override grid side (testing only)")
    ap.add_argument("--batch", type=int, default=0)
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--ckpt", type=int, default=0)
    ap.add_argument("--spc", type=int, default=0, help="shots per CTA (TMA kernels)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched, serving and inversion samples")
    ap.add_argument("--nprob", type=int, default=0, help="uneven: problems (default 64)")
    ap.add_argument("--nreq", type=int, default=0, help="serving: requests (default 650)")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="invert: the experiment in scaled units (grid / scale)")
    ap.add_argument("--scheme", default="", choices=sorted(SCHEMES),
                    help="breast2d / skull3d in an extended scheme (default: leapfrog, sponge, "
                         "bilinear points)")
    return ap.parse_args()


# Extended schemes of the solver for the breast2d / skull3d lines (--scheme):
# the plan options and the attenuation (alpha0, y) they set.
SCHEMES = {
    "": "leapfrog (CFL 0.4), sponge, bilinear points",
    "t4": "fourth order in time at CFL 0.8 in 2D / 0.66 in 3D (the same record in fewer steps)",
    "att0": "power-law attenuation y = 0, alpha0 = 5.8 Np/m (0.5 dB/cm of soft tissue at 1 MHz)",
    "att2": "power-law attenuation y = 2, alpha0 = 5.8 Np/m at 1 MHz",
    "sinc": "Kaiser-windowed sinc sources and receivers",
    "pml": "perfectly matched layer over the 20-point absorbing layer",
}


def scheme_setup(scheme):
    """(plan options, (alpha0, y) or None) of an extended scheme."""
    opts = {"t4": {"time_order": 4}, "sinc": {"interp": 1}, "pml": {"boundary": 1}}.get(scheme, {})
    att = {"att0": (5.8, 0), "att2": (5.8 / (2 * np.pi * 1e6) ** 2, 2)}.get(scheme)
    return opts, att


def t4_time_axis(p):
    """The fourth-order scheme's larger step on the same record: CFL 0.8 in 2D
    (2x the leapfrog's 0.4), 0.66 in 3D (the paper's 3D constant), the
    wavelet resampled."""
    from paper_2110_03345_gb300 import inputs
    f = 2.0 if p.ndim == 2 else 0.66 / 0.4
    T = (p.nt - 1) * p.dt
    p.dt = p.dt * f
    p.nt = int(T / p.dt) + 1
    w = inputs.ricker(500e3, p.dt, p.nt)
    p.wavelet = np.broadcast_to(w, (p.nshots,) + p.wavelet.shape[1:2] + (p.nt,)).copy()
    return p


def make_problem(args, rank=0, world=1):
    """The workload of one rank.  A multi-GPU run processes world x 128 (2D)
    or world x 32 (3D) distinct shots, sharded by distributed.shard: in 2D
    firing f is element 2 (f mod 128) of the ring turned by (f div 128) /
    world element pitches (a rotated acquisition of the same phantom), in 3D
    firing f is receiver 16 (f mod 32) + (f div 32) of the sphere (distinct
    for up to 16 ranks)."""
    from paper_2110_03345_gb300 import inputs
    from paper_2110_03345_gb300.distributed import shard
    if args.workload == "breast2d":
        n = args.n or 1024
        nt = args.nt or 4000
        dx = 0.1e-3 * 1024 / n
        fires = shard(128 * world, rank, world)
        turns = sorted({f // 128 for f in fires})
        assert len(turns) == 1 and len(fires) == 128
        p = inputs.config_breast_2d(n=n, dx=dx, nt=nt, shots=[2 * (f % 128) for f in fires],
                                    rotation=turns[0] / world)
    elif args.workload == "invert":
        p = inputs.config_inversion_2d(scale=args.scale)
    else:
        n = args.n or 256
        nt = args.nt or 2000
        dx = 0.25e-3 * 256 / n
        fires = shard(32 * world, rank, world)
        shots = [16 * (f % 32) + f // 32 for f in fires]
        assert world <= 16 and len(shots) == 32
        p = inputs.config_skull_3d(n=n, dx=dx, nt=nt, shots=shots)
    if args.shots:
        p.src_xyz = p.src_xyz[:args.shots]
        p.wavelet = p.wavelet[:args.shots]
    if getattr(args, "scheme", "") == "t4" and args.workload in ("breast2d", "skull3d"):
        p = t4_time_axis(p)
    return p


PROFILE_EVERY = 32   # stencil launches per CUDA-event-timed launch in the timed region


def kernel_name(ndim, tile):
    """Stencil kernel of a resolved tile variant."""
    if ndim == 2:
        return "k_step2d" if tile <= 4 else "k_step2d_tma"
    return "k_step3d" if tile <= 4 else ("k_step3d_tma" if tile <= 8 else "k_step3d_x2")


def useful_updates(p) -> int:
    """2 propagations x grid points x leapfrog steps x shots."""
    return 2 * p.npoints * (p.nt - 1) * p.nshots


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples (every 200 ms) during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        cmd = ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200"]
        if uuid:
            cmd += ["-i", uuid]
        try:
            self.p = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [l.strip().split(", ") for l in self.f.read().splitlines() if l.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for name, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def gpu_uuid():
    try:
        import torch
        u = torch.cuda.get_device_properties(torch.cuda.current_device()).uuid
        s = str(u)
        return s if s.startswith("GPU-") else "GPU-" + s
    except Exception:
        return None


def measured_hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def traffic_record(kernel_kind, tile):
    """DRAM bytes per point of the dominant kernel from a committed ncu summary,
    or None when absent, taken on another kernel variant or on a different
    kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path)).get(kernel_kind)
    except Exception:
        return None
    if not rec or rec.get("tile") != tile:
        return None
    import hashlib
    srcs = rec.get("source", "kernels2d.cu")
    hs = hashlib.sha256()
    try:
        for f in ([srcs] if isinstance(srcs, str) else srcs):   # the kernel's source files, in order
            hs.update(open(os.path.join(ROOT, "paper_2110_03345_gb300", "csrc", f), "rb").read())
    except OSError:
        return None
    h = hs.hexdigest()[:16]
    if h != rec.get("source_sha256_16"):
        return None
    return rec


# ---------------------------------------------------------------- CPU baseline

def cpu_baseline(p, budget_s: float):
    """The FP64 oracle, as it stands, on one shot of the workload with the time
    axis cut so that the run takes about budget_s seconds."""
    import oracle
    oracle.build()
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))

    def run(nt):
        g = oracle.Grid(p.shape, p.spacing, dt=p.dt, nt=nt, order=p.order, nb=p.nb, c_ref=p.c_ref)
        obs = np.zeros((1, p.rec_xyz.shape[0], nt))
        t0 = time.perf_counter()
        oracle.gradient(g, p.vp, p.rho, p.src_xyz[:1], p.wavelet[:1, :, :nt], p.rec_xyz, obs,
                        ckpt_every=max(2, int(np.sqrt(2 * nt))))
        return time.perf_counter() - t0

    t_small = run(12)
    per_step = t_small / 11
    nt = int(min(p.nt, max(12, budget_s / max(per_step, 1e-6))))
    t = run(nt)
    upd = 2 * p.npoints * (nt - 1)
    return {"value": upd / t / 1e9, "unit": "Gpts/s", "cores": cores, "kind": "oracle",
            "seconds": t,
            "sample": f"1 shot of {p.nshots}, {nt} of {p.nt} steps, full grid "
                      f"{'x'.join(map(str, p.shape))}, FP64 C oracle (OpenMP), observed data = 0, "
                      f"checkpointed gradient; {t:.1f} s"}


# ---------------------------------------------------------------- reference arm

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    if args.workload in ("uneven", "serving"):
        print(json.dumps({"impl": "reference", "unavailable":
                          "the oracle arm times the breast2d, skull3d and invert workloads only"}))
        return 0
    p = make_problem(args)
    steps = []
    per = max(3.0, min(args.cpu_seconds, 150.0 / max(1, args.steps + args.warmup)))
    for i in range(args.warmup + args.steps):
        r = cpu_baseline(p, per)
        if i >= args.warmup:
            steps.append(r)
    val = statistics.median(s["value"] for s in steps)
    upd = useful_updates(p)
    if args.workload == "invert":                     # same metric as the GPU arm's invert line
        per_grad = 2 * p.npoints * (p.nt - 1)
        v = val * 1e9 / per_grad
        line = {"impl": "reference",
                "metric": "shot gradients/s in the inversion loop (low-pass, gradient, update)",
                "value": v, "unit": "shot gradients/s", "n_gpus": args.gpus, "steps": args.steps,
                "warmup": args.warmup, "higher_is_better": True, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOADS["invert"], "scale": args.scale,
                           "sample": steps[-1]["sample"]},
                "cpu_baseline": {"value": v, "unit": "shot gradients/s", "cores": steps[-1]["cores"],
                                 "kind": "oracle", "sample": steps[-1]["sample"]},
                "e2e": {"value": v, "unit": "shot gradients/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0
    sample_ms = statistics.median(s["seconds"] for s in steps) * 1e3
    line = {
        "impl": "reference", "metric": "Gpts/s (grid-point updates per second, gradient: forward + adjoint)",
        "value": val, "unit": "Gpts/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sample_ms, "higher_is_better": True,
        "step": "one bounded sample of the workload: " + steps[-1]["sample"],
        "extrapolated": True,
        "extrapolation": {"ms_per_full_step": upd / (val * 1e9) * 1e3,
                          "basis": "the measured Gpts/s applied to the full workload's updates "
                                   f"({upd} per step: {p.nshots} shots x {p.nt} steps); "
                                   "the full step is not run"},
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "shots": p.nshots, "nt": p.nt,
                   "grid": list(p.shape), "sample": steps[-1]["sample"]},
        "cpu_baseline": {"value": val, "unit": "Gpts/s", "cores": steps[-1]["cores"],
                         "kind": "oracle", "sample": steps[-1]["sample"]},
        "e2e": {"value": val, "unit": "Gpts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- batched and serving

def uneven_batch(nprob=64, seed=4, reps=2, **kw):
    """Uneven set of independent 2D problems: one multi-problem launch per
    step captured in one CUDA graph (tile variant and shots per CTA from the
    batch autotuner), against the plain solver run problem after problem with
    one shot per launch ("plain") and with all of a problem's shots per launch
    ("per_problem").  Inputs and workspaces resident (created outside the
    timed region)."""
    import torch
    from paper_2110_03345_gb300 import binding, inputs
    ps = inputs.config_uneven_batch(nprob=nprob, seed=seed, **kw)
    dev = torch.device("cuda", torch.cuda.current_device())
    f32 = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device=dev)
    entries = [dict(shape=p.shape, spacing=p.spacing, nt=p.nt, dt=p.dt, order=p.order, sponge=p.nb,
                    c_ref=p.c_ref, vp=f32(p.vp), rho=f32(p.rho),
                    geometry=binding.Geometry(p.src_xyz, p.rec_xyz), wavelet=f32(p.wavelet))
               for p in ps]
    shots = sum(p.nshots for p in ps)
    updates = sum(p.nshots * p.npoints * (p.nt - 1) for p in ps)
    from paper_2110_03345_gb300 import autotune
    tuned = autotune.tune_batch(entries)
    batch = binding.Batch(entries, use_graph=True, **tuned)
    batch.run()
    t_b = []
    for _ in range(reps):
        batch.run()
        t_b.append(batch.stats()["run_ms"] * 1e-3)
    nodes = batch.stats()["launches"]
    batch.close()

    def plain(per_launch, nrep):
        """Each problem on its own plan, one problem after another: all its
        shots per launch (per_launch = 0) or one shot per launch (1)."""
        plans = []
        for e in entries:
            pl = binding.Plan(e["shape"], e["spacing"], e["nt"], e["dt"], order=e["order"],
                              sponge=e["sponge"], c_ref=e["c_ref"])
            pl.set_options(batch=per_launch or e["geometry"].nshots)
            plans.append(pl)
        outs = [torch.empty((e["geometry"].nshots, e["geometry"].nrec, e["nt"]), device=dev)
                for e in entries]
        for pl, e, o in zip(plans, entries, outs):
            pl.forward(e["vp"], e["rho"], e["geometry"], e["wavelet"], traces=o)
        t_p = []
        launches = 0
        for _ in range(nrep):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for pl, e, o in zip(plans, entries, outs):
                pl.forward(e["vp"], e["rho"], e["geometry"], e["wavelet"], traces=o)
                launches += pl.stats()["launches"]
            torch.cuda.synchronize()
            t_p.append(time.perf_counter() - t0)
        for pl in plans:
            pl.close()
        tp = min(t_p)
        return {"shots_per_s": shots / tp, "gpts": updates / tp / 1e9, "s": tp,
                "launches": launches // nrep}

    per_problem = plain(0, reps)
    one_shot = plain(1, 1)
    tb = min(t_b)
    return {"problems": nprob, "shots": shots, "updates": updates,
            "batched": {"shots_per_s": shots / tb, "gpts": updates / tb / 1e9, "s": tb,
                        "graph_nodes": nodes, "launches": 1, "options": tuned},
            "plain": one_shot, "per_problem": per_problem,
            "speedup": one_shot["s"] / tb, "speedup_vs_per_problem": per_problem["s"] / tb}


def uneven_gradient(nprob=64, seed=4, lanes=4, **kw):
    """Gradient variant of the uneven set: every problem's gradient (misfit
    against zero data), (a) submitted at once to the serving loop, which runs
    them concurrently on `lanes` streams within the HBM budget and while their
    GPU-fill weights sum to at most one, one plan per problem with all its
    shots per launch; (b) one plan per problem, problems one after another
    (each plan's own shots per CTA, and six); (c) the plain solver with one
    shot per launch; (d) gradient batches (one CUDA graph each, shot groups
    sized for the batch)."""
    import torch
    from paper_2110_03345_gb300 import binding, inputs, serve
    ps = inputs.config_uneven_batch(nprob=nprob, seed=seed, **kw)
    dev = torch.device("cuda", torch.cuda.current_device())
    f32 = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device=dev)
    reqs = [dict(shape=p.shape, spacing=p.spacing, nt=p.nt, dt=p.dt, vp=f32(p.vp), rho=f32(p.rho),
                 geometry=binding.Geometry(p.src_xyz, p.rec_xyz), wavelet=f32(p.wavelet),
                 observed=torch.zeros((p.nshots, p.rec_xyz.shape[0], p.nt), device=dev),
                 order=p.order, sponge=p.nb, c_ref=p.c_ref) for p in ps]
    shots = sum(p.nshots for p in ps)
    updates = sum(2 * p.nshots * p.npoints * (p.nt - 1) for p in ps)
    budget = int(0.7 * binding.mem_available())

    def served(spc=0):
        # requests that each fill the GPU (>= 8 M points x shots) run one at a
        # time, and a request may take the whole budget (as in the sequential
        # arms), so no plan is pushed into checkpointing by a per-request cap
        server = serve.Server(budget_bytes=budget, lanes=lanes, fill_points=8 << 20,
                              request_cap=budget, shots_per_cta=spc)
        objs = [serve.Request(**r) for r in reqs]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        futs = [server.submit(o) for o in objs]
        for f in futs:
            f.result()
        server.drain()
        t = time.perf_counter() - t0
        server.close()
        return t

    def sequential(per_launch, spc=0):
        stream = torch.cuda.current_stream()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for r in reqs:
            pl = binding.Plan(r["shape"], r["spacing"], r["nt"], r["dt"], order=r["order"],
                              sponge=r["sponge"], c_ref=r["c_ref"], stream=stream,
                              budget=budget)
            pl.set_options(batch=per_launch, shots_per_cta=spc)
            pl.gradient(r["vp"], r["rho"], r["geometry"], r["wavelet"], r["observed"])
            pl.close()
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    def batched():
        """(d) gradient batches: the problems packed (first fit, largest
        first) into batches whose full histories fit the budget, each one CUDA graph with
        one branch per problem (its forward, misfit, adjoint with imaging and
        finalisation on a stream of its own); a problem whose history alone
        exceeds the budget runs on its own (checkpointed) plan.  Batches are
        prepared outside the timed region, as in the forward arm."""
        stream = torch.cuda.current_stream()
        est = []
        for r in reqs:
            pl = binding.Plan(r["shape"], r["spacing"], r["nt"], r["dt"], order=r["order"],
                              sponge=r["sponge"], c_ref=r["c_ref"], stream=stream)
            pl.set_options(batch=r["geometry"].nshots, ckpt_every=-1)
            est.append(pl.estimate(r["geometry"], True))
            pl.close()
        # first-fit decreasing on the workspace sizes: few graphs, each with
        # as many concurrent branches as the budget holds
        order = sorted(range(len(reqs)), key=lambda i: -est[i])
        groups, used, alone = [], [], []
        for i in order:
            if est[i] > budget:
                alone.append(i)
                continue
            for g in range(len(groups)):
                if used[g] + est[i] <= budget:
                    groups[g].append(i)
                    used[g] += est[i]
                    break
            else:
                groups.append([i])
                used.append(est[i])
        t = 0.0
        for gidx in groups:
            b = binding.Batch([reqs[i] for i in gidx], budget=budget, gradient=True)
            b.run()   # warm-up
            b.run()
            t += b.stats()["run_ms"] * 1e-3
            b.close()
            torch.cuda.empty_cache()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in alone:
            r = reqs[i]
            pl = binding.Plan(r["shape"], r["spacing"], r["nt"], r["dt"], order=r["order"],
                              sponge=r["sponge"], c_ref=r["c_ref"], stream=stream, budget=budget)
            pl.gradient(r["vp"], r["rho"], r["geometry"], r["wavelet"], r["observed"])
            pl.close()
        torch.cuda.synchronize()
        return t + time.perf_counter() - t0, len(groups), len(alone)

    served()   # warm-up (allocator pool, kernel attributes)
    out = {}
    # per_problem_s6: the same with six shots per CTA in every plan (the shot
    # groups the batches take), against each plan's own choice
    for name, fn in (("served", served), ("served_s6", lambda: served(6)),
                     ("per_problem", lambda: sequential(0)),
                     ("per_problem_s6", lambda: sequential(0, 6)),
                     ("plain", lambda: sequential(1))):
        t = fn()
        out[name] = {"shots_per_s": shots / t, "gpts": updates / t / 1e9, "s": t}
    t, ngroups, nalone = batched()
    out["batched"] = {"shots_per_s": shots / t, "gpts": updates / t / 1e9, "s": t,
                      "graphs": ngroups, "problems_on_own_plan": nalone}
    out.update({"problems": nprob, "shots": shots, "updates": updates, "lanes": lanes,
                "speedup": out["plain"]["s"] / out["served"]["s"],
                "speedup_vs_per_problem": out["per_problem"]["s"] / out["served"]["s"],
                "batched_vs_per_problem": out["per_problem"]["s"] / out["batched"]["s"]})
    return out


def serving_stream(nreq=650, warm=50, seed=5, lanes=4, rate=20.0, **kw):
    """Poisson request stream through the serving loop (continuous admission
    onto `lanes` concurrent streams under an HBM budget) and through the plain
    solver (one request at a time, first come first served).  Latency =
    completion - arrival (host clock); the first `warm` requests are not
    counted."""
    import torch
    from paper_2110_03345_gb300 import binding, inputs, serve
    dev = torch.device("cuda", torch.cuda.current_device())
    f32 = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device=dev)
    stream = inputs.config_serving(nreq=nreq, seed=seed, rate=rate, **kw)
    models = {}
    reqs = []
    for t, kind, p in stream:
        key = (p.shape, id(p))
        vp, rho = f32(p.vp), f32(p.rho)          # device-resident models
        obs = None
        if kind == "gradient":
            obs = torch.zeros((p.nshots, p.rec_xyz.shape[0], p.nt), device=dev)
        reqs.append((t, dict(shape=p.shape, spacing=p.spacing, nt=p.nt, dt=p.dt, vp=vp, rho=rho,
                             geometry=binding.Geometry(p.src_xyz, p.rec_xyz), wavelet=f32(p.wavelet),
                             observed=obs, order=p.order, sponge=p.nb, c_ref=p.c_ref)))
    budget = int(0.7 * binding.mem_available())

    def play(nlanes):
        server = serve.Server(budget_bytes=budget, lanes=nlanes, request_cap=budget // 4)
        objs = [serve.Request(**r) for _, r in reqs]
        futs = []
        t0 = time.perf_counter()
        for (t, _), o in zip(reqs, objs):
            now = time.perf_counter() - t0
            if now < t:
                time.sleep(t - now)
            futs.append(server.submit(o))
        for f in futs:
            f.result()
        server.drain()
        server.close()
        counted = objs[warm:] if len(objs) > warm else objs
        st = serve.latency_stats(counted)
        st["peak_running"] = server.peak_running
        return st

    cont = play(lanes)
    plain = play(1)
    return {"requests": nreq, "warmup": warm, "rate_per_s": rate, "lanes": lanes,
            "continuous": cont, "plain": plain}


# ---------------------------------------------------------------- GPU arm

def roofline(acc, steps, ms, vd, ndim, tile, scheme=""):
    """Roofline record of the dominant stencil kernel from the plan's counters
    summed over the timed steps (CUDA events around every PROFILE_EVERY-th
    launch on the plan's stream; an extended scheme's step of two passes is
    timed as one launch)."""
    per_launch = {k: acc[f"{k}_ms"] / max(acc[f"{k}_timed"], 1) for k in ("fwd", "adj")}
    kind = "adj" if per_launch["adj"] * acc["adj_launches"] >= per_launch["fwd"] * acc["fwd_launches"] \
        else "fwd"
    n_l = max(acc[f"{kind}_launches"], 1)
    t_launch = per_launch[kind] * 1e-3
    pts_launch = acc[f"{kind}_points"] / n_l
    ext = scheme in ("t4", "att0", "att2", "pml")
    if ext:
        bpu = SCHEME_BYTES[(scheme, kind)] + (4 if vd else 0)   # + ln rho
        # 2D sponge-boundary schemes run on the TMA shot-loop kernels
        kern = ("k_pml%dd" % ndim if scheme == "pml" else
                "k_step2d_tma_ext" if ndim == 2 else
                "k_step3d_x2" if scheme in ("t4", "att0") else "k_ext3d")
        kname = "%s %s step (%s)" % (kern, "adjoint+imaging" if kind == "adj" else "forward+store",
                                     scheme)
    else:
        bpu = BYTES_PER_UPDATE[(kind, vd)]
        kname = "%s %s" % (kernel_name(ndim, tile), "adjoint+imaging" if kind == "adj" else "forward+store")
    achieved = bpu * pts_launch / t_launch / 1e9
    peak, peak_src = measured_hbm_peak()
    tr = traffic_record(f"{ndim}d-{kind}" + (f"-{scheme}" if scheme else ""), tile)
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": (tr["dram_bytes_per_point"] * pts_launch) if tr else None,
            "kernel": kname,
            "bytes_per_update": bpu, "points_per_launch": int(pts_launch),
            "launch_ms": t_launch * 1e3, "peak_source": peak_src,
            "timed_launches": int(acc[f"{kind}_timed"]),
            "share_of_step": per_launch[kind] * n_l / steps / ms}


# Algorithmic HBM bytes per point update of the extended schemes' steps, as
# fused single passes (FP32 fields, constant density; variable density adds
# the ln rho field, 4 B): fourth order in time: u^n, u^{n-1}, k read, u^{n+1},
# F, k w written (adjoint: lambda^k, lambda^{k+1}, k, F, k w, g read,
# lambda^{k-1}, g written); attenuation adds its coefficient (y = 0) or the
# coefficient and the Laplacian state read and written (y = 2).
SCHEME_BYTES = {("t4", "fwd"): 24, ("t4", "adj"): 32, ("att0", "fwd"): 24, ("att0", "adj"): 32,
                ("att2", "fwd"): 32, ("att2", "adj"): 40,
                # the PML step is the leapfrog's away from the layer (its fields
                # are touched in the layer only, a small fraction of the grid)
                ("pml", "fwd"): 20, ("pml", "adj"): 28}


def scheme_sample(kind, shots=30, steps=1, warmup=1):
    """The 2D breast workload (1024^2, 0.1 mm, vd, o8, 256 receivers, 100 us
    record) with `shots` of its 128 shots, in an extended scheme: "t4" the
    fourth-order time scheme at CFL 0.8 (2000 steps of 50 ns) against the
    leapfrog at CFL 0.4 (4000 steps of 25 ns) on the same shots
    (time-to-solution of the same record); "att0" / "att2" the attenuation
    term of Eq. 10 with alpha0 of soft tissue (0.5 dB/cm at 1 MHz: 5.8 Np/m
    for y = 0, 5.8 Np/m / (2 pi 1e6)^2 for y = 2); "sinc" Kaiser-windowed sinc
    points; "pml" the perfectly matched layer.  Gradient Gpts/s (useful
    updates: 2 x points x steps x shots) and
    the roofline of the dominant kernel, inputs resident."""
    import torch
    from paper_2110_03345_gb300 import binding, inputs
    p = inputs.config_breast_2d(shots=list(range(0, 2 * shots, 2)))
    dev = torch.device("cuda", torch.cuda.current_device())
    f32 = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)
    geo = binding.Geometry(p.src_xyz, p.rec_xyz)
    vp, rho = f32(p.vp), f32(p.rho)
    stream = torch.cuda.current_stream()

    def run(nt, dt, opts, alpha=None, y=0):
        w = inputs.ricker(500e3, dt, nt)
        wav = f32(np.broadcast_to(w, (p.nshots, 1, nt)))
        plan = binding.Plan(p.shape, p.spacing, nt, dt, order=p.order, sponge=p.nb, c_ref=p.c_ref,
                            stream=stream)
        plan.set_options(profile=PROFILE_EVERY, **opts)
        if alpha is not None:
            plan.set_attenuation(f32(np.full(p.shape, alpha)), y)
        obs = plan.forward(f32(p.vp_true), rho, geo, wav)
        grad = torch.empty(p.shape, device=dev, dtype=torch.float32)
        for _ in range(warmup):
            plan.gradient(vp, rho, geo, wav, obs, grad=grad)
        acc = dict.fromkeys(STAT_KEYS, 0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            plan.gradient(vp, rho, geo, wav, obs, grad=grad)
            st = plan.stats()
            for k in acc:
                acc[k] += st[k]
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        st = plan.stats()
        plan.close()
        upd = 2 * p.npoints * (nt - 1) * p.nshots
        return {"nt": nt, "dt_ns": dt * 1e9, "s_per_gradient": ms * 1e-3,
                "value": upd / (ms * 1e-3) / 1e9, "unit": "Gpts/s", "batch": st["batch"],
                "gpu_launches": int(acc["launches"]), "acc": acc, "ms": ms}

    def with_roof(r, key):
        acc, ms = r.pop("acc"), r.pop("ms")
        r["roofline"] = roofline(acc, steps, ms, True, 2, 6, key or "")
        return r

    out = {"workload": f"breast2d 1024^2, {p.nshots} of the 128 shots, vd, o8, 100 us record",
           "scheme": kind}
    if kind == "t4":
        lf = with_roof(run(p.nt, p.dt, {}), None)
        t4 = with_roof(run((p.nt - 1) // 2 + 1, 2 * p.dt, {"time_order": 4}), "t4")
        out.update({"leapfrog_cfl_0.4": lf, "time4_cfl_0.8": t4,
                    "time_to_solution_speedup": lf["s_per_gradient"] / t4["s_per_gradient"]})
    else:
        opts, att = scheme_setup(kind)
        alpha, y = att if att else (None, 0)
        out.update(with_roof(run(p.nt, p.dt, opts, alpha=alpha, y=y), kind if kind != "sinc" else None))
        if att:
            out["alpha0"] = alpha
    return out


STAT_KEYS = ("fwd_ms", "adj_ms", "fwd_launches", "adj_launches", "fwd_points", "adj_points",
             "launches", "fwd_timed", "adj_timed")


def skull3d_sample(shots=2, steps=2, warmup=1, scheme="", **opts):
    """The 3D workload at full grid size and time axis (256^3, 0.25 mm,
    10th order, variable density, 2000 steps, 512 receivers) with `shots`
    of its 32 shots: gradient Gpts/s and the roofline of its dominant kernel,
    device-timed like the main line (inputs resident).  `scheme`: an extended
    scheme of SCHEMES (the fourth-order scheme on the same record at CFL
    0.66)."""
    import torch
    from paper_2110_03345_gb300 import binding, inputs
    p = inputs.config_skull_3d(shots=list(range(0, 16 * shots, 16)))
    sopts, satt = scheme_setup(scheme)
    if scheme == "t4":
        p = t4_time_axis(p)
    dev = torch.device("cuda", torch.cuda.current_device())
    f32 = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)
    vp, rho, wav = f32(p.vp), f32(p.rho), f32(p.wavelet)
    geo = binding.Geometry(p.src_xyz, p.rec_xyz)
    stream = torch.cuda.current_stream()
    plan = binding.Plan(p.shape, p.spacing, p.nt, p.dt, order=p.order, sponge=p.nb, c_ref=p.c_ref,
                        stream=stream)
    plan.set_options(**sopts)
    if satt is not None:
        plan.set_attenuation(f32(np.full(p.shape, satt[0])), satt[1])
    obs = plan.forward(f32(p.vp_true), rho, geo, wav)
    grad = torch.empty(p.shape, device=dev, dtype=torch.float32)
    plan.set_options(profile=PROFILE_EVERY, **sopts, **opts)
    for _ in range(warmup):
        plan.gradient(vp, rho, geo, wav, obs, grad=grad)
    acc = dict.fromkeys(STAT_KEYS, 0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        plan.gradient(vp, rho, geo, wav, obs, grad=grad)
        st = plan.stats()
        for k in acc:
            acc[k] += st[k]
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    st = plan.stats()
    plan.close()
    upd = useful_updates(p)
    out = {"workload": f"skull3d 256^3 x 2000 steps, {shots} of the 32 shots, vd, o10, 512 receivers",
           "value": upd / (ms * 1e-3) / 1e9, "unit": "Gpts/s", "ms_per_gradient": ms,
           "steps": steps, "warmup": warmup, "batch": st["batch"], "ckpt_every": st["ckpt_every"],
           "tile": st["tile"], "gpu_launches": int(acc["launches"]),
           "roofline": roofline(acc, steps, ms, True, 3, st["tile"], scheme)}
    if scheme:
        out.update({"scheme": scheme, "nt": p.nt, "dt_ns": p.dt * 1e9})
    return out


def run_mine(args):
    import torch
    from paper_2110_03345_gb300 import binding

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    def barrier():
        if dist is not None:
            dist.barrier()

    p = make_problem(args, rank, world)
    vd = p.rho is not None
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    vp_h = torch.from_numpy(f32(p.vp)).pin_memory()
    rho_h = torch.from_numpy(f32(p.rho)).pin_memory()
    wav_h = torch.from_numpy(f32(p.wavelet)).pin_memory()
    vp, rho, wav = vp_h.to(dev), rho_h.to(dev), wav_h.to(dev)
    geo = binding.Geometry(p.src_xyz, p.rec_xyz)
    stream = torch.cuda.current_stream()
    plan = binding.Plan(p.shape, p.spacing, p.nt, p.dt, order=p.order, sponge=p.nb, c_ref=p.c_ref,
                        stream=stream)
    sopts, satt = scheme_setup(args.scheme)
    if satt is not None:
        alpha0 = torch.full(p.shape, satt[0], device=dev, dtype=torch.float32)
        plan.set_attenuation(alpha0, satt[1])
    plan.set_options(**sopts)
    # observed data: the same solver on the perturbed model (bench input only)
    obs = plan.forward(torch.from_numpy(f32(p.vp_true)).to(dev), rho, geo, wav)
    obs_h = obs.cpu().pin_memory()
    grad = torch.empty(p.shape, device=dev, dtype=torch.float32)
    # CUDA events around every PROFILE_EVERY-th stencil launch (the events
    # stay in the timed region; sampling keeps their cost small)
    plan.set_options(batch=args.batch, tile=args.tile, ckpt_every=args.ckpt, profile=PROFILE_EVERY,
                     shots_per_cta=args.spc, **sopts)
    plan.gradient(vp, rho, geo, wav, obs, grad=grad)      # first warm-up: sets the batch size
    tuned = None
    if not args.tile and not args.spc and not args.scheme:
        # kernel variant and shots per CTA from the autotuner at the real batch size
        from paper_2110_03345_gb300 import autotune
        b_real = plan.stats()["batch"]
        tuned = autotune.tune(p.shape, p.spacing, p.dt, p.order, p.nb, p.c_ref, vp, rho, geo,
                              wav, observed=obs, steps=60, batch=b_real)
        plan.set_options(batch=args.batch, ckpt_every=args.ckpt, profile=PROFILE_EVERY, **tuned)
    for _ in range(max(args.warmup - 1, 1)):
        plan.gradient(vp, rho, geo, wav, obs, grad=grad)
    torch.cuda.synchronize()

    clocks = ClockSampler(gpu_uuid())
    acc = dict.fromkeys(STAT_KEYS, 0)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    from paper_2110_03345_gb300 import distributed as fwi_dist
    J = None
    for _ in range(args.steps):
        J, _, _ = plan.gradient(vp, rho, geo, wav, obs, grad=grad)
        s = plan.stats()
        for k in acc:
            acc[k] += s[k]
        # the exchange step of a multi-GPU run: the gradient and misfit of all
        # ranks' shots are summed (the paper's sum over shots); no-op on one GPU
        J = fwi_dist.sum_over_ranks(grad, J)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1) / args.steps
    clk = clocks.stop()
    if dist is not None:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    stats = plan.stats()

    upd = useful_updates(p)
    value = world * upd / (ms * 1e-3) / 1e9
    roof = roofline(acc, args.steps, ms, vd, p.ndim, stats["tile"], args.scheme)

    e2e = None
    if not args.no_e2e:
        gh = torch.empty(p.shape, dtype=torch.float32).pin_memory()
        nb = vp_h.numel() * 4 + rho_h.numel() * 4 + wav_h.numel() * 4 + obs_h.numel() * 4
        ke = 3
        te_all = []
        for _ in range(ke):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            vp_d = vp_h.to(dev, non_blocking=True)
            rho_d = rho_h.to(dev, non_blocking=True)
            wav_d = wav_h.to(dev, non_blocking=True)
            obs_d = obs_h.to(dev, non_blocking=True)
            Je, gd, _ = plan.gradient(vp_d, rho_d, geo, wav_d, obs_d)
            gh.copy_(gd, non_blocking=True)
            torch.cuda.synchronize()
            te_all.append(time.perf_counter() - t0)
        te = statistics.median(te_all)
        e2e = {"value": world * upd / te / 1e9, "unit": "Gpts/s", "h2d_bytes_per_step": nb,
               "d2h_bytes_per_step": gh.numel() * 4 + 8, "steps": ke, "statistic": "median",
               "samples_s": te_all}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(p, args.cpu_seconds)
    # the samples below admit work by free device memory: release this workload's
    plan.close()
    del vp, rho, wav, obs, grad
    torch.cuda.empty_cache()
    extras = {}
    if rank == 0 and world == 1 and not args.no_extras:
        # reduced samples of the uneven-batch and serving patterns (full size:
        # --workload uneven / serving)
        if args.workload == "breast2d" and not args.scheme:
            extras["skull3d"] = skull3d_sample()
            extras["schemes"] = {k: scheme_sample(k) for k in ("t4", "att0", "att2", "sinc", "pml")}
            # the 3D schemes on the plane-ring kernels (one timed gradient each)
            extras["schemes3d"] = {k: skull3d_sample(steps=1, scheme=k) for k in ("t4", "att0")}
        extras["batched"] = uneven_batch(nprob=16, seed=4, reps=1)
        extras["serving"] = serving_stream(nreq=80, warm=10, seed=5)
        try:                               # the full Sec. 3.2 loop: ~3 s on one GB300
            extras["inversion"] = inversion_run()
        except Exception as ex:            # reported, not fatal to the gradient line
            extras["inversion"] = {"error": f"{type(ex).__name__}: {ex}"}

    if rank == 0:
        line = {
            "metric": "Gpts/s (grid-point updates per second, gradient: forward + adjoint)",
            "value": value, "unit": "Gpts/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "scheme": SCHEMES[args.scheme],
                       "dt_ns": p.dt * 1e9, "grid": list(p.shape),
                       "shots": p.nshots, "nt": p.nt, "receivers": int(p.rec_xyz.shape[0]),
                       "order": p.order, "variable_density": vd,
                       "batch": stats["batch"], "ckpt_every": stats["ckpt_every"], "tile": stats["tile"],
                       "autotuned": tuned,
                       "l2": "inputs larger than L2 (history of every batch streams through HBM)",
                       "misfit": J},
            "shots_per_s": world * p.nshots / (ms * 1e-3),
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(acc["launches"]),
            "clocks": clk,
        }
        line.update(extras)
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------- inversion loop

def inversion_run(scale=1.0, step=5.0, blocks=None):
    """The imaging experiment of Sec. 3.2 through invert.Inversion: frequency
    blocks, 16 random shots per iteration (each shot once per block), one
    normalised gradient-descent step per iteration.  Observed data come from
    the same solver on the true phantom.  Reports the loop's wall time (every
    iteration: two low-pass launches, the gradient of 16 shots, the update),
    its throughput and the error to the true model (epsilon of Sec. 3.2)."""
    import torch
    from paper_2110_03345_gb300 import binding, inputs, invert
    p = inputs.config_inversion_2d(scale=scale)
    dev = torch.device("cuda", torch.cuda.current_device())

    def f32(a):
        return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)

    plan = binding.Plan(p.shape, p.spacing, p.nt, p.dt, order=p.order, sponge=p.nb, c_ref=p.c_ref)
    geo = binding.Geometry(p.src_xyz, p.rec_xyz)
    wav = f32(p.wavelet)
    obs = plan.forward(f32(p.vp_true), None, geo, wav)
    freqs = tuple(p.extra["freqs"]) if blocks is None else tuple(p.extra["freqs"][:blocks])
    sched = p.extra["schedule"][:len(freqs)]
    per_iter = max(len(ids) for b in sched for ids in b)
    run = invert.Inversion(plan, p.src_xyz, p.rec_xyz, wav, obs, mask=f32(p.extra["mask"]),
                           bounds=(1400.0, 1600.0), filter_cycles=p.extra["filter_cycles"],
                           max_shots=per_iter)
    run.iterate(f32(p.vp), sched[0][0], freqs[0], step)          # warm-up on a copy
    per_call = []                                                  # kernels of each gradient call
    vp = f32(p.vp)
    rec = run.run(vp, freqs, sched, step,
                  callback=lambda b, i, J: per_call.append(plan.stats()["launches"]))
    iters = sum(len(b) for b in sched)
    launches = sum(per_call) + 4 * iters                           # + 2 low-pass, 2 update kernels
    vp_h = vp.cpu().numpy().astype(np.float64)
    region = p.extra["mask"] > 0

    def eps(v, where=None):
        d = np.abs(v - p.vp_true)
        return float(d[where].mean() if where is not None else d.mean())

    # device time of the loop's own kernels, for one iteration of the first block
    st = plan.stream
    M = invert.half_width(freqs[0], p.dt, p.extra["filter_cycles"])
    ids = sched[0][0]
    out = torch.empty((len(ids),) + tuple(obs.shape[1:]), device=dev, dtype=torch.float32)
    vp_t = f32(p.vp)
    work = torch.empty(1, device=dev, dtype=torch.float32)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    with torch.cuda.stream(st):
        e[0].record(st)
        for _ in range(5):
            binding.lowpass(obs, ids, p.dt, freqs[0], M, out=out, stream=st)
        e[1].record(st)
        for _ in range(5):
            binding.vp_update(vp_t, run.grad, step, 1400.0, 1600.0, work=work, stream=st)
        e[2].record(st)
    st.synchronize()
    lp_ms, up_ms = e[0].elapsed_time(e[1]) / 5, e[1].elapsed_time(e[2]) / 5
    lp_bytes = 2 * 4 * out.numel()
    plan.close()
    return {"grid": list(p.shape), "nt": p.nt, "shots": p.nshots, "blocks_khz": [f / 1e3 for f in freqs],
            "iterations": iters, "shots_per_iteration": per_iter, "step_m_per_s": step,
            "seconds": rec.seconds, "shot_gradients": rec.shot_gradients,
            "shot_gradients_per_s": rec.shot_gradients / rec.seconds,
            "gpts": rec.point_updates / rec.seconds / 1e9,
            "s_per_iteration": rec.seconds / iters,
            "epsilon_start": eps(p.vp), "epsilon_final": eps(vp_h),
            "epsilon_start_in_ring": eps(p.vp, region), "epsilon_final_in_ring": eps(vp_h, region),
            "misfit_first_iteration_per_block": [Jb[0] for Jb in rec.misfits],
            "misfit_last_iteration_per_block": [Jb[-1] for Jb in rec.misfits],
            "lowpass_ms": lp_ms, "lowpass_gbs": lp_bytes / (lp_ms * 1e-3) / 1e9,
            "update_ms": up_ms, "gpu_launches": int(launches), "scale": scale}


def run_extra_workload(args):
    """--workload uneven | serving: one JSON line for that workload alone."""
    import torch
    torch.cuda.set_device(0)
    if args.workload == "invert":
        from paper_2110_03345_gb300 import inputs
        r = inversion_run(scale=args.scale)
        cpu = None
        if not args.no_cpu_baseline:
            p = inputs.config_inversion_2d(scale=args.scale)
            c = cpu_baseline(p, args.cpu_seconds)
            per_grad = 2 * p.npoints * (p.nt - 1)
            cpu = dict(c, value=c["value"] * 1e9 / per_grad, unit="shot gradients/s")
        line = {"metric": "shot gradients/s in the inversion loop (low-pass, gradient, update)",
                "value": r["shot_gradients_per_s"], "unit": "shot gradients/s", "n_gpus": 1,
                "higher_is_better": True, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOADS["invert"], "scale": args.scale},
                "gpu_launches": r["gpu_launches"], "cpu_baseline": cpu, "inversion": r}
        print(json.dumps(line))
        return 0
    if args.workload == "uneven":
        r = uneven_batch(nprob=args.nprob or 64)
        rg = uneven_gradient(nprob=args.nprob or 64)
        line = {"metric": "shots/s (uneven batch, one CUDA graph vs one plan per problem)",
                "value": r["batched"]["shots_per_s"], "unit": "shots/s", "n_gpus": 1,
                "higher_is_better": True, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOADS["uneven"]}, "uneven": r, "uneven_gradient": rg}
    else:
        r = serving_stream(nreq=args.nreq or 650)
        line = {"metric": "p99 latency (s) and shots/s, continuous admission vs plain",
                "value": r["continuous"]["p99_s"], "unit": "s", "n_gpus": 1,
                "higher_is_better": False, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOADS["serving"]}, "serving": r}
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in ("uneven", "serving", "invert"):
        return run_extra_workload(args)
    return run_mine(args)


if __name__ == "__main__":
    sys.exit(main())
