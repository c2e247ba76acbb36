#!/usr/bin/env python3
"""Benchmark of the surfel ray tracer's hot path on one or more B300s.

One step is one pass of the whole path over the one-bounce workload (a
200k-surfel room: background shell + 4 objects, 800x800, 16 spp, 256x512
environment): full LBVH build, environment sampling tables, a rigid object
edit (transform + BLAS refit + TLAS), primary trace, one-bounce shading and
the path-replay adjoint to all surfel attributes and environment texels.

Metric: Mrays/s of forward + backward (rays traced by the forward pass /
time of the whole step); the forward-only figure is reported beside it.
Inputs are synthetic (seeded); the scene (~17 MB of packed records and
nodes) fits in L2, so L2 is flushed between timed steps.

`--impl reference` times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (the reference arm of this comparison).
`--serve` runs the served-vs-plain latency sweep on the 1M-surfel scene and
`--multistate` the multi-state relighting workload (3 environments x 8
layouts assembled from one canonical scene); each prints its own JSON line.
Multi-GPU: every rank renders its own replica (no collective on the data
path), timing is the max over ranks, `value` counts the rays of all ranks.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mrays/s fwd+bwd (one-bounce surfel ray tracing)"
UNIT = "Mrays/s"
def workload(size=800, spp=16):
    return dict(workload=f"one-bounce room: 200k surfels (10k/face shell + 4x35k objects), {size}x{size}, {spp} spp, "
                         "256x512 sky+sun env, fwd+bwd, full LBVH build + rigid edit per step",
                surfels=200_000, width=size, height=size, spp=spp, env="256x512")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lightfuse", choices=["lightfuse", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    ap.add_argument("--size", type=int, default=800)
    ap.add_argument("--spp", type=int, default=16)
    ap.add_argument("--serve", action="store_true", help="served vs plain loop sweep only (C5-style)")
    ap.add_argument("--no-serving", action="store_true", help="skip the small served-vs-plain comparison")
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--rates", default="0.5,1,2")
    ap.add_argument("--serve-scene", default="c4", choices=["c2", "c4"])
    ap.add_argument("--multistate", action="store_true",
                    help="multi-state relighting on the 1M-surfel scene only (3 environments x layouts)")
    ap.add_argument("--ms-size", type=int, default=1024)
    ap.add_argument("--ms-spp", type=int, default=64)
    ap.add_argument("--ms-layouts", type=int, default=8)
    ap.add_argument("--no-multistate", action="store_true",
                    help="skip the bounded multi-state relighting object of the default line")
    ap.add_argument("--ms-default-layouts", type=int, default=2,
                    help="layouts of the bounded multi-state object (x 3 environments, 1024^2, 64 spp)")
    return ap.parse_args()


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------- workload
def make_workload(size, spp, seed):
    from synthetic import scenes as S
    sc = S.scene_c2(seed)
    cam = S.camera_c2(size, size)
    env = S.env_sky_sun(seed)
    return sc, cam, env


class Step:
    """Device buffers and the hot-path step on one GPU."""

    def __init__(self, sc, cam, env, spp, seed):
        import numpy as np
        import torch
        from paper_2608_29269_b300 import SceneTensors, Tracer
        from paper_2608_29269_b300._native import LF_GBUF_CHANNELS
        self.torch = torch
        self.cam, self.spp, self.seed = cam, spp, seed
        self.tr = Tracer()
        self.st = SceneTensors.from_numpy(sc)
        self.env = torch.as_tensor(env.rgb, device="cuda").contiguous()
        self.tr.build(self.st)
        self.tr.set_env(0, self.env)
        P = cam.width * cam.height
        self.gbuf = torch.empty((LF_GBUF_CHANNELS, cam.height, cam.width), device="cuda")
        self.rgb = torch.empty((cam.height, cam.width, 3), device="cuda")
        self.samples = self.tr.alloc_samples(cam, spp)
        self.scratch = torch.empty((9 * P * 4 + 256 + 3) // 4, device="cuda")
        self.d_surfel = torch.zeros((sc.n, 17), device="cuda")
        self.d_env = torch.zeros_like(self.env)
        self.rays = torch.zeros(1, dtype=torch.int64, device="cuda")
        g = torch.Generator(device="cpu").manual_seed(seed)
        self.dL = (torch.rand((cam.height, cam.width, 3), generator=g) - 0.5).to("cuda").contiguous()
        # rigid edit of object 1 (rotation about +y through its centre, shift); alternate with its inverse
        lo, hi = sc.object_offsets[1], sc.object_offsets[2]
        from synthetic.scenes import rigid_motion
        R, t = rigid_motion(np.random.default_rng(seed), sc.mu[lo:hi].mean(0))
        self.T = (R, t)
        self.Tinv = (R.T.copy(), (-(R.T @ t)).astype(np.float32))
        self.k = 0
        self.ev = None

    def run(self, events=None):
        """One step; `events` (dict name -> (start, end)) records phase times."""
        torch, tr, cam = self.torch, self.tr, self.cam
        rec = (lambda name, i: events[name][i].record()) if events is not None else (lambda name, i: None)
        rec("build", 0)
        tr.build(self.st)
        tr.set_env(0, self.env)
        R, t = self.T if self.k % 2 == 0 else self.Tinv
        tr.refit(1, R, t)
        self.k += 1
        rec("build", 1)
        rec("primary", 0)
        tr.trace_primary(cam, 0, out=self.gbuf)
        rec("primary", 1)
        rec("shade", 0)
        tr.shade(cam, self.gbuf, 0, self.spp, self.seed, out=self.rgb, ray_count=self.rays, samples=self.samples)
        rec("shade", 1)
        rec("backward", 0)
        self.d_surfel.zero_()
        self.d_env.zero_()
        tr.backward(cam, self.gbuf, 0, self.spp, self.seed, dL_drgb=self.dL, d_surfel=self.d_surfel,
                    d_env=self.d_env, scratch=self.scratch, fwd_samples=self.samples)
        rec("backward", 1)


KERNELS_PER_STEP = {  # launches of this library's kernels in one step
    # bounds init + reduce, morton, radix 5 x (hist, scan, scatter), hierarchy, fit (pack + wide boxes),
    # collapse, wide boxes
    "build": 2 + 1 + 5 * 3 + 1 + 2 + 1 + 1,
    "env": 2,
    "refit": 3,  # rigid transform, pack + fit, wide boxes
    "primary": 1,
    "shade": 7,  # gen, shadow A, continue, secondary sampling, shadow C, count, combine
    "backward": 2,  # combine adjoint, trace backward
}


def oracle_sample(sc, cam, env, spp, seed, target_s, include_grad=True):
    """Time the FP64 oracle on a bounded pixel sample (~target_s seconds)."""
    import numpy as np
    import oracle
    from synthetic.scenes import pixel_subset
    threads = os.cpu_count() or 1
    n = 8
    while True:
        pix = pixel_subset(cam.width, cam.height, n, seed=seed)
        t0 = time.perf_counter()
        out = oracle.render(sc, cam, env, pix, spp=spp, seed=seed, threads=threads)
        if include_grad:
            oracle.grad(sc, cam, env, pix, spp, seed, np.ones((len(pix), 3)), None, threads=threads)
        dt = time.perf_counter() - t0
        if dt >= 0.25 * target_s or n >= cam.width * cam.height:
            scale = target_s / max(dt, 1e-3)
            if scale > 1.5 and n < cam.width * cam.height:
                n = int(min(cam.width * cam.height, n * scale))
                continue
            return dict(rays=out["rays"], seconds=dt, pixels=len(pix), threads=threads)
        n *= 4


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    sc, cam, env = make_workload(args.size, args.spp, 0)
    import oracle
    oracle.build()
    per_step = max(1.0, 60.0 / max(1, args.steps + args.warmup))
    probe = oracle_sample(sc, cam, env, args.spp, 0, per_step)
    from synthetic.scenes import pixel_subset
    import numpy as np
    pix = pixel_subset(cam.width, cam.height, probe["pixels"], seed=0)
    times, rays = [], 0
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        out = oracle.render(sc, cam, env, pix, spp=args.spp, seed=k, threads=probe["threads"])
        oracle.grad(sc, cam, env, pix, args.spp, k, np.ones((len(pix), 3)), None, threads=probe["threads"])
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
            rays += out["rays"]
    total = sum(times)
    value = rays / total / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
            "config": dict(workload(args.size, args.spp), sample_pixels=len(pix)),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": probe["threads"], "kind": "oracle",
                             "sample": f"{len(pix)} seeded pixels of the {cam.width}x{cam.height} frame, "
                                       f"{args.spp} spp, fwd + gradient per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def serving_compare(sc, envs, n_req, rate, resolutions, spps, seed, budget=40 << 30, max_slots=8, n_streams=4):
    """Served loop vs the plain per-request rebuild-and-render loop on the same
    request stream: p50 / p99 edit-to-frame latency (ms) and Mrays/s."""
    import numpy as np
    import torch
    from paper_2608_29269_b300 import SceneTensors, Tracer
    from paper_2608_29269_b300.serve import Server, run_plain, run_served
    from synthetic.requests import request_stream
    reqs = request_stream(n_req, rate, sc, n_envs=len(envs), resolutions=resolutions, spps=spps, seed=seed)
    out = {}
    tr = Tracer()
    st = SceneTensors.from_numpy(sc)
    tr.build(st)
    env_t = [torch.as_tensor(e.rgb, device="cuda").contiguous() for e in envs]
    for i, e in enumerate(env_t):
        tr.set_env(i, e)
    srv = Server(tr, budget_bytes=budget, max_slots=max_slots, n_streams=n_streams)
    # untimed warm-up of both loops (lazy module loading, memory pools, pinned frames)
    warm = [dataclasses.replace(r, arrival=0.0) for r in reqs[:4]]
    run_served(srv, warm)
    t0 = time.perf_counter()
    served = run_served(srv, reqs)
    wall = time.perf_counter() - t0
    srv.close()
    lat = np.array([r["latency"] for r in served if r["status"] == 0]) * 1e3
    # rays per request: shading rays of its launch group are shared; estimate from the plain loop's counts below
    ok = [r for r in served if r["status"] == 0]
    phases = {name: [1e3 * (r[b] - r[a]) for r in ok] for name, a, b in
              [("queue", "t_submit", "t_admit"), ("admit", "t_admit", "t_start"), ("gpu", "t_start", "t_done")]}
    out["served"] = {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                     "completed": int(len(lat)), "failed": int(len(served) - len(lat)), "wall_s": wall,
                     "mean_ms": {k: float(np.mean(v)) for k, v in phases.items()},
                     "max_ms": {k: float(np.max(v)) for k, v in phases.items()}}
    rays = torch.zeros(1, dtype=torch.int64, device="cuda")
    run_plain(tr, warm)  # after the server is closed: the plain loop edits the context's own scene
    t0 = time.perf_counter()
    plain = run_plain_counted(tr, reqs, rays)
    wall_p = time.perf_counter() - t0
    latp = np.array([r["latency"] for r in plain]) * 1e3
    total_rays = float(rays.item()) + sum(r.cam.width * r.cam.height for r in reqs)
    out["plain"] = {"p50_ms": float(np.percentile(latp, 50)), "p99_ms": float(np.percentile(latp, 99)),
                    "completed": int(len(latp)), "wall_s": wall_p, "mrays_s": total_rays / wall_p / 1e6}
    out["served"]["mrays_s"] = total_rays / wall / 1e6
    out["requests"] = n_req
    out["rate_per_s"] = rate
    tr.close()
    return out


def run_plain_counted(tracer, requests, rays):
    """The plain loop (edit, full rebuild, render, frame to host, sync) counting shading rays."""
    env_state = dict(env=0)
    from paper_2608_29269_b300.serve import apply_edit
    t0 = time.perf_counter()
    out = []
    for rq in requests:
        arrival = t0 + rq.arrival
        now = time.perf_counter()
        if now < arrival:
            time.sleep(arrival - now)
        apply_edit(tracer, rq.edit, env_state)
        tracer.build(tracer.scene)
        g = tracer.trace_primary(rq.cam, env_state["env"])
        rgb = tracer.shade(rq.cam, g, env_state["env"], rq.spp, rq.seed, ray_count=rays)
        rgb.cpu()
        tracer.sync()
        out.append(dict(latency=time.perf_counter() - arrival))
    return out


def run_serve_sweep(args):
    from synthetic import scenes as S
    sc = S.scene_c4(0) if args.serve_scene == "c4" else S.scene_c2(0)
    envs = [S.env_sky_sun(i) for i in range(3)]
    res = {}
    for rate in [float(x) for x in args.rates.split(",")]:
        res[str(rate)] = serving_compare(sc, envs, args.requests, rate, (256, 512, 800, 1024), (4, 8, 16, 32), seed=5)
    line = {"metric": "p50/p99 edit-to-frame ms, served vs plain loop", "unit": "ms", "higher_is_better": False,
            "scene": f"{args.serve_scene}: {sc.n} surfels, {sc.n_objects} objects", "budget_gb": 40,
            "requests_per_rate": args.requests, "rates": res, "data": "synthetic (seeded)"}
    print(json.dumps(line))


def run_multistate(args):
    line = multistate(args.ms_size, args.ms_spp, args.ms_layouts)
    print(json.dumps(line))


def multistate(size, spp, n_layouts, stage_prefix="multi-state"):
    """Multi-state relighting (cross-state supervision, Sec. 3.2): the 1M-surfel
    scene (shell + 12 objects) as one canonical scene, 3 environment states x
    `n_layouts` layouts, each layout moving 1-4 random objects (rotation
    about +y through the object's centre, x/z shift U[-0.5, 0.5]).  Per
    (environment, layout): the state is assembled from the canonical scene
    (Eq. 2, every BLAS refit), traced at size^2, shaded at spp,
    differentiated, and its surfel gradient carried back to the canonical
    parameters.  One warm-up state, then every state timed with CUDA events.
    Returns the JSON object of the measurement."""
    import numpy as np
    import torch
    from synthetic import scenes as S
    from paper_2608_29269_b300 import SceneTensors, Tracer
    stage(f"{stage_prefix} workload")
    sc = S.scene_c4(0)
    cam = S.camera_c4(size, size)
    envs = [S.env_sky_sun(i) for i in range(3)]
    tr = Tracer()
    can = SceneTensors.from_numpy(sc)
    world = SceneTensors.from_numpy(sc)
    for k in ["scale", "opacity", "albedo", "metallic", "roughness"]:  # shared with the canonical scene
        setattr(world, k, getattr(can, k))
    tr.build(world)
    env_t = [torch.as_tensor(e.rgb, device="cuda").contiguous() for e in envs]
    for i, e in enumerate(env_t):
        tr.set_env(i, e)
    rng = np.random.default_rng(7)
    M = sc.n_objects - 1
    layouts = []
    for _ in range(n_layouts):
        R = np.stack([np.eye(3, dtype=np.float32)] * M)
        t = np.zeros((M, 3), np.float32)
        for o in rng.choice(np.arange(1, M + 1), size=int(rng.integers(1, 5)), replace=False):
            lo, hi = sc.object_offsets[o], sc.object_offsets[o + 1]
            R[o - 1], t[o - 1] = S.rigid_motion(rng, sc.mu[lo:hi].mean(0), max_shift=0.5)
        layouts.append((R, t))
    P = cam.width * cam.height
    from paper_2608_29269_b300._native import LF_GBUF_CHANNELS
    gbuf = torch.empty((LF_GBUF_CHANNELS, cam.height, cam.width), device="cuda")
    rgb = torch.empty((cam.height, cam.width, 3), device="cuda")
    samples = tr.alloc_samples(cam, spp)
    scratch = torch.empty((9 * P * 4 + 256 + 3) // 4, device="cuda")
    d_world = torch.zeros((sc.n, 17), device="cuda")
    d_can = torch.zeros((sc.n, 17), device="cuda")
    d_env = [torch.zeros_like(e) for e in env_t]
    g = torch.Generator(device="cpu").manual_seed(3)
    dL = ((torch.rand((cam.height, cam.width, 3), generator=g) > 0.5).float() * 2 - 1).div_(3 * P).to("cuda")
    rays = torch.zeros(1, dtype=torch.int64, device="cuda")
    names = ["assemble", "primary", "shade", "backward", "pullback"]
    states = [(e, l) for e in range(len(envs)) for l in range(len(layouts))]

    def run_state(e, l, ev):
        R, t = layouts[l]
        rec = (lambda n, i: ev[n][i].record()) if ev else (lambda n, i: None)
        seed = 100 + 17 * e + l
        rec("assemble", 0); tr.assemble_state(can, R, t); rec("assemble", 1)
        rec("primary", 0); tr.trace_primary(cam, e, out=gbuf); rec("primary", 1)
        rec("shade", 0)
        tr.shade(cam, gbuf, e, spp, seed, out=rgb, ray_count=rays if ev else None, samples=samples)
        rec("shade", 1)
        rec("backward", 0)
        d_world.zero_()
        tr.backward(cam, gbuf, e, spp, seed, dL_drgb=dL, d_surfel=d_world, d_env=d_env[e], scratch=scratch,
                    fwd_samples=samples)
        rec("backward", 1)
        rec("pullback", 0); tr.state_pullback(R, d_world, d_can); rec("pullback", 1)

    stage(f"{stage_prefix} warm-up")
    run_state(0, 0, None)
    tr.sync()
    stage(f"{stage_prefix} timed")
    evs = []
    for e, l in states:
        ev = {n: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for n in names}
        run_state(e, l, ev)
        evs.append(ev)
    tr.sync()
    per_state = [ev["assemble"][0].elapsed_time(ev["pullback"][1]) for ev in evs]
    phase = {n: statistics.mean(ev[n][0].elapsed_time(ev[n][1]) for ev in evs) for n in names}
    total_rays = int(rays.item()) + len(states) * P
    total_ms = sum(per_state)
    line = {"metric": "Mrays/s fwd+bwd, multi-state relighting (canonical scene, per-state assembly)",
            "value": total_rays / (total_ms * 1e-3) / 1e6, "unit": "Mrays/s", "higher_is_better": True,
            "states": len(states), "ms_per_state": total_ms / len(states),
            "state_ms": {"median": statistics.median(per_state), "min": min(per_state), "max": max(per_state)},
            "rays_per_state": total_rays / len(states), "phase_ms": {n: round(v, 3) for n, v in phase.items()},
            "dtype": "f32", "data": "synthetic (seeded)",
            "config": {"workload": f"multi-state relighting: {sc.n} surfels (shell 6x40k + {M} objects), "
                                   f"{cam.width}x{cam.height}, {spp} spp, 3 env states x {len(layouts)} layouts "
                                   "(1-4 objects moved each), fwd+bwd + pullback to the canonical scene",
                       "surfels": sc.n, "width": cam.width, "height": cam.height, "spp": spp,
                       "states": len(states)},
            "canonical_grad_abs_sum": float(d_can.abs().sum().item())}
    tr.close()
    return line


def stage(msg):
    """Progress of the run on stderr (the JSON line alone goes to stdout)."""
    print(f"[bench {time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


def main():
    args = parse()
    if args.serve:
        run_serve_sweep(args)
        return
    if args.multistate:
        run_multistate(args)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2608_29269_b300.build import build
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0:
        build()
    if world > 1:
        dist.barrier()
    stage("workload")
    sc, cam, env = make_workload(args.size, args.spp, 0)
    step = Step(sc, cam, env, args.spp, seed=1234 + rank)
    names = ["build", "primary", "shade", "backward"]

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    stage("warm-up")
    for _ in range(args.warmup):
        step.run()
    step.tr.sync()
    stage("counted run")

    # counted run (outside the timed region): traversal counters per kernel slot
    cnt20 = torch.zeros(20, dtype=torch.int64, device="cuda")
    step.tr.set_counters(cnt20)
    step.run()
    step.tr.sync()
    step.tr.set_counters(None)
    c = [int(v) for v in cnt20.tolist()]
    counters = {name: c[4 * k:4 * k + 4] for k, name in
                enumerate(["primary", "nee_shadow", "continuation", "secondary_shadow", "trace_backward"])}

    stage("timed steps")
    flush = torch.empty(int(256e6) // 4, dtype=torch.float32, device="cuda")
    step.rays.zero_()
    clocks = ClockSampler(local)
    per_step_ms, phase_ms = [], {n: [] for n in names}
    kern_names = ["primary", "gen", "nee_shadow", "continuation", "secondary_shadow", "combine", "shade_adjoint",
                  "trace_backward"]
    kern_ms = {n: [] for n in kern_names}
    step.tr.profile(True)  # CUDA events around the library's kernels, on its stream
    barrier()
    clocks.start()
    for k in range(args.steps):
        flush.fill_(float(k))  # evict the scene from L2 between steps
        events = {n: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for n in names}
        barrier()
        step.run(events)
        torch.cuda.synchronize()
        for n in names:
            phase_ms[n].append(events[n][0].elapsed_time(events[n][1]))
        per_step_ms.append(events["build"][0].elapsed_time(events["backward"][1]))
        for n, v in zip(kern_names, step.tr.profile_read()):
            kern_ms[n].append(v)
    barrier()
    clk = clocks.stop()
    step.tr.profile(False)
    step.tr.sync()
    total_ms = sum(per_step_ms)
    shade_rays = int(step.rays.item())
    rays = shade_rays + args.steps * cam.width * cam.height
    fwd_ms = sum(phase_ms["primary"]) + sum(phase_ms["shade"])
    total_ms, fwd_ms, rays_all = reduce_over_ranks(total_ms, fwd_ms, rays, "cuda")
    value = rays_all / (total_ms * 1e-3) / 1e6
    fwd_value = rays_all / (fwd_ms * 1e-3) / 1e6

    # ---------------------------------------------------------------- e2e through the public API
    stage("end to end")
    e2e = e2e_run(step, sc, env, args, world)

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return
    # ---------------------------------------------------------------- roofline of the dominant kernel
    hbm, peak_kind = read_peaks()
    avg = {n: statistics.mean(v) for n, v in phase_ms.items()}
    kavg = {n: statistics.mean(v) for n, v in kern_ms.items()}
    # Algorithmic bytes per launch with the unit costs of the hot-path scope
    # (per ray: 64 B per node visit, 48 B per surfel test, 32 B per composited
    # hit, plus the ray's own inputs and outputs; the adjoint adds 17 x 4 B of
    # gradient atomics per hit it scatters).  Per-ray I/O: primary 88 B of
    # G-buffer output (22 floats); NEE shadow 44 B (queue
    # entry, origin from the G-buffer, direction, visibility), continuation
    # 112 B (queue entry, origin, direction, secondary record, two NEE
    # samples), secondary shadow 32 B, adjoint 136 B per pixel (25 G-buffer and
    # 9 shading-gradient floats).  The wide-node layout actually reads all 32
    # child slots of a node (lf_bvh_wide_node_bytes per visit) and 80 B per
    # composited hit, and a primary ray writes all 32 G-buffer planes (the
    # residuals included); that accounting is kept beside it.
    unit = {"node": 64, "test": 48, "hit": 32, "grad_atomics": 68}
    per_ray_io = {"primary": 88, "nee_shadow": 44, "continuation": 112, "secondary_shadow": 32,
                  "trace_backward": 136}
    hit_cost = {n: unit["hit"] + (unit["grad_atomics"] if n == "trace_backward" else 0) for n in per_ray_io}
    kbytes = {n: unit["node"] * counters[n][0] + unit["test"] * counters[n][1] + hit_cost[n] * counters[n][2] +
              per_ray_io[n] * counters[n][3] for n in per_ray_io}
    wnode = step.tr.lib.lf_bvh_wide_node_bytes()
    wide_io = dict(per_ray_io, primary=4 * 32)
    wide_hit = {n: (196 if n == "trace_backward" else 80) for n in per_ray_io}
    kbytes_wide = {n: wnode * counters[n][0] + 48 * counters[n][1] + wide_hit[n] * counters[n][2] +
                   wide_io[n] * counters[n][3] for n in per_ray_io}
    kernels = {n: {"ms": round(kavg[n], 3), "algorithmic_bytes": kbytes.get(n),
                   "achieved_gbs": (kbytes[n] / (kavg[n] * 1e-3) / 1e9) if n in kbytes else None,
                   "wide_node_bytes": kbytes_wide.get(n)}
               for n in kern_names}
    dom = max(per_ray_io, key=lambda n: kavg[n])
    achieved = kbytes[dom] / (kavg[dom] * 1e-3) / 1e9
    traffic = read_traffic(KERNEL_NAMES[dom])
    # the working set sits in L2: L2 bytes of the same kernel (ncu) against the L2 read bandwidth measured here
    l2_peak = step.tr.measure_l2_read()
    l2_bytes = read_traffic(KERNEL_NAMES[dom], "l2_bytes_per_launch")
    l2 = {"peak": l2_peak, "unit": "GB/s", "peak_kind": "measured in this run (ld.global.cg read loop over 32 MB)",
          "bytes_per_launch": l2_bytes, "bytes_kind": "ncu lts__t_sectors x 32 B of the same kernel",
          "achieved": l2_bytes / (kavg[dom] * 1e-3) / 1e9 if l2_bytes else None,
          "frac": l2_bytes / (kavg[dom] * 1e-3) / 1e9 / l2_peak if l2_bytes else None,
          "algorithmic_frac": achieved / l2_peak}
    # the trace kernels are bound by instruction issue: warp instructions of
    # the same kernel (ncu smsp__inst_executed, scaled per ray) against the
    # issue rate of the SMs, one warp instruction per cycle per scheduler
    # (148 SMs x 4 schedulers) at the SM clock sampled under load
    insts = read_traffic(KERNEL_NAMES[dom], "warp_inst_per_launch")
    sm_mhz = (clk or {}).get("sm_mhz") or 2032.0
    issue_peak = 148 * 4 * sm_mhz * 1e6
    issue = {"peak": issue_peak, "unit": "warp instructions/s",
             "peak_kind": f"148 SMs x 4 schedulers x 1 warp instruction/cycle at {sm_mhz:.0f} MHz",
             "inst_per_launch": insts, "inst_kind": "ncu smsp__inst_executed.sum of the same kernel, scaled per ray",
             "achieved": insts / (kavg[dom] * 1e-3) if insts else None,
             "frac": insts / (kavg[dom] * 1e-3) / issue_peak if insts else None}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded)",
        "config": dict(workload(args.size, args.spp), parallelism=f"replicas x{world}",
                       l2="flushed between steps (256 MB write)"),
        "fwd_mrays_s": fwd_value,
        "step_ms": {"median": statistics.median(per_step_ms), "min": min(per_step_ms), "max": max(per_step_ms)},
        "rays_per_step": rays_all / args.steps / world,
        "phase_ms": {n: round(v, 3) for n, v in avg.items()},
        "roofline": {"bound": "l2", "kernel": KERNEL_NAMES[dom], "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "peak_kind": f"{peak_kind} HBM copy (burst)", "traffic": traffic,
                     "traffic_kind": "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch",
                     "algorithmic_bytes_per_launch": kbytes[dom], "unit_costs": dict(unit, io_per_ray=per_ray_io),
                     "launch_ms": kavg[dom], "l2": l2, "issue": issue,
                     "wide_node_accounting": {"bytes_per_launch": kbytes_wide[dom], "node_bytes": wnode,
                                              "achieved": kbytes_wide[dom] / (kavg[dom] * 1e-3) / 1e9}},
        "kernels": kernels,
        "counters": dict(counters, fields=["node visits", "surfel tests", "composited hits", "rays"]),
        "clocks": clk,
        "e2e": e2e,
        "gpu_launches": args.steps * sum(KERNELS_PER_STEP.values()),
    }
    if not args.no_multistate:
        try:
            line["multistate"] = multistate(1024, 64, args.ms_default_layouts, stage_prefix="multi-state (bounded)")
        except Exception as exc:
            line["multistate"] = {"error": str(exc)}
    if not args.no_serving:
        stage("serving comparison")
        try:
            from synthetic import scenes as S
            line["serving"] = dict(serving_compare(sc, [env, S.env_sky_sun(1), S.env_sky_sun(2)], 24, 4.0,
                                                   (256, 512), (4, 8), seed=11),
                                   scene="200k-surfel room", resolutions=[256, 512], spp=[4, 8])
        except Exception as exc:
            line["serving"] = {"error": str(exc)}
    if not args.no_cpu_baseline:
        stage("cpu baseline")
        try:
            import oracle
            oracle.build()
            cb = oracle_sample(sc, cam, env, args.spp, 0, args.cpu_seconds)
            line["cpu_baseline"] = {"value": cb["rays"] / cb["seconds"] / 1e6, "unit": UNIT, "cores": cb["threads"],
                                    "kind": "oracle",
                                    "sample": f"{cb['pixels']} seeded pixels of the frame, {args.spp} spp, "
                                              f"forward + gradient, {cb['seconds']:.1f} s"}
        except Exception as exc:  # the bench line must still print
            line["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                    "sample": f"failed: {exc}"}
    print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def reduce_over_ranks(total_ms, fwd_ms, rays, device):
    """Replicas: the job's time is the slowest rank's, its rays the sum of all ranks'."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([total_ms, fwd_ms], dtype=torch.float64, device=device)
    r = torch.tensor([float(rays)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(r, op=dist.ReduceOp.SUM)
    return float(t[0]), float(t[1]), float(r[0])


KERNEL_NAMES = {"primary": "k_trace_primary", "nee_shadow": "k_wf_shadow (NEE)",
                "continuation": "k_wf_continue", "secondary_shadow": "k_wf_shadow (secondary)",
                "trace_backward": "k_trace_backward"}


def read_traffic(kernel, field="dram_bytes_per_launch"):
    """DRAM (or L2) bytes per launch of `kernel` at the bench workload, from the
    committed ncu summary, when it was taken on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
        if t.get("sources_sha") != sources_sha():
            return None
        return t.get(field, {}).get(kernel)
    except Exception:
        return None


def sources_sha():
    """Hash of the kernel sources with comments and blank lines removed, so
    a committed ncu summary stays attached to the code it measured."""
    import hashlib
    import re
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2608_29269_b300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(csrc, name)) as f:
                text = re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)
            lines = [re.sub(r"//.*$", "", line).rstrip() for line in text.splitlines()]
            h.update("\n".join(line for line in lines if line).encode())
    return h.hexdigest()[:16]


def e2e_run(step, sc, env, args, world):
    """Same step through the public API with host inputs: every step copies
    its scene, environment and upstream gradient from pinned host memory to
    the device and its image and gradients back, inside the timed region.
    The copies run on a side stream over two buffer sets (two contexts), so
    step k+1's inputs go up and step k's outputs come down while the other
    set computes, as a stream of renders would."""
    import torch
    names = ["mu", "tu", "tv", "scale", "opacity", "albedo", "metallic", "roughness"]
    host = {k: torch.as_tensor(getattr(sc, k)).pin_memory() for k in names}
    h_env = torch.as_tensor(env.rgb).pin_memory()
    h_dL = step.dL.cpu().pin_memory()
    out_rgb = torch.empty(step.rgb.shape, dtype=torch.float32).pin_memory()
    out_ds = torch.empty(step.d_surfel.shape, dtype=torch.float32).pin_memory()
    out_de = torch.empty(step.d_env.shape, dtype=torch.float32).pin_memory()
    h2d = sum(t.numel() * 4 for t in host.values()) + h_env.numel() * 4 + h_dL.numel() * 4
    d2h = (out_rgb.numel() + out_ds.numel() + out_de.numel()) * 4
    other = Step(sc, step.cam, env, step.spp, step.seed)
    sets = [step, other]
    n = max(2, args.steps)
    copy = torch.cuda.Stream()
    compute = torch.cuda.current_stream()
    up = [torch.cuda.Event() for _ in range(n)]
    done = [torch.cuda.Event() for _ in range(n)]

    def upload(k):
        st = sets[k % 2]
        with torch.cuda.stream(copy):
            for name, t in host.items():
                getattr(st.st, name).copy_(t, non_blocking=True)
            st.env.copy_(h_env, non_blocking=True)
            st.dL.copy_(h_dL, non_blocking=True)
            up[k].record(copy)

    for st in sets:
        st.rays.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    upload(0)
    upload(1)
    for k in range(n):
        st = sets[k % 2]
        compute.wait_event(up[k])
        st.run()
        done[k].record(compute)
        with torch.cuda.stream(copy):
            copy.wait_event(done[k])
            out_rgb.copy_(st.rgb, non_blocking=True)
            out_ds.copy_(st.d_surfel, non_blocking=True)
            out_de.copy_(st.d_env, non_blocking=True)
        if k + 2 < n:
            upload(k + 2)  # after this set's outputs, in copy-stream order
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    rays = sum(int(st.rays.item()) for st in sets) + n * step.cam.width * step.cam.height
    other.tr.close()
    return {"value": rays / dt / 1e6 * world, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "steps": n, "copies": "side stream, two buffer sets: step k+1 uploads and step k downloads overlap compute"}


if __name__ == "__main__":
    main()
