"""Benchmark: AO ray-tracing throughput (Mrays/s, fps) of the paper-sized scene.

Default workload: the 26,318-object globule (13,500 spheres + 12,818 bonds)
at 965x1137 with 16 AO samples per pixel, FP32 path (FP64 primary ray, hit
refined in its object's frame). A step renders one whole frame. Rays = primary rays (one per
pixel) + AO rays actually cast (samples x pixels whose primary ray hits).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload paper_1mp|paper_17mp|small|orbit64|serve] [--precision fp32|fp64]

Under torchrun (N > 1) every rank renders its own frames (frames are
independent; no collective on the data path): value = all ranks' rays / the
slowest rank's time, "scaling": "weak".

``--impl reference`` times the FP64 CPU oracle (the only other place this
script runs it) on a bounded row sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_0801_1500_gb300 import scenes as S  # noqa: E402

# Algorithmic flops of one step of each kind, the roofline's fixed convention
# (an FMA counts 2, a square root or reciprocal 1): grid-walk step 8,
# ray-sphere test 20 (the sphere's own formula), ray-cylinder test 50.
FLOPS_CELL, FLOPS_SPHERE, FLOPS_CYLINDER = 8, 20, 50
# The same counts taken from the device code's one branch-free test, which
# runs the cylinder formula for spheres too (reported beside the roofline).
FLOPS_SPHERE_DEVICE, FLOPS_CYLINDER_DEVICE = 24, 58
# bytes a walk reads per step: a cell record (8 B), an item id (4 B), a sphere
# record (16 B) or a cylinder record (32 B)
BYTES_CELL, BYTES_ITEM, BYTES_SPHERE, BYTES_CYLINDER = 8, 4, 16, 32
L2_FLUSH_BYTES = 512 << 20   # > 126 MB L2
PROFILE_EVERY = 10           # timed steps per step with per-kernel events


def workload(name, precision):
    prec = S.PRECISION_FP64 if precision == "fp64" else S.PRECISION_FP32
    if name == "paper_1mp":
        return S.paper_1mp(precision=prec)
    if name == "paper_17mp":
        return S.paper_17mp(precision=prec)
    if name == "small":
        w = S.small_fp64()
        w.params.precision = prec
        return w
    raise SystemExit(f"unknown workload {name}")


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


KERNEL_SOURCES = ("gbrt_device.cuh", "gbrt_types.h", "render.cu")


def _code_only(text):
    """C++ source without its comments and blank space (comment edits do not
    change a kernel)."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def sources_hash():
    """Hash of the code (comments stripped) of the sources that define the
    render kernels."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_0801_1500_gb300", "csrc")
    for f in KERNEL_SOURCES:
        h.update(_code_only(open(os.path.join(d, f)).read()).encode())
    return h.hexdigest()[:16]


def committed_profile(workload_name, precision):
    """Figures of the AO walk kernel from the committed ncu summary, if it was
    taken on the current kernel sources (else {})."""
    p = os.path.join(ROOT, "profiles", f"k_ao_walk_{precision}_{workload_name}.txt")
    if not os.path.exists(p):
        return {}
    kv = {}
    for line in open(p):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("sources_hash") != sources_hash():
        return {}
    out = {}
    for key in ("dram_bytes_per_launch", "issue_active_pct", "warp_instructions_per_launch", "grid_lambda",
                "refill", "block"):
        try:
            out[key] = float(kv[key])
        except (KeyError, ValueError):
            pass
    return out


def committed_traffic(workload_name, precision):
    """DRAM bytes per launch of the AO walk kernel from the committed ncu
    summary, if it was taken on the current kernel sources (else None)."""
    return committed_profile(workload_name, precision).get("dram_bytes_per_launch")


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p)), "measured"
        except ValueError:
            pass
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        # nvidia-smi names the GPU by its UUID: its own indices need not match
        # CUDA's when CUDA_VISIBLE_DEVICES remaps devices
        self.index = str(index)
        try:
            import torch
            u = str(torch.cuda.get_device_properties(index).uuid)
            self.index = u if u.startswith("GPU-") else "GPU-" + u
        except Exception:
            pass
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.index, f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # the timed region starts once the sampler is running
            t_end = time.time() + 3.0
            while not self.lines and time.time() < t_end and self.proc.poll() is None:
                time.sleep(0.01)
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_sample(w, lam, budget_s=15.0, threads=0):
    """Time the oracle on evenly spaced rows of the frame (about budget_s of CPU work)."""
    import oracle
    W, H = w.width, w.height
    stride = max(1, H // 8)
    rows = np.arange(stride // 2, H, stride)
    pix = (rows[:, None] * W + np.arange(W)[None, :]).ravel()
    t0 = time.perf_counter()
    out = oracle.render(w.scene, w.camera, W, H, w.lights, w.params, pixels=pix, mode="grid", lam=lam,
                        threads=threads)
    el = time.perf_counter() - t0
    if el < budget_s / 4 and stride > 1:
        # grow the sample toward the budget
        stride = max(1, int(stride * el / budget_s * 4))
        rows = np.arange(stride // 2, H, stride)
        pix = (rows[:, None] * W + np.arange(W)[None, :]).ravel()
        t0 = time.perf_counter()
        out = oracle.render(w.scene, w.camera, W, H, w.lights, w.params, pixels=pix, mode="grid", lam=lam,
                            threads=threads)
        el = time.perf_counter() - t0
    c = out["counters"]
    rays = c["primary_rays"] + c["ao_rays"]
    return dict(rays=rays, seconds=el, rows=len(rows), pixels=len(pix), counters=c,
                cores=oracle.max_threads() if threads <= 0 else threads)


def per_ray_work(c, kind="ao", device_formulas=False):
    """Algorithmic flops and walk bytes per ray (of one kind: "ao" or
    "primary") from the oracle's grid-walk counters."""
    rays = max(1, c[f"{kind}_rays"])
    cells = c[f"{kind}_cells"]
    sph = c[f"{kind}_sphere_tests"]
    cyl = c[f"{kind}_cylinder_tests"]
    fs, fc = (FLOPS_SPHERE_DEVICE, FLOPS_CYLINDER_DEVICE) if device_formulas else (FLOPS_SPHERE, FLOPS_CYLINDER)
    flops = (cells * FLOPS_CELL + sph * fs + cyl * fc) / rays
    nbytes = (cells * BYTES_CELL + (sph + cyl) * BYTES_ITEM + sph * BYTES_SPHERE + cyl * BYTES_CYLINDER) / rays
    return flops, nbytes


def run_reference(args, w):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    lam = args.lam
    times, rays = [], 0
    # each step a bounded row sample: the whole run stays within a few minutes
    budget = min(args.ref_budget, 150.0 / (args.warmup + args.steps))
    for k in range(args.warmup + args.steps):
        s = oracle_sample(w, lam, budget_s=budget)
        if k >= args.warmup:
            times.append(s["seconds"])
            rays += s["rays"]
    total = sum(times)
    v = rays / total / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "Mrays/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * total / max(1, len(times)), 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "sample": f"{s['rows']} evenly spaced rows of {w.height}"},
            "cpu_baseline": {"value": round(v, 4), "unit": "Mrays/s", "cores": s["cores"], "kind": "oracle",
                             "sample": f"{s['rows']} rows x {w.width} px per step"},
            "e2e": {"value": round(v, 4), "unit": "Mrays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


METRIC = "AO Mrays/s & fps at 1.1/17.6 MP, FP32 vs FP64 on GPU; serving p50/p99 latency"


def orbit_items(G, torch, dev, scene_h, grid_h, sc, lights, precision, n_frames=64):
    """The 64-frame orbit: render items plus their rays (primary + AO of hit pixels)."""
    frames = S.orbit_frames(sc, n_frames)
    items, outs = [], []
    for f in frames:
        p = S.Params(ao_samples=f["spp"], seed=f["seed"], frame=f["frame"], precision=precision)
        dt = torch.float64 if precision == S.PRECISION_FP64 else torch.float32
        o = (torch.empty((f["height"], f["width"], 3), dtype=dt, device=dev),
             torch.empty((f["height"], f["width"]), dtype=torch.int32, device=dev))
        outs.append(o)
        items.append(G.make_item(scene_h, grid_h, f["camera"], f["width"], f["height"], f["spp"], lights, p, *o))
    return frames, items, outs


def time_steps(torch, stream, flush, step, steps, warmup, after=None, before=None, every=1):
    """Per-step device times (ms): L2 flush outside the events. On every
    `every`-th step, `before(True)` runs before it and `after()` after it
    (their results are returned); `before(False)` before the others."""
    for _ in range(warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    extra = []
    for k in range(steps):
        picked = k % every == 0
        if before is not None:
            before(picked)
        flush.zero_()
        starts[k].record(stream)
        step()
        ends[k].record(stream)
        if after is not None and picked:
            extra.append(after())
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in zip(starts, ends)], extra


def animation_extra(G, torch, r, w, lam, stream, flush, dev, n_frames=16):
    """Molecular-dynamics animation of the paper scene at 965x1137, 16 spp:
    gbrt_scene_update (page-locked host arrays) + gbrt_grid_rebuild + render
    per frame, camera fixed while the molecule turns and vibrates."""
    W, H, spp = w.width, w.height, w.params.ao_samples
    traj = S.MDTrajectory(w.scene, amplitude=0.3, seed=0)
    frames = [traj.frame(k) for k in range(1, n_frames + 1)]
    pinned = [(torch.from_numpy(f.spheres).pin_memory().numpy(), torch.from_numpy(f.cylinders).pin_memory().numpy())
              for f in frames]
    scene, grid = r.upload(w.scene, lam=lam)
    G.gbrt_grid_rebuild(r.ctx, grid, scene)   # the first rebuild allocates its buffers
    G.gbrt_sync(r.ctx)
    cam, li, pa = G.make_camera(w.camera), G.make_lights(w.lights), G.make_params(w.params)
    out = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
    ids = torch.empty((H, W), dtype=torch.int32, device=dev)
    rays = 0
    for sp, cy in pinned:
        G.gbrt_scene_update(r.ctx, scene, sp, cy, G.HOST_PTRS)
        G.gbrt_grid_rebuild(r.ctx, grid, scene)
        G.gbrt_render(r.ctx, scene, grid, cam, W, H, spp, li, pa, out, ids)
        G.gbrt_sync(r.ctx)
        rays += W * H + spp * int((ids.cpu().numpy().view(np.uint32) != G.MISS).sum())

    def whole():
        for sp, cy in pinned:
            G.gbrt_scene_update(r.ctx, scene, sp, cy, G.HOST_PTRS)
            G.gbrt_grid_rebuild(r.ctx, grid, scene)
            G.gbrt_render(r.ctx, scene, grid, cam, W, H, spp, li, pa, out)

    def rebuild_only():
        for sp, cy in pinned:
            G.gbrt_scene_update(r.ctx, scene, sp, cy, G.HOST_PTRS)
            G.gbrt_grid_rebuild(r.ctx, grid, scene)

    ms_all, _ = time_steps(torch, stream, flush, whole, 3, 1)
    ms_reb, _ = time_steps(torch, stream, flush, rebuild_only, 3, 1)
    G.gbrt_sync(r.ctx)
    r.free(scene, grid)
    per = sum(ms_all) / len(ms_all) / n_frames
    reb = sum(ms_reb) / len(ms_reb) / n_frames
    return {"frames": n_frames, "ms_per_frame": round(per, 4), "fps": round(1e3 / per, 2),
            "Mrays_s": round(rays / n_frames / per / 1e3, 2), "update_rebuild_ms_per_frame": round(reb, 4),
            "h2d_bytes_per_frame": int(pinned[0][0].nbytes + pinned[0][1].nbytes), "dtype": "f32"}


def replay(srv, SV, reqs_spec, scenes, precision):
    """Submit a trace in real time (arrival offsets in seconds); wait for all."""
    import torch
    reqs, futs = [], []
    t0 = time.perf_counter()
    for spec in reqs_spec:
        delay = spec["arrival_s"] - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        sc = scenes[spec["scene"]]
        cam = S.ortho_camera(sc, spec["width"], spec["height"], angle_deg=spec.get("angle_deg", 0.0))
        rq = SV.Request(scene=spec["scene"], camera=cam, width=spec["width"], height=spec["height"],
                        spp=spec["spp"], precision=precision, seed=spec["id"], want_ids=True)
        reqs.append(rq)
        futs.append(srv.submit(rq))
    done = []
    rays = 0
    for rq, f in zip(reqs, futs):
        try:
            rgb, ids = f.result(timeout=3600)
        except SV.RejectedError:
            continue
        hits = int((ids != -1).sum().item())
        rays += rq.width * rq.height + hits * rq.spp
        done.append(rq)
    t1 = time.perf_counter()
    lat = np.array([r.t_done - r.t_submit for r in done]) if done else np.zeros(1)
    return {"requests": len(reqs_spec), "completed": len(done), "rejected": len(reqs_spec) - len(done),
            "p50_ms": round(float(np.percentile(lat, 50)) * 1e3, 2),
            "p99_ms": round(float(np.percentile(lat, 99)) * 1e3, 2),
            "max_ms": round(float(lat.max()) * 1e3, 2), "wall_s": round(t1 - t0, 3),
            "Mrays_s": round(rays / (t1 - t0) / 1e6, 1), "waves": srv.stats()["waves"]}


def serving_extra(args, local, paper_scene, stream_s=3.0, trace_s=1.0, rate=200.0):
    """Bounded serving figures for the default run: the paper-sized scene at
    965x1137, 16 spp streamed at 30 requests/s for stream_s seconds; then
    trace_s seconds of the Poisson trace at `rate` requests/s over the 8
    serving scenes (it offers far more rays than one GPU renders, so the
    queue grows and the latencies include the wait)."""
    from paper_0801_1500_gb300 import serve as SV
    lam = args.lam or 8.0
    out = {}
    be = SV.GpuBackend(local, lam=lam)
    srv = SV.Server(be, [paper_scene], hbm_budget=int(args.hbm_gb * (1 << 30)), wave_rays=24e6, band_rows=1137)
    n = int(round(30.0 * stream_s))
    trace = [dict(id=k, arrival_s=k / 30.0, scene=0, width=965, height=1137, spp=16, angle_deg=0.0) for k in range(n)]
    res = replay(srv, SV, trace, [paper_scene], S.PRECISION_FP32)
    srv.close()
    be.close()
    # a throttled stream: it is sustained when every frame is done within a
    # frame interval of its arrival
    res["offered_fps"] = 30.0
    res["sustained"] = res["completed"] == n and res["max_ms"] < 1e3 / 30.0
    out["paper_scene_1.1MP_16spp_30fps"] = res
    scenes = S.serving_scenes(8, 1000, 250000, seed=0)
    be = SV.GpuBackend(local, lam=lam)
    srv = SV.Server(be, scenes, hbm_budget=int(args.hbm_gb * (1 << 30)))
    trace = S.poisson_trace(int(round(rate * trace_s)), rate, len(scenes), seed=0)
    res = replay(srv, SV, trace, scenes, S.PRECISION_FP32)
    srv.close()
    be.close()
    res["rate_req_s"] = rate
    res["arrivals_s"] = trace_s
    out["poisson_trace_segment"] = res
    return out


def run_serve(args):
    """Serving stream over 8 resident scenes (1k-250k objects): Poisson
    arrivals, mixed resolutions and sample counts, admitted by HBM footprint."""
    import torch
    from paper_0801_1500_gb300 import serve as SV
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    prec = S.PRECISION_FP64 if args.precision == "fp64" else S.PRECISION_FP32
    scenes = S.serving_scenes(8, 1000, 250000, seed=0)
    out = {"metric": METRIC, "unit": "ms", "higher_is_better": False, "n_gpus": ws, "data": "synthetic",
           "dtype": "f32" if prec == S.PRECISION_FP32 else "f64",
           "config": {"workload": "serve_8scenes_1k-250k_poisson", "objects": [s.n_objects for s in scenes],
                      "resolutions": S.SERVE_RESOLUTIONS, "spp": S.SERVE_SPP, "hbm_budget_GB": args.hbm_gb,
                      "grid_lambda": args.lam or 8.0}}
    with ClockSampler(local) as clk:
        # the offered stream at several rates (the highest is the configured rate)
        sweep = []
        for rate in args.rates:
            be = SV.GpuBackend(local, lam=args.lam or 8.0)
            srv = SV.Server(be, scenes, hbm_budget=int(args.hbm_gb * (1 << 30)))
            trace = S.poisson_trace(args.requests, rate, len(scenes), seed=0)
            res = replay(srv, SV, trace, scenes, prec)
            srv.close()
            be.close()
            res["rate_req_s"] = rate
            sweep.append(res)
        # a steady 1.1 MP, 16-sample stream on the paper-sized scene at 30 frames/s, then unthrottled
        paper = [S.paper_scene(0)]
        steady = {}
        for label, rate, n in (("30fps", 30.0, 90), ("unthrottled", 1e6, 240)):
            be = SV.GpuBackend(local, lam=args.lam or 8.0)
            srv = SV.Server(be, paper, hbm_budget=int(args.hbm_gb * (1 << 30)), wave_rays=24e6, band_rows=1137)
            trace = [dict(id=k, arrival_s=k / rate, scene=0, width=965, height=1137, spp=16, angle_deg=0.0)
                     for k in range(n)]
            res = replay(srv, SV, trace, paper, prec)
            srv.close()
            be.close()
            res["fps"] = round(res["completed"] / res["wall_s"], 1)
            steady[label] = res
    main_res = sweep[-1]
    out.update(value=main_res["p99_ms"], steps=len(sweep), warmup=0,
               serving={"rate_sweep": sweep, "paper_scene_1.1MP_16spp": steady}, clocks=clk.summary())
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=0,
                    help="timed steps (0: about a second of device time for the workload)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="paper_1mp", help="paper_1mp | paper_17mp | small | orbit64")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--lam", type=float, default=0.0, help="grid cells per object (0 = autotune)")
    ap.add_argument("--refill", type=int, default=0, help="AO lane refill threshold (0 = autotune)")
    ap.add_argument("--block", type=int, default=0, help="threads per CTA of the persistent kernels")
    ap.add_argument("--tile", default="", help="primary tile WxH, product 32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64 and 17.6 MP side measurements")
    ap.add_argument("--ref-budget", type=float, default=8.0)
    ap.add_argument("--requests", type=int, default=200, help="serve: requests per offered rate")
    ap.add_argument("--rates", type=float, nargs="+", default=[25.0, 50.0, 100.0, 200.0],
                    help="serve: offered request rates (req/s)")
    ap.add_argument("--hbm-gb", type=float, default=16.0, help="serve: HBM budget for outputs")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.steps <= 0:
        # a timed region of about a second, so the clock sampler (every 200 ms)
        # sees it several times
        args.steps = {"paper_1mp": 500, "small": 500, "paper_17mp": 40, "orbit64": 12}.get(args.workload, 20)
    if args.workload == "serve" and args.impl == "ours":
        run_serve(args)
        return
    orbit = args.workload == "orbit64"
    w = workload("paper_1mp" if orbit else args.workload, args.precision)

    if args.impl == "reference":
        if not args.lam:
            args.lam = 2.0
        run_reference(args, w)
        return

    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    from paper_0801_1500_gb300 import gbrt as G
    from paper_0801_1500_gb300 import autotune as AT

    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    r = G.Renderer(local, stream)
    W, H, p = w.width, w.height, w.params
    spp = p.ao_samples
    manual = args.lam or args.refill or args.block or args.tile
    if manual:
        tun = G.gbrt_get_tuning(r.ctx)
        if args.refill:
            tun["refill"] = args.refill
        if args.block:
            tun["block"] = args.block
        if args.tile:
            tun["tile_w"], tun["tile_h"] = (int(x) for x in args.tile.split("x"))
        G.gbrt_set_tuning(r.ctx, **tun)
        lam = args.lam or 2.0
        scene, grid = r.upload(w.scene, lam=lam)
        tuned = {"source": "command line"}
    else:
        best, scene, grid = AT.autotune(r, w.scene, w.camera, W, H, w.lights, p)
        lam = best["lambda"]
        tuned = {"source": "autotuner", "trials": best.get("trials", 0)}
    args.lam = lam
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    launches0 = G.gbrt_launch_count(r.ctx)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    if orbit:
        frames, items, outs = orbit_items(G, torch, dev, scene, grid, w.scene, w.lights, p.precision)
        G.gbrt_render_batch(r.ctx, items, G.BATCH_GRAPH)
        G.gbrt_sync(r.ctx)
        hits = sum(int((o[1].cpu().numpy().view(np.uint32) != G.MISS).sum()) for o in outs)
        rays_per_step = sum(f["width"] * f["height"] for f in frames) + sum(
            int((o[1].cpu().numpy().view(np.uint32) != G.MISS).sum()) * f["spp"] for f, o in zip(frames, outs))
        frames_per_step = len(frames)
        barrier()
        launches0 = G.gbrt_launch_count(r.ctx)
        with ClockSampler(local) as clk:
            t0 = time.perf_counter()
            ms, _ = time_steps(torch, stream, flush, lambda: G.gbrt_render_batch(r.ctx, items, G.BATCH_GRAPH),
                               args.steps, args.warmup)
            barrier()
            wall = time.perf_counter() - t0
        phases = phases_all = None
    else:
        rgb, ids, _ = r.render(scene, grid, w.camera, W, H, w.lights, p, ids=True)
        G.gbrt_sync(r.ctx)
        hits = int((ids.cpu().numpy().view(np.uint32) != G.MISS).sum())
        rays_per_step = W * H + hits * spp
        frames_per_step = 1
        out = torch.empty((H, W, 3), dtype=torch.float64 if p.precision == S.PRECISION_FP64 else torch.float32,
                          device=dev)
        cam, li, pa = G.make_camera(w.camera), G.make_lights(w.lights), G.make_params(p)
        # per-kernel CUDA events on every PROFILE_EVERY-th step of the timed
        # region (the roofline's AO-walk time and the split per kernel): an
        # event between two kernels costs a few microseconds and the overlap
        # of the dependent launch, so the other steps run without them
        barrier()
        launches0 = G.gbrt_launch_count(r.ctx)
        with ClockSampler(local) as clk:
            t0 = time.perf_counter()
            ms, phases = time_steps(torch, stream, flush,
                                    lambda: G.gbrt_render(r.ctx, scene, grid, cam, W, H, spp, li, pa, out),
                                    args.steps, args.warmup, after=lambda: G.gbrt_phase_times(r.ctx),
                                    before=lambda on: G.gbrt_set_profiling(r.ctx, on), every=PROFILE_EVERY)
            barrier()
            wall = time.perf_counter() - t0
        launches1 = G.gbrt_launch_count(r.ctx)
        G.gbrt_set_profiling(r.ctx, False)
        phases_all = phases
    rc = G.gbrt_sync(r.ctx, check=False)
    if rc != G.OK:
        raise SystemExit(f"render reported {G.strerror(rc)}")
    # kernels the library launched per timed step (warm-up steps ran in the same window;
    # the separate per-kernel pass after it is not counted)
    if orbit:
        launches1 = G.gbrt_launch_count(r.ctx)
    launches = (launches1 - launches0) * args.steps // (args.steps + args.warmup)
    dev_s = sum(ms) / 1e3
    from paper_0801_1500_gb300 import partition
    t_max = partition.max_over_ranks(dev_s)
    value = rays_per_step * args.steps * ws / t_max / 1e6
    ms_step = 1e3 * t_max / args.steps

    # e2e through the C ABI from host memory, wall-clocked, per step: the
    # frame's geometry from page-locked host arrays -> gbrt_scene_update ->
    # gbrt_grid_rebuild -> render into a page-locked host image. The colours
    # and palette are uploaded once. A second figure ("cold") creates the scene
    # and builds its grid from host arrays every step, then frees them.
    e2e = None
    if rank == 0 and not orbit:
        pinned = {k: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).pin_memory().numpy().view(a.dtype)
                  for k, a in (("s", w.scene.spheres), ("c", w.scene.cylinders),
                               ("i", w.scene.color_idx), ("p", w.scene.palette))}
        host_out = torch.empty(out.shape, dtype=out.dtype).pin_memory().numpy()
        pa_host = G.make_params(p, out_flags=G.HOST_PTRS)
        n_e2e = max(3, min(args.steps, 10))
        sc2 = G.gbrt_scene_upload(r.ctx, pinned["s"], pinned["c"], pinned["i"], pinned["p"], G.HOST_PTRS)
        gr2 = G.gbrt_grid_build(r.ctx, sc2, lam)
        G.gbrt_grid_rebuild(r.ctx, gr2, sc2)   # the first rebuild allocates its buffers
        G.gbrt_sync(r.ctx)
        # (a) a stream of frames: each step enqueues its geometry copy, rebuild,
        #     render and image copy-back (asynchronous host outputs); the host
        #     waits once, after the last step. Frames alternate between two
        #     contexts (each its own CUDA stream, scene and grid), so one
        #     frame's geometry update and grid rebuild overlap the other's
        #     render; "one_context" is the same stream of frames on one context.
        pa_async = G.make_params(p, out_flags=G.HOST_PTRS | G.HOST_ASYNC)
        outs_async = [torch.empty(out.shape, dtype=out.dtype).pin_memory().numpy() for _ in range(2)]
        r_b = G.Renderer(local, torch.cuda.Stream(dev))
        sc_b = G.gbrt_scene_upload(r_b.ctx, pinned["s"], pinned["c"], pinned["i"], pinned["p"], G.HOST_PTRS)
        gr_b = G.gbrt_grid_build(r_b.ctx, sc_b, lam)
        G.gbrt_grid_rebuild(r_b.ctx, gr_b, sc_b)
        G.gbrt_sync(r_b.ctx)

        def stream_steps(n, lanes):
            for k in range(n):
                c, sc_k, gr_k = lanes[k % len(lanes)]
                G.gbrt_scene_update(c, sc_k, pinned["s"], pinned["c"], G.HOST_PTRS)
                G.gbrt_grid_rebuild(c, gr_k, sc_k)
                G.gbrt_render(c, sc_k, gr_k, cam, W, H, spp, li, pa_async, outs_async[k % 2])
            for c, _, _ in lanes:
                G.gbrt_sync(c)

        two = [(r.ctx, sc2, gr2), (r_b.ctx, sc_b, gr_b)]
        n_stream = max(10, args.steps)
        t_lanes = {}
        for name, lanes in (("two", two), ("one", two[:1])):
            stream_steps(3, lanes)
            torch.cuda.synchronize(dev)
            t1 = time.perf_counter()
            stream_steps(n_stream, lanes)
            t_lanes[name] = (time.perf_counter() - t1) / n_stream
            assert np.array_equal(outs_async[0], outs_async[1])  # the same frame, copied back each step
        t_stream = t_lanes["two"]
        G.gbrt_grid_free(r_b.ctx, gr_b)
        G.gbrt_scene_free(r_b.ctx, sc_b)
        r_b.close()
        # (b) one frame at a time: the host waits for every image
        tt = []
        for k in range(n_e2e + 2):
            torch.cuda.synchronize(dev)
            t1 = time.perf_counter()
            G.gbrt_scene_update(r.ctx, sc2, pinned["s"], pinned["c"], G.HOST_PTRS)
            G.gbrt_grid_rebuild(r.ctx, gr2, sc2)
            G.gbrt_render(r.ctx, sc2, gr2, cam, W, H, spp, li, pa_host, host_out)   # waits for the image
            t2 = time.perf_counter()
            if k >= 2:
                tt.append(t2 - t1)
        assert np.array_equal(host_out, outs_async[0])
        G.gbrt_grid_free(r.ctx, gr2)
        G.gbrt_scene_free(r.ctx, sc2)
        tc = []
        for k in range(n_e2e + 2):
            torch.cuda.synchronize(dev)
            t1 = time.perf_counter()
            sc2 = G.gbrt_scene_upload(r.ctx, pinned["s"], pinned["c"], pinned["i"], pinned["p"], G.HOST_PTRS)
            gr2 = G.gbrt_grid_build(r.ctx, sc2, lam)
            G.gbrt_render(r.ctx, sc2, gr2, cam, W, H, spp, li, pa_host, host_out)
            G.gbrt_grid_free(r.ctx, gr2)
            G.gbrt_scene_free(r.ctx, sc2)
            t2 = time.perf_counter()
            if k >= 2:
                tc.append(t2 - t1)
        h2d = pinned["s"].nbytes + pinned["c"].nbytes
        e2e = {"value": round(rays_per_step / t_stream / 1e6, 3), "unit": "Mrays/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(host_out.nbytes),
               "ms_per_step": round(1e3 * t_stream, 3), "fps": round(1.0 / t_stream, 2),
               "path": "scene_update + grid_rebuild + render with asynchronous host image, per step; "
                       f"{n_stream} steps alternating between two contexts, one wait at the end",
               "one_context": {"ms_per_step": round(1e3 * t_lanes["one"], 3),
                               "Mrays_s": round(rays_per_step / t_lanes["one"] / 1e6, 3),
                               "path": "the same stream of frames on one context"},
               "per_frame_wait": {"ms_per_step": round(1e3 * sum(tt) / len(tt), 3),
                                  "Mrays_s": round(rays_per_step / (sum(tt) / len(tt)) / 1e6, 3),
                                  "path": "the same calls, the host waiting for each image"},
               "cold": {"ms_per_step": round(1e3 * sum(tc) / len(tc), 3),
                        "Mrays_s": round(rays_per_step / (sum(tc) / len(tc)) / 1e6, 3),
                        "h2d_bytes_per_step": int(sum(a.nbytes for a in pinned.values())),
                        "path": "scene_upload + grid_build + render (host image) + free, per step"}}

    if rank != 0:
        r.close()
        if ws > 1:
            torch.distributed.destroy_process_group()
        return

    props = torch.cuda.get_device_properties(dev)
    peaks, peak_src = measured_peaks()
    # live calibration of the ALU roofline on this GPU at its current clock
    calib = {"fp32_fma_tflops": round(G.gbrt_microbench(r.ctx, G.MB_FP32_FMA), 2),
             "fp64_fma_tflops": round(G.gbrt_microbench(r.ctx, G.MB_FP64_FMA), 3),
             "l2_read_gbs": round(G.gbrt_microbench(r.ctx, G.MB_L2_READ), 1)}
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12  # TFLOP/s

    # side measurements on the same GPU: the plain FP64 path and 17.6 MP
    extras = {}
    if not args.no_extras and not orbit and args.workload == "paper_1mp":
        other = S.PRECISION_FP64 if p.precision == S.PRECISION_FP32 else S.PRECISION_FP32
        mid = S.Workload("paper_26318obj_1930x2274_spp16", w.scene, 1930, 2274, S.Params(ao_samples=16),
                         w.lights, S.ortho_camera(w.scene, 1930, 2274))
        shadowed = S.paper_1mp(scene=w.scene)
        shadowed.params.shadows = True
        pin_aa = S.Workload("paper_26318obj_965x1137_pinhole_aa2x2_spp16", w.scene, W, H, S.Params(ao_samples=16),
                            w.lights, S.pinhole_camera(w.scene, W, H, fov_deg=30.0, aa=2))
        side = (("fp64_path_1.1MP", S.paper_1mp(precision=other, scene=w.scene), 20),
                ("fp32_path_1.1MP_direct_light_shadows", shadowed, 5),
                ("fp32_path_1.1MP_pinhole_2x2_supersampled", pin_aa, 3),
                ("fp32_path_4.4MP", mid, 3),
                ("fp32_path_17.6MP", S.paper_17mp(precision=S.PRECISION_FP32, scene=w.scene), 3),
                ("fp64_path_17.6MP", S.paper_17mp(precision=S.PRECISION_FP64, scene=w.scene), 1))
        for name, wk, nsteps in side:
            o2 = torch.empty((wk.height, wk.width, 3),
                             dtype=torch.float64 if wk.params.precision == S.PRECISION_FP64 else torch.float32,
                             device=dev)
            aa2 = max(1, wk.camera.aa)  # hit ids per sub-sample
            i2 = torch.empty((aa2 * wk.height, aa2 * wk.width), dtype=torch.int32, device=dev)
            c2, l2, p2 = G.make_camera(wk.camera), G.make_lights(wk.lights), G.make_params(wk.params)
            G.gbrt_render(r.ctx, scene, grid, c2, wk.width, wk.height, 16, l2, p2, o2, i2)
            G.gbrt_sync(r.ctx)
            h2 = int((i2.cpu().numpy().view(np.uint32) != G.MISS).sum())
            # rays counted: primary + AO samples of hit pixels (shadow rays, at most one per
            # light per hit, are not counted: Mrays/s of the shadow run is a lower bound)
            rays2 = aa2 * aa2 * wk.width * wk.height + 16 * h2
            profile = name == "fp64_path_1.1MP"
            G.gbrt_set_profiling(r.ctx, profile)
            ms2, ph2 = time_steps(torch, stream, flush,
                                  lambda: G.gbrt_render(r.ctx, scene, grid, c2, wk.width, wk.height, 16, l2, p2, o2),
                                  nsteps, 2, after=(lambda: G.gbrt_phase_times(r.ctx)) if profile else None)
            G.gbrt_set_profiling(r.ctx, False)
            m2 = sum(ms2) / len(ms2)
            extras[name] = {"Mrays_s": round(rays2 / m2 / 1e3, 2), "ms_per_frame": round(m2, 4),
                            "fps": round(1e3 / m2, 2), "rays_per_frame": rays2, "steps": nsteps,
                            "dtype": "f64" if wk.params.precision == S.PRECISION_FP64 else "f32"}
            if profile:
                extras[name]["phases_ms"] = {k: round(sum(ph[k] for ph in ph2) / len(ph2), 4) for k in G.PHASES}
                extras[name]["ao_rays_per_frame"] = 16 * h2
        # animated scene: per frame, new geometry from page-locked host memory,
        # a device-side grid rebuild and the render, with no host round trip
        extras["fp32_path_1.1MP_md_animation"] = animation_extra(G, torch, r, w, lam, stream, flush, dev)
        # weak-scaling analogue of the paper's Table 4 (1.1 / 4.4 / 17.6 MP), on one GPU
        extras["resolution_sweep_Mrays_s"] = {"1.1MP": round(value, 1),
                                              "4.4MP": extras["fp32_path_4.4MP"]["Mrays_s"],
                                              "17.6MP": extras["fp32_path_17.6MP"]["Mrays_s"]}
        # serving: the paper scene streamed at 30 frames/s, and a segment of
        # the Poisson serving trace (8 resident scenes, 1k-250k objects)
        extras["serving"] = serving_extra(args, local, w.scene)

    cpu = None
    roof = None
    if not args.no_cpu_baseline:
        s = oracle_sample(w, lam, budget_s=10.0)
        cpu = {"value": round(s["rays"] / s["seconds"] / 1e6, 4), "unit": "Mrays/s", "cores": s["cores"],
               "kind": "oracle", "sample": f"{s['rows']} evenly spaced rows ({s['pixels']} px, {s['rays']} rays) "
                                           f"of the 965x1137 frame, FP64 grid walk, lambda {lam}"}
        s1 = oracle_sample(w, lam, budget_s=4.0, threads=1)
        cpu["single_core"] = {"value": round(s1["rays"] / s1["seconds"] / 1e6, 4), "cores": 1,
                              "sample": f"{s1['rows']} evenly spaced rows ({s1['rays']} rays)"}
        if not args.no_extras and args.workload == "paper_1mp":
            w17 = S.paper_17mp(precision=p.precision, scene=w.scene)
            s17 = oracle_sample(w17, lam, budget_s=10.0)
            cpu["17.6MP"] = {"value": round(s17["rays"] / s17["seconds"] / 1e6, 4), "cores": s17["cores"],
                             "seconds": round(s17["seconds"], 2),
                             "sample": f"{s17['rows']} evenly spaced rows of 4548 ({s17['rays']} rays)"}
        if phases:
            # dominant kernel: the AO walk; its algorithmic work per launch is the
            # AO rays of one frame x the oracle's AO flops per ray (same grid lambda)
            fpr, bpr = per_ray_work(s["counters"], "ao")
            fpr_dev, _ = per_ray_work(s["counters"], "ao", device_formulas=True)
            ao_rays = rays_per_step - W * H
            ao_s = sum(ph["ao_walk"] for ph in phases) / len(phases) / 1e3
            achieved = fpr * ao_rays / ao_s / 1e12
            l2_gbs = bpr * ao_rays / ao_s / 1e9
            prof = committed_profile(args.workload, args.precision)
            roof = {"bound": "alu", "kernel": "k_ao_walk", "achieved": round(achieved, 3),
                    "peak": round(fp32_peak, 2), "unit": "TFLOP/s", "frac": round(achieved / fp32_peak, 4),
                    "traffic": committed_traffic(args.workload, args.precision),
                    "peak_source": f"{props.multi_processor_count} SMs x 128 FP32 lanes x 2 flop x "
                                   f"{sm_max:.0f} MHz ({peak_src} max clock)",
                    "flops_per_ray": round(fpr, 1),
                    "flops_convention": f"per AO ray: oracle cells x {FLOPS_CELL} + sphere tests x {FLOPS_SPHERE} "
                                        f"+ cylinder tests x {FLOPS_CYLINDER} (same lambda)",
                    "flops_per_ray_device_formulas": round(fpr_dev, 1),
                    "frac_device_formulas": round(fpr_dev * ao_rays / ao_s / 1e12 / fp32_peak, 4),
                    "issue_slots_busy_ncu": (round(prof["issue_active_pct"] / 100.0, 3)
                                             if "issue_active_pct" in prof else None),
                    "fma_measured_tflops": calib["fp32_fma_tflops"],
                    "frac_of_measured_fma": round(achieved / calib["fp32_fma_tflops"], 4),
                    "kernel_ms": round(ao_s * 1e3, 4),
                    "l2": {"bound": "l2", "achieved": round(l2_gbs, 1), "peak": calib["l2_read_gbs"],
                           "unit": "GB/s", "frac": round(l2_gbs / calib["l2_read_gbs"], 4),
                           "bytes_per_ray": round(bpr, 1),
                           "peak_source": "16-byte reads of a buffer of half the L2 (gbrt_microbench, this GPU)"}}
            tun = G.gbrt_get_tuning(r.ctx)
            if ("warp_instructions_per_launch" in prof and prof.get("grid_lambda") == lam
                    and prof.get("refill") == tun["refill"] and prof.get("block") == tun["block"]):
                # the instruction-issue bound: ncu's warp instructions of one
                # launch (same kernel sources and launch shape) over the live
                # kernel time, against one instruction a clock per scheduler
                inst = prof["warp_instructions_per_launch"]
                issue_peak = 4 * props.multi_processor_count * sm_max * 1e6 / 1e9
                issue = inst / ao_s / 1e9
                roof["issue"] = {"bound": "issue", "achieved": round(issue, 1), "peak": round(issue_peak, 1),
                                 "unit": "G warp instructions/s", "frac": round(issue / issue_peak, 4),
                                 "warp_instructions_per_launch": int(inst),
                                 "warp_instructions_per_ao_ray": round(inst / ao_rays, 2),
                                 "peak_source": f"4 warp schedulers x {props.multi_processor_count} SMs x "
                                                f"{sm_max:.0f} MHz",
                                 "count_source": "ncu smsp__inst_executed.sum from the committed summary of this "
                                                 "kernel, workload and launch shape"}
            fp64 = extras.get("fp64_path_1.1MP")
            if fp64 and "phases_ms" in fp64:
                # the plain FP64 path's AO walk against the FP64 FMA rate measured
                # on this GPU (same algorithmic work per AO ray, its own AO rays)
                ao64_s = fp64["phases_ms"]["ao_walk"] / 1e3
                ach64 = fpr * fp64["ao_rays_per_frame"] / ao64_s / 1e12
                fp64["roofline"] = {"bound": "alu_fp64", "kernel": "k_ao_walk<double>", "achieved": round(ach64, 4),
                                    "peak": calib["fp64_fma_tflops"], "unit": "TFLOP/s",
                                    "frac": round(ach64 / calib["fp64_fma_tflops"], 4),
                                    "peak_source": "FP64 FMA rate measured by gbrt_microbench on this GPU",
                                    "kernel_ms": round(ao64_s * 1e3, 4), "flops_per_ray": round(fpr, 1),
                                    "nominal_fp64_tflops": 1.25,
                                    "frac_of_nominal": round(ach64 / 1.25, 4)}
                fp64["fp32_path_speedup"] = round(fp64["ms_per_frame"] / ms_step, 2)

    config = {"workload": ("orbit64_" if orbit else "") + w.name, "precision": args.precision,
              "grid_lambda": lam, "tuning": G.gbrt_get_tuning(r.ctx), "tuned_by": tuned,
              "rays_per_step": rays_per_step, "frames_per_step": frames_per_step, "hit_pixels": hits,
              "l2": "flushed between steps (512 MB write outside the timed events)"}
    if not orbit:
        config.update(width=W, height=H, ao_samples=spp, objects=w.scene.n_objects)
    line = {"metric": METRIC, "value": round(value, 3), "unit": "Mrays/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
            "fps": round(frames_per_step * 1e3 / ms_step, 2), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
            "config": config, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
            "phases_ms": ({k: round(sum(ph[k] for ph in phases_all) / len(phases_all), 4) for k in G.PHASES}
                          if phases else None),
            "phases_note": (f"CUDA events between the kernels on every {PROFILE_EVERY}th timed step "
                            "(the roofline's kernel_ms is their AO-walk mean)") if phases else None,
            "extras": extras or None, "calibration": calib, "wall_s_timed_region": round(wall, 4),
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    r.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
