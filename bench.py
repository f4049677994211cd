"""Benchmark: AO ray-tracing throughput (Mrays/s, fps) of the paper-sized scene.

Default workload: the 26,318-object globule (13,500 spheres + 12,818 bonds)
at 965x1137 with 16 AO samples per pixel, FP32 path with FP64 root and
re-projection. A step renders one whole frame. Rays = primary rays (one per
pixel) + AO rays actually cast (samples x pixels whose primary ray hits).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload paper_1mp|paper_17mp|small] [--precision fp32|fp64]

Under torchrun (N > 1) every rank renders its own frames (frames are
independent; no collective on the data path): value = all ranks' rays / the
slowest rank's time, "scaling": "weak".

``--impl reference`` times the FP64 CPU oracle (the only other place this
script runs it) on a bounded row sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
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

# FP32 flops of one step of each kind, counted from the formulas of the device
# code (an FMA counts 2, sqrt / reciprocal 1): grid-walk step, ray-sphere test,
# ray-cylinder test.
FLOPS_CELL, FLOPS_SPHERE, FLOPS_CYLINDER = 8, 24, 58
# bytes a walk reads per step: a cell record (8 B), an item id (4 B), a sphere
# record (16 B) or a cylinder record (32 B)
BYTES_CELL, BYTES_ITEM, BYTES_SPHERE, BYTES_CYLINDER = 8, 4, 16, 32
L2_FLUSH_BYTES = 512 << 20   # > 126 MB L2


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


def sources_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_0801_1500_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def committed_traffic(workload_name, precision):
    """DRAM bytes per launch of the AO walk kernel from the committed ncu
    summary, if it was taken on the current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", f"k_ao_walk_{precision}_{workload_name}.txt")
    if not os.path.exists(p):
        return None
    kv = {}
    for line in open(p):
        if ":" in line:
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("sources_hash") != sources_hash():
        return None
    try:
        return float(kv["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


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
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
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


def per_ray_work(c, kind="ao"):
    """Algorithmic FP32 flops and walk bytes per ray (of one kind: "ao" or
    "primary") from the oracle's grid-walk counters."""
    rays = max(1, c[f"{kind}_rays"])
    cells = c[f"{kind}_cells"]
    sph = c[f"{kind}_sphere_tests"]
    cyl = c[f"{kind}_cylinder_tests"]
    flops = (cells * FLOPS_CELL + sph * FLOPS_SPHERE + cyl * FLOPS_CYLINDER) / rays
    nbytes = (cells * BYTES_CELL + (sph + cyl) * BYTES_ITEM + sph * BYTES_SPHERE + cyl * BYTES_CYLINDER) / rays
    return flops, nbytes


def run_reference(args, w):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    lam = args.lam
    times, rays = [], 0
    for k in range(args.warmup + args.steps):
        s = oracle_sample(w, lam, budget_s=args.ref_budget)
        if k >= args.warmup:
            times.append(s["seconds"])
            rays += s["rays"]
    total = sum(times)
    v = rays / total / 1e6
    line = {"impl": "reference", "metric": "AO Mrays/s (FP64 CPU oracle)", "value": round(v, 4), "unit": "Mrays/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * total / max(1, len(times)), 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "sample": f"{s['rows']} evenly spaced rows of {w.height}"},
            "cpu_baseline": {"value": round(v, 4), "unit": "Mrays/s", "cores": s["cores"], "kind": "oracle",
                             "sample": f"{s['rows']} rows x {w.width} px per step"},
            "e2e": {"value": round(v, 4), "unit": "Mrays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="paper_1mp")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--lam", type=float, default=2.0)
    ap.add_argument("--refill", type=int, default=0, help="AO lane refill threshold (0 = library default)")
    ap.add_argument("--block", type=int, default=0, help="threads per CTA of the persistent kernels")
    ap.add_argument("--tile", default="", help="primary tile WxH, product 32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-budget", type=float, default=8.0)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    w = workload(args.workload, args.precision)

    if args.impl == "reference":
        run_reference(args, w)
        return

    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    from paper_0801_1500_gb300 import gbrt as G

    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    r = G.Renderer(local, stream)
    tun = G.gbrt_get_tuning(r.ctx)
    if args.refill:
        tun["refill"] = args.refill
    if args.block:
        tun["block"] = args.block
    if args.tile:
        tun["tile_w"], tun["tile_h"] = (int(x) for x in args.tile.split("x"))
    G.gbrt_set_tuning(r.ctx, **tun)
    scene, grid = r.upload(w.scene, lam=args.lam)
    W, H, p = w.width, w.height, w.params
    spp = p.ao_samples

    # rays per frame (pixels + AO rays of hit pixels), from one untimed render
    rgb, ids, _ = r.render(scene, grid, w.camera, W, H, w.lights, p, ids=True)
    G.gbrt_sync(r.ctx)
    hits = int((ids.cpu().numpy().view(np.uint32) != G.MISS).sum())
    rays_per_frame = W * H + hits * spp
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    out = torch.empty((H, W, 3), dtype=torch.float64 if p.precision == S.PRECISION_FP64 else torch.float32,
                      device=dev)
    cam, li, pa = G.make_camera(w.camera), G.make_lights(w.lights), G.make_params(p)

    def render_once():
        G.gbrt_render(r.ctx, scene, grid, cam, W, H, spp, li, pa, out)

    for _ in range(args.warmup):
        flush.zero_()
        render_once()
    G.gbrt_sync(r.ctx)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    phases = []
    G.gbrt_set_profiling(r.ctx, True)
    launches0 = G.gbrt_launch_count(r.ctx)
    barrier()
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()                      # L2 flush between steps, outside the events
            starts[k].record(stream)
            render_once()
            ends[k].record(stream)
            phases.append(G.gbrt_phase_times(r.ctx))   # the library's events between its kernels
        barrier()
        wall = time.perf_counter() - t0
    G.gbrt_set_profiling(r.ctx, False)
    rc = G.gbrt_sync(r.ctx, check=False)
    if rc != G.OK:
        raise SystemExit(f"render reported {G.strerror(rc)}")
    launches = G.gbrt_launch_count(r.ctx) - launches0
    ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    dev_s = sum(ms) / 1e3
    t_rank = torch.tensor([dev_s], dtype=torch.float64, device=dev)
    if ws > 1:
        torch.distributed.all_reduce(t_rank, op=torch.distributed.ReduceOp.MAX)
    t_max = float(t_rank.item())
    total_rays = rays_per_frame * args.steps * ws
    value = total_rays / t_max / 1e6
    ms_step = 1e3 * t_max / args.steps

    # e2e: host arrays -> upload -> grid build -> render -> host image, per step
    e2e = None
    if rank == 0:
        pinned = {k: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).pin_memory().numpy().view(a.dtype)
                  for k, a in (("s", w.scene.spheres), ("c", w.scene.cylinders),
                               ("i", w.scene.color_idx), ("p", w.scene.palette))}
        host_out = torch.empty(out.shape, dtype=out.dtype).pin_memory().numpy()
        pa_host = G.make_params(p, out_flags=G.HOST_PTRS)
        e2e_steps = max(3, min(args.steps, 10))
        tt = []
        for k in range(e2e_steps + 2):
            torch.cuda.synchronize(dev)
            t1 = time.perf_counter()
            sc2 = G.gbrt_scene_upload(r.ctx, pinned["s"], pinned["c"], pinned["i"], pinned["p"], G.HOST_PTRS)
            gr2 = G.gbrt_grid_build(r.ctx, sc2, args.lam)
            G.gbrt_render(r.ctx, sc2, gr2, cam, W, H, spp, li, pa_host, host_out)
            t2 = time.perf_counter()
            G.gbrt_grid_free(r.ctx, gr2)
            G.gbrt_scene_free(r.ctx, sc2)
            if k >= 2:
                tt.append(t2 - t1)
        h2d = sum(a.nbytes for a in pinned.values())
        e2e = {"value": round(rays_per_frame / (sum(tt) / len(tt)) / 1e6, 3), "unit": "Mrays/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(host_out.nbytes),
               "ms_per_step": round(1e3 * sum(tt) / len(tt), 3)}

    if rank != 0:
        r.close()
        if ws > 1:
            torch.distributed.destroy_process_group()
        return

    props = torch.cuda.get_device_properties(dev)
    peaks, peak_src = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12  # TFLOP/s

    cpu = None
    roof = None
    if not args.no_cpu_baseline:
        s = oracle_sample(w, args.lam, budget_s=15.0)
        cpu = {"value": round(s["rays"] / s["seconds"] / 1e6, 4), "unit": "Mrays/s", "cores": s["cores"],
               "kind": "oracle", "sample": f"{s['rows']} evenly spaced rows ({s['pixels']} px, {s['rays']} rays) "
                                           f"of the same frame, FP64 grid walk, lambda {args.lam}"}
        # dominant kernel: the AO walk; its algorithmic work per launch is the
        # AO rays of one frame x the oracle's AO flops per ray (same grid lambda)
        fpr, bpr = per_ray_work(s["counters"], "ao")
        ao_rays = rays_per_frame - W * H
        ao_s = sum(ph["ao_walk"] for ph in phases) / len(phases) / 1e3
        achieved = fpr * ao_rays / ao_s / 1e12
        roof = {"bound": "alu", "kernel": "k_ao_walk", "achieved": round(achieved, 3), "peak": round(fp32_peak, 2),
                "unit": "TFLOP/s", "frac": round(achieved / fp32_peak, 4),
                "traffic": committed_traffic(args.workload, args.precision),
                "peak_source": f"{props.multi_processor_count} SMs x 128 FP32 lanes x 2 flop x {sm_max:.0f} MHz "
                               f"({peak_src} max clock)",
                "kernel_ms": round(ao_s * 1e3, 4), "flops_per_ray": round(fpr, 1),
                "walk_bytes_per_ray": round(bpr, 1), "walk_GBps": round(bpr * ao_rays / ao_s / 1e9, 1)}

    line = {"metric": "AO Mrays/s (primary + AO rays) at 1.1 MP, 16 spp", "value": round(value, 3),
            "unit": "Mrays/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms_step, 4), "fps": round(1e3 / ms_step, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64",
            "data": "synthetic",
            "config": {"workload": w.name, "width": W, "height": H, "ao_samples": spp,
                       "objects": w.scene.n_objects, "precision": args.precision, "grid_lambda": args.lam,
                       "tuning": G.gbrt_get_tuning(r.ctx),
                       "rays_per_frame": rays_per_frame, "hit_pixels": hits,
                       "l2": "flushed between steps (512 MB write outside the timed events)"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
            "phases_ms": {k: round(sum(ph[k] for ph in phases) / len(phases), 4) for k in G.PHASES},
            "wall_s_timed_region": round(wall, 4), "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    r.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
