"""Benchmark of the null-collision path tracer on one GB300 (or N replicas).

Workload (one step = the whole hot path on one batch of synthetic input):
512 x 512 x 160 voxels of 25 m shaped like a shallow-cumulus LES field
(20 % cover, log-normal LWC, ssa 0.999, HG g = 0.86, ground albedo 0.1,
sun zenith 60 deg); per step: brick relayout + level-1 max of the field,
3-level majorant pyramid, leaf map, a 1024 x 1024 nadir image at 64 paths
per pixel (67,108,864 paths), mean/SE finalize.

  value      paths/s with the field resident in HBM (device-timed, CUDA events)
  e2e        the same through the C ABI from a pinned host field, host->device
             copy of the field and device->host read of the image (mean, SE)
             inside the timed region
  roofline   trace kernel: algorithmic bytes (4 B per voxel read at a
             tentative collision + 8 B per leaf entered, counted by a separate
             counting run with the same seed) / kernel time, over measured HBM
  cpu_baseline  the CPU oracle on a bounded pixel sample of the same image

``--impl reference`` times the CPU oracle alone on the same workload.
Multi-GPU (torchrun): every rank renders an independent replica of the image
with its own seed (paths are independent: weak scaling, no collective on the
data path); rank 0 prints the max-over-ranks timing.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "paths/s and 1/(variance x time) at 1% rel. std err, learned vs plain, 1 GB300"
WORKLOAD = "cumulus 512x512x160 @25m, 3-level majorants, 1024x1024 nadir image x 64 spp, sun 60 deg"
W, H, SPP = 1024, 1024, 64


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        load = sorted(sm)[len(sm) // 4:] if len(sm) >= 4 else sm
        return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def make_workload():
    import scenes
    spec = scenes.cumulus(512, 512, 160, seed=0)
    cam = scenes.nadir_camera(spec, W, H)
    return spec, cam


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample
# ---------------------------------------------------------------------------
def oracle_sample(spec, cam, target_s=12.0, seed=0):
    """Time the oracle on whole image rows until about target_s seconds of
    work; returns (paths/s, cores, sample description, paths)."""
    import oracle
    oracle.build()
    osc = oracle.Scene(k=spec.k, dx=spec.dx, dy=spec.dy, dz=spec.dz, levels=spec.levels, k_clear=spec.k_clear,
                       ssa_clear=spec.ssa_clear, ssa_cloud=spec.ssa_cloud, g=spec.g,
                       ground_albedo=spec.ground_albedo, sun_zenith_deg=spec.sun_zenith_deg)
    ocam = oracle.Camera(cam.pos, cam.target, cam.up, cam.fov_deg, cam.width, cam.height)
    cores = oracle.default_threads()
    # calibrate on rows spread over the image
    rows = 1
    r0 = H // 2
    t0 = time.perf_counter()
    oracle.trace_camera(osc, ocam, SPP, seed, pix_range=(r0 * W, (r0 + rows) * W), nthreads=cores)
    dt = time.perf_counter() - t0
    rows = max(1, min(H, int(rows * target_s / max(dt, 1e-3))))
    step = max(1, H // rows)
    picked = list(range(0, H, step))[:rows]
    paths = 0
    t0 = time.perf_counter()
    for r in picked:
        oracle.trace_camera(osc, ocam, SPP, seed, pix_range=(r * W, (r + 1) * W), nthreads=cores)
        paths += W * SPP
    dt = time.perf_counter() - t0
    desc = "%d image rows (every %d-th) x %d px x %d spp = %d paths" % (len(picked), step, W, SPP, paths)
    return paths / dt, cores, desc, paths, dt


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    spec, cam = make_workload()
    vals = []
    for _ in range(args.warmup):
        oracle_sample(spec, cam, target_s=2.0)
    descs = []
    cores = 1
    for _ in range(args.steps):
        v, cores, desc, paths, dt = oracle_sample(spec, cam, target_s=args.ref_seconds)
        vals.append(v)
        descs.append(desc)
    value = statistics.median(vals)
    line = {"metric": METRIC, "value": value, "unit": "paths/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": W * H * SPP / value * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "timed": "CPU oracle on a row sample, paths/s extrapolated"},
            "cpu_baseline": {"value": value, "unit": "paths/s", "cores": cores, "kind": "oracle",
                             "sample": descs[0]},
            "e2e": {"value": value, "unit": "paths/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gpu(args):
    import torch
    import paper_1902_01137_gb300 as m

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    spec, cam = make_workload()
    nx, ny, nz = spec.shape_xyz
    k_host = torch.from_numpy(spec.k).pin_memory()
    k_dev = k_host.to(dev, non_blocking=False)
    flush_buf = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)
    ctx = m.Context(local)
    stream = torch.cuda.current_stream(dev)

    def new_scene(k):
        return m.Scene(ctx, k, spec.dx, spec.dy, spec.dz, k_clear=spec.k_clear, ssa_clear=spec.ssa_clear,
                       ssa_cloud=spec.ssa_cloud, g=spec.g, levels=spec.levels, albedo=spec.ground_albedo,
                       sun_zenith_deg=spec.sun_zenith_deg, sun_azimuth_deg=spec.sun_azimuth_deg)

    cd = m.CameraDesc()
    for i in range(3):
        cd.pos[i], cd.target[i], cd.up[i] = cam.pos[i], cam.target[i], cam.up[i]
    cd.fov_deg, cd.width, cd.height = cam.fov_deg, cam.width, cam.height
    opts = m.mcrt_trace_opts_default()
    tally = [None]

    def step(seed, k):
        sc = new_scene(k)
        try:
            t = m.mcrt_trace_camera(ctx.h, sc.h, cd, SPP, seed, opts, tally[0])
            tally[0] = t
            return m.mcrt_tally_kernel_ms(ctx.h, t)
        finally:
            sc.close()

    base_seed = 1000 * (rank + 1)
    for i in range(args.warmup):
        step(base_seed + i, k_dev)
    torch.cuda.synchronize()

    # counting run (same seed as the first timed step) for algorithmic bytes
    copts = m.mcrt_trace_opts_default()
    copts.count_events = 1
    sc = new_scene(k_dev)
    ct = m.mcrt_trace_camera(ctx.h, sc.h, cd, SPP, base_seed + 100, copts)
    cnt = m.mcrt_tally_counters(ctx.h, ct)
    m.mcrt_tally_destroy(ct)
    sc.close()

    # timed region: device-resident input
    clocks = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = ctx.launches
    step_ms, kern_ms = [], []
    for i in range(args.steps):
        flush_buf.fill_(float(i))                     # evict L2 between steps
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        kern_ms.append(step(base_seed + 100 + i, k_dev))
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    launches = ctx.launches - launches0
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
        torch.distributed.barrier()
    clk = clocks.stop()
    paths_per_step = W * H * SPP
    value = world * paths_per_step * args.steps / (total_ms / 1e3)

    # e2e: pinned host field in, image mean/SE out, through the C ABI
    e2e_val = None
    h2d = spec.k.nbytes
    d2h = W * H * 16
    if not args.no_e2e:
        e2e_ms = []
        for i in range(max(1, min(args.steps, 3))):
            flush_buf.fill_(float(i))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sc = new_scene(k_host)                     # H2D copy of the field inside
            try:
                t = m.mcrt_trace_camera(ctx.h, sc.h, cd, SPP, base_seed + 200 + i, opts, tally[0])
                mean, se, _ = m.mcrt_tally_read(ctx.h, t)   # D2H of the image
            finally:
                sc.close()
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
        e2e_val = world * paths_per_step * len(e2e_ms) / (sum(e2e_ms) / 1e3)

    # roofline of the trace kernel
    pk = peaks()
    leaf_entries = cnt["leaf_steps"] + cnt["sun_leaf_steps"] + cnt["sun_rays"] + cnt.get("flights", 0)
    vox_reads = cnt["tentative"] + cnt["sun_tentative"]
    alg_bytes = 4 * vox_reads + 8 * leaf_entries
    kavg = statistics.mean(kern_ms)
    achieved = alg_bytes / (kavg / 1e3) / 1e9
    peak = pk["hbm_gbs"] if pk else 6800.0
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": args.traffic_bytes if args.traffic_bytes else None,
            "peak_source": "measured" if pk else "fallback",
            "kernel": "trace_kernel<camera,f32>", "kernel_ms": kavg,
            "alg_bytes_per_launch": alg_bytes, "vox_reads": vox_reads, "leaf_entries": leaf_entries}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, desc, paths, dt = oracle_sample(spec, cam, target_s=args.ref_seconds)
        cpu = {"value": v, "unit": "paths/s", "cores": cores, "kind": "oracle", "sample": desc}

    events = cnt["tentative"] + cnt["sun_tentative"]
    line = {"metric": METRIC, "value": value, "unit": "paths/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "paths_per_step": paths_per_step, "l2": "flushed between steps",
                       "parallelism": "replicas" if world > 1 else "single"},
            "roofline": roof, "cpu_baseline": cpu,
            "e2e": {"value": e2e_val, "unit": "paths/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches, "clocks": clk,
            "collision_events_per_s": events / (kavg / 1e3),
            "counters": cnt}
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-seconds", type=float, default=12.0)
    ap.add_argument("--traffic-bytes", type=float, default=0.0,
                    help="ncu dram bytes per trace launch, if captured for this kernel version")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
