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
  roofline   trace kernel against instruction issue, the ceiling that binds
             it: warp instructions per launch (ncu count per path x paths) /
             kernel time, over 152 SMs x 4 schedulers x the sampled SM clock
  roofline_hbm  the memory roofline: algorithmic bytes (4 B per voxel read at
             a tentative collision + 4 B of majorant per leaf entered, counted
             by a separate counting run with the same seed) / kernel time,
             over measured HBM
  cpu_baseline  the CPU oracle on a bounded pixel sample of the same image
  octree     the same steps over the paper's 2^L octree (built in each step)
  wavefront  the same steps (same seeds, same path scores) scheduled as a
             wavefront: SoA queues of flights and vertices, one kernel per
             stage and round, instead of the persistent loop

  fom        1/(relative variance x time) of the learned proposal against
             plain HG sampling on the bench field at sun zenith 60 deg, each
             run until its median pixel relative SE is 1 %: a 512 x 512
             image and the domain-mean ground flux T_tot, frozen network and
             with its online training time counted

``--workload batch``: 96 flux problems (fields 64^2x32 ... 1024^2x160 with
1-16 gas bands each, sun zenith 0-75 deg) in one persistent launch, launch
shape chosen by the autotuner.  ``--workload sweep``: the refinement sweep
(128^2x40 ... 2048^2x640 over a 4096^2 heightfield, 1e8 flux paths per
point, FP32 and BF16 storage, FP64 oracle difference at the two smallest).

``--impl reference`` times the CPU oracle alone on the same workload.
Multi-GPU (torchrun): the job is one image with 64 x N samples per pixel;
rank r traces every N-th pixel of the claim order (64 x W x H paths per rank:
weak scaling) and the ranks' per-pixel FP64 sums are added in rank order at
the end of each step (the only collective); rank 0 prints the max-over-ranks
timing.  The line's `strong` figure splits the single 64-spp image instead.
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

from scenes.configs import CUMULUS, REFINEMENT_SWEEP  # noqa: E402

METRIC = "paths/s and 1/(variance x time) at 1% rel. std err, learned vs plain, 1 GB300"
WORKLOAD = "cumulus 512x512x160 @25m, 3-level majorants, 1024x1024 nadir image x 64 spp, sun 60 deg"
W, H, SPP = CUMULUS.image.width, CUMULUS.image.height, CUMULUS.image.spp
# DRAM traffic of the trace kernel from the last full ncu capture (profiles/),
# valid only while the kernel's sources are the ones that were captured
PROFILED_TRACE_SHA = "a98ee57872041750"
PROFILED_DRAM_BYTES_PER_PATH = 23.62
# issue figures: warp instructions per path and threads per warp instruction
# from a one-pass count of a bench launch (1024^2 x 64 spp), the small
# capture's issue-active fraction; the kernel is issue-bound, so these
# locate it against its real ceiling: 152 SMs x 4 schedulers x 1 warp
# instruction per cycle
PROFILED_ISSUE_ACTIVE = 0.7237
PROFILED_THREADS_PER_INST = 16.53
PROFILED_WARP_INST_PER_PATH = 4877.3
PROFILED_SOURCE = "profiles/trace_kernel_cumulus_1024px64spp_launches.md"
# the same capture over the octree (profiles/trace_kernel_octree_cumulus_512px16spp_ncu_full.md)
PROFILED_OCTREE_DRAM_BYTES_PER_PATH = 39.87
# one-pass count of the bench's octree launches (same profile as the pyramid's)
PROFILED_OCTREE_WARP_INST_PER_PATH = 3704.2
PROFILED_OCTREE_THREADS_PER_INST = 15.35


def trace_sources_sha() -> str:
    """sha256 prefix over the trace kernel's sources (trace.cu, mcrt_device.cuh)."""
    import hashlib
    h = hashlib.sha256()
    for f in ("trace.cu", "mcrt_device.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1902_01137_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(paths_per_launch):
    try:
        sha = trace_sources_sha()
    except OSError:
        return None
    return PROFILED_DRAM_BYTES_PER_PATH * paths_per_launch if sha == PROFILED_TRACE_SHA else None


def issue_roofline(kernel_ms, paths, sm_mhz, traffic, inst_per_path=PROFILED_WARP_INST_PER_PATH,
                   threads_per_inst=PROFILED_THREADS_PER_INST):
    """Roofline of the trace kernel against the ceiling that binds it,
    instruction issue: warp instructions per launch (the committed ncu
    capture's count per path times the launch's paths) over the live kernel
    time, against 152 SMs x 4 schedulers x 1 warp instruction per cycle at
    the SM clock sampled during the timed steps.  None once the kernel's
    sources differ from the captured ones."""
    try:
        if trace_sources_sha() != PROFILED_TRACE_SHA:
            return None
    except OSError:
        return None
    mhz = sm_mhz or 2070.0
    peak = 152 * 4 * mhz * 1e6
    achieved = inst_per_path * paths / (kernel_ms / 1e3)
    return {"bound": "alu", "resource": "warp-instruction issue", "achieved": achieved, "peak": peak,
            "unit": "warp instructions/s", "frac": achieved / peak, "traffic": traffic,
            "simt_efficiency": threads_per_inst / 32.0,
            "lane_frac": achieved / peak * threads_per_inst / 32.0,
            "inst_per_path": inst_per_path, "sm_mhz": mhz,
            "peak_derivation": "152 SMs x 4 schedulers x 1 warp instruction/cycle x sampled SM clock",
            "source": "instructions per path from " + PROFILED_SOURCE}


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
    spec = CUMULUS.scene()
    return spec, CUMULUS.camera(spec)


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
    """The CPU oracle on the bench workload: each step traces a bounded row
    sample of the image (the whole run stays within a few minutes); value is
    the paths per second over what ran, ms_per_step the time a step took.
    The time a whole image would take is only extrapolated, in its own
    labelled field."""
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    spec, cam = make_workload()
    per_step = max(2.0, min(args.ref_seconds, 150.0 / max(1, args.steps)))
    for _ in range(args.warmup):
        oracle_sample(spec, cam, target_s=min(2.0, per_step))
    descs, paths_all, dts = [], 0, []
    cores = 1
    for _ in range(args.steps):
        v, cores, desc, paths, dt = oracle_sample(spec, cam, target_s=per_step)
        descs.append(desc)
        paths_all += paths
        dts.append(dt)
    value = paths_all / sum(dts)
    line = {"metric": METRIC, "value": value, "unit": "paths/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(dts) / len(dts), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD,
                       "timed": "each step: the CPU oracle on a row sample of the image (about %.0f s of work)"
                                % per_step,
                       "paths_per_step": paths_all // max(1, args.steps)},
            "full_image_ms_extrapolated": W * H * SPP / value * 1e3,
            "cpu_baseline": {"value": value, "unit": "paths/s", "cores": cores, "kind": "oracle",
                             "sample": descs[0]},
            "e2e": {"value": value, "unit": "paths/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def ctx_octree_levels(spec) -> int:
    n = max(spec.shape_xyz)
    L = 1
    while (1 << L) < n:
        L += 1
    return L


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
    # N > 1: one image whose samples grow with the ranks (SPP x N per pixel,
    # weak scaling: every rank traces SPP x W x H paths), split by pixels
    # (every N-th pixel of the claim order per rank) and combined by a
    # rank-ordered FP64 reduction of the per-pixel sums
    spp_job = SPP * world
    if world > 1:
        opts.shard_index, opts.shard_count = rank, world
    from paper_1902_01137_gb300 import shard

    def step(seed, k, spp=None, o=None):
        spp = spp_job if spp is None else spp
        o = opts if o is None else o
        sc = new_scene(k)
        try:
            t = m.mcrt_trace_camera(ctx.h, sc.h, cd, spp, seed, o, tally[0])
            tally[0] = t
            if o.shard_count > 1:
                s1, s2 = m.mcrt_tally_read_sums(ctx.h, t)
                shard.combine_image(s1[:, 0], s2[:, 0], spp)
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
    copts.shard_index, copts.shard_count = opts.shard_index, opts.shard_count
    sc = new_scene(k_dev)
    ct = m.mcrt_trace_camera(ctx.h, sc.h, cd, spp_job, base_seed + 100, copts)
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
        from paper_1902_01137_gb300 import shard
        total_ms = shard.max_over_ranks(total_ms)
        torch.distributed.barrier()
    clk = clocks.stop()
    paths_per_step = W * H * SPP
    value = world * paths_per_step * args.steps / (total_ms / 1e3)

    # N > 1 also: the single SPP image split over the ranks (strong scaling)
    strong = None
    if world > 1:
        for i in range(args.warmup):
            step(base_seed + 400 + i, k_dev, spp=SPP)
        torch.distributed.barrier()
        torch.cuda.synchronize()
        st_ms = []
        for i in range(args.steps):
            flush_buf.fill_(float(i))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(base_seed + 500 + i, k_dev, spp=SPP)
            e1.record(stream)
            e1.synchronize()
            st_ms.append(e0.elapsed_time(e1))
        st_total = shard.max_over_ranks(sum(st_ms))
        strong = {"value": paths_per_step * args.steps / (st_total / 1e3), "unit": "paths/s",
                  "ms_per_step": st_total / args.steps,
                  "workload": "the %dx%d x %d spp image split by pixels over %d ranks" % (W, H, SPP, world)}

    # the same steps over the paper's 2^L octree (Sec. 3.1.1), built in each
    # step beside the pyramid, leaves at tau~ = 1 with 2^3-voxel cells as the
    # finest level; timed like the steps above
    oopts = m.mcrt_trace_opts_default()
    oopts.grid = m.MCRT_GRID_OCTREE
    oopts.finest_level = 1
    oopts.shard_index, oopts.shard_count = opts.shard_index, opts.shard_count

    def octree_step(seed, k):
        sc = new_scene(k)
        try:
            sc.build_octree()
            t = m.mcrt_trace_camera(ctx.h, sc.h, cd, spp_job, seed, oopts, tally[0])
            tally[0] = t
            if oopts.shard_count > 1:
                s1, s2 = m.mcrt_tally_read_sums(ctx.h, t)
                shard.combine_image(s1[:, 0], s2[:, 0], spp_job)
            return m.mcrt_tally_kernel_ms(ctx.h, t)
        finally:
            sc.close()

    octree = None
    if not args.no_octree:
        for i in range(args.warmup):
            octree_step(base_seed + 300 + i, k_dev)
        torch.cuda.synchronize()
        oct_step_ms, oct_kern_ms = [], []
        for i in range(args.steps):
            flush_buf.fill_(float(i))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            oct_kern_ms.append(octree_step(base_seed + 100 + i, k_dev))
            e1.record(stream)
            e1.synchronize()
            oct_step_ms.append(e0.elapsed_time(e1))
        oct_total = sum(oct_step_ms)
        if world > 1:
            from paper_1902_01137_gb300 import shard
            oct_total = shard.max_over_ranks(oct_total)
        # its own roofline: algorithmic bytes from a counting run on the same seed
        sc = new_scene(k_dev)
        try:
            sc.build_octree()
            oc = m.mcrt_trace_opts_default()
            oc.grid, oc.finest_level, oc.count_events = m.MCRT_GRID_OCTREE, 1, 1
            oc.shard_index, oc.shard_count = opts.shard_index, opts.shard_count
            ct = m.mcrt_trace_camera(ctx.h, sc.h, cd, spp_job, base_seed + 100, oc)
            ocnt = m.mcrt_tally_counters(ctx.h, ct)
            m.mcrt_tally_destroy(ct)
        finally:
            sc.close()
        o_alg = 4 * (ocnt["tentative"] + ocnt["sun_tentative"]) + 4 * (ocnt["leaf_steps"] + ocnt["sun_leaf_steps"] +
                                                                      ocnt["sun_rays"] + ocnt.get("flights", 0))
        o_kavg = statistics.mean(oct_kern_ms)
        o_ach = o_alg / (o_kavg / 1e3) / 1e9
        o_peak = peaks()["hbm_gbs"] if peaks() else 6800.0
        o_traffic = None
        try:
            if trace_sources_sha() == PROFILED_TRACE_SHA:
                o_traffic = PROFILED_OCTREE_DRAM_BYTES_PER_PATH * paths_per_step
        except OSError:
            pass
        octree = {"value": world * paths_per_step * args.steps / (oct_total / 1e3), "unit": "paths/s",
                  "ms_per_step": oct_total / args.steps, "kernel_ms": o_kavg,
                  "grid": "2^L octree (Sec. 3.1.1), %d levels, tau~ 1, finest level 1" % ctx_octree_levels(spec),
                  "steps": args.steps, "l2": "flushed between steps",
                  "roofline_hbm": {"bound": "hbm", "achieved": o_ach, "peak": o_peak, "unit": "GB/s",
                                   "frac": o_ach / o_peak, "traffic": o_traffic, "alg_bytes_per_launch": o_alg,
                                   "leaf_steps_per_path": (ocnt["leaf_steps"] + ocnt["sun_leaf_steps"]) / paths_per_step,
                                   "tentative_per_path": (ocnt["tentative"] + ocnt["sun_tentative"]) / paths_per_step}}
        # against instruction issue, the ceiling that binds it too (the
        # octree's own one-pass count; the SM clock sampled during the steps)
        o_issue = issue_roofline(o_kavg, paths_per_step, clk.get("sm_mhz") if clk else None, o_traffic,
                                 PROFILED_OCTREE_WARP_INST_PER_PATH, PROFILED_OCTREE_THREADS_PER_INST)
        octree["roofline"] = o_issue or octree["roofline_hbm"]

    # the same steps (same seeds, so the same path scores) scheduled as a
    # wavefront: SoA queues of flights and vertices in device memory, one
    # kernel per stage and round, instead of the persistent loop
    wavefront = None
    if not args.no_wavefront and world == 1:
        wopts = m.mcrt_trace_opts_default()
        wopts.schedule = m.MCRT_SCHEDULE_WAVEFRONT
        for i in range(args.warmup):
            step(base_seed + 600 + i, k_dev, o=wopts)
        torch.cuda.synchronize()
        wf_step_ms, wf_kern_ms = [], []
        for i in range(args.steps):
            flush_buf.fill_(float(i))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            wf_kern_ms.append(step(base_seed + 100 + i, k_dev, o=wopts))
            e1.record(stream)
            e1.synchronize()
            wf_step_ms.append(e0.elapsed_time(e1))
        wf_total = sum(wf_step_ms)
        wavefront = {"value": paths_per_step * args.steps / (wf_total / 1e3), "unit": "paths/s",
                     "ms_per_step": wf_total / args.steps, "kernel_ms": statistics.mean(wf_kern_ms),
                     "schedule": "wavefront: SoA queues, flight / vertex+sun ray / start kernels per round, "
                                 "2^21 paths in flight", "steps": args.steps, "l2": "flushed between steps",
                     "persistent_kernel_ms": statistics.mean(kern_ms)}

    # e2e: pinned host field in, image mean/SE out, through the C ABI
    e2e_val = None
    h2d = spec.k.nbytes
    d2h = W * H * 16
    if not args.no_e2e:
        e2e_ms = []
        for i in range(args.steps):
            flush_buf.fill_(float(i))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sc = new_scene(k_host)                     # H2D copy of the field inside
            try:
                t = m.mcrt_trace_camera(ctx.h, sc.h, cd, spp_job, base_seed + 200 + i, opts, tally[0])
                if world > 1:                              # D2H of this rank's sums, then the reduction
                    s1, s2 = m.mcrt_tally_read_sums(ctx.h, t)
                    shard.combine_image(s1[:, 0], s2[:, 0], spp_job)
                else:
                    mean, se, _ = m.mcrt_tally_read(ctx.h, t)   # D2H of the image
            finally:
                sc.close()
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
        e2e_val = world * paths_per_step * len(e2e_ms) / (sum(e2e_ms) / 1e3)

    # roofline of the trace kernel
    pk = peaks()
    leaf_entries = cnt["leaf_steps"] + cnt["sun_leaf_steps"] + cnt["sun_rays"] + cnt.get("flights", 0)
    vox_reads = cnt["tentative"] + cnt["sun_tentative"]
    alg_bytes = 4 * vox_reads + 4 * leaf_entries
    kavg = statistics.mean(kern_ms)
    achieved = alg_bytes / (kavg / 1e3) / 1e9
    peak = pk["hbm_gbs"] if pk else 6800.0
    traffic = args.traffic_bytes if args.traffic_bytes else profiled_traffic(W * H * SPP)
    roof_hbm = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_source": "measured" if pk else "fallback",
                "kernel": "trace_kernel<camera,f32>", "kernel_ms": kavg,
                "alg_bytes_per_launch": alg_bytes, "vox_reads": vox_reads, "leaf_entries": leaf_entries}
    # the kernel is bound by instruction issue, not by HBM: the line's
    # roofline is the issue ceiling, the memory roofline is reported beside it
    roof = issue_roofline(kavg, W * H * SPP, clk.get("sm_mhz") if clk else None, traffic) or roof_hbm
    roof["kernel"], roof["kernel_ms"] = "trace_kernel<camera,f32>", kavg

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, desc, paths, dt = oracle_sample(spec, cam, target_s=args.ref_seconds)
        cpu = {"value": v, "unit": "paths/s", "cores": cores, "kind": "oracle", "sample": desc}

    fom = None
    if world == 1 and not args.no_fom:         # the learned proposal's FOM: one GPU (minutes of tracing)
        fom = learned_fom(m, ctx)
    events = cnt["tentative"] + cnt["sun_tentative"]
    line = {"metric": METRIC, "value": value, "unit": "paths/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD if world == 1 else
                       WORKLOAD.replace("x %d spp" % SPP, "x %d spp (%d per rank)" % (spp_job, SPP)),
                       "paths_per_step": paths_per_step, "l2": "flushed between steps",
                       "parallelism": "pixel shards over %d ranks, rank-ordered FP64 reduction" % world
                       if world > 1 else "single"},
            "strong": strong,
            "roofline": roof, "roofline_hbm": roof_hbm,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_val, "unit": "paths/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches, "clocks": clk,
            "collision_events_per_s": events / (kavg / 1e3),
            "octree": octree, "wavefront": wavefront,
            "fom": fom,
            "counters": cnt}
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def _fom(rel, ms):
    return 1.0 / (rel * rel * ms / 1e3)


# The learned proposal's configuration in the bench line: 2 learned vertices,
# MIS share 0.75 for HG (the best figure of merit of the alpha / vertex sweep
# of --workload fom at 256 spp), network trained online on the image's own
# kind of path.
FOM_ALPHA, FOM_NL = 0.75, 2
FOM_TARGET = 0.01


def _img_stats(r):
    """Mean pixel relative variance and median pixel relative SE over the
    pixels brighter than 1e-3 of the image maximum."""
    ok = r.mean > 1e-3 * r.mean.max()
    rel = r.se[ok] / r.mean[ok]
    return float(np.mean(rel * rel)), float(np.median(rel))


def _sum_stats(s1, s2, n):
    mean = s1 / n
    var = np.maximum(s2 / n - mean * mean, 0.0) * n / max(n - 1, 1)
    se = np.sqrt(var / n)
    ok = mean > 1e-3 * mean.max()
    rel = se[ok] / mean[ok]
    return float(np.mean(rel * rel)), float(np.median(rel)), float(mean.mean())


def _run_to_target(trace, pilot_spp, seed, max_rounds=8):
    """Trace the image in segments (fresh seeds), adding their per-pixel FP64
    sums, until the median pixel relative SE is at most FOM_TARGET: each
    next segment is sized from the current median (10 % margin).  The FOM is
    1 / (mean pixel relative variance x the time of all segments)."""
    s1 = s2 = 0.0
    n, ms, segs = 0, 0.0, []
    spp = pilot_spp
    rv = med = mean = float("nan")
    for r in range(max_rounds):
        a1, a2, t = trace(spp, seed + r)
        s1, s2, n, ms = s1 + a1, s2 + a2, n + spp, ms + t
        segs.append(spp)
        rv, med, mean = _sum_stats(s1, s2, n)
        if med <= FOM_TARGET:
            break
        spp = max(pilot_spp, int(math.ceil(n * (med / FOM_TARGET) ** 2 * 1.1)) - n)
    return {"spp": n, "segments_spp": segs, "ms": ms, "rel_var": rv, "median_rel_se": med,
            "fom": 1.0 / (rv * ms / 1e3), "paths": n * int(np.size(s1)), "mean": mean}


def _flux_to_target(trace, seed):
    p = trace(1 << 20, seed)
    rel = p.se[2] / p.mean[2]
    n = max(1024, int(math.ceil((1 << 20) * (rel / FOM_TARGET) ** 2 * 1.1)))
    r = trace(n, seed + 1)
    rel = r.se[2] / r.mean[2]
    return {"paths": n, "ms": r.kernel_ms, "rel_se": rel, "fom": _fom(rel, r.kernel_ms)}


def learned_fom(m, ctx, sweep=False):
    """Learned proposal against plain HG sampling, 1/(relative variance x
    time) at 1 % relative standard error (the metric), on the bench's cumulus
    field (512x512x160 at 25 m), sun zenith 60 deg.

    Image: a 512 x 512 nadir image traced until its median pixel relative SE
    is at most 1 % (pixels brighter than 1e-3 of the maximum); FOM = 1 /
    (mean pixel relative variance x time).  The learned form's network is
    first trained online on camera paths of the same image (2^26 paths in
    batches of 2^20, two Adam steps each); 'online' counts that training in
    the time, 'frozen' does not.  Flux: T_tot to 1 % relative SE (a few
    thousand paths, where fixed launch costs dominate) and, beside it, at
    2^26 paths.  sweep: the image FOM for MIS shares 0.25 / 0.5 / 0.75 and
    2 / 8 learned vertices at 256 spp (the FOM of a frozen network does not
    depend on the run's length) instead of the full 1 % runs."""
    import scenes
    import torch
    spec, _ = make_workload()
    sc = m.Scene.from_spec(ctx, spec, k=torch.from_numpy(spec.k).cuda())
    cam = scenes.nadir_camera(spec, 512, 512)
    out = {"field": "cumulus 512x512x160 @25m (the bench field), sun 60 deg",
           "protocol": "median pixel relative SE <= 1 %% (pixels > 1e-3 of max), FOM = 1/(mean pixel rel. "
                       "variance x time); learned: alpha %.2f, %d learned vertices" % (FOM_ALPHA, FOM_NL)}
    try:
        sc.trace_camera(cam, 16, seed=1)
        cd = m.CameraDesc()
        for i in range(3):
            cd.pos[i], cd.target[i], cd.up[i] = cam.pos[i], cam.target[i], cam.up[i]
        cd.fov_deg, cd.width, cd.height = cam.fov_deg, cam.width, cam.height

        def sums(spp, seed, **kw):
            t = m.mcrt_trace_camera(ctx.h, sc.h, cd, spp, seed, m.Scene._opts(**kw))
            try:
                a1, a2 = m.mcrt_tally_read_sums(ctx.h, t)
                return a1[:, 0], a2[:, 0], m.mcrt_tally_kernel_ms(ctx.h, t)
            finally:
                m.mcrt_tally_destroy(t)

        def plain(spp, seed):
            return sc.trace_camera(cam, spp, seed=seed)

        def train(alpha, nl):
            prop = m.Proposal(ctx, seed=7)
            t = sc.trace_camera(cam, 256, seed=4, proposal=prop, learn=1, batch_paths=1 << 20, n_learned=nl,
                                mis_alpha=alpha, train_steps=2)
            return prop, t.kernel_ms

        if sweep:
            base = plain(256, 3)
            rv0, _ = _img_stats(base)
            f0 = 1.0 / (rv0 * base.kernel_ms / 1e3)
            out["plain_256spp"] = {"ms": base.kernel_ms, "rel_var": rv0, "fom": f0}
            for alpha in (0.25, 0.5, 0.75):
                for nl in (2, 8):
                    prop, tms = train(alpha, nl)
                    try:
                        r = sc.trace_camera(cam, 256, seed=5, proposal=prop, learn=0, n_learned=nl,
                                            mis_alpha=alpha)
                    finally:
                        prop.close()
                    rv, _ = _img_stats(r)
                    f = 1.0 / (rv * r.kernel_ms / 1e3)
                    out["alpha%.2f_nl%d" % (alpha, nl)] = {"ms": r.kernel_ms, "rel_var": rv, "fom": f,
                                                           "ratio": f / f0, "var_gain": rv0 / rv,
                                                           "time_ratio": r.kernel_ms / base.kernel_ms,
                                                           "train_ms": tms}
            return out
        pl = _run_to_target(lambda spp, seed: sums(spp, seed), 256, 10)
        out["plain_image"] = pl
        prop, tms = train(FOM_ALPHA, FOM_NL)
        try:
            lf = _run_to_target(lambda spp, seed: sums(spp, seed, proposal=prop, learn=0, n_learned=FOM_NL,
                                                      mis_alpha=FOM_ALPHA), 256, 20)
            lf["train_ms"] = tms
            out["learned_image"] = lf
            online = 1.0 / (lf["rel_var"] * (lf["ms"] + tms) / 1e3)
            out["ratio_image_vs_plain"] = lf["fom"] / pl["fom"]
            out["ratio_online_image_vs_plain"] = online / pl["fom"]
            out["image_means_agree_rel"] = abs(lf["mean"] - pl["mean"]) / pl["mean"]

            # ground flux T_tot: its own network, trained on flux paths
            fprop = m.Proposal(ctx, seed=7)
            try:
                ft = sc.trace_flux(1 << 26, seed=4, proposal=fprop, learn=1, batch_paths=1 << 20, n_learned=FOM_NL,
                                   mis_alpha=FOM_ALPHA, train_steps=2)
                pf = _flux_to_target(lambda n, s_: sc.trace_flux(n, seed=s_), 30)
                lfx = _flux_to_target(lambda n, s_: sc.trace_flux(n, seed=s_, proposal=fprop, learn=0,
                                                                  n_learned=FOM_NL, mis_alpha=FOM_ALPHA), 40)
                big = 1 << 26
                pb = sc.trace_flux(big, seed=50)
                lb = sc.trace_flux(big, seed=51, proposal=fprop, learn=0, n_learned=FOM_NL, mis_alpha=FOM_ALPHA)
                fp_b = _fom(pb.se[2] / pb.mean[2], pb.kernel_ms)
                fl_b = _fom(lb.se[2] / lb.mean[2], lb.kernel_ms)
                out["flux"] = {"plain_1pct": pf, "learned_1pct": lfx, "train_ms": ft.kernel_ms,
                               "ratio_1pct": lfx["fom"] / pf["fom"],
                               "ratio_online_1pct": 1.0 / ((lfx["rel_se"] ** 2) * (lfx["ms"] + ft.kernel_ms) / 1e3)
                               / pf["fom"],
                               "plain_2p26": {"fom": fp_b, "ms": pb.kernel_ms, "rel_se": pb.se[2] / pb.mean[2]},
                               "learned_2p26": {"fom": fl_b, "ms": lb.kernel_ms, "rel_se": lb.se[2] / lb.mean[2]},
                               "ratio_2p26": fl_b / fp_b}
            finally:
                fprop.close()
        finally:
            prop.close()
    finally:
        sc.close()
    return out


# ---------------------------------------------------------------------------
# Batching workload
# ---------------------------------------------------------------------------
BATCH_METRIC_NOTE = "96 flux problems (1-16 gas bands each) in one persistent launch"


def run_batch(args):
    import torch
    import scenes
    import paper_1902_01137_gb300 as m
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ctx = m.Context(local)
    stream = torch.cuda.current_stream(dev)
    inst = scenes.batch_instances(0)
    specs = [scenes.cumulus(b.nx, b.nx, b.nz, seed=b.field_seed, device=dev) for b in inst]
    field_bytes = sum(int(s.k.numel()) * 4 for s in specs)

    def make_scenes(fields):
        return [m.Scene(ctx, f, sp.dx, sp.dy, sp.dz, k_clear=sp.k_clear, ssa_clear=sp.ssa_clear,
                        ssa_cloud=sp.ssa_cloud, g=sp.g, levels=sp.levels, albedo=sp.ground_albedo)
                for f, sp in zip(fields, specs)]

    dev_fields = [sp.k for sp in specs]
    sc = make_scenes(dev_fields)
    # the batch configuration names no grid depth: the timed steps track the
    # paper's 2^L octree (tau~ 1, finest leaves 2^3 voxels), the faster grid;
    # the 8^L pyramid is timed beside it
    for s_ in sc:
        s_.build_octree()
    items = scenes.batch_items(inst, lambda i: sc[i])
    seeds0 = [it[5] for it in items]
    paths = sum(it[4] for it in items)
    topts = m.mcrt_trace_opts_default()
    topts.grid = m.MCRT_GRID_OCTREE
    topts.finest_level = 1
    opts, best = m.mcrt_autotune_batch(ctx.h, m.make_batch_items(items), 0.25, topts)
    shape = dict(chunk=opts.chunk, rare_batch=opts.rare_batch, block_size=opts.block_size)
    grid_kw = dict(grid=m.MCRT_GRID_OCTREE, finest_level=1)
    cr = m.trace_batch(ctx, items, count_events=1, **shape, **grid_kw)
    cnt = cr.counters
    flush_buf = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    # the same batch as a CUDA-graph plan over these scenes (set up once):
    # one graph launch per step, new seeds each step
    plan_fig = None
    plan = m.BatchPlan(ctx, items, **shape, **grid_kw)
    try:
        base = np.array(seeds0, dtype=np.uint64)
        for i in range(args.warmup):
            plan.set_seeds(base + np.uint64(7000 * (rank + 1) + i))
            plan.run()
        torch.cuda.synchronize()
        p_ms, g_ms = [], []
        for i in range(args.steps):
            flush_buf.fill_(float(i))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan.set_seeds(base + np.uint64(1000 * (rank + 1) + 100 + i))
            r = plan.run()
            e1.record(stream)
            e1.synchronize()
            p_ms.append(e0.elapsed_time(e1))
            g_ms.append(r.kernel_ms)
        p_total = sum(p_ms)
        if world > 1:
            from paper_1902_01137_gb300 import shard
            p_total = shard.max_over_ranks(p_total)
        plan_fig = {"value": world * paths * args.steps / (p_total / 1e3), "unit": "paths/s",
                    "ms_per_step": p_total / args.steps, "graph_ms": statistics.mean(g_ms),
                    "step": "new seeds + one graph launch (tally reset, trace, finalize, copies); scenes set up once"}
    finally:
        plan.close()
    for s_ in sc:
        s_.close()

    def step(fields, seed_off, octree=True):
        scs = make_scenes(fields)
        try:
            kw = dict(shape)
            if octree:
                # the paper's 2^L octree (Sec. 3.1.1) per field, finest leaves 2^3 voxels
                for s_ in scs:
                    s_.build_octree()
                kw.update(grid_kw)
            its = [(scs[i], kg, z, a, n, seed + seed_off)
                   for i, (_, kg, z, a, n, seed) in zip(_item_instance(inst), items)]
            r = m.trace_batch(ctx, its, **kw)
        finally:
            for s_ in scs:
                s_.close()
        return r

    for i in range(args.warmup):
        step(dev_fields, 1000 * (rank + 1) + i)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    l0 = ctx.launches
    step_ms, kern_ms = [], []
    for i in range(args.steps):
        flush_buf.fill_(float(i))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = step(dev_fields, 1000 * (rank + 1) + 100 + i)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        kern_ms.append(r.kernel_ms)
    torch.cuda.synchronize()
    launches = ctx.launches - l0
    total_ms = sum(step_ms)
    if world > 1:
        from paper_1902_01137_gb300 import shard
        total_ms = shard.max_over_ranks(total_ms)
    clk = clocks.stop()
    value = world * paths * args.steps / (total_ms / 1e3)
    pyramid = None
    if not args.no_octree:
        for i in range(args.warmup):
            step(dev_fields, 3000 * (rank + 1) + i, octree=False)
        torch.cuda.synchronize()
        o_ms, o_kern = [], []
        for i in range(args.steps):
            flush_buf.fill_(float(i))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = step(dev_fields, 1000 * (rank + 1) + 100 + i, octree=False)
            e1.record(stream)
            e1.synchronize()
            o_ms.append(e0.elapsed_time(e1))
            o_kern.append(r.kernel_ms)
        o_total = sum(o_ms)
        if world > 1:
            from paper_1902_01137_gb300 import shard
            o_total = shard.max_over_ranks(o_total)
        pyramid = {"value": world * paths * args.steps / (o_total / 1e3), "unit": "paths/s",
                   "ms_per_step": o_total / args.steps, "kernel_ms": statistics.mean(o_kern),
                   "grid": "8^L pyramid per field, tau~ 1, finest level 0 (same launch shape)",
                   "step": "96 scenes (relayout, pyramid, leaf maps) + one batch trace"}
    # e2e: fields from pinned host memory, tallies back to the host
    e2e = None
    if not args.no_e2e:
        host_fields = [f.cpu().pin_memory() for f in dev_fields]
        ems = []
        for i in range(max(1, min(args.steps, 2))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = step(host_fields, 5000 + i)
            _ = r.mean.sum()
            ems.append((time.perf_counter() - t0) * 1e3)
        del host_fields
        e2e = world * paths * len(ems) / (sum(ems) / 1e3)
    pk = peaks()
    leaf_entries = cnt["leaf_steps"] + cnt["sun_leaf_steps"] + cnt["sun_rays"] + cnt.get("flights", 0)
    vox_reads = cnt["tentative"] + cnt["sun_tentative"]
    alg = 4 * vox_reads + 4 * leaf_entries
    kavg = statistics.mean(kern_ms)
    ach = alg / (kavg / 1e3) / 1e9
    peak = pk["hbm_gbs"] if pk else 6800.0
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = batch_oracle_sample(inst, target_s=args.ref_seconds)
    line = {"metric": METRIC, "value": value, "unit": "paths/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch: " + BATCH_METRIC_NOTE, "items": len(items), "instances": len(inst),
                       "paths_per_step": paths, "field_bytes": field_bytes, "launch_shape": shape,
                       "autotune_best_ms_on_quarter": best, "l2": "flushed between steps",
                       "grid": "2^L octree per field (Sec. 3.1.1), tau~ 1, finest level 1",
                       "step": "96 scenes (relayout, pyramid, octree, leaf maps) + one batch trace"},
            "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                         "traffic": None, "peak_source": "measured" if pk else "fallback",
                         "kernel": "trace_kernel<flux,f32,batch>", "kernel_ms": kavg, "alg_bytes_per_launch": alg},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e, "unit": "paths/s", "h2d_bytes_per_step": field_bytes,
                    "d2h_bytes_per_step": len(items) * 4 * 16},
            "gpu_launches": launches, "clocks": clk, "pyramid": pyramid, "graph_plan": plan_fig, "counters": cnt}
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def _item_instance(inst):
    """Instance index of each flattened item (one per band)."""
    out = []
    for i, b in enumerate(inst):
        out += [i] * len(b.k_gas)
    return out


def batch_oracle_sample(inst, target_s=12.0):
    """The oracle on the batch's smallest fields (64^2x32 and 128^2x40
    instances, all bands), paths/s over about target_s seconds."""
    import oracle
    import scenes
    oracle.build()
    cores = oracle.default_threads()
    small = [(i, b) for i, b in enumerate(inst) if b.nx <= 128][:4]
    jobs = []
    for i, b in small:
        sp = scenes.cumulus(b.nx, b.nx, b.nz, seed=b.field_seed)
        for kg in b.k_gas:
            osc = oracle.Scene(k=sp.k, dx=sp.dx, dy=sp.dy, dz=sp.dz, levels=sp.levels, k_clear=sp.k_clear,
                               ssa_clear=sp.ssa_clear, ssa_cloud=sp.ssa_cloud, g=sp.g,
                               ground_albedo=sp.ground_albedo, sun_zenith_deg=b.sun_zenith_deg,
                               sun_azimuth_deg=b.sun_azimuth_deg, k_gas=kg)
            jobs.append(osc)
    n = 2000
    t0 = time.perf_counter()
    oracle.trace_flux(jobs[0], n, seed=1, nthreads=cores)
    dt = time.perf_counter() - t0
    per = max(1000, int(n * target_s / max(dt, 1e-3) / len(jobs)))
    t0 = time.perf_counter()
    for j, osc in enumerate(jobs):
        oracle.trace_flux(osc, per, seed=j, nthreads=cores)
    dt = time.perf_counter() - t0
    return {"value": per * len(jobs) / dt, "unit": "paths/s", "cores": cores, "kind": "oracle",
            "sample": "%d paths on each of %d items (all bands of the first %d instances with 64^2x32 or 128^2x40 "
                      "fields)" % (per, len(jobs), len(small))}


# ---------------------------------------------------------------------------
# Refinement sweep with a heightfield ground
# ---------------------------------------------------------------------------
SWEEP = REFINEMENT_SWEEP.sizes


def run_sweep(args):
    import torch
    import scenes
    import paper_1902_01137_gb300 as m
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ctx = m.Context(local)
    hf = scenes.heightfield(4096, 0.3, seed=0)
    npaths = args.sweep_paths
    points = []
    clocks = ClockSampler(local)
    clocks.start()
    for nx, nz in SWEEP:
        spec = scenes.cumulus(nx, nx, nz, seed=0, device=dev)
        spec.sun_zenith_deg = 60.0
        row = {"field": "%dx%dx%d" % (nx, nx, nz), "dx_m": 12800.0 / nx, "voxels": nx * nx * nz, "paths": npaths}
        for name, storage in (("f32", m.MCRT_STORAGE_F32), ("bf16", m.MCRT_STORAGE_BF16)):
            sc = m.Scene.from_spec(ctx, spec, storage=storage)
            try:
                sc.set_heightfield(hf, spec.ground_albedo)
                sc.trace_flux(1 << 20, seed=1)
                r = sc.trace_flux(npaths, seed=7)
                row[name] = {"ms": r.kernel_ms, "paths_per_s": npaths / (r.kernel_ms / 1e3),
                             "ns_per_path": r.kernel_ms * 1e6 / npaths, "mean": list(map(float, r.mean)),
                             "se": list(map(float, r.se))}
                if storage == m.MCRT_STORAGE_F32:
                    # the same paths over the paper's 2^L octree (Sec. 3.1.1)
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    sc.build_octree()
                    torch.cuda.synchronize()
                    build_ms = (time.perf_counter() - t0) * 1e3
                    kw = dict(grid=m.MCRT_GRID_OCTREE, finest_level=1)
                    sc.trace_flux(1 << 20, seed=1, **kw)
                    r = sc.trace_flux(npaths, seed=7, **kw)
                    row["f32_octree"] = {"ms": r.kernel_ms, "paths_per_s": npaths / (r.kernel_ms / 1e3),
                                         "ns_per_path": r.kernel_ms * 1e6 / npaths, "build_ms": build_ms,
                                         "mean": list(map(float, r.mean)), "se": list(map(float, r.se))}
            finally:
                sc.close()
        f, b = row["f32"], row["bf16"]
        row["bf16_minus_f32_in_se"] = [(b["mean"][q] - f["mean"][q]) / math.hypot(b["se"][q], f["se"][q])
                                       for q in range(3)]
        if nx <= 256 and not args.no_cpu_baseline:
            import oracle
            hspec = scenes.cumulus(nx, nx, nz, seed=0)
            osc = oracle.Scene(k=hspec.k, dx=hspec.dx, dy=hspec.dy, dz=hspec.dz, levels=hspec.levels,
                               k_clear=hspec.k_clear, ssa_clear=hspec.ssa_clear, ssa_cloud=hspec.ssa_cloud,
                               g=hspec.g, ground_albedo=hspec.ground_albedo, sun_zenith_deg=60.0, heights=hf)
            no = 1 << 20
            t0 = time.perf_counter()
            o, _ = oracle.trace_flux(osc, no, seed=7)
            row["oracle_fp64"] = {"paths": no, "s": time.perf_counter() - t0, "mean": list(map(float, o.mean[:3])),
                                  "se": list(map(float, o.se[:3])),
                                  "f32_minus_oracle_in_se": [(f["mean"][q] - o.mean[q]) / math.hypot(f["se"][q], o.se[q])
                                                             for q in range(3)],
                                  "note": "host field from numpy FFT (the device field differs by FFT rounding)"}
        points.append(row)
        del spec
        torch.cuda.empty_cache()
    clk = clocks.stop()
    line = {"metric": METRIC, "workload": "refinement sweep, 4096^2 heightfield (0-300 m), sun 60 deg, flux",
            "unit": "paths/s", "points": points, "clocks": clk, "data": "synthetic"}
    print(json.dumps(line))
    ctx.close()
    return 0


def run_tau(args):
    """The merge threshold sweep (Sec. 4.2, Sec. 5): the bench image traced
    with leaves chosen at several tau~ (finest level 0 and 1), over the 8^L
    pyramid and over the paper's 2^L octree (Sec. 3.1.1); per point the
    trace time and, from a counting run, the traversal work (leaf steps of
    flights and sun rays) and the collision work (tentative collisions, null
    ones among them) -- the paper's partition of the time between the
    acceleration structure and null collisions.  tau~ = 0 (voxel leaves) and
    infinity (one global cell) are the same leaves on both grids and are
    run once."""
    import torch
    import paper_1902_01137_gb300 as m
    spec, cam = make_workload()
    ctx = m.Context(0)
    sc = m.Scene.from_spec(ctx, spec, k=torch.from_numpy(spec.k).cuda())
    points = []
    clocks = ClockSampler(0)
    clocks.start()
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sc.build_octree()
        torch.cuda.synchronize()
        octree_build_ms = (time.perf_counter() - t0) * 1e3
        sc.trace_camera(cam, 4, seed=1)
        sc.trace_camera(cam, 4, seed=1, grid=m.MCRT_GRID_OCTREE)
        for grid, fin in [(g, f) for g in (m.MCRT_GRID_PYRAMID, m.MCRT_GRID_OCTREE) for f in (0, 1)]:
            for tau in (0.0, 0.1, 0.3, 1.0, 3.0, 10.0, 100.0, float("inf")):
                if fin == 1 and tau == 0.0:
                    continue
                if grid == m.MCRT_GRID_OCTREE and (tau == 0.0 or not math.isfinite(tau)):
                    continue
                kw = dict(tau_merge=tau, finest_level=fin, grid=grid)
                ms = [sc.trace_camera(cam, SPP, seed=10 + i, **kw).kernel_ms for i in range(2)]
                c = sc.trace_camera(cam, SPP, seed=10, count_events=1, **kw).counters
                P = c["paths"]
                points.append({"grid": "octree 2^L" if grid == m.MCRT_GRID_OCTREE else "pyramid 8^L",
                               "tau_merge": tau if math.isfinite(tau) else "inf", "finest_level": fin,
                               "ms": min(ms), "paths_per_s": W * H * SPP / (min(ms) / 1e3),
                               "leaf_steps_per_path": (c["leaf_steps"] + c["sun_leaf_steps"]) / P,
                               "tentative_per_path": (c["tentative"] + c["sun_tentative"]) / P,
                               "null_per_path": (c["tentative"] - c["real"]) / P,
                               "sun_tentative_per_path": c["sun_tentative"] / P})
    finally:
        sc.close()
        ctx.close()
    clk = clocks.stop()
    print(json.dumps({"metric": METRIC, "workload": "tau~ sweep: " + WORKLOAD, "unit": "paths/s",
                      "octree_build_ms": octree_build_ms, "points": points, "clocks": clk,
                      "data": "synthetic"}))
    return 0


def run_fom_sweep(args):
    """The learned proposal's image FOM for each MIS share and learned-vertex
    count (256 spp; see learned_fom), as one JSON line."""
    import paper_1902_01137_gb300 as m
    ctx = m.Context(0)
    out = learned_fom(m, ctx, sweep=True)
    print(json.dumps({"metric": METRIC, "workload": "learned-proposal sweep", "fom": out}))
    ctx.close()
    return 0


def run_profile_case(grid="pyramid", schedule="persistent"):
    """A small case of the bench kernel for ncu: the same 512x512x160 field
    (160 MiB, larger than L2), a 512 x 512 image at 16 spp (4,194,304
    paths), two launches; over the 8^L pyramid (the bench line) or over the
    paper's 2^L octree (the line's `octree` figure: tau~ 1, finest level 1).
    schedule "wavefront": one trace of the bench image itself (1024 x 1024
    x 64 spp) with the wavefront schedule, whose round count is set by the
    longest path rather than by the image size."""
    import torch
    import paper_1902_01137_gb300 as m
    spec, bench_cam = make_workload()
    import scenes
    cam = scenes.nadir_camera(spec, 512, 512)
    ctx = m.Context(0)
    sc = m.Scene.from_spec(ctx, spec, k=torch.from_numpy(spec.k).cuda())
    if schedule == "wavefront":
        l0 = ctx.launches
        r = sc.trace_camera(bench_cam, SPP, seed=7, schedule=m.MCRT_SCHEDULE_WAVEFRONT)
        print("wavefront kernel_ms", r.kernel_ms, "launches", ctx.launches - l0, "mean", float(r.mean.mean()),
              flush=True)
        sc.close()
        ctx.close()
        return 0
    kw = dict(chunk=4)            # the bench launch's claim size (the default at its size)
    if grid == "octree":
        sc.build_octree()
        kw.update(grid=m.MCRT_GRID_OCTREE, finest_level=1)
    for i in range(2):
        r = sc.trace_camera(cam, 16, seed=7 + i, **kw)
        print("launch", i, "kernel_ms", r.kernel_ms, "mean", float(r.mean.mean()), flush=True)
    sc.close()
    ctx.close()
    return 0


def run_profile_learned():
    """A case of the learned proposal's passes for ncu: the bench field, a
    512 x 512 image at 16 spp, 8 learned vertices, MIS alpha 0.5, a fixed
    (Xavier-initialised, seed 7) network, one batch: trace launches 0..8 are
    passes 0..8, with a network evaluation before each resumed pass."""
    import torch
    import paper_1902_01137_gb300 as m
    import scenes
    spec, _ = make_workload()
    cam = scenes.nadir_camera(spec, 512, 512)
    ctx = m.Context(0)
    sc = m.Scene.from_spec(ctx, spec, k=torch.from_numpy(spec.k).cuda())
    prop = m.Proposal(ctx, seed=7)
    r = sc.trace_camera(cam, 16, seed=5, proposal=prop, learn=0, batch_paths=1 << 22, n_learned=8, mis_alpha=0.5)
    print("learned image kernel_ms", r.kernel_ms, "mean", float(r.mean.mean()), flush=True)
    prop.close()
    sc.close()
    ctx.close()
    return 0


def run_profile_train():
    """The proposal network's training kernels for ncu: 2^20 synthetic
    records (features in the tracer's ranges, unit directions, exponential
    targets; seed 1), one Adam-free gradient step per call, five calls per
    mode (FP32 SIMT, then BF16 tensor cores) after one warm-up call on 4096
    records."""
    import paper_1902_01137_gb300 as m
    r = np.random.default_rng(1)
    n = 1 << 20
    x = np.concatenate([r.uniform(-1, 1, (n, 3)), r.normal(size=(n, 3)), r.uniform(-8, 6, (n, 3))], axis=1)
    x[:, 3:6] /= np.linalg.norm(x[:, 3:6], axis=1, keepdims=True)
    d = r.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    t = r.exponential(size=n)
    ctx = m.Context(0)
    for mode in (m.MCRT_TRAIN_FP32, m.MCRT_TRAIN_TENSOR):
        prop = m.Proposal(ctx, seed=3, training=mode)
        prop.train_step(x[:4096], d[:4096], t[:4096])
        for _ in range(5):
            loss, _g = prop.train_step(x, d, t)
        print("mode", mode, "loss", loss, flush=True)
        prop.close()
    ctx.close()
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
    ap.add_argument("--workload", default="image", choices=["image", "batch", "sweep", "tau", "fom"])
    ap.add_argument("--sweep-paths", type=int, default=100_000_000)
    ap.add_argument("--no-fom", action="store_true")
    ap.add_argument("--no-octree", action="store_true")
    ap.add_argument("--no-wavefront", action="store_true")
    ap.add_argument("--profile-case", action="store_true",
                    help="trace one 512x512 x 16 spp image of the cumulus field twice and exit (for ncu captures)")
    ap.add_argument("--profile-learned", action="store_true",
                    help="trace one learned-proposal image (8 learned vertices, fixed network) and exit (for ncu)")
    ap.add_argument("--profile-train", action="store_true",
                    help="run the network's training kernels on 2^20 synthetic records and exit (for ncu)")
    ap.add_argument("--profile-grid", default="pyramid", choices=["pyramid", "octree"],
                    help="grid the profile case traces over")
    ap.add_argument("--profile-schedule", default="persistent", choices=["persistent", "wavefront"],
                    help="schedule the profile case traces with")
    ap.add_argument("--traffic-bytes", type=float, default=0.0,
                    help="ncu dram bytes per trace launch, if captured for this kernel version")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_case:
        return run_profile_case(args.profile_grid, args.profile_schedule)
    if args.profile_learned:
        return run_profile_learned()
    if args.profile_train:
        return run_profile_train()
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "sweep":
        return run_sweep(args)
    if args.workload == "tau":
        return run_tau(args)
    if args.workload == "fom":
        return run_fom_sweep(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
