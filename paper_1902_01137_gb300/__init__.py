"""Python binding of the GB300 null-collision radiative-transfer library.

Thin ctypes marshalling around ``libmcrt.so`` (the C ABI of
``include/mcrt.h``): every step of the method runs in the library's CUDA
kernels.  PyTorch is used only for device memory and streams (a CUDA tensor
can be passed as the extinction field; the context can run on torch's current
stream).  Importing this package fails loudly when the library has not been
built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

# MCRT_LIBRARY selects another build of the same library (e.g. the
# bounds-checked variant, build(checked=True)); default: the in-tree build.
LIB_PATH = os.environ.get("MCRT_LIBRARY") or _build.LIB

MCRT_OK = 0
MCRT_ERR_ARG = -1
MCRT_ERR_OOM = -2
MCRT_ERR_CUDA = -3
MCRT_ERR_TIMEOUT = -4
MCRT_ERR_CANCELLED = -5
MCRT_ERR_STATE = -6
MCRT_ERR_BOUNDS = -7
MCRT_ERR_UNSUPPORTED = -8
MCRT_MEM_HOST = 0
MCRT_MEM_DEVICE = 1
MCRT_STORAGE_F32 = 0
MCRT_STORAGE_BF16 = 1
MCRT_SUN_RATIO = 0
MCRT_SUN_DELTA = 1
MCRT_SUN_DECOMP = 2
MCRT_PHASE_HG = 0
MCRT_PHASE_RAYLEIGH = 1
MCRT_TRAIN_TENSOR = 0
MCRT_TRAIN_FP32 = 1
MCRT_GRID_PYRAMID = 0
MCRT_GRID_OCTREE = 1
MCRT_ORDER_COST = 0
MCRT_ORDER_RASTER = 1
# the struct layouts below match include/mcrt.h at this ABI version
ABI_VERSION = 2
MCRT_SCHEDULE_PERSISTENT = 0
MCRT_SCHEDULE_WAVEFRONT = 1

COUNTER_NAMES = ("paths", "tentative", "real", "ground", "leaf_steps", "sun_tentative", "sun_leaf_steps",
                 "sun_rays", "aborted", "flights", "max_path_iters", "warp_ns_to_dry", "warp_ns_total",
                 "clk_top", "clk_philox", "clk_start", "clk_begin", "clk_step", "clk_vertex", "clk_load",
                 "clk_after", "clk_end", "occ_iters", "occ_busy", "occ_step", "occ_tent", "occ_rare", "occ_wait",
                 "occ_rare_iters", "occ_empty")


class McrtError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (%d): %s" % (_status_name(status), status, msg))
        self.status = status


class FieldDesc(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("dx", C.c_float), ("dy", C.c_float), ("dz", C.c_float),
                ("ext", C.c_void_p), ("ext_mem", C.c_int32),
                ("k_clear", C.c_float), ("ssa_clear", C.c_float), ("ssa_cloud", C.c_float),
                ("hg_g", C.c_float), ("storage", C.c_int32)]


class CameraDesc(C.Structure):
    _fields_ = [("pos", C.c_float * 3), ("target", C.c_float * 3), ("up", C.c_float * 3),
                ("fov_deg", C.c_float), ("width", C.c_int32), ("height", C.c_int32)]


class BatchItem(C.Structure):
    _fields_ = [("scene", C.c_void_p), ("k_gas", C.c_float), ("sun_zenith_deg", C.c_float),
                ("sun_azimuth_deg", C.c_float), ("npaths", C.c_uint64), ("seed", C.c_uint64)]


class TraceOpts(C.Structure):
    _fields_ = [("tau_merge", C.c_float), ("finest_level", C.c_int32), ("max_order", C.c_int32),
                ("sun_mode", C.c_int32), ("chunk", C.c_int32), ("block_size", C.c_int32),
                ("grid_size", C.c_int32), ("count_events", C.c_int32), ("rare_batch", C.c_int32),
                ("proposal", C.c_void_p), ("n_learned", C.c_int32), ("mis_alpha", C.c_float),
                ("learn", C.c_int32), ("batch_paths", C.c_int32), ("learning_rate", C.c_float),
                ("train_steps", C.c_int32),
                ("deadline_ms", C.c_double),
                ("cancel_flag", C.c_void_p),
                ("batch_dalpha", C.c_int32),
                ("grid", C.c_int32),
                ("pixel_order", C.c_int32),
                ("shard_index", C.c_int32),
                ("shard_count", C.c_int32),
                ("schedule", C.c_int32),
                ("wavefront_slots", C.c_int32)]


_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libmcrt.so is not built (%s); run __graft_entry__.build() or "
                          "python -m paper_1902_01137_gb300.build" % LIB_PATH)
    L = C.CDLL(LIB_PATH)
    vp, i32, u32, u64, f32, f64 = C.c_void_p, C.c_int32, C.c_uint32, C.c_uint64, C.c_float, C.c_double
    P = C.POINTER
    sig = {
        "mcrt_version": [P(i32)],
        "mcrt_status_string": [C.c_int],
        "mcrt_create": [P(vp), C.c_int, vp],
        "mcrt_destroy": [vp],
        "mcrt_last_error": [vp],
        "mcrt_launch_count": [vp, P(u64)],
        "mcrt_scene_create": [vp, P(FieldDesc), P(vp)],
        "mcrt_scene_destroy": [vp],
        "mcrt_scene_build_majorants": [vp, i32],
        "mcrt_scene_levels": [vp, P(i32)],
        "mcrt_scene_majorant_dims": [vp, i32, P(i32)],
        "mcrt_scene_read_majorants": [vp, i32, P(f32), C.c_size_t],
        "mcrt_scene_read_minorants": [vp, i32, P(f32), C.c_size_t],
        "mcrt_scene_build_octree": [vp, i32],
        "mcrt_scene_octree_levels": [vp, P(i32)],
        "mcrt_scene_octree_dims": [vp, i32, P(i32)],
        "mcrt_scene_read_octree": [vp, i32, P(f32), P(f32), C.c_size_t],
        "mcrt_scene_set_ground_flat": [vp, f32],
        "mcrt_scene_set_clear_sky_phase": [vp, i32],
        "mcrt_scene_set_ground_heightfield": [vp, vp, i32, i32, i32, f32],
        "mcrt_debug_terrain": [vp, i32, P(f32), P(f32), P(f32)],
        "mcrt_debug_terrain_height": [vp, i32, P(f32), P(f32)],
        "mcrt_scene_set_sun": [vp, f32, f32],
        "mcrt_trace_opts_default": [P(TraceOpts)],
        "mcrt_trace_camera": [vp, P(CameraDesc), u32, u64, P(TraceOpts), P(vp)],
        "mcrt_trace_flux": [vp, u64, u64, P(TraceOpts), P(vp)],
        "mcrt_trace_camera_noalloc": [vp, P(CameraDesc), u32, u64, P(TraceOpts), vp, vp],
        "mcrt_tally_shape": [vp, P(i32), P(i32)],
        "mcrt_tally_read": [vp, P(f64), P(f64), P(u64), C.c_size_t],
        "mcrt_tally_read_sums": [vp, P(f64), P(f64), C.c_size_t],
        "mcrt_tally_counters": [vp, P(u64), C.c_size_t],
        "mcrt_tally_kernel_ms": [vp, P(f32)],
        "mcrt_tally_destroy": [vp],
        "mcrt_debug_dda": [vp, P(f32), P(f32), f32, i32, P(i32), P(f32), i32, P(i32), P(i32)],
        "mcrt_debug_dda_grid": [vp, P(f32), P(f32), f32, i32, i32, P(i32), P(f32), i32, P(i32), P(i32)],
        "mcrt_debug_philox": [vp, P(u32), P(u32), P(u32), C.c_size_t],
        "mcrt_debug_bounds_violations": [vp, P(i32), P(u64), P(i32)],
        "mcrt_debug_pool_usage": [vp, i32, P(u64), P(u64)],
        "mcrt_debug_learned_records": [vp, vp, u64, u64, P(TraceOpts), i32, P(f32), P(f32), P(f32), P(u64), P(i32)],
        "mcrt_trace_batch": [vp, P(BatchItem), i32, P(TraceOpts), P(vp)],
        "mcrt_autotune_batch": [vp, P(BatchItem), i32, C.c_double, P(TraceOpts), P(f32)],
        "mcrt_batch_plan_create": [vp, P(BatchItem), i32, P(TraceOpts), P(vp)],
        "mcrt_batch_plan_set_seeds": [vp, P(C.c_uint64), i32],
        "mcrt_batch_plan_run": [vp, P(C.c_double), P(C.c_double), C.c_size_t, P(f32)],
        "mcrt_batch_plan_tally": [vp, P(vp)],
        "mcrt_batch_plan_destroy": [vp],
        "mcrt_proposal_nparams": [P(i32)],
        "mcrt_proposal_create": [vp, u64, P(vp)],
        "mcrt_proposal_destroy": [vp],
        "mcrt_proposal_set_params": [vp, P(f32), C.c_size_t],
        "mcrt_proposal_get_params": [vp, P(f32), C.c_size_t],
        "mcrt_proposal_eval": [vp, P(f32), C.c_size_t, P(f32), P(f32)],
        "mcrt_proposal_train_step": [vp, P(f32), P(f32), P(f32), C.c_size_t, f32, P(f32), P(f32)],
        "mcrt_proposal_apply_gradient": [vp, P(f32), f32],
        "mcrt_proposal_get_adam": [vp, P(f32), P(f32), C.c_size_t, P(C.c_int64)],
        "mcrt_proposal_set_adam": [vp, P(f32), P(f32), C.c_size_t, C.c_int64],
        "mcrt_proposal_set_training": [vp, i32],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = C.c_int
    L.mcrt_status_string.restype = C.c_char_p
    L.mcrt_last_error.restype = C.c_char_p
    abi = C.c_int32()
    L.mcrt_version(C.byref(abi))
    if abi.value != ABI_VERSION:
        raise ImportError("libmcrt.so has ABI version %d, this binding expects %d: rebuild it" % (abi.value, ABI_VERSION))
    _lib = L
    return L


def lib():
    return _load()


def exported_names():
    """Names of the C entry points the binding uses."""
    _load()
    return sorted(n for n in dir(_lib) if n.startswith("mcrt_"))


def _status_name(s):
    try:
        return _load().mcrt_status_string(int(s)).decode()
    except Exception:  # pragma: no cover
        return "status"


def _ptr(a, t):
    return a.ctypes.data_as(C.POINTER(t))


# ---------------------------------------------------------------------------
# Same-name wrappers of the C entry points (argument marshalling only)
# ---------------------------------------------------------------------------
def _check(rc, ctx=None):
    if rc != MCRT_OK:
        msg = _load().mcrt_last_error(ctx).decode() if ctx is not None else _load().mcrt_last_error(None).decode()
        raise McrtError(rc, msg)


def mcrt_create(device: int = 0, stream=None):
    h = C.c_void_p()
    if stream is None:
        try:
            import torch
            stream = torch.cuda.current_stream(device).cuda_stream
        except Exception:
            stream = 0
    _check(_load().mcrt_create(C.byref(h), device, C.c_void_p(int(stream) if stream else None)))
    return h


def mcrt_destroy(ctx):
    _check(_load().mcrt_destroy(ctx))


def mcrt_launch_count(ctx) -> int:
    v = C.c_uint64()
    _check(_load().mcrt_launch_count(ctx, C.byref(v)), ctx)
    return v.value


def mcrt_scene_create(ctx, desc: FieldDesc):
    h = C.c_void_p()
    _check(_load().mcrt_scene_create(ctx, C.byref(desc), C.byref(h)), ctx)
    return h


def mcrt_scene_destroy(scene):
    _check(_load().mcrt_scene_destroy(scene))


def mcrt_scene_build_majorants(ctx, scene, levels: int):
    _check(_load().mcrt_scene_build_majorants(scene, levels), ctx)


def mcrt_scene_levels(scene) -> int:
    v = C.c_int32()
    _check(_load().mcrt_scene_levels(scene, C.byref(v)))
    return v.value


def mcrt_scene_majorant_dims(ctx, scene, level: int):
    d = (C.c_int32 * 3)()
    _check(_load().mcrt_scene_majorant_dims(scene, level, d), ctx)
    return (d[0], d[1], d[2])


def mcrt_scene_read_majorants(ctx, scene, level: int) -> np.ndarray:
    dx, dy, dz = mcrt_scene_majorant_dims(ctx, scene, level)
    out = np.zeros(dx * dy * dz, dtype=np.float32)
    _check(_load().mcrt_scene_read_majorants(scene, level, _ptr(out, C.c_float), out.size), ctx)
    return out.reshape(dz, dy, dx)


def mcrt_scene_read_minorants(ctx, scene, level: int) -> np.ndarray:
    dx, dy, dz = mcrt_scene_majorant_dims(ctx, scene, level)
    out = np.zeros(dx * dy * dz, dtype=np.float32)
    _check(_load().mcrt_scene_read_minorants(scene, level, _ptr(out, C.c_float), out.size), ctx)
    return out.reshape(dz, dy, dx)


def mcrt_scene_build_octree(ctx, scene, levels: int = 0):
    _check(_load().mcrt_scene_build_octree(scene, levels), ctx)


def mcrt_scene_octree_levels(scene) -> int:
    v = C.c_int32()
    _check(_load().mcrt_scene_octree_levels(scene, C.byref(v)))
    return v.value


def mcrt_scene_octree_dims(ctx, scene, level: int):
    d = (C.c_int32 * 3)()
    _check(_load().mcrt_scene_octree_dims(scene, level, d), ctx)
    return (d[0], d[1], d[2])


def mcrt_scene_read_octree(ctx, scene, level: int):
    """(max, min) of octree level ``level``, each [z][y][x]."""
    dx, dy, dz = mcrt_scene_octree_dims(ctx, scene, level)
    mx = np.zeros(dx * dy * dz, dtype=np.float32)
    mn = np.zeros(dx * dy * dz, dtype=np.float32)
    _check(_load().mcrt_scene_read_octree(scene, level, _ptr(mx, C.c_float), _ptr(mn, C.c_float), mx.size), ctx)
    return mx.reshape(dz, dy, dx), mn.reshape(dz, dy, dx)


def mcrt_scene_set_clear_sky_phase(ctx, scene, phase: int):
    _check(_load().mcrt_scene_set_clear_sky_phase(scene, phase), ctx)


def mcrt_scene_set_ground_flat(ctx, scene, albedo: float):
    _check(_load().mcrt_scene_set_ground_flat(scene, albedo), ctx)


def mcrt_scene_set_ground_heightfield(ctx, scene, heights, albedo: float):
    """heights: [hny][hnx] km, numpy array or CUDA tensor."""
    if hasattr(heights, "is_cuda") and heights.is_cuda:
        import torch
        hh = heights.contiguous().to(torch.float32)
        ptr, mem = C.c_void_p(hh.data_ptr()), MCRT_MEM_DEVICE
    else:
        hh = np.ascontiguousarray(heights, dtype=np.float32)
        ptr, mem = C.c_void_p(hh.ctypes.data), MCRT_MEM_HOST
    hny, hnx = hh.shape
    _check(_load().mcrt_scene_set_ground_heightfield(scene, ptr, hnx, hny, mem, albedo), ctx)


def mcrt_debug_terrain(ctx, scene, o, d):
    oo = np.ascontiguousarray(o, dtype=np.float32).reshape(-1, 3)
    dd = np.ascontiguousarray(d, dtype=np.float32).reshape(-1, 3)
    t = np.zeros(oo.shape[0], dtype=np.float32)
    _check(_load().mcrt_debug_terrain(scene, oo.shape[0], _ptr(oo, C.c_float), _ptr(dd, C.c_float),
                                      _ptr(t, C.c_float)), ctx)
    return t


def mcrt_debug_terrain_height(ctx, scene, xy):
    p = np.ascontiguousarray(xy, dtype=np.float32).reshape(-1, 2)
    out = np.zeros((p.shape[0], 4), dtype=np.float32)
    _check(_load().mcrt_debug_terrain_height(scene, p.shape[0], _ptr(p, C.c_float), _ptr(out, C.c_float)), ctx)
    return out[:, 0], out[:, 1:]


def mcrt_scene_set_sun(ctx, scene, zenith_deg: float, azimuth_deg: float):
    _check(_load().mcrt_scene_set_sun(scene, zenith_deg, azimuth_deg), ctx)


def mcrt_trace_opts_default() -> TraceOpts:
    o = TraceOpts()
    _check(_load().mcrt_trace_opts_default(C.byref(o)))
    return o


def mcrt_trace_camera(ctx, scene, cam: CameraDesc, spp: int, seed: int, opts: TraceOpts, tally=None):
    h = tally if tally is not None else C.c_void_p()
    _check(_load().mcrt_trace_camera(scene, C.byref(cam), spp, seed, C.byref(opts), C.byref(h)), ctx)
    return h


def mcrt_trace_flux(ctx, scene, npaths: int, seed: int, opts: TraceOpts, tally=None):
    h = tally if tally is not None else C.c_void_p()
    _check(_load().mcrt_trace_flux(scene, npaths, seed, C.byref(opts), C.byref(h)), ctx)
    return h


def mcrt_trace_camera_noalloc(ctx, scene, cam: CameraDesc, spp: int, seed: int, opts: TraceOpts,
                              d_mean: int, d_stderr: int):
    """Camera trace writing mean / SE into caller-owned device buffers
    (addresses), with no device allocation inside the library."""
    _check(_load().mcrt_trace_camera_noalloc(scene, C.byref(cam), spp, seed, C.byref(opts),
                                             C.c_void_p(d_mean), C.c_void_p(d_stderr)), ctx)


def mcrt_tally_shape(ctx, tally):
    a, b = C.c_int32(), C.c_int32()
    _check(_load().mcrt_tally_shape(tally, C.byref(a), C.byref(b)), ctx)
    return a.value, b.value


def mcrt_tally_read(ctx, tally):
    nc, nq = mcrt_tally_shape(ctx, tally)
    m = nc * nq
    mean = np.zeros(m)
    se = np.zeros(m)
    n = np.zeros(m, dtype=np.uint64)
    _check(_load().mcrt_tally_read(tally, _ptr(mean, C.c_double), _ptr(se, C.c_double), _ptr(n, C.c_uint64), m), ctx)
    return mean.reshape(nc, nq), se.reshape(nc, nq), n.reshape(nc, nq)


def mcrt_tally_read_sums(ctx, tally):
    nc, nq = mcrt_tally_shape(ctx, tally)
    m = nc * nq
    s1 = np.zeros(m)
    s2 = np.zeros(m)
    _check(_load().mcrt_tally_read_sums(tally, _ptr(s1, C.c_double), _ptr(s2, C.c_double), m), ctx)
    return s1.reshape(nc, nq), s2.reshape(nc, nq)


def mcrt_tally_counters(ctx, tally) -> dict:
    c = np.zeros(len(COUNTER_NAMES), dtype=np.uint64)
    _check(_load().mcrt_tally_counters(tally, _ptr(c, C.c_uint64), c.size), ctx)
    return {k: int(v) for k, v in zip(COUNTER_NAMES, c)}


def mcrt_tally_kernel_ms(ctx, tally) -> float:
    v = C.c_float()
    _check(_load().mcrt_tally_kernel_ms(tally, C.byref(v)), ctx)
    return v.value


def mcrt_tally_destroy(tally):
    _check(_load().mcrt_tally_destroy(tally))


def mcrt_debug_dda(ctx, scene, o, d, tau_merge=1.0, finest_level=1, cap=4096, grid=MCRT_GRID_PYRAMID):
    o32 = np.ascontiguousarray(o, dtype=np.float32)
    d32 = np.ascontiguousarray(d, dtype=np.float32)
    cells = np.zeros((cap, 4), dtype=np.int32)
    tio = np.zeros((cap, 2), dtype=np.float32)
    n, st = C.c_int32(), C.c_int32()
    _check(_load().mcrt_debug_dda_grid(scene, _ptr(o32, C.c_float), _ptr(d32, C.c_float), tau_merge, finest_level,
                                       grid, _ptr(cells, C.c_int32), _ptr(tio, C.c_float), cap, C.byref(n),
                                       C.byref(st)), ctx)
    return cells[:n.value].copy(), tio[:n.value].copy(), st.value


def mcrt_debug_bounds_violations(ctx):
    """(checked build?, violations since the last call, first code)."""
    chk, n, code = C.c_int32(), C.c_uint64(), C.c_int32()
    _check(_load().mcrt_debug_bounds_violations(ctx, C.byref(chk), C.byref(n), C.byref(code)), ctx)
    return bool(chk.value), int(n.value), int(code.value)


def mcrt_debug_learned_records(ctx, scene, cam, n: int, seed: int, opts, cap: int = 1 << 16):
    """Online-training records of one learned trace (no training): a dict of
    feat (k x 9), dir (k x 3), before, w_omega, own, target, path, and the
    number of records the trace produced.  ``cam`` a CameraDesc (n = spp) or
    None for ground flux (n = paths)."""
    feat = np.zeros((cap, 9), np.float32)
    dirs = np.zeros((cap, 3), np.float32)
    val = np.zeros((cap, 4), np.float32)
    path = np.zeros(cap, np.uint64)
    cnt = C.c_int32()
    camp = C.byref(cam) if cam is not None else None
    _check(_load().mcrt_debug_learned_records(scene, camp, n, seed, C.byref(opts), cap, _ptr(feat, C.c_float),
                                              _ptr(dirs, C.c_float), _ptr(val, C.c_float),
                                              _ptr(path, C.c_uint64), C.byref(cnt)), ctx)
    k = min(cap, cnt.value)
    return {"feat": feat[:k], "dir": dirs[:k], "before": val[:k, 0], "w_omega": val[:k, 1], "own": val[:k, 2],
            "target": val[:k, 3], "path": path[:k], "count": int(cnt.value)}


def mcrt_debug_pool_usage(ctx, reset_high: bool = False):
    """(bytes in use, most bytes in use since the last reset) of the device's
    stream-ordered memory pool; reset_high then resets the high mark."""
    cur, high = C.c_uint64(), C.c_uint64()
    _check(_load().mcrt_debug_pool_usage(ctx, 1 if reset_high else 0, C.byref(cur), C.byref(high)), ctx)
    return int(cur.value), int(high.value)


def mcrt_debug_philox(ctx, ctr, key) -> np.ndarray:
    ctr = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(-1, 4))
    key = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(-1, 2))
    out = np.zeros_like(ctr)
    _check(_load().mcrt_debug_philox(ctx, _ptr(ctr, C.c_uint32), _ptr(key, C.c_uint32), _ptr(out, C.c_uint32),
                                     ctr.shape[0]), ctx)
    return out


# ---------------------------------------------------------------------------
# Convenience objects
# ---------------------------------------------------------------------------
class Context:
    def __init__(self, device: int = 0, stream=None):
        self.device = device
        self.h = mcrt_create(device, stream)

    def close(self):
        if self.h:
            mcrt_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def launches(self) -> int:
        return mcrt_launch_count(self.h)


@dataclass
class Result:
    mean: np.ndarray
    se: np.ndarray
    n: np.ndarray
    kernel_ms: float
    counters: dict


class Scene:
    """A field on the device with its majorant pyramid."""

    def __init__(self, ctx: Context, k, dx, dy, dz, k_clear=0.0, ssa_clear=1.0, ssa_cloud=1.0, g=0.85,
                 storage=MCRT_STORAGE_F32, levels=0, albedo=0.0, sun_zenith_deg=0.0, sun_azimuth_deg=0.0):
        self.ctx = ctx
        desc = FieldDesc()
        if hasattr(k, "is_cuda") and k.is_cuda:
            import torch
            kk = k.contiguous().to(torch.float32)
            nz, ny, nx = kk.shape
            desc.ext = C.c_void_p(kk.data_ptr())
            desc.ext_mem = MCRT_MEM_DEVICE
            self._keep = kk
        else:
            if hasattr(k, "numpy"):
                k = k.numpy()
            kk = np.ascontiguousarray(k, dtype=np.float32)
            nz, ny, nx = kk.shape
            desc.ext = C.c_void_p(kk.ctypes.data)
            desc.ext_mem = MCRT_MEM_HOST
            self._keep = kk
        desc.nx, desc.ny, desc.nz = nx, ny, nz
        desc.dx, desc.dy, desc.dz = dx, dy, dz
        desc.k_clear, desc.ssa_clear, desc.ssa_cloud, desc.hg_g = k_clear, ssa_clear, ssa_cloud, g
        desc.storage = storage
        self.shape_xyz = (nx, ny, nz)
        self.h = mcrt_scene_create(ctx.h, desc)
        self._keep = None
        mcrt_scene_build_majorants(ctx.h, self.h, levels)
        mcrt_scene_set_ground_flat(ctx.h, self.h, albedo)
        mcrt_scene_set_sun(ctx.h, self.h, sun_zenith_deg, sun_azimuth_deg)

    @classmethod
    def from_spec(cls, ctx: Context, spec, storage=MCRT_STORAGE_F32, k=None):
        return cls(ctx, spec.k if k is None else k, spec.dx, spec.dy, spec.dz, k_clear=spec.k_clear,
                   ssa_clear=spec.ssa_clear, ssa_cloud=spec.ssa_cloud, g=spec.g, storage=storage,
                   levels=spec.levels, albedo=spec.ground_albedo, sun_zenith_deg=spec.sun_zenith_deg,
                   sun_azimuth_deg=spec.sun_azimuth_deg)

    def close(self):
        if self.h:
            mcrt_scene_destroy(self.h)
            self.h = None

    @property
    def levels(self):
        return mcrt_scene_levels(self.h)

    def majorants(self, level):
        return mcrt_scene_read_majorants(self.ctx.h, self.h, level)

    def minorants(self, level):
        return mcrt_scene_read_minorants(self.ctx.h, self.h, level)

    def build_octree(self, levels=0):
        """Build the paper's 2^L octree beside the pyramid (traces select it
        with grid=MCRT_GRID_OCTREE)."""
        mcrt_scene_build_octree(self.ctx.h, self.h, levels)

    @property
    def octree_levels(self):
        return mcrt_scene_octree_levels(self.h)

    def octree(self, level):
        return mcrt_scene_read_octree(self.ctx.h, self.h, level)

    def set_heightfield(self, heights, albedo):
        mcrt_scene_set_ground_heightfield(self.ctx.h, self.h, heights, albedo)

    def terrain_hit(self, o, d):
        return mcrt_debug_terrain(self.ctx.h, self.h, o, d)

    def terrain_height(self, xy):
        return mcrt_debug_terrain_height(self.ctx.h, self.h, xy)

    def dda(self, o, d, tau_merge=1.0, finest_level=1, cap=4096, grid=MCRT_GRID_PYRAMID):
        return mcrt_debug_dda(self.ctx.h, self.h, o, d, tau_merge, finest_level, cap, grid)

    @staticmethod
    def _opts(**kw):
        o = mcrt_trace_opts_default()
        for k, v in kw.items():
            if k == "cancel_flag":
                o.cancel_flag = C.c_void_p(v)
            elif k == "proposal":
                o.proposal = v.h if hasattr(v, "h") else v
            else:
                setattr(o, k, v)
        return o

    def _result(self, t, read_counters):
        mean, se, n = mcrt_tally_read(self.ctx.h, t)
        ms = mcrt_tally_kernel_ms(self.ctx.h, t)
        cnt = mcrt_tally_counters(self.ctx.h, t) if read_counters else {}
        return Result(mean, se, n, ms, cnt)

    def learned_records(self, cam, n, seed, cap=1 << 16, **opts):
        """Online-training records of one learned trace (no training) of a
        camera (``cam``, n = spp) or of ground flux (``cam`` None, n paths)."""
        cd = None
        if cam is not None:
            cd = CameraDesc()
            for i in range(3):
                cd.pos[i], cd.target[i], cd.up[i] = cam.pos[i], cam.target[i], cam.up[i]
            cd.fov_deg, cd.width, cd.height = cam.fov_deg, cam.width, cam.height
        return mcrt_debug_learned_records(self.ctx.h, self.h, cd, n, seed, self._opts(**opts), cap)

    def trace_camera(self, cam, spp, seed, tally=None, **opts):
        cd = CameraDesc()
        for i in range(3):
            cd.pos[i], cd.target[i], cd.up[i] = cam.pos[i], cam.target[i], cam.up[i]
        cd.fov_deg, cd.width, cd.height = cam.fov_deg, cam.width, cam.height
        o = self._opts(**opts)
        t = mcrt_trace_camera(self.ctx.h, self.h, cd, spp, seed, o, tally)
        try:
            r = self._result(t, o.count_events)
        finally:
            if tally is None:
                mcrt_tally_destroy(t)
        r.mean = r.mean.reshape(cam.height, cam.width)
        r.se = r.se.reshape(cam.height, cam.width)
        r.n = r.n.reshape(cam.height, cam.width)
        return r

    def trace_flux(self, npaths, seed, tally=None, **opts):
        o = self._opts(**opts)
        t = mcrt_trace_flux(self.ctx.h, self.h, npaths, seed, o, tally)
        try:
            r = self._result(t, o.count_events)
        finally:
            if tally is None:
                mcrt_tally_destroy(t)
        r.mean = r.mean.reshape(3)
        r.se = r.se.reshape(3)
        r.n = r.n.reshape(3)
        return r


# ---------------------------------------------------------------------------
# Learned proposal
# ---------------------------------------------------------------------------
def mcrt_proposal_create(ctx, seed: int):
    h = C.c_void_p()
    _check(_load().mcrt_proposal_create(ctx, seed, C.byref(h)), ctx)
    return h


def mcrt_proposal_destroy(prop):
    _check(_load().mcrt_proposal_destroy(prop))


def mcrt_proposal_set_params(ctx, prop, params):
    p = np.ascontiguousarray(params, dtype=np.float32)
    _check(_load().mcrt_proposal_set_params(prop, _ptr(p, C.c_float), p.size), ctx)


def mcrt_proposal_get_params(ctx, prop) -> np.ndarray:
    n = C.c_int32()
    _load().mcrt_proposal_nparams(C.byref(n))
    p = np.zeros(n.value, dtype=np.float32)
    _check(_load().mcrt_proposal_get_params(prop, _ptr(p, C.c_float), p.size), ctx)
    return p


def mcrt_proposal_eval(ctx, prop, features):
    f = np.ascontiguousarray(features, dtype=np.float32).reshape(-1, 9)
    mix = np.zeros((f.shape[0], 40), dtype=np.float32)
    raw = np.zeros((f.shape[0], 40), dtype=np.float32)
    _check(_load().mcrt_proposal_eval(prop, _ptr(f, C.c_float), f.shape[0], _ptr(mix, C.c_float),
                                      _ptr(raw, C.c_float)), ctx)
    return mix, raw


def mcrt_proposal_train_step(ctx, prop, features, dirs, targets, lr=0.0):
    f = np.ascontiguousarray(features, dtype=np.float32).reshape(-1, 9)
    d = np.ascontiguousarray(dirs, dtype=np.float32).reshape(-1, 3)
    t = np.ascontiguousarray(targets, dtype=np.float32).reshape(-1)
    g = np.zeros(11560, dtype=np.float32)
    loss = C.c_float()
    _check(_load().mcrt_proposal_train_step(prop, _ptr(f, C.c_float), _ptr(d, C.c_float), _ptr(t, C.c_float),
                                            f.shape[0], lr, C.byref(loss), _ptr(g, C.c_float)), ctx)
    return loss.value, g


class Proposal:
    """Learned scattering proposal network on the device."""

    def __init__(self, ctx: Context, seed: int = 0, params=None, training=MCRT_TRAIN_TENSOR):
        self.ctx = ctx
        self.h = mcrt_proposal_create(ctx.h, seed)
        if params is not None:
            mcrt_proposal_set_params(ctx.h, self.h, params)
        _check(_load().mcrt_proposal_set_training(self.h, training), ctx.h)

    def close(self):
        if self.h:
            mcrt_proposal_destroy(self.h)
            self.h = None

    @property
    def params(self):
        return mcrt_proposal_get_params(self.ctx.h, self.h)

    @params.setter
    def params(self, p):
        mcrt_proposal_set_params(self.ctx.h, self.h, p)

    def eval(self, features):
        return mcrt_proposal_eval(self.ctx.h, self.h, features)

    def train_step(self, features, dirs, targets, lr=0.0):
        return mcrt_proposal_train_step(self.ctx.h, self.h, features, dirs, targets, lr)

    @property
    def adam_state(self):
        """(first moments, second moments, step count) of Adam."""
        mm = np.zeros(11560, dtype=np.float32)
        vv = np.zeros(11560, dtype=np.float32)
        st = C.c_int64()
        _check(_load().mcrt_proposal_get_adam(self.h, _ptr(mm, C.c_float), _ptr(vv, C.c_float), 11560,
                                              C.byref(st)), self.ctx.h)
        return mm, vv, int(st.value)

    @adam_state.setter
    def adam_state(self, state):
        mm, vv, st = state
        mm = np.ascontiguousarray(mm, dtype=np.float32)
        vv = np.ascontiguousarray(vv, dtype=np.float32)
        _check(_load().mcrt_proposal_set_adam(self.h, _ptr(mm, C.c_float), _ptr(vv, C.c_float), mm.size, int(st)),
               self.ctx.h)

    def apply_gradient(self, grad, lr=1e-3):
        """One Adam step with a given gradient (data-parallel training)."""
        g = np.ascontiguousarray(grad, dtype=np.float32).ravel()
        if g.size != 11560:
            raise ValueError("gradient must have 11,560 entries")
        _check(_load().mcrt_proposal_apply_gradient(self.h, _ptr(g, C.c_float), float(lr)), self.ctx.h)


# ---------------------------------------------------------------------------
# Batches
# ---------------------------------------------------------------------------
def make_batch_items(items):
    """items: sequence of (scene handle, k_gas, sun zenith, sun azimuth, npaths, seed)."""
    arr = (BatchItem * len(items))()
    for i, (sc, kg, z, a, n, seed) in enumerate(items):
        arr[i].scene = sc.h if hasattr(sc, "h") else sc
        if arr[i].scene is None:
            arr[i].scene = 0
        arr[i].k_gas, arr[i].sun_zenith_deg, arr[i].sun_azimuth_deg = kg, z, a
        arr[i].npaths, arr[i].seed = n, seed
    return arr


def mcrt_trace_batch(ctx, items, opts: TraceOpts, tally=None):
    arr = items if isinstance(items, C.Array) else make_batch_items(items)
    h = tally if tally is not None else C.c_void_p()
    _check(_load().mcrt_trace_batch(ctx, arr, len(arr), C.byref(opts), C.byref(h)), ctx)
    return h


def mcrt_autotune_batch(ctx, items, fraction: float, opts: TraceOpts):
    arr = items if isinstance(items, C.Array) else make_batch_items(items)
    best = C.c_float()
    _check(_load().mcrt_autotune_batch(ctx, arr, len(arr), fraction, C.byref(opts), C.byref(best)), ctx)
    return opts, best.value


def trace_batch(ctx: Context, items, tally=None, **kw):
    """Returns Result with mean / se of shape (n_items, 5):
    T_dir, T_dif, T_tot, dT_tot/dg, dT_tot/dalpha."""
    o = Scene._opts(**kw)
    t = mcrt_trace_batch(ctx.h, items, o, tally)
    try:
        mean, se, n = mcrt_tally_read(ctx.h, t)
        ms = mcrt_tally_kernel_ms(ctx.h, t)
        cnt = mcrt_tally_counters(ctx.h, t) if o.count_events else {}
    finally:
        if tally is None:
            mcrt_tally_destroy(t)
    return Result(mean.reshape(-1, 5), se.reshape(-1, 5), n.reshape(-1, 5), ms, cnt)


def mcrt_batch_plan_create(ctx, items, opts: TraceOpts):
    arr = items if isinstance(items, C.Array) else make_batch_items(items)
    h = C.c_void_p()
    _check(_load().mcrt_batch_plan_create(ctx, arr, len(arr), C.byref(opts), C.byref(h)), ctx)
    return h


def mcrt_batch_plan_set_seeds(ctx, plan, seeds):
    s = np.ascontiguousarray(seeds, dtype=np.uint64)
    _check(_load().mcrt_batch_plan_set_seeds(plan, _ptr(s, C.c_uint64), s.size), ctx)


def mcrt_batch_plan_run(ctx, plan, n_items: int):
    mean = np.zeros(n_items * 5)
    se = np.zeros(n_items * 5)
    ms = C.c_float()
    _check(_load().mcrt_batch_plan_run(plan, _ptr(mean, C.c_double), _ptr(se, C.c_double), mean.size,
                                       C.byref(ms)), ctx)
    return mean.reshape(n_items, 5), se.reshape(n_items, 5), ms.value


def mcrt_batch_plan_destroy(plan):
    _check(_load().mcrt_batch_plan_destroy(plan))


class BatchPlan:
    """A batch captured into a CUDA graph; ``run()`` replays it."""

    def __init__(self, ctx: Context, items, **kw):
        self.ctx = ctx
        self.n = len(items)
        self.h = mcrt_batch_plan_create(ctx.h, items, Scene._opts(**kw))

    def set_seeds(self, seeds):
        mcrt_batch_plan_set_seeds(self.ctx.h, self.h, seeds)

    def run(self):
        mean, se, ms = mcrt_batch_plan_run(self.ctx.h, self.h, self.n)
        return Result(mean, se, None, ms, {})

    def close(self):
        if self.h:
            mcrt_batch_plan_destroy(self.h)
            self.h = None
