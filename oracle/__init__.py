"""FP64 CPU oracle of the null-collision path tracer -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it and
shares no code with it; both sides only see the same seeded scene arrays.

The C source (``mcrt_oracle.c``) is compiled with plain gcc, ``-O2
-ffp-contract=off`` (no fused multiply-add, so the FP32 traversal spec is
reproduced operation by operation).  This module is argument marshalling
around it plus small pure-Python/numpy helpers that follow the paper:

* Sec. 2.3 (steps 1-5, Eq. 2): null-collision direct transmissivity.
* Sec. 2.4 / 3.1.1: piecewise-uniform majorant, max over merged voxels.
* Sec. 4.1: backward rendering with local estimates toward the sun.
* Sec. 5.2: forward analog flux, diffuse once scattered.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mcrt_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (no CUDA involved)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class OrcScene(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("dx", C.c_float), ("dy", C.c_float), ("dz", C.c_float),
        ("k", C.POINTER(C.c_float)),
        ("levels", C.c_int32),
        ("pyr", C.POINTER(C.c_float)),
        ("tau_merge", C.c_float),
        ("finest_level", C.c_int32),
        ("k_clear", C.c_double),
        ("ssa_clear", C.c_double), ("ssa_cloud", C.c_double),
        ("g", C.c_double),
        ("ground_albedo", C.c_double),
        ("sun", C.c_double * 3),
        ("sun_mode", C.c_int32),
        ("max_order", C.c_int32),
        ("k_gas", C.c_double),
        ("max_steps", C.c_int64),
        ("mlp", C.POINTER(C.c_double)),
        ("n_learned", C.c_int32),
        ("mis_alpha", C.c_double),
        ("hf", C.POINTER(C.c_float)),
        ("hnx", C.c_int32), ("hny", C.c_int32),
        ("hmax", C.c_double),
        ("pyr_min", C.POINTER(C.c_float)),
        ("clear_phase", C.c_int32),
        ("grid", C.c_int32),
        ("oct_levels", C.c_int32),
        ("oct", C.POINTER(C.c_float)),
        ("oct_min", C.POINTER(C.c_float)),
    ]


class OrcCamera(C.Structure):
    _fields_ = [
        ("pos", C.c_double * 3), ("target", C.c_double * 3), ("up", C.c_double * 3),
        ("fov_deg", C.c_double),
        ("width", C.c_int32), ("height", C.c_int32),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            f32p = C.POINTER(C.c_float)
            f64p = C.POINTER(C.c_double)
            u32p = C.POINTER(C.c_uint32)
            i32p = C.POINTER(C.c_int32)
            i64p = C.POINTER(C.c_int64)
            sp = C.POINTER(OrcScene)
            L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.orc_philox_batch.argtypes = [u32p, u32p, u32p, C.c_int64]
            L.orc_u01_from_u32.argtypes = [C.c_uint32]
            L.orc_u01_from_u32.restype = C.c_double
            L.orc_bf16_round_nearest.argtypes = [C.c_float]
            L.orc_bf16_round_nearest.restype = C.c_float
            L.orc_bf16_round_up.argtypes = [C.c_float]
            L.orc_bf16_round_up.restype = C.c_float
            L.orc_level_dims.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int)]
            L.orc_pyramid_size.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int]
            L.orc_pyramid_size.restype = C.c_int64
            L.orc_build_pyramid.argtypes = [f32p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, f32p]
            L.orc_build_pyramid_min.argtypes = [f32p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, f32p]
            L.orc_octree_dims.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int)]
            L.orc_octree_size.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int]
            L.orc_octree_size.restype = C.c_int64
            L.orc_build_octree.argtypes = [f32p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, f32p, f32p]
            L.orc_bf16_round_down.argtypes = [C.c_float]
            L.orc_bf16_round_down.restype = C.c_float
            L.orc_dda_spec.argtypes = [sp, f32p, f32p, C.c_int, i32p, f32p, i32p]
            L.orc_dda_bruteforce.argtypes = [sp, f64p, f64p, C.c_double, C.c_int, i32p, f64p, i32p]
            L.orc_hg_pdf.argtypes = [C.c_double, C.c_double]
            L.orc_hg_pdf.restype = C.c_double
            L.orc_hg_sample_mu.argtypes = [C.c_double, C.c_double]
            L.orc_hg_sample_mu.restype = C.c_double
            L.orc_rayleigh_pdf.argtypes = [C.c_double]
            L.orc_rayleigh_pdf.restype = C.c_double
            L.orc_rayleigh_sample_mu.argtypes = [C.c_double]
            L.orc_rayleigh_sample_mu.restype = C.c_double
            L.orc_hg_sample_dirs.argtypes = [C.c_double, f64p, f64p, C.c_int64, f64p]
            L.orc_transmissivity.argtypes = [sp, f64p, f64p, C.c_uint64, C.c_uint64]
            L.orc_transmissivity.restype = C.c_double
            L.orc_first_collision_distance.argtypes = [sp, f64p, f64p, C.c_uint64, C.c_uint64]
            L.orc_first_collision_distance.restype = C.c_double
            L.orc_trace_camera.argtypes = [sp, C.POINTER(OrcCamera), C.c_uint32, C.c_uint64,
                                           C.c_int64, C.c_int64, f64p, C.c_int, i64p]
            L.orc_trace_flux.argtypes = [sp, C.c_uint64, C.c_uint64, C.c_uint64, f64p, C.c_int, i64p]
            L.orc_trace_forward.argtypes = [sp, C.c_uint64, C.c_uint64, C.c_uint64, f64p, C.c_int, i64p]
            L.orc_forward_balance_residual.argtypes = [sp, C.c_uint64, C.c_uint64, C.c_uint64]
            L.orc_terrain_height.argtypes = [sp, C.c_double, C.c_double, f64p]
            L.orc_terrain_height.restype = C.c_double
            L.orc_terrain_hit.argtypes = [sp, f64p, f64p, f64p, i64p, C.POINTER(C.c_int)]
            L.orc_terrain_hit.restype = C.c_int
            L.orc_forward_balance_residual.restype = C.c_double
            _lib = L
    return _lib


def _ptr(a, t):
    return a.ctypes.data_as(C.POINTER(t))


def default_threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return max(1, os.cpu_count() or 1)


# --------------------------------------------------------------------------
# Philox and uniforms
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 on arrays of counters (n, 4) and keys (n, 2)."""
    ctr = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(-1, 4))
    key = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(-1, 2))
    out = np.zeros_like(ctr)
    lib().orc_philox_batch(_ptr(ctr, C.c_uint32), _ptr(key, C.c_uint32), _ptr(out, C.c_uint32), ctr.shape[0])
    return out


def u01(x) -> np.ndarray:
    """Uniform in (0, 1] from a 32-bit word: ((x >> 8) + 1) * 2^-24."""
    x = np.asarray(x, dtype=np.uint32)
    return ((x >> np.uint32(8)).astype(np.float64) + 1.0) * 2.0 ** -24


# --------------------------------------------------------------------------
# Majorant pyramid
# --------------------------------------------------------------------------
def level_dims(shape_xyz, level):
    d = (C.c_int * 3)()
    lib().orc_level_dims(shape_xyz[0], shape_xyz[1], shape_xyz[2], level, d)
    return (d[0], d[1], d[2])


def build_pyramid(k_zyx: np.ndarray, levels: int, round_up_bf16: bool = False):
    """Majorant pyramid of a field stored [z][y][x]; returns a list of
    arrays [z][y][x] for levels 1..levels (exact FP32 max, Sec. 3.1.1)."""
    k = np.ascontiguousarray(k_zyx, dtype=np.float32)
    nz, ny, nx = k.shape
    tot = lib().orc_pyramid_size(nx, ny, nz, levels)
    out = np.zeros(tot, dtype=np.float32)
    rc = lib().orc_build_pyramid(_ptr(k, C.c_float), nx, ny, nz, levels, int(round_up_bf16), _ptr(out, C.c_float))
    if rc != 0:
        raise ValueError("bad pyramid request")
    res, off = [], 0
    for l in range(1, levels + 1):
        dx, dy, dz = level_dims((nx, ny, nz), l)
        n = dx * dy * dz
        res.append(out[off:off + n].reshape(dz, dy, dx))
        off += n
    return res


def build_pyramid_min(k_zyx: np.ndarray, levels: int, round_nearest_bf16: bool = False):
    """Minorant pyramid (exact FP32 min per cell over its existing children;
    with round_nearest_bf16, the min of the BF16-rounded voxels)."""
    k = np.ascontiguousarray(k_zyx, dtype=np.float32)
    nz, ny, nx = k.shape
    tot = lib().orc_pyramid_size(nx, ny, nz, levels)
    out = np.zeros(tot, dtype=np.float32)
    rc = lib().orc_build_pyramid_min(_ptr(k, C.c_float), nx, ny, nz, levels, int(round_nearest_bf16),
                                     _ptr(out, C.c_float))
    if rc != 0:
        raise ValueError("bad pyramid request")
    res, off = [], 0
    for l in range(1, levels + 1):
        dx, dy, dz = level_dims((nx, ny, nz), l)
        n = dx * dy * dz
        res.append(out[off:off + n].reshape(dz, dy, dx))
        off += n
    return res


def octree_levels(shape_xyz) -> int:
    """Octree levels above the voxels up to the first level with one cell."""
    L = 0
    while (1 << L) < max(shape_xyz):
        L += 1
    return max(L, 1)


def octree_dims(shape_xyz, level):
    d = (C.c_int * 3)()
    lib().orc_octree_dims(shape_xyz[0], shape_xyz[1], shape_xyz[2], level, d)
    return (d[0], d[1], d[2])


def build_octree(k_zyx: np.ndarray, levels: int, round_nearest_bf16: bool = False):
    """The paper's octree (Sec. 3.1.1): per level 1..levels, the max and the
    min over each aligned block of 2^L voxels per axis.  Returns two lists
    of arrays [z][y][x]."""
    k = np.ascontiguousarray(k_zyx, dtype=np.float32)
    nz, ny, nx = k.shape
    tot = lib().orc_octree_size(nx, ny, nz, levels)
    mx = np.zeros(tot, dtype=np.float32)
    mn = np.zeros(tot, dtype=np.float32)
    rc = lib().orc_build_octree(_ptr(k, C.c_float), nx, ny, nz, levels, int(round_nearest_bf16),
                                _ptr(mx, C.c_float), _ptr(mn, C.c_float))
    if rc != 0:
        raise ValueError("bad octree request")
    rmax, rmin, off = [], [], 0
    for l in range(1, levels + 1):
        dx, dy, dz = octree_dims((nx, ny, nz), l)
        n = dx * dy * dz
        rmax.append(mx[off:off + n].reshape(dz, dy, dx))
        rmin.append(mn[off:off + n].reshape(dz, dy, dx))
        off += n
    return rmax, rmin


def bf16_round_down(x: float) -> float:
    return lib().orc_bf16_round_down(float(x))


def bf16_round_nearest(x: float) -> float:
    return lib().orc_bf16_round_nearest(float(x))


def bf16_round_up(x: float) -> float:
    return lib().orc_bf16_round_up(float(x))


# --------------------------------------------------------------------------
# Scene
# --------------------------------------------------------------------------
@dataclass
class Scene:
    """Oracle view of a scene.  ``k`` is [z][y][x] FP32 extinction [km^-1]."""
    k: np.ndarray
    dx: float
    dy: float
    dz: float
    levels: int
    tau_merge: float = 1.0
    finest_level: int = 0
    k_clear: float = 0.0
    ssa_clear: float = 1.0
    ssa_cloud: float = 1.0
    g: float = 0.85
    ground_albedo: float = 0.0
    sun_zenith_deg: float = 0.0
    sun_azimuth_deg: float = 0.0
    sun_mode: int = 0
    max_order: int = 0
    k_gas: float = 0.0
    max_steps: int = 1 << 22
    bf16: bool = False
    mlp: object = None            # learned proposal parameters (11,560 float64) or None
    n_learned: int = 8
    mis_alpha: float = 0.5
    heights: object = None        # heightfield ground [hny][hnx] float32 km (periodic), or None: flat
    clear_phase: int = 0          # clear-air phase function: 0 HG (the cloud's g), 1 Rayleigh
    grid: int = 0                 # tracked grid: 0 the 8^L pyramid, 1 the paper's 2^L octree
    _keep: list = field(default_factory=list, repr=False)

    def sun_dir(self):
        th = math.radians(self.sun_zenith_deg)
        ph = math.radians(self.sun_azimuth_deg)
        return (math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th))

    def struct(self) -> OrcScene:
        k = np.ascontiguousarray(self.k, dtype=np.float32)
        if self.bf16:
            k = bf16_round_nearest_array(k)
        nz, ny, nx = k.shape
        pyr = build_pyramid(k, self.levels, round_up_bf16=False) if not self.bf16 else \
            build_pyramid(np.ascontiguousarray(self.k, dtype=np.float32), self.levels, round_up_bf16=True)
        flat = np.ascontiguousarray(np.concatenate([p.ravel() for p in pyr]).astype(np.float32))
        pmin = build_pyramid_min(np.ascontiguousarray(self.k, dtype=np.float32), self.levels,
                                 round_nearest_bf16=bool(self.bf16))
        flat_min = np.ascontiguousarray(np.concatenate([p.ravel() for p in pmin]).astype(np.float32))
        self._keep = [k, flat, flat_min]
        s = OrcScene()
        s.nx, s.ny, s.nz = nx, ny, nz
        s.dx, s.dy, s.dz = self.dx, self.dy, self.dz
        s.k = _ptr(k, C.c_float)
        s.levels = self.levels
        s.pyr = _ptr(flat, C.c_float)
        s.pyr_min = _ptr(flat_min, C.c_float)
        s.tau_merge = self.tau_merge
        s.finest_level = self.finest_level
        s.k_clear = self.k_clear
        s.ssa_clear = self.ssa_clear
        s.ssa_cloud = self.ssa_cloud
        s.g = self.g
        s.ground_albedo = self.ground_albedo
        sd = self.sun_dir()
        for i in range(3):
            s.sun[i] = sd[i]
        s.sun_mode = self.sun_mode
        s.max_order = self.max_order
        s.k_gas = self.k_gas
        s.max_steps = self.max_steps
        if self.mlp is not None:
            mp = np.ascontiguousarray(self.mlp, dtype=np.float64)
            self._keep.append(mp)
            s.mlp = _ptr(mp, C.c_double)
        s.n_learned = self.n_learned
        s.mis_alpha = self.mis_alpha
        s.clear_phase = self.clear_phase
        s.grid = self.grid
        if self.grid == 1:
            ol = octree_levels((nx, ny, nz))
            omax, omin = build_octree(np.ascontiguousarray(self.k, dtype=np.float32), ol,
                                      round_nearest_bf16=bool(self.bf16))
            fo = np.ascontiguousarray(np.concatenate([a.ravel() for a in omax]))
            fm = np.ascontiguousarray(np.concatenate([a.ravel() for a in omin]))
            self._keep += [fo, fm]
            s.oct_levels = ol
            s.oct = _ptr(fo, C.c_float)
            s.oct_min = _ptr(fm, C.c_float)
        if self.heights is not None:
            hf = np.ascontiguousarray(self.heights, dtype=np.float32)
            self._keep.append(hf)
            s.hf = _ptr(hf, C.c_float)
            s.hny, s.hnx = hf.shape
            s.hmax = float(hf.max())
        return s


def bf16_round_nearest_array(k: np.ndarray) -> np.ndarray:
    """Round-to-nearest-even to bfloat16, values kept as float32 (numpy)."""
    u = np.ascontiguousarray(k, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).reshape(k.shape)


@dataclass
class Camera:
    pos: tuple
    target: tuple
    up: tuple
    fov_deg: float
    width: int
    height: int

    def struct(self) -> OrcCamera:
        c = OrcCamera()
        for i in range(3):
            c.pos[i] = self.pos[i]
            c.target[i] = self.target[i]
            c.up[i] = self.up[i]
        c.fov_deg = self.fov_deg
        c.width, c.height = self.width, self.height
        return c


# --------------------------------------------------------------------------
# Traversal
# --------------------------------------------------------------------------
def dda_spec(scene: Scene, o, d, cap: int = 4096):
    """FP32 traversal spec: leaves (level, ix, iy, iz) and (t_in, t_out)."""
    s = scene.struct()
    o32 = np.asarray(o, dtype=np.float32)
    d32 = np.asarray(d, dtype=np.float32)
    cells = np.zeros((cap, 4), dtype=np.int32)
    tio = np.zeros((cap, 2), dtype=np.float32)
    st = C.c_int32(0)
    n = lib().orc_dda_spec(C.byref(s), _ptr(o32, C.c_float), _ptr(d32, C.c_float), cap,
                           _ptr(cells, C.c_int32), _ptr(tio, C.c_float), C.byref(st))
    return cells[:n].copy(), tio[:n].copy(), st.value


def dda_bruteforce(scene: Scene, o, d, tmax: float = 1e30, cap: int = 4096):
    s = scene.struct()
    o64 = np.asarray(o, dtype=np.float64)
    d64 = np.asarray(d, dtype=np.float64)
    cells = np.zeros((cap, 4), dtype=np.int32)
    tio = np.zeros((cap, 2), dtype=np.float64)
    st = C.c_int32(0)
    n = lib().orc_dda_bruteforce(C.byref(s), _ptr(o64, C.c_double), _ptr(d64, C.c_double), tmax, cap,
                                 _ptr(cells, C.c_int32), _ptr(tio, C.c_double), C.byref(st))
    return cells[:n].copy(), tio[:n].copy(), st.value


# --------------------------------------------------------------------------
# Estimators
# --------------------------------------------------------------------------
def hg_pdf(g, mu):
    return lib().orc_hg_pdf(float(g), float(mu))


def rayleigh_pdf(mu):
    return lib().orc_rayleigh_pdf(float(mu))


def rayleigh_sample_mu(xi):
    return lib().orc_rayleigh_sample_mu(float(xi))


def hg_sample_mu(g, xi):
    return lib().orc_hg_sample_mu(float(g), float(xi))


def hg_sample_dirs(g, d, xi):
    d = np.ascontiguousarray(d, dtype=np.float64).reshape(-1, 3)
    xi = np.ascontiguousarray(xi, dtype=np.float64).reshape(-1, 2)
    out = np.zeros_like(d)
    lib().orc_hg_sample_dirs(float(g), _ptr(d, C.c_double), _ptr(xi, C.c_double), d.shape[0],
                             _ptr(out, C.c_double))
    return out


def transmissivity(scene: Scene, p, s, seed: int, path: int) -> float:
    st = scene.struct()
    p64 = np.asarray(p, dtype=np.float64)
    s64 = np.asarray(s, dtype=np.float64)
    return lib().orc_transmissivity(C.byref(st), _ptr(p64, C.c_double), _ptr(s64, C.c_double), seed, path)


def transmissivity_many(scene: Scene, p, s, seed: int, n: int) -> np.ndarray:
    st = scene.struct()
    p64 = np.asarray(p, dtype=np.float64)
    s64 = np.asarray(s, dtype=np.float64)
    f = lib().orc_transmissivity
    return np.array([f(C.byref(st), _ptr(p64, C.c_double), _ptr(s64, C.c_double), seed, i) for i in range(n)])


def first_collision_distances(scene: Scene, p, d, seed: int, n: int) -> np.ndarray:
    st = scene.struct()
    p64 = np.asarray(p, dtype=np.float64)
    d64 = np.asarray(d, dtype=np.float64)
    f = lib().orc_first_collision_distance
    return np.array([f(C.byref(st), _ptr(p64, C.c_double), _ptr(d64, C.c_double), seed, i) for i in range(n)])


@dataclass
class Tally:
    """Mean and standard error from FP64 sums (sum s, sum s^2, N)."""
    s1: np.ndarray
    s2: np.ndarray
    n: np.ndarray

    @property
    def mean(self):
        with np.errstate(invalid="ignore", divide="ignore"):      # cells with no paths: nan
            return self.s1 / self.n

    @property
    def se(self):
        with np.errstate(invalid="ignore", divide="ignore"):
            m = self.s1 / self.n
            var = np.maximum(self.s2 / self.n - m * m, 0.0) * self.n / np.maximum(self.n - 1, 1)
            return np.sqrt(var / self.n)


def trace_camera(scene: Scene, cam: Camera, spp: int, seed: int, pix_range=None, nthreads: int = 0,
                 pixels=None):
    """Per-pixel radiance tallies [height][width] (units of F0 per sr).
    ``pix_range`` (begin, end) or ``pixels`` (flat indices) restrict the
    trace to those pixels (same path ids as the whole image); the others
    are left at zero with a path count of 0."""
    st = scene.struct()
    cs = cam.struct()
    npix = cam.width * cam.height
    sums = np.zeros((npix, 2), dtype=np.float64)
    stats = np.zeros(4, dtype=np.int64)
    n = np.zeros(npix)
    ranges = [(0, npix) if pix_range is None else tuple(pix_range)]
    if pixels is not None:
        ranges = [(int(p), int(p) + 1) for p in pixels]
    for p0, p1 in ranges:
        st_i = np.zeros(4, dtype=np.int64)
        rc = lib().orc_trace_camera(C.byref(st), C.byref(cs), spp, seed, p0, p1, _ptr(sums, C.c_double),
                                    nthreads or default_threads(), _ptr(st_i, C.c_int64))
        if rc != 0:
            raise ValueError("bad camera request")
        stats += st_i
        n[p0:p1] = spp
    t = Tally(sums[:, 0].reshape(cam.height, cam.width), sums[:, 1].reshape(cam.height, cam.width),
              n.reshape(cam.height, cam.width))
    return t, stats


def trace_flux(scene: Scene, npaths: int, seed: int, begin: int = 0, nthreads: int = 0):
    """Domain-mean ground transmittance tallies (T_dir, T_dif, T_tot, dT/dg,
    dT/dalpha)."""
    st = scene.struct()
    sums = np.zeros(10, dtype=np.float64)
    stats = np.zeros(4, dtype=np.int64)
    rc = lib().orc_trace_flux(C.byref(st), seed, begin, begin + npaths, _ptr(sums, C.c_double),
                              nthreads or default_threads(), _ptr(stats, C.c_int64))
    if rc != 0:
        raise ValueError("bad flux request")
    return Tally(sums[0::2].copy(), sums[1::2].copy(), np.full(5, float(npaths))), stats


def terrain_height(scene: Scene, x: float, y: float):
    """Surface height of the heightfield ground at (x, y) and its normal."""
    st = scene.struct()
    n = np.zeros(3)
    z = lib().orc_terrain_height(C.byref(st), x, y, _ptr(n, C.c_double))
    return z, n


def terrain_hit(scene: Scene, o, d):
    """First hit of the ray o + t d with the heightfield: (t, (i, j), tri)
    with the unwrapped cell and triangle (0: u >= v, 1: u < v), or None."""
    st = scene.struct()
    oo = np.ascontiguousarray(o, dtype=np.float64)
    dd = np.ascontiguousarray(d, dtype=np.float64)
    t = np.zeros(1)
    cell = np.zeros(2, dtype=np.int64)
    tri = C.c_int()
    if not lib().orc_terrain_hit(C.byref(st), _ptr(oo, C.c_double), _ptr(dd, C.c_double), _ptr(t, C.c_double),
                                 _ptr(cell, C.c_int64), C.byref(tri)):
        return None
    return float(t[0]), (int(cell[0]), int(cell[1])), int(tri.value)


def trace_forward(scene: Scene, nphotons: int, seed: int, nthreads: int = 0):
    """Forward analog: (R, T_dir, T_dif, A_vol, A_ground, cutoff) per photon."""
    st = scene.struct()
    sums = np.zeros(12, dtype=np.float64)
    stats = np.zeros(1, dtype=np.int64)
    lib().orc_trace_forward(C.byref(st), seed, 0, nphotons, _ptr(sums, C.c_double),
                            nthreads or default_threads(), _ptr(stats, C.c_int64))
    return Tally(sums[0::2].copy(), sums[1::2].copy(), np.full(6, float(nphotons))), stats


def forward_balance_residual(scene: Scene, seed: int, nphotons: int) -> float:
    st = scene.struct()
    return lib().orc_forward_balance_residual(C.byref(st), seed, 0, nphotons)


# --------------------------------------------------------------------------
# Learned proposal (MLP -> vMF mixture, one-sample MIS with HG)
# --------------------------------------------------------------------------
def _learned_sigs():
    L = lib()
    f64p = C.POINTER(C.c_double)
    L.orc_mlp_nparam.restype = C.c_int
    L.orc_mlp_forward.argtypes = [f64p, f64p, C.c_int64, f64p]
    L.orc_mixture.argtypes = [f64p, f64p, f64p, f64p]
    L.orc_vmf_pdf.argtypes = [f64p, C.c_double, f64p]
    L.orc_vmf_pdf.restype = C.c_double
    L.orc_vmf_sample.argtypes = [f64p, C.c_double, C.c_double, C.c_double, f64p]
    L.orc_mis_sample.argtypes = [f64p, C.c_double, C.c_double, f64p, f64p, f64p, f64p, f64p]
    L.orc_mis_sample.restype = C.c_double
    L.orc_mixture_pdf.argtypes = [f64p, f64p]
    L.orc_mixture_pdf.restype = C.c_double
    L.orc_mlp_loss_grad.argtypes = [f64p, f64p, f64p, f64p, C.c_int64, f64p]
    L.orc_mlp_loss_grad.restype = C.c_double
    L.orc_adam_step.argtypes = [f64p, f64p, f64p, f64p, C.c_int64, C.c_int64, C.c_double, C.c_double, C.c_double,
                                C.c_double]
    return L


MLP_SHAPES = [(64, 9), (64,), (64, 64), (64,), (64, 64), (64,), (40, 64), (40,)]

# One online-training record of a learned vertex (orc_record in the C file).
RECORD_DTYPE = np.dtype([("path", np.uint64), ("vertex", np.int32), ("pad", np.int32), ("x", np.float64, 9),
                         ("dir", np.float64, 3), ("before", np.float64), ("w_omega", np.float64),
                         ("own", np.float64), ("target", np.float64)])


def learned_records(scene: Scene, cam, spp: int, seed: int, begin: int, end: int, cap: int = 1 << 20):
    """The learned proposal's online-training records of camera paths
    [begin, end) (``cam`` a Camera, ``spp`` samples per pixel) or of ground
    flux paths (``cam`` None), in path order, plus each path's backward
    score.  Each record holds the vertex's features, the sampled direction,
    the score before the vertex, w * omega, the vertex's own estimate and the
    KL target (score after the vertex excluding its own estimate, over
    w * omega)."""
    if scene.mlp is None:
        raise ValueError("learned_records needs a scene with a network (mlp=...)")
    L = lib()
    L.orc_learned_records.restype = C.c_int64
    L.orc_learned_records.argtypes = [C.c_void_p, C.c_void_p, C.c_uint32, C.c_uint64, C.c_uint64, C.c_uint64,
                                      C.c_void_p, C.c_int64, C.POINTER(C.c_double)]
    st = scene.struct()
    cs = cam.struct() if cam is not None else None
    out = np.zeros(cap, dtype=RECORD_DTYPE)
    scores = np.zeros(end - begin, dtype=np.float64)
    n = L.orc_learned_records(C.addressof(st), C.addressof(cs) if cs is not None else None, spp if cam else 0,
                              seed, begin, end, out.ctypes.data, cap, _ptr(scores, C.c_double))
    if n < 0:
        raise ValueError("bad learned-records request")
    return out[:min(n, cap)].copy(), scores


def mlp_nparam() -> int:
    return _learned_sigs().orc_mlp_nparam()


def mlp_split(params):
    """Views of the flat parameter vector in layer order (W1, b1, ..., W4, b4)."""
    out, off = [], 0
    for sh in MLP_SHAPES:
        n = int(np.prod(sh))
        out.append(np.asarray(params[off:off + n]).reshape(sh))
        off += n
    return out


def mlp_forward(params, x):
    p = np.ascontiguousarray(params, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 9)
    out = np.zeros((x.shape[0], 40))
    _learned_sigs().orc_mlp_forward(_ptr(p, C.c_double), _ptr(x, C.c_double), x.shape[0], _ptr(out, C.c_double))
    return out


def mixture(raw):
    raw = np.ascontiguousarray(raw, dtype=np.float64)
    mu = np.zeros((8, 3)); ka = np.zeros(8); pi = np.zeros(8)
    _learned_sigs().orc_mixture(_ptr(raw, C.c_double), _ptr(mu, C.c_double), _ptr(ka, C.c_double),
                                _ptr(pi, C.c_double))
    return mu, ka, pi


def vmf_pdf(mu, kappa, x):
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    return _learned_sigs().orc_vmf_pdf(_ptr(mu, C.c_double), float(kappa), _ptr(x, C.c_double))


def vmf_sample(mu, kappa, xi1, xi2):
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    out = np.zeros(3)
    _learned_sigs().orc_vmf_sample(_ptr(mu, C.c_double), float(kappa), float(xi1), float(xi2), _ptr(out, C.c_double))
    return out


def mis_sample(raw, g, alpha, d, u):
    """Returns (direction, weight factor p_HG/q, q, p_HG)."""
    raw = np.ascontiguousarray(raw, dtype=np.float64)
    d = np.ascontiguousarray(d, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(3)
    q = C.c_double(); ph = C.c_double()
    f = _learned_sigs().orc_mis_sample(_ptr(raw, C.c_double), float(g), float(alpha), _ptr(d, C.c_double),
                                       _ptr(u, C.c_double), _ptr(out, C.c_double), C.byref(q), C.byref(ph))
    return out, f, q.value, ph.value


def mixture_pdf(raw, x):
    raw = np.ascontiguousarray(raw, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    return _learned_sigs().orc_mixture_pdf(_ptr(raw, C.c_double), _ptr(x, C.c_double))


def mlp_loss_grad(params, x, dirs, t):
    p = np.ascontiguousarray(params, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 9)
    dirs = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 3)
    t = np.ascontiguousarray(t, dtype=np.float64).reshape(-1)
    g = np.zeros(p.size)
    loss = _learned_sigs().orc_mlp_loss_grad(_ptr(p, C.c_double), _ptr(x, C.c_double), _ptr(dirs, C.c_double),
                                             _ptr(t, C.c_double), x.shape[0], _ptr(g, C.c_double))
    return loss, g


def adam_step(params, m, v, grad, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """In-place Adam update of float64 arrays params, m, v."""
    _learned_sigs().orc_adam_step(_ptr(params, C.c_double), _ptr(m, C.c_double), _ptr(v, C.c_double),
                                  _ptr(np.ascontiguousarray(grad, dtype=np.float64), C.c_double), params.size, t,
                                  lr, b1, b2, eps)


def xavier_init(seed: int):
    """Xavier-uniform weights, zero biases (float64)."""
    r = np.random.Generator(np.random.Philox(seed))
    parts = []
    for sh in MLP_SHAPES:
        if len(sh) == 2:
            lim = math.sqrt(6.0 / (sh[0] + sh[1]))
            parts.append(r.uniform(-lim, lim, sh).ravel())
        else:
            parts.append(np.zeros(sh))
    return np.concatenate(parts)
