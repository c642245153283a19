"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

* Philox4x32-10, majorant pyramid (FP32 and BF16 round-up) and the leaf
  traversal: bit-exact.
* Monte Carlo tallies: within 4 combined standard errors of the oracle, on
  the same seeds (the two sides draw the same random numbers, so most paths
  coincide up to FP32 rounding; a paired check makes that explicit).
* Closed forms met by the GPU directly (Beer, black sky, single scattering).
* Edge cases: ragged sizes, a one-voxel field, an empty field, tau~ = 0 and
  infinity, voxel tracking, delta tracking, order cut, bad arguments,
  deadline and cancel flag.
"""
import math

import numpy as np
import pytest

import scenes
from parity_util import close_4se, image_parity, ocam, oscene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1902_01137_gb300 as mod
    from paper_1902_01137_gb300 import build
    build.build()
    return mod


@pytest.fixture(scope="module")
def ctx(m):
    c = m.Context(0)
    yield c
    c.close()


# ---------------------------------------------------------------------------
# bit-exact parts
# ---------------------------------------------------------------------------
def test_philox_bit_exact(m, ctx, orc):
    r = np.random.default_rng(5)
    ctr = r.integers(0, 2 ** 32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    key = r.integers(0, 2 ** 32, size=(4096, 2), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    key[0] = 0
    g = m.mcrt_debug_philox(ctx.h, ctr, key)
    o = orc.philox4x32_10(ctr, key)
    assert np.array_equal(g, o)


@pytest.mark.parametrize("shape,levels", [((32, 64, 64), 2), ((21, 29, 37), 2), ((1, 1, 1), 1),
                                          ((40, 72, 72), 3), ((9, 8, 65), 3)])
@pytest.mark.parametrize("bf16", [False, True])
def test_majorants_bit_exact(m, ctx, orc, shape, levels, bf16):
    r = np.random.default_rng(sum(shape))
    k = (r.lognormal(0.0, 2.0, shape) * (r.uniform(size=shape) < 0.4)).astype(np.float32)
    sc = m.Scene(ctx, k, 0.1, 0.1, 0.1, levels=levels, storage=m.MCRT_STORAGE_BF16 if bf16 else 0)
    try:
        want = orc.build_pyramid(k, levels, round_up_bf16=bf16)
        want_min = orc.build_pyramid_min(k, levels, round_nearest_bf16=bf16)
        for L in range(1, levels + 1):
            got = sc.majorants(L)
            assert got.shape == want[L - 1].shape
            assert np.array_equal(got.view(np.uint32), want[L - 1].view(np.uint32)), L
            gmin = sc.minorants(L)
            assert np.array_equal(gmin.view(np.uint32), want_min[L - 1].view(np.uint32)), ("min", L)
    finally:
        sc.close()


def _dda_field():
    sp = scenes.random_voxels(72, 64, 40, 0.1, 3.0, seed=2, sparsity=0.5)
    k = sp.k.copy()
    k[:, :, 32:64] = 0.0
    k[24:, :, :] *= 0.01
    return sp, k


@pytest.mark.parametrize("tau,finest", [(1.0, 1), (0.3, 0), (float("inf"), 1), (0.0, 0), (5.0, 0)])
def test_dda_bit_exact(m, ctx, orc, tau, finest):
    sp, k = _dda_field()
    sc = m.Scene(ctx, k, sp.dx, sp.dy, sp.dz, levels=2)
    osc = orc.Scene(k=k, dx=sp.dx, dy=sp.dy, dz=sp.dz, levels=2, tau_merge=tau, finest_level=finest)
    try:
        o, d = scenes.random_rays(sp, 200, seed=17)
        # add rays from faces and along axes
        o = np.concatenate([o, np.array([[0.85, 0.85, 0.0], [0.85, 0.85, 4.0], [0.0, 1.05, 1.05]], np.float32)])
        d = np.concatenate([d, np.array([[0, 0, 1], [0, 0, -1], [0.6, 0.8, 0.0]], np.float32)])
        for i in range(len(o)):
            cg, tg, sg = sc.dda(o[i], d[i], tau, finest, cap=2000)
            co, to, so = orc.dda_spec(osc, o[i], d[i], cap=2000)
            assert sg == so, i
            assert np.array_equal(cg, co), i
            assert np.array_equal(tg.view(np.uint32), to.view(np.uint32)), i
    finally:
        sc.close()


# ---------------------------------------------------------------------------
# statistical parity on the small config (64x64x32 blobs)
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def small(m, ctx):
    sp = scenes.blobs_small(0)
    sc = m.Scene.from_spec(ctx, sp)
    yield sp, sc
    sc.close()


def test_flux_small_vs_oracle(m, orc, small):
    sp, sc = small
    n = 100000
    g = sc.trace_flux(n, seed=0)
    o, _ = orc.trace_flux(oscene(orc, sp), n, seed=0)
    for q in range(3):
        assert close_4se(g.mean[q], g.se[q], o.mean[q], o.se[q]), (q, g.mean[q], o.mean[q], g.se[q], o.se[q])
    # same random numbers: the two estimates differ by far less than their noise
    assert abs(g.mean[2] - o.mean[2]) < 0.25 * o.se[2]


def test_camera_small_vs_oracle(m, orc, small):
    sp, sc = small
    cam = scenes.nadir_camera(sp, 64, 64)
    g = sc.trace_camera(cam, 16, seed=0)
    o, _ = orc.trace_camera(oscene(orc, sp), ocam(orc, cam), 16, seed=0)
    ok, info = image_parity(g.mean, g.se, o.mean, o.se, 16)
    assert ok, info
    # paired: identical random numbers give near-identical pixels
    rel = np.abs(g.mean - o.mean) / np.maximum(np.abs(o.mean), 1e-3)
    assert np.median(rel) < 1e-3, np.median(rel)


@pytest.mark.parametrize("opts", [dict(tau_merge=0.0, finest_level=0), dict(tau_merge=float("inf")),
                                  dict(tau_merge=1.0, finest_level=1), dict(tau_merge=0.5, finest_level=1),
                                  dict(tau_merge=10.0), dict(sun_mode=1), dict(sun_mode=2),
                                  dict(sun_mode=2, tau_merge=1.0, finest_level=1), dict(chunk=1), dict(chunk=64),
                                  dict(block_size=64, grid_size=7)])
def test_flux_options_vs_oracle(m, orc, small, opts):
    sp, sc = small
    n = 40000
    g = sc.trace_flux(n, seed=3, **opts)
    okw = {}
    if "tau_merge" in opts:
        okw["tau_merge"] = opts["tau_merge"]
    if "finest_level" in opts:
        okw["finest_level"] = opts["finest_level"]
    if "sun_mode" in opts:
        okw["sun_mode"] = opts["sun_mode"]
    o, _ = orc.trace_flux(oscene(orc, sp, **okw), n, seed=3)
    for q in range(3):
        assert close_4se(g.mean[q], g.se[q], o.mean[q], o.se[q]), (opts, q, g.mean[q], o.mean[q])


def test_decomposition_tracking_closed_form_and_variance(m, ctx, orc, small):
    """Decomposition tracking on the GPU: exp(-tau) with zero variance through
    a uniform slab whose extinction is a bfloat16 value (the leaves'
    minorant equals it) and tau < ln 10; on the blob field the same
    expectation as ratio tracking with a smaller diffuse variance, paired
    with the oracle's decomposition tracking."""
    k, th = 0.75, 40.0
    sp = scenes.homogeneous(16, 16, 16, 0.1, k, levels=2, sun_zenith_deg=th)
    sc = m.Scene.from_spec(ctx, sp)
    try:
        r = sc.trace_flux(20000, seed=2, sun_mode=2)
        want = math.exp(-k * 16 * float(np.float32(0.1)) / math.cos(math.radians(th)))
        assert r.mean[0] == pytest.approx(want, rel=2e-6) and r.se[0] < 1e-6 * want
    finally:
        sc.close()
    sp, sc = small
    n = 200000
    a = sc.trace_flux(n, seed=31, sun_mode=0)
    b = sc.trace_flux(n, seed=31, sun_mode=2)
    o, _ = orc.trace_flux(oscene(orc, sp, sun_mode=2), n, seed=31)
    for q in range(3):
        assert close_4se(a.mean[q], a.se[q], b.mean[q], b.se[q])
        assert close_4se(b.mean[q], b.se[q], o.mean[q], o.se[q])
    assert abs(b.mean[2] - o.mean[2]) < 0.25 * o.se[2]
    assert b.se[1] < a.se[1]


def test_launch_shape_does_not_change_results(m, small):
    """Path i always draws the same numbers, so the launch shape only changes
    how the per-path scores are summed: FP32 partial sums over a chunk (at
    most 64 terms, relative rounding <= 64 * 2^-24 ~ 4e-6) then FP64 atomics."""
    sp, sc = small
    a = sc.trace_flux(30000, seed=9)
    b = sc.trace_flux(30000, seed=9, block_size=32, grid_size=3, chunk=5)
    np.testing.assert_allclose(a.mean, b.mean, rtol=4e-6)
    cam = scenes.nadir_camera(sp, 32, 32)
    c = sc.trace_camera(cam, 16, seed=9)
    d = sc.trace_camera(cam, 16, seed=9, chunk=1, block_size=64)
    np.testing.assert_allclose(c.mean, d.mean, rtol=4e-6, atol=1e-12)


def test_rare_phase_batching_does_not_change_results(m, ctx, small):
    """When a lane's path start, ray start or vertex runs (how many lanes of
    its warp must be waiting for one) is launch shape only: a path start or
    vertex that runs on into its ray start takes the same numbers it would
    take in a later iteration, so every path's score is the same and only
    the order of the FP64 adds of the chunk sums differs.  Covers the plain
    kernel, decomposition tracking (its own variant) and a heightfield
    (whose ground walks are a rare kind of their own)."""
    sp, sc = small
    cam = scenes.nadir_camera(sp, 32, 32)
    for kw in ({}, {"sun_mode": m.MCRT_SUN_DECOMP}):
        ref = sc.trace_flux(40000, seed=11, **kw)
        for rb in (1, 4, 32):
            r = sc.trace_flux(40000, seed=11, rare_batch=rb, **kw)
            np.testing.assert_allclose(r.mean, ref.mean, rtol=1e-10, atol=1e-14)
    ci = sc.trace_camera(cam, 16, seed=12)
    for rb in (1, 32):
        r = sc.trace_camera(cam, 16, seed=12, rare_batch=rb)
        np.testing.assert_allclose(r.mean, ci.mean, rtol=1e-10, atol=1e-14)
    ts = m.Scene.from_spec(ctx, sp)
    try:
        ts.set_heightfield(scenes.heightfield(128, 0.3, seed=5), sp.ground_albedo)
        ref = ts.trace_flux(20000, seed=13)
        for rb in (1, 32):
            r = ts.trace_flux(20000, seed=13, rare_batch=rb)
            np.testing.assert_allclose(r.mean, ref.mean, rtol=1e-10, atol=1e-14)
    finally:
        ts.close()


def test_event_counters(m, small):
    sp, sc = small
    r = sc.trace_flux(20000, seed=4, count_events=1)
    c = r.counters
    assert c["paths"] == 20000
    assert c["tentative"] >= c["real"] > 0
    assert c["sun_rays"] == c["paths"] + c["real"] + c["ground"]  # the direct ray plus one per vertex
    assert c["aborted"] == 0
    q = sc.trace_flux(20000, seed=4)
    np.testing.assert_allclose(q.mean, r.mean, rtol=1e-12)


# ---------------------------------------------------------------------------
# closed forms on the GPU directly
# ---------------------------------------------------------------------------
def test_beer_gpu(m, ctx):
    k, th = 1.7, 40.0
    sp = scenes.homogeneous(16, 16, 16, 0.1, k, levels=2, sun_zenith_deg=th)
    sc = m.Scene.from_spec(ctx, sp)
    try:
        r = sc.trace_flux(200000, seed=5)
        want = math.exp(-k * 1.6 / math.cos(math.radians(th)))
        assert abs(r.mean[0] - want) < 3 * r.se[0]
    finally:
        sc.close()


def test_black_sky_gpu(m, ctx):
    rho, th = 0.3, 35.0
    sp = scenes.homogeneous(16, 16, 8, 0.1, 0.0, levels=1, ground_albedo=rho, sun_zenith_deg=th)
    sc = m.Scene.from_spec(ctx, sp)
    try:
        cam = scenes.nadir_camera(sp, 8, 8)
        r = sc.trace_camera(cam, 64, seed=2)
        want = rho * math.cos(math.radians(th)) / math.pi
        np.testing.assert_allclose(r.mean, want, rtol=2e-6)
    finally:
        sc.close()


def test_single_scattering_gpu(m, ctx):
    k, g, om, th0, thv = 2.0, 0.7, 0.9, 30.0, 50.0
    sp = scenes.homogeneous(16, 16, 8, 0.1, k, levels=1, g=g, ssa_cloud=om, ssa_clear=om, sun_zenith_deg=th0)
    sc = m.Scene.from_spec(ctx, sp)
    try:
        d = np.array([math.sin(math.radians(thv)), 0.0, -math.cos(math.radians(thv))])
        pos = np.array([0.8, 0.8, 0.8]) - 20.0 * d
        cam = scenes.CameraSpec(tuple(pos), (0.8, 0.8, 0.8), (0.0, 0.0, 1.0), 1e-3, 1, 1)
        r = sc.trace_camera(cam, 1 << 20, seed=4, max_order=1)
        mu0, mu = math.cos(math.radians(th0)), math.cos(math.radians(thv))
        s = np.array([math.sin(math.radians(th0)), 0.0, mu0])
        cosang = float(d @ s)
        p = (1 - g * g) / (4 * math.pi * (1 + g * g - 2 * g * cosang) ** 1.5)
        want = om * p * mu0 / (mu0 + mu) * (1 - math.exp(-k * 0.8 * (1 / mu0 + 1 / mu)))
        assert abs(r.mean[0, 0] - want) < 3 * r.se[0, 0], (r.mean[0, 0], want, r.se[0, 0])
    finally:
        sc.close()


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------
def test_ragged_field_vs_oracle(m, ctx, orc):
    sp = scenes.random_voxels(37, 29, 21, 0.1, 6.0, seed=8, levels=2, sparsity=0.7, ground_albedo=0.4,
                              sun_zenith_deg=20.0, g=0.6, ssa_cloud=0.95, ssa_clear=0.95)
    sc = m.Scene.from_spec(ctx, sp)
    try:
        n = 60000
        g = sc.trace_flux(n, seed=12)
        o, _ = orc.trace_flux(oscene(orc, sp), n, seed=12)
        for q in range(3):
            assert close_4se(g.mean[q], g.se[q], o.mean[q], o.se[q]), (q, g.mean[q], o.mean[q])
        cam = scenes.nadir_camera(sp, 24, 16)
        gi = sc.trace_camera(cam, 32, seed=13)
        oi, _ = orc.trace_camera(oscene(orc, sp), ocam(orc, cam), 32, seed=13)
        ok, info = image_parity(gi.mean, gi.se, oi.mean, oi.se, 32)
        assert ok, info
    finally:
        sc.close()


def test_one_voxel_field(m, ctx, orc):
    sp = scenes.homogeneous(1, 1, 1, 0.5, 1.3, levels=1, ground_albedo=0.5, sun_zenith_deg=10.0, g=0.3)
    sc = m.Scene.from_spec(ctx, sp)
    try:
        g = sc.trace_flux(50000, seed=1)
        o, _ = orc.trace_flux(oscene(orc, sp), 50000, seed=1)
        for q in range(3):
            assert close_4se(g.mean[q], g.se[q], o.mean[q], o.se[q])
    finally:
        sc.close()


def test_empty_field(m, ctx):
    sp = scenes.homogeneous(16, 16, 16, 0.1, 0.0, levels=2, ground_albedo=0.0, sun_zenith_deg=0.0)
    sc = m.Scene.from_spec(ctx, sp)
    try:
        r = sc.trace_flux(10000, seed=1)
        np.testing.assert_allclose(r.mean, [1.0, 0.0, 1.0], atol=0)
        cam = scenes.nadir_camera(sp, 4, 4)
        img = sc.trace_camera(cam, 4, seed=1)
        assert np.all(img.mean == 0.0)
    finally:
        sc.close()


def test_bad_arguments(m, ctx, small):
    sp, sc = small
    with pytest.raises(m.McrtError) as e:
        sc.trace_flux(0, seed=1)
    assert e.value.status == m.MCRT_ERR_ARG
    with pytest.raises(m.McrtError) as e:
        m.mcrt_scene_set_sun(ctx.h, sc.h, 95.0, 0.0)
    assert e.value.status == m.MCRT_ERR_ARG
    with pytest.raises(m.McrtError) as e:
        sc.trace_flux(10, seed=1, finest_level=3)
    assert e.value.status == m.MCRT_ERR_ARG
    with pytest.raises(m.McrtError) as e:
        m.Scene(ctx, np.zeros((4, 4, 4), np.float32), -0.1, 0.1, 0.1)
    assert e.value.status == m.MCRT_ERR_ARG
    with pytest.raises(m.McrtError) as e:
        m.mcrt_scene_read_majorants(ctx.h, sc.h, 9)
    assert e.value.status == m.MCRT_ERR_ARG


def test_deadline_and_cancel(m, ctx, small):
    torch = pytest.importorskip("torch")
    sp, sc = small
    cam = scenes.nadir_camera(sp, 256, 256)
    with pytest.raises(m.McrtError) as e:
        sc.trace_camera(cam, 4096, seed=1, deadline_ms=2.0)
    assert e.value.status == m.MCRT_ERR_TIMEOUT
    flag = torch.ones(1, dtype=torch.int32).pin_memory()
    with pytest.raises(m.McrtError) as e:
        sc.trace_camera(cam, 4096, seed=1, cancel_flag=flag.data_ptr())
    assert e.value.status == m.MCRT_ERR_CANCELLED
    # the context is still usable afterwards
    r = sc.trace_flux(1000, seed=2)
    assert np.isfinite(r.mean).all()


# ---------------------------------------------------------------------------
# precision: BF16 voxel storage with majorants rounded up
# ---------------------------------------------------------------------------
def test_bf16_storage_vs_oracle_bf16(m, ctx, orc):
    """BF16 storage traces the nearest-BF16 field exactly (majorants rounded
    up stay bounds); the oracle traces the same rounded field in FP64."""
    sp = scenes.blobs_small(0)
    sc = m.Scene.from_spec(ctx, sp, storage=m.MCRT_STORAGE_BF16)
    try:
        n = 100000
        g = sc.trace_flux(n, seed=5)
        o, _ = orc.trace_flux(oscene(orc, sp, bf16=True), n, seed=5)
        for q in range(3):
            assert close_4se(g.mean[q], g.se[q], o.mean[q], o.se[q]), (q, g.mean[q], o.mean[q])
        assert abs(g.mean[2] - o.mean[2]) < 0.25 * o.se[2]
        cam = scenes.nadir_camera(sp, 64, 64)
        gi = sc.trace_camera(cam, 16, seed=6)
        oi, _ = orc.trace_camera(oscene(orc, sp, bf16=True), ocam(orc, cam), 16, seed=6)
        ok, info = image_parity(gi.mean, gi.se, oi.mean, oi.se, 16)
        assert ok, info
        rel = np.abs(gi.mean - oi.mean) / np.maximum(np.abs(oi.mean), 1e-3)
        assert np.median(rel) < 1e-3
    finally:
        sc.close()


def test_bf16_error_against_fp64_oracle_of_fp32_field(m, ctx, orc, capsys):
    """Error of the BF16-stored field against the FP64 oracle of the FP32
    field.  Rounding to nearest BF16 changes each voxel by at most 2^-9
    relative, so an optical depth tau moves by at most 2^-9 tau and a
    transmissivity by at most a factor exp(2^-9 tau); the direct part
    (tau_sun of the blobs <= 40) is bounded accordingly, and every tally must
    also stay within that bound plus 4 combined SE.  The measured
    differences are printed (the report of the precision row)."""
    sp = scenes.blobs_small(0)
    n = 200000
    o, _ = orc.trace_flux(oscene(orc, sp), n, seed=8)
    res = {}
    for storage, name in [(m.MCRT_STORAGE_F32, "f32"), (m.MCRT_STORAGE_BF16, "bf16")]:
        sc = m.Scene.from_spec(ctx, sp, storage=storage)
        try:
            res[name] = sc.trace_flux(n, seed=8)
        finally:
            sc.close()
    tau_max = 40.0
    for name, g in res.items():
        for q in range(3):
            d = abs(g.mean[q] - o.mean[q])
            bound = 4.0 * math.hypot(g.se[q], o.se[q])
            if name == "bf16":
                bound += o.mean[q] * (math.exp(tau_max * 2.0 ** -9) - 1.0)
            assert d <= bound, (name, q, g.mean[q], o.mean[q], bound)
    with capsys.disabled():
        print("\n[precision] flux T_dir/T_dif/T_tot: fp64 oracle %s | f32 %s | bf16 %s | "
              "bf16-oracle %s (se %s)" % (np.round(o.mean[:3], 6), np.round(res["f32"].mean, 6),
                                           np.round(res["bf16"].mean, 6),
                                           np.round(res["bf16"].mean - o.mean[:3], 6), np.round(o.se[:3], 6)))


def test_scene_from_pinned_host_field(m, ctx, orc):
    """A page-locked host field is read by the relayout kernel in place (no
    staging copy): bricks and majorants equal those of the same field from
    pageable host memory and from device memory, and the oracle's."""
    torch = pytest.importorskip("torch")
    r = np.random.default_rng(77)
    shape = (40, 72, 72)
    k = (r.lognormal(0.0, 2.0, shape) * (r.uniform(size=shape) < 0.4)).astype(np.float32)
    pinned = torch.from_numpy(k).pin_memory()
    assert pinned.is_pinned()
    want = orc.build_pyramid(k, 3)
    for src in (pinned, k, torch.from_numpy(k).cuda()):
        sc = m.Scene(ctx, src, 0.1, 0.1, 0.1, levels=3)
        try:
            for L in range(1, 4):
                assert np.array_equal(sc.majorants(L).view(np.uint32), want[L - 1].view(np.uint32)), (type(src), L)
            cam = scenes.nadir_camera(scenes.homogeneous(72, 72, 40, 0.1, 1.0), 16, 16)
            res = sc.trace_camera(cam, 4, seed=3)
            if src is pinned:
                ref = res.mean
            else:
                np.testing.assert_allclose(res.mean, ref, rtol=1e-12, atol=0)   # FP64 atomics: order only
        finally:
            sc.close()


def test_pixel_order_changes_speed_not_results(m, small):
    """Cost-ordered claims (the default) and raster claims trace the same
    paths with the same draws: equal images up to the order of the FP64
    atomic adds, equal event counts.  A ragged image (tiles cut at the
    edges) and an oblique camera."""
    sp, sc = small
    for cam in (scenes.nadir_camera(sp, 37, 21),
                scenes.CameraSpec((1.0, -4.0, 6.0), (3.2, 3.2, 0.8), (0.0, 0.0, 1.0), 50.0, 45, 30)):
        a = sc.trace_camera(cam, 8, seed=5)
        b = sc.trace_camera(cam, 8, seed=5, pixel_order=m.MCRT_ORDER_RASTER)
        np.testing.assert_allclose(a.mean, b.mean, rtol=1e-12, atol=0)
        np.testing.assert_allclose(a.se, b.se, rtol=1e-9, atol=1e-15)
        ca = sc.trace_camera(cam, 8, seed=5, count_events=1).counters
        cb = sc.trace_camera(cam, 8, seed=5, count_events=1, pixel_order=m.MCRT_ORDER_RASTER).counters
        for k in ("paths", "tentative", "real", "ground", "leaf_steps", "sun_tentative", "sun_rays"):
            assert ca[k] == cb[k], k
    with pytest.raises(m.McrtError):
        sc.trace_camera(scenes.nadir_camera(sp, 8, 8), 1, seed=1, pixel_order=5)


def test_shards_add_up_to_the_whole_trace(m, ctx, small):
    """One image or flux traced as shards (one per process in a multi-GPU
    run): every path keeps its global id, so the shards' per-pixel sums add
    up to the unsharded trace's (to the order of the FP64 adds) and their
    pixel sets partition the image, in cost and in raster claim order; the
    flux shards cover [0, n) with no path twice."""
    sp, sc = small
    cam = scenes.nadir_camera(sp, 37, 21)
    cd = m.CameraDesc()
    for i in range(3):
        cd.pos[i], cd.target[i], cd.up[i] = cam.pos[i], cam.target[i], cam.up[i]
    cd.fov_deg, cd.width, cd.height = cam.fov_deg, cam.width, cam.height

    def sums(fn, **kw):
        o = m.Scene._opts(**kw)
        t = fn(o)
        try:
            return m.mcrt_tally_read_sums(ctx.h, t)
        finally:
            m.mcrt_tally_destroy(t)

    cam_fn = lambda o: m.mcrt_trace_camera(ctx.h, sc.h, cd, 8, 5, o)
    for order in (m.MCRT_ORDER_COST, m.MCRT_ORDER_RASTER):
        w1, w2 = sums(cam_fn, pixel_order=order)
        parts = [sums(cam_fn, pixel_order=order, shard_index=r, shard_count=3) for r in range(3)]
        owner = np.stack([(p[0][:, 0] != 0) | (p[1][:, 0] != 0) for p in parts])
        assert owner.sum(axis=0).max() <= 1                 # no pixel in two shards
        if order == m.MCRT_ORDER_RASTER:
            for r in range(3):                              # raster shards: every third pixel
                assert not owner[r][np.setdiff1d(np.arange(37 * 21), np.arange(r, 37 * 21, 3))].any()
        np.testing.assert_allclose(sum(p[0] for p in parts), w1, rtol=1e-12, atol=0)
        np.testing.assert_allclose(sum(p[1] for p in parts), w2, rtol=1e-12, atol=0)
    flux_fn = lambda o: m.mcrt_trace_flux(ctx.h, sc.h, 10007, 6, o)
    f1, f2 = sums(flux_fn)
    parts = [sums(flux_fn, shard_index=r, shard_count=4) for r in range(4)]
    np.testing.assert_allclose(sum(p[0] for p in parts), f1, rtol=1e-12, atol=0)
    np.testing.assert_allclose(sum(p[1] for p in parts), f2, rtol=1e-12, atol=0)
    with pytest.raises(m.McrtError) as e:
        sums(flux_fn, shard_index=4, shard_count=4)
    assert e.value.status == m.MCRT_ERR_ARG
    # more shards than pixels: the surplus shards trace nothing
    tiny = scenes.nadir_camera(sp, 3, 2)
    td = m.CameraDesc()
    for i in range(3):
        td.pos[i], td.target[i], td.up[i] = tiny.pos[i], tiny.target[i], tiny.up[i]
    td.fov_deg, td.width, td.height = tiny.fov_deg, tiny.width, tiny.height
    tiny_fn = lambda o: m.mcrt_trace_camera(ctx.h, sc.h, td, 16, 7, o)
    t1, t2 = sums(tiny_fn)
    parts = [sums(tiny_fn, shard_index=r, shard_count=9) for r in range(9)]
    assert all(not p[0].any() for p in parts[6:])
    np.testing.assert_allclose(sum(p[0] for p in parts), t1, rtol=1e-12, atol=0)
    # shards are for plain traces: not with a proposal or in batches
    prop = m.Proposal(ctx, seed=1)
    try:
        with pytest.raises(m.McrtError) as e:
            sums(flux_fn, shard_index=0, shard_count=2, proposal=prop.h)
        assert e.value.status == m.MCRT_ERR_UNSUPPORTED
    finally:
        prop.close()
