"""Heightfield ground on the GPU against the oracle.

* Ray-surface distances (the GPU's FP32 max-pyramid walk against the
  oracle's FP64 cell-by-cell walk) and surface heights and normals: within
  FP32 rounding, except for rays grazing an edge or the surface (a small,
  bounded fraction).
* Flux and image tallies over a cloud field on fractal terrain: within 4
  combined SE of the oracle (same random numbers, paired).
* Closed forms on the GPU: with no atmosphere the direct irradiance is 1 on
  average at any sun (exactly 1 per path with the sun overhead); a flat
  heightfield reproduces the flat ground.
* Bad heights and unsupported combinations are refused.
"""
import math

import numpy as np
import pytest

import scenes

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


def oscene(orc, sp, heights, **kw):
    a = dict(k=sp.k, dx=sp.dx, dy=sp.dy, dz=sp.dz, levels=sp.levels, k_clear=sp.k_clear, ssa_clear=sp.ssa_clear,
             ssa_cloud=sp.ssa_cloud, g=sp.g, ground_albedo=sp.ground_albedo, sun_zenith_deg=sp.sun_zenith_deg,
             sun_azimuth_deg=sp.sun_azimuth_deg, heights=heights)
    a.update(kw)
    return orc.Scene(**a)


def close_4se(a, sa, b, sb):
    return abs(a - b) <= 4.0 * math.hypot(sa, sb) + 1e-12


@pytest.mark.parametrize("hn", [(64, 48), (256, 256), (30, 21)])
def test_terrain_hits_vs_oracle(m, ctx, orc, hn):
    sp = scenes.blobs_small(0)
    r = np.random.default_rng(sum(hn))
    h = scenes.heightfield(max(hn), 0.3, seed=hn[0])[:hn[1], :hn[0]].copy()
    h[r.uniform(size=h.shape) < 0.02] = 0.3                   # a few spikes
    sc = m.Scene.from_spec(ctx, sp)
    try:
        sc.set_heightfield(h, 0.2)
        osc = oscene(orc, sp, h)
        Lx = float(np.float32(64) * np.float32(0.1))
        n = 2000
        o = np.stack([r.uniform(0, Lx, n), r.uniform(0, Lx, n), r.uniform(0.31, 3.2, n)], 1)
        d = r.normal(size=(n, 3))
        d[:, 2] = -np.abs(d[:, 2]) - 0.02
        # a quarter start just above the surface in any direction
        q = n // 4
        zs, _ = sc.terrain_height(o[:q, :2])
        o[:q, 2] = zs + r.uniform(0.002, 0.05, q)
        d[:q] = r.normal(size=(q, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        o = o.astype(np.float32)
        d = d.astype(np.float32)
        t = sc.terrain_hit(o, d)
        bad = 0
        for i in range(n):
            ref = orc.terrain_hit(osc, o[i].astype(np.float64), d[i].astype(np.float64))
            tr = math.inf if ref is None else ref[0]
            if math.isinf(tr) and math.isinf(t[i]):
                continue
            if not (abs(t[i] - tr) <= 2e-4 + 2e-5 * tr):
                bad += 1
        assert bad <= max(2, n // 200), bad
        assert np.isfinite(t).sum() > n // 2
        # heights and normals
        xy = np.stack([r.uniform(0, Lx, 500), r.uniform(0, Lx, 500)], 1).astype(np.float32)
        z, nn = sc.terrain_height(xy)
        for i in range(500):
            oz, on = orc.terrain_height(osc, float(xy[i, 0]), float(xy[i, 1]))
            assert abs(z[i] - oz) <= 2e-6 + 1e-5 * oz
            assert np.abs(nn[i] - on).max() <= 2e-5
    finally:
        sc.close()


@pytest.fixture(scope="module")
def terrain_scene(m, ctx):
    sp = scenes.blobs_small(0)
    sp.sun_zenith_deg = 50.0
    sp.sun_azimuth_deg = 30.0
    h = scenes.heightfield(256, 0.3, seed=7)
    sc = m.Scene.from_spec(ctx, sp)
    sc.set_heightfield(h, sp.ground_albedo)
    yield sp, h, sc
    sc.close()


def test_terrain_flux_vs_oracle(m, orc, terrain_scene):
    sp, h, sc = terrain_scene
    n = 60000
    g = sc.trace_flux(n, seed=11)
    o, _ = orc.trace_flux(oscene(orc, sp, h), n, seed=11)
    for q in range(3):
        assert close_4se(g.mean[q], g.se[q], o.mean[q], o.se[q]), (q, g.mean, o.mean, g.se, o.se)
    assert abs(g.mean[2] - o.mean[2]) < 0.5 * o.se[2]


def test_terrain_camera_vs_oracle(m, orc, terrain_scene):
    sp, h, sc = terrain_scene
    cam = scenes.nadir_camera(sp, 32, 32)
    g = sc.trace_camera(cam, 16, seed=12)
    oc = orc.Camera(cam.pos, cam.target, cam.up, cam.fov_deg, cam.width, cam.height)
    o, _ = orc.trace_camera(oscene(orc, sp, h), oc, 16, seed=12)
    blocks = lambda x: x.reshape(4, 8, 4, 8).sum(axis=(1, 3))
    z = np.abs(blocks(g.mean) - blocks(o.mean)) / np.hypot(np.sqrt(blocks(g.se ** 2)), np.sqrt(blocks(o.se ** 2)))
    assert int((z > 4).sum()) <= 1, z
    sg = math.sqrt((g.se ** 2).sum()) / g.se.size
    so = math.sqrt((o.se ** 2).sum()) / o.se.size
    assert close_4se(g.mean.mean(), sg, o.mean.mean(), so)


@pytest.mark.parametrize("zenith", [0.0, 45.0, 72.0])
def test_terrain_direct_sunlight_conserved_gpu(m, ctx, zenith):
    sp = scenes.homogeneous(32, 32, 16, 0.1, 0.0, levels=2, ground_albedo=0.0, sun_zenith_deg=zenith,
                            sun_azimuth_deg=120.0)
    sc = m.Scene.from_spec(ctx, sp)
    try:
        sc.set_heightfield(scenes.heightfield(128, 0.3, seed=3), 0.0)
        r = sc.trace_flux(400000, seed=13)
        if zenith == 0.0:
            assert r.mean[0] == pytest.approx(1.0, abs=2e-6) and r.se[0] < 1e-6
        else:
            assert abs(r.mean[0] - 1.0) <= 3 * r.se[0], (r.mean[0], r.se[0])
            assert r.se[0] > 1e-4
        assert r.mean[1] == 0.0
    finally:
        sc.close()


def test_flat_heightfield_is_flat_ground_gpu(m, ctx):
    sp = scenes.blobs_small(0)
    a = m.Scene.from_spec(ctx, sp)
    b = m.Scene.from_spec(ctx, sp)
    try:
        b.set_heightfield(np.zeros((64, 64), np.float32), sp.ground_albedo)
        ra = a.trace_flux(100000, seed=21)
        rb = b.trace_flux(100000, seed=21)
        for q in range(3):
            assert close_4se(ra.mean[q], ra.se[q], rb.mean[q], rb.se[q])
            assert abs(ra.mean[q] - rb.mean[q]) <= 0.1 * ra.se[q] + 1e-9
    finally:
        a.close()
        b.close()


def test_terrain_bad_arguments(m, ctx):
    sp = scenes.blobs_small(0)
    sc = m.Scene.from_spec(ctx, sp)
    try:
        for bad in (np.full((8, 8), -0.01, np.float32), np.full((8, 8), np.nan, np.float32),
                    np.full((8, 8), 10.0, np.float32)):
            with pytest.raises(m.McrtError) as e:
                sc.set_heightfield(bad, 0.2)
            assert e.value.status == m.MCRT_ERR_ARG
        with pytest.raises(m.McrtError) as e:
            sc.terrain_hit(np.zeros((1, 3)), np.ones((1, 3)))
        assert e.value.status == m.MCRT_ERR_STATE
        sc.set_heightfield(np.full((8, 8), 0.1, np.float32), 0.2)
        prop = m.Proposal(ctx, seed=1)
        try:
            with pytest.raises(m.McrtError) as e:
                sc.trace_flux(100, seed=1, proposal=prop)
            assert e.value.status == m.MCRT_ERR_UNSUPPORTED
        finally:
            prop.close()
        with pytest.raises(m.McrtError) as e:
            m.trace_batch(ctx, [(sc, 0.0, 30.0, 0.0, 100, 1)])
        assert e.value.status == m.MCRT_ERR_UNSUPPORTED
        # back to the flat ground
        m.mcrt_scene_set_ground_flat(ctx.h, sc.h, 0.2)
        assert np.isfinite(sc.trace_flux(1000, seed=1).mean).all()
    finally:
        sc.close()
