"""The paper's octree (Sec. 3.1.1, 2^3 groups merged recursively) on the GPU
against the oracle.

* Octree maxima and minima, FP32 and BF16 storage, ragged sizes: bit-exact.
* Leaf sequences and distances over the octree (several tau~, finest
  levels): bit-exact with the oracle's FP32 traversal spec.
* Flux and image tallies over the octree within 4 combined SE of the
  oracle over the same octree, on the same seeds (paired).
* Octree and pyramid tallies agree (any valid majorant, Sec. 2.3-2.4);
  batches over the octree equal single traces; the no-allocation entry
  point takes it too.
* Refusals: the octree selected before it is built, a bad grid value.
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


def oscene(orc, sp, **kw):
    a = dict(k=sp.k, dx=sp.dx, dy=sp.dy, dz=sp.dz, levels=sp.levels, k_clear=sp.k_clear, ssa_clear=sp.ssa_clear,
             ssa_cloud=sp.ssa_cloud, g=sp.g, ground_albedo=sp.ground_albedo, sun_zenith_deg=sp.sun_zenith_deg,
             sun_azimuth_deg=sp.sun_azimuth_deg)
    a.update(kw)
    return orc.Scene(**a)


def close_4se(a, sa, b, sb):
    return abs(a - b) <= 4.0 * math.hypot(sa, sb) + 1e-12


@pytest.mark.parametrize("shape", [(32, 64, 64), (21, 29, 37), (1, 1, 1), (9, 8, 65), (40, 72, 72)])
@pytest.mark.parametrize("bf16", [False, True])
def test_octree_bit_exact(m, ctx, orc, shape, bf16):
    r = np.random.default_rng(sum(shape) + 7)
    k = (r.lognormal(0.0, 2.0, shape) * (r.uniform(size=shape) < 0.4)).astype(np.float32)
    sc = m.Scene(ctx, k, 0.1, 0.1, 0.1, levels=1, storage=m.MCRT_STORAGE_BF16 if bf16 else 0)
    try:
        sc.build_octree()
        levels = orc.octree_levels(shape[::-1])
        assert sc.octree_levels == levels
        wmax, wmin = orc.build_octree(k, levels, round_nearest_bf16=bf16)
        for L in range(1, levels + 1):
            gmax, gmin = sc.octree(L)
            assert gmax.shape == wmax[L - 1].shape
            assert np.array_equal(gmax.view(np.uint32), wmax[L - 1].view(np.uint32)), L
            assert np.array_equal(gmin.view(np.uint32), wmin[L - 1].view(np.uint32)), ("min", L)
    finally:
        sc.close()


def _dda_field():
    sp = scenes.random_voxels(72, 64, 40, 0.1, 3.0, seed=2, sparsity=0.5)
    k = sp.k.copy()
    k[:, :, 32:64] = 0.0
    k[24:, :, :] *= 0.01
    k[:, 40:44, :] *= 0.2
    return sp, k


@pytest.mark.parametrize("tau,finest", [(1.0, 0), (0.3, 0), (5.0, 1), (float("inf"), 1), (0.0, 0), (1.0, 1)])
def test_octree_dda_bit_exact(m, ctx, orc, tau, finest):
    sp, k = _dda_field()
    sc = m.Scene(ctx, k, sp.dx, sp.dy, sp.dz, levels=2)
    osc = orc.Scene(k=k, dx=sp.dx, dy=sp.dy, dz=sp.dz, levels=2, tau_merge=tau, finest_level=finest, grid=1)
    try:
        sc.build_octree()
        o, d = scenes.random_rays(sp, 200, seed=23)
        o = np.concatenate([o, np.array([[0.85, 0.85, 0.0], [0.85, 0.85, 4.0], [0.0, 1.05, 1.05]], np.float32)])
        d = np.concatenate([d, np.array([[0, 0, 1], [0, 0, -1], [0.6, 0.8, 0.0]], np.float32)])
        for i in range(len(o)):
            cg, tg, sg = sc.dda(o[i], d[i], tau, finest, cap=4000, grid=m.MCRT_GRID_OCTREE)
            co, to, so = orc.dda_spec(osc, o[i], d[i], cap=4000)
            assert sg == so, i
            assert np.array_equal(cg, co), i
            assert np.array_equal(tg.view(np.uint32), to.view(np.uint32)), i
        # the pyramid is still there and unchanged beside it
        cg, tg, sg = sc.dda(o[0], d[0], tau, finest, cap=4000)
        co, to, so = orc.dda_spec(orc.Scene(k=k, dx=sp.dx, dy=sp.dy, dz=sp.dz, levels=2, tau_merge=tau,
                                            finest_level=finest), o[0], d[0], cap=4000)
        assert np.array_equal(cg, co) and sg == so
    finally:
        sc.close()


@pytest.fixture(scope="module")
def small(m, ctx):
    sp = scenes.blobs_small(0)
    sc = m.Scene.from_spec(ctx, sp)
    sc.build_octree()
    yield sp, sc
    sc.close()


@pytest.mark.parametrize("opts", [dict(tau_merge=1.0), dict(tau_merge=0.1), dict(tau_merge=10.0),
                                  dict(tau_merge=1.0, finest_level=1), dict(tau_merge=float("inf")),
                                  dict(tau_merge=1.0, sun_mode=2), dict(tau_merge=1.0, sun_mode=1)])
def test_octree_flux_vs_oracle(m, orc, small, opts):
    sp, sc = small
    n = 60000
    g = sc.trace_flux(n, seed=11, grid=m.MCRT_GRID_OCTREE, **opts)
    o, _ = orc.trace_flux(oscene(orc, sp, grid=1, **opts), n, seed=11)
    for q in range(3):
        assert close_4se(g.mean[q], g.se[q], o.mean[q], o.se[q]), (opts, q, g.mean[q], o.mean[q])
    # same random numbers over the same leaves: far closer than the noise
    assert abs(g.mean[2] - o.mean[2]) < 0.25 * o.se[2], (opts, g.mean[2], o.mean[2], o.se[2])


def test_octree_camera_vs_oracle(m, orc, small):
    sp, sc = small
    cam = scenes.nadir_camera(sp, 64, 64)
    g = sc.trace_camera(cam, 16, seed=12, grid=m.MCRT_GRID_OCTREE)
    o, _ = orc.trace_camera(oscene(orc, sp, grid=1), orc.Camera(cam.pos, cam.target, cam.up, cam.fov_deg,
                                                                 cam.width, cam.height), 16, seed=12)
    rel = np.abs(g.mean - o.mean) / np.maximum(np.abs(o.mean), 1e-3)
    assert np.median(rel) < 1e-3, np.median(rel)
    mg, mo = g.mean.mean(), o.mean.mean()
    sg = math.sqrt(np.sum(g.se ** 2)) / g.mean.size
    so = math.sqrt(np.sum(o.se ** 2)) / o.mean.size
    assert close_4se(mg, sg, mo, so), (mg, mo, sg, so)


def test_octree_and_pyramid_agree(m, small):
    sp, sc = small
    n = 400000
    a = sc.trace_flux(n, seed=21)
    b = sc.trace_flux(n, seed=22, grid=m.MCRT_GRID_OCTREE)
    for q in range(3):
        assert close_4se(a.mean[q], a.se[q], b.mean[q], b.se[q]), (q, a.mean[q], b.mean[q])


def test_octree_batch_matches_single_traces(m, ctx, small):
    sp, sc = small
    items = [(sc, 0.0, 20.0, 10.0, 30001, 5), (sc, 0.02, 45.0, 0.0, 20000, 6)]
    r = m.trace_batch(ctx, items, grid=m.MCRT_GRID_OCTREE)
    try:
        for i, (s, kg, z, az, npaths, seed) in enumerate(items):
            if kg:
                continue
            m.mcrt_scene_set_sun(ctx.h, s.h, z, az)
            single = s.trace_flux(npaths, seed=seed, grid=m.MCRT_GRID_OCTREE)
            np.testing.assert_allclose(r.mean[i, :3], single.mean, rtol=4e-6, atol=1e-12)
    finally:
        m.mcrt_scene_set_sun(ctx.h, sc.h, sp.sun_zenith_deg, sp.sun_azimuth_deg)


def test_octree_noalloc_matches_allocating_trace(m, ctx, small):
    torch = pytest.importorskip("torch")
    sp, sc = small
    cam = scenes.nadir_camera(sp, 32, 32)
    g = sc.trace_camera(cam, 8, seed=31, grid=m.MCRT_GRID_OCTREE)
    sc.trace_flux(1000, seed=1)            # leaves the pyramid's leaf map current
    cd = m.CameraDesc()
    for i in range(3):
        cd.pos[i], cd.target[i], cd.up[i] = cam.pos[i], cam.target[i], cam.up[i]
    cd.fov_deg, cd.width, cd.height = cam.fov_deg, cam.width, cam.height
    opts = m.mcrt_trace_opts_default()
    opts.grid = m.MCRT_GRID_OCTREE
    mean = torch.zeros(32 * 32, dtype=torch.float64, device="cuda")
    se = torch.zeros_like(mean)
    m.mcrt_trace_camera_noalloc(ctx.h, sc.h, cd, 8, 31, opts, mean.data_ptr(), se.data_ptr())
    np.testing.assert_allclose(mean.cpu().numpy().reshape(32, 32), g.mean, rtol=4e-6, atol=1e-12)


def test_octree_refusals(m, ctx):
    sp = scenes.blobs_small(0)
    sc = m.Scene.from_spec(ctx, sp)
    try:
        with pytest.raises(m.McrtError) as e:
            sc.trace_flux(100, seed=1, grid=m.MCRT_GRID_OCTREE)
        assert e.value.status == m.MCRT_ERR_STATE
        with pytest.raises(m.McrtError) as e:
            sc.trace_flux(100, seed=1, grid=7)
        assert e.value.status == m.MCRT_ERR_ARG
        with pytest.raises(m.McrtError) as e:
            m.mcrt_scene_build_octree(ctx.h, sc.h, 21)
        assert e.value.status == m.MCRT_ERR_ARG
        sc.build_octree(2)
        assert sc.octree_levels == 2
        r = sc.trace_flux(1000, seed=1, grid=m.MCRT_GRID_OCTREE, tau_merge=float("inf"))
        assert np.all(np.isfinite(r.mean))
    finally:
        sc.close()


# ---------------------------------------------------------------------------
# the other kernel variants over the octree (terrain walk, Rayleigh species,
# learned proposal): the grid changes only the leaves, so each must still
# match the oracle over the same octree
# ---------------------------------------------------------------------------
def test_octree_with_terrain_vs_oracle(m, ctx, orc):
    sp = scenes.blobs_small(0)
    sp.sun_zenith_deg = 50.0
    sp.sun_azimuth_deg = 30.0
    h = scenes.heightfield(256, 0.3, seed=7)
    sc = m.Scene.from_spec(ctx, sp)
    try:
        sc.set_heightfield(h, sp.ground_albedo)
        sc.build_octree()
        n = 60000
        g = sc.trace_flux(n, seed=13, grid=m.MCRT_GRID_OCTREE)
        o, _ = orc.trace_flux(oscene(orc, sp, heights=h, grid=1), n, seed=13)
        for q in range(3):
            assert close_4se(g.mean[q], g.se[q], o.mean[q], o.se[q]), (q, g.mean, o.mean)
        assert abs(g.mean[2] - o.mean[2]) < 0.5 * o.se[2]
    finally:
        sc.close()


def test_octree_with_rayleigh_vs_oracle(m, ctx, orc):
    sp = scenes.blobs_small(0)
    sp.k = sp.k + np.float32(0.04)
    sp.k_clear = 0.05
    sc = m.Scene.from_spec(ctx, sp)
    try:
        m.mcrt_scene_set_clear_sky_phase(ctx.h, sc.h, m.MCRT_PHASE_RAYLEIGH)
        sc.build_octree()
        n = 60000
        g = sc.trace_flux(n, seed=15, grid=m.MCRT_GRID_OCTREE, tau_merge=3.0)
        o, _ = orc.trace_flux(oscene(orc, sp, clear_phase=1, grid=1, tau_merge=3.0), n, seed=15)
        for q in range(3):
            assert close_4se(g.mean[q], g.se[q], o.mean[q], o.se[q]), (q, g.mean, o.mean)
        assert abs(g.mean[2] - o.mean[2]) < 0.25 * o.se[2]
    finally:
        sc.close()


def test_octree_with_learned_proposal_vs_oracle(m, ctx, orc):
    """A fixed network over the octree (its features still read the
    pyramid's levels 1 and 2): the oracle with the same parameters over the
    same octree agrees within 4 combined SE."""
    sp = scenes.blobs_small(0)
    p = orc.xavier_init(21)
    r = np.random.default_rng(21)
    p[p.size - 40:] = r.normal(size=40) * 0.5
    p = p.astype(np.float32).astype(np.float64)
    sc = m.Scene.from_spec(ctx, sp)
    prop = m.Proposal(ctx, params=p)
    try:
        sc.build_octree()
        n = 100000
        g = sc.trace_flux(n, seed=42, proposal=prop, batch_paths=30000, grid=m.MCRT_GRID_OCTREE)
        o, _ = orc.trace_flux(oscene(orc, sp, mlp=p, grid=1), n, seed=42)
        for q in range(3):
            assert close_4se(g.mean[q], g.se[q], o.mean[q], o.se[q]), (q, g.mean, o.mean)
    finally:
        prop.close()
        sc.close()


def test_batch_plan_survives_scene_changes(m, ctx):
    """A plan keeps its own options: a trace with another tau~ or grid in
    between, or the octree rebuilt elsewhere in memory, does not change
    what the plan traces (its records are remade before the launch)."""
    sp = scenes.blobs_small(0)
    sc = m.Scene.from_spec(ctx, sp)
    try:
        sc.build_octree()
        items = [(sc, 0.0, 20.0, 10.0, 20000, 5), (sc, 0.01, 40.0, 0.0, 9000, 6)]
        for grid in (m.MCRT_GRID_PYRAMID, m.MCRT_GRID_OCTREE):
            plan = m.BatchPlan(ctx, items, grid=grid, tau_merge=1.0)
            try:
                r1 = plan.run()
                sc.trace_flux(5000, seed=3, tau_merge=10.0, grid=m.MCRT_GRID_OCTREE)
                sc.trace_flux(5000, seed=3, tau_merge=0.0)
                r2 = plan.run()
                np.testing.assert_allclose(r2.mean, r1.mean, rtol=4e-6, atol=1e-12)
                sc.build_octree()                  # new device buffers for the octree
                r3 = plan.run()
                np.testing.assert_allclose(r3.mean, r1.mean, rtol=4e-6, atol=1e-12)
                direct = m.trace_batch(ctx, items, grid=grid, tau_merge=1.0)
                np.testing.assert_allclose(r1.mean, direct.mean, rtol=4e-6, atol=1e-12)
            finally:
                plan.close()
    finally:
        sc.close()
