"""Parity at the full sizes the bench times, in its launch configuration.

The oracle cannot trace whole full-size workloads in seconds, so each check
takes outputs it can compute one by one, or properties that hold at any
size:

* The bench image (cumulus 512x512x160 at 25 m, 1024 x 1024 nadir image at
  64 spp, default options): the majorant pyramid and the octree of the
  whole field bit-exact; 512 sampled pixels traced by the oracle with the
  same path ids, paired per pixel (same random numbers) and within 4
  combined SE over the sample -- over the pyramid (the headline) and over
  the octree (the line's octree figure).
* The bench batch (96 instances, 814 items, autotuned launch shape, over
  the octree as the bench traces it): sampled items against the oracle's
  trace of the same item's first paths over the same octree (same seeds
  and path ids), within 4 combined SE.
* The largest sweep field (2048^2 x 640, 2.7e9 voxels, over the 4096^2
  heightfield): sampled pyramid and octree cells bit-exact against the
  oracle's reduction of their voxel blocks; the pyramid, the octree and
  BF16 storage give the same flux within 4 combined SE.
"""
import math

import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1902_01137_gb300 as m
    from paper_1902_01137_gb300 import build
    build.build()
    ctx = m.Context(0)
    yield torch, m, ctx
    ctx.close()


def close_4se(a, sa, b, sb):
    return abs(a - b) <= 4.0 * math.hypot(sa, sb) + 1e-12


def _oscene(orc, sp, **kw):
    a = dict(k=sp.k, dx=sp.dx, dy=sp.dy, dz=sp.dz, levels=sp.levels, k_clear=sp.k_clear, ssa_clear=sp.ssa_clear,
             ssa_cloud=sp.ssa_cloud, g=sp.g, ground_albedo=sp.ground_albedo, sun_zenith_deg=sp.sun_zenith_deg,
             sun_azimuth_deg=sp.sun_azimuth_deg)
    a.update(kw)
    return orc.Scene(**a)


def test_bench_image_full_size(env, orc):
    import bench
    torch, m, ctx = env
    spec, cam = bench.make_workload()
    assert spec.k.shape == (160, 512, 512) and (cam.width, cam.height) == (1024, 1024)
    sc = m.Scene.from_spec(ctx, spec)
    try:
        # the whole field's grids, bit for bit
        want = orc.build_pyramid(spec.k, spec.levels)
        want_min = orc.build_pyramid_min(spec.k, spec.levels)
        for L in range(1, spec.levels + 1):
            assert np.array_equal(sc.majorants(L).view(np.uint32), want[L - 1].view(np.uint32)), L
            assert np.array_equal(sc.minorants(L).view(np.uint32), want_min[L - 1].view(np.uint32)), L
        sc.build_octree()
        levels = orc.octree_levels(spec.shape_xyz)
        omax, omin = orc.build_octree(spec.k, levels)
        for L in range(1, levels + 1):
            gmax, gmin = sc.octree(L)
            assert np.array_equal(gmax.view(np.uint32), omax[L - 1].view(np.uint32)), L
            assert np.array_equal(gmin.view(np.uint32), omin[L - 1].view(np.uint32)), L
        # the bench step's trace (default options), sampled pixels
        seed = 1101
        g = sc.trace_camera(cam, bench.SPP, seed=seed)
        r = np.random.default_rng(8)
        pix = np.sort(r.choice(cam.width * cam.height, size=512, replace=False))
        oc = orc.Camera(cam.pos, cam.target, cam.up, cam.fov_deg, cam.width, cam.height)
        o, stats = orc.trace_camera(_oscene(orc, spec), oc, bench.SPP, seed, pixels=pix)
        assert stats[0] == 0
        gm, gs = g.mean.ravel()[pix], g.se.ravel()[pix]
        om, os_ = o.mean.ravel()[pix], o.se.ravel()[pix]
        # same random numbers: most pixels agree far below their noise
        rel = np.abs(gm - om) / np.maximum(np.abs(om), 1e-3)
        assert np.median(rel) < 1e-3, np.median(rel)
        z = np.abs(gm - om) / np.maximum(np.hypot(gs, os_), 1e-300)
        assert int(np.sum(z > 4.0)) <= max(1, int(3 * pix.size * 6.33e-5)), np.sort(z)[-5:]
        sg = math.sqrt(np.sum(gs ** 2)) / pix.size
        so = math.sqrt(np.sum(os_ ** 2)) / pix.size
        assert close_4se(gm.mean(), sg, om.mean(), so), (gm.mean(), om.mean(), sg, so)
        # the bench line's octree figure: the same image over the octree,
        # finest leaves 2^3 voxels, against the oracle over the same octree
        g2 = sc.trace_camera(cam, bench.SPP, seed=seed, grid=m.MCRT_GRID_OCTREE, finest_level=1)
        o2, st2 = orc.trace_camera(_oscene(orc, spec, grid=1, finest_level=1), oc, bench.SPP, seed, pixels=pix)
        assert st2[0] == 0
        gm2, gs2 = g2.mean.ravel()[pix], g2.se.ravel()[pix]
        om2, os2 = o2.mean.ravel()[pix], o2.se.ravel()[pix]
        rel2 = np.abs(gm2 - om2) / np.maximum(np.abs(om2), 1e-3)
        assert np.median(rel2) < 1e-3, np.median(rel2)
        sg2 = math.sqrt(np.sum(gs2 ** 2)) / pix.size
        so2 = math.sqrt(np.sum(os2 ** 2)) / pix.size
        assert close_4se(gm2.mean(), sg2, om2.mean(), so2), (gm2.mean(), om2.mean(), sg2, so2)
    finally:
        sc.close()


def test_bench_batch_full_size(env, orc):
    import bench
    torch, m, ctx = env
    dev = torch.device("cuda", 0)
    inst = scenes.batch_instances(0)
    assert len(inst) == 96
    specs = [scenes.cumulus(b.nx, b.nx, b.nz, seed=b.field_seed, device=dev) for b in inst]
    scs = [m.Scene(ctx, sp.k, sp.dx, sp.dy, sp.dz, k_clear=sp.k_clear, ssa_clear=sp.ssa_clear,
                   ssa_cloud=sp.ssa_cloud, g=sp.g, levels=sp.levels, albedo=sp.ground_albedo) for sp in specs]
    try:
        for s in scs:
            s.build_octree()
        items = scenes.batch_items(inst, lambda i: scs[i])
        assert len(items) == 814
        topts = m.mcrt_trace_opts_default()
        topts.grid = m.MCRT_GRID_OCTREE
        topts.finest_level = 1
        opts, _ = m.mcrt_autotune_batch(ctx.h, m.make_batch_items(items), 0.25, topts)
        shape = dict(chunk=opts.chunk, rare_batch=opts.rare_batch, block_size=opts.block_size)
        res = m.trace_batch(ctx, items, grid=m.MCRT_GRID_OCTREE, finest_level=1, **shape)
        owner = bench._item_instance(inst)
        r = np.random.default_rng(4)
        # sampled items: two of the smallest fields, one mid-size, one of the largest
        small = [i for i in range(len(items)) if inst[owner[i]].nx <= 128]
        mid = [i for i in range(len(items)) if inst[owner[i]].nx == 256]
        large = [i for i in range(len(items)) if inst[owner[i]].nx == 1024]
        picks = list(r.choice(small, 2, replace=False)) + [int(r.choice(mid))] + [int(r.choice(large))]
        for i in picks:
            _, kg, z, az, npaths, seed = items[i]
            sp = specs[owner[i]]
            k = sp.k.cpu().numpy()
            osc = orc.Scene(k=k, dx=sp.dx, dy=sp.dy, dz=sp.dz, levels=sp.levels, k_clear=sp.k_clear,
                            ssa_clear=sp.ssa_clear, ssa_cloud=sp.ssa_cloud, g=sp.g, ground_albedo=sp.ground_albedo,
                            sun_zenith_deg=z, sun_azimuth_deg=az, k_gas=kg, grid=1, finest_level=1)
            n = min(npaths, 20000)
            o, st = orc.trace_flux(osc, n, seed=seed)
            assert st[0] == 0
            for q in range(4):          # T_dir, T_dif, T_tot, dT/dg
                assert close_4se(res.mean[i, q], res.se[i, q], o.mean[q], o.se[q]), \
                    (i, q, res.mean[i, :4], o.mean[:4], res.se[i, :4], o.se[:4])
    finally:
        for s in scs:
            s.close()
        del specs
        torch.cuda.empty_cache()


def test_largest_sweep_field(env, orc):
    torch, m, ctx = env
    dev = torch.device("cuda", 0)
    spec = scenes.cumulus(2048, 2048, 640, seed=0, device=dev)
    spec.sun_zenith_deg = 60.0
    hf = scenes.heightfield(4096, 0.3, seed=0)
    nz, ny, nx = spec.k.shape
    assert (nx, ny, nz) == (2048, 2048, 640)
    sc = m.Scene.from_spec(ctx, spec)
    sb = None
    try:
        sc.set_heightfield(hf, spec.ground_albedo)
        sc.build_octree()
        r = np.random.default_rng(12)
        # sampled pyramid cells of levels 1 and 2 (8^3 and 64^3 voxels) and
        # octree cells of levels 1, 3 and 6 (2^3, 8^3, 64^3 voxels): the
        # oracle reduces each cell's voxel block on the host
        for L, count in ((1, 24), (2, 6)):
            got = sc.majorants(L)
            gmin = sc.minorants(L)
            f = 8 ** L
            for _ in range(count):
                cz, cy, cx = (int(r.integers(0, d)) for d in got.shape)
                blk = spec.k[cz * f:(cz + 1) * f, cy * f:(cy + 1) * f, cx * f:(cx + 1) * f].cpu().numpy()
                w = orc.build_pyramid(blk, L)[-1]
                wm = orc.build_pyramid_min(blk, L)[-1]
                assert w.size == 1 and got[cz, cy, cx].view(np.uint32) == w.ravel()[0].view(np.uint32)
                assert gmin[cz, cy, cx].view(np.uint32) == wm.ravel()[0].view(np.uint32)
        for L, count in ((1, 24), (3, 12), (6, 4)):
            gmax, gmin = sc.octree(L)
            f = 1 << L
            for _ in range(count):
                cz, cy, cx = (int(r.integers(0, d)) for d in gmax.shape)
                blk = spec.k[cz * f:(cz + 1) * f, cy * f:(cy + 1) * f, cx * f:(cx + 1) * f].cpu().numpy()
                omax, omin = orc.build_octree(blk, L)
                assert gmax[cz, cy, cx].view(np.uint32) == omax[-1].ravel()[0].view(np.uint32)
                assert gmin[cz, cy, cx].view(np.uint32) == omin[-1].ravel()[0].view(np.uint32)
        # any valid majorant, either storage: the same flux
        n = 10_000_000
        a = sc.trace_flux(n, seed=7)
        b = sc.trace_flux(n, seed=8, grid=m.MCRT_GRID_OCTREE, finest_level=1)
        sc.close()
        sc = None
        sb = m.Scene.from_spec(ctx, spec, storage=m.MCRT_STORAGE_BF16)
        sb.set_heightfield(hf, spec.ground_albedo)
        c = sb.trace_flux(n, seed=9)
        for q in range(3):
            assert close_4se(a.mean[q], a.se[q], b.mean[q], b.se[q]), ("octree", q, a.mean, b.mean)
            assert close_4se(a.mean[q], a.se[q], c.mean[q], c.se[q]), ("bf16", q, a.mean, c.mean)
        assert 0.0 < a.mean[0] < 1.0 and 0.0 < a.mean[1] < 1.0
    finally:
        if sc is not None:
            sc.close()
        if sb is not None:
            sb.close()
        del spec
        torch.cuda.empty_cache()


def test_lane_sums_stay_within_their_fp32_bound(env):
    """Each lane sums the scores x and x^2 of its chunk (at most 8 paths) in
    FP32 before one FP64 atomic add, so a pixel's sums may differ from exact
    FP64 sums of the same FP32 path scores by at most (chunk - 1) 2^-24 of
    themselves (all terms are >= 0).  Tracing the same paths with one path
    per claim (every score reaches the FP64 sums alone) and with 8 per claim
    checks that bound pixel by pixel on the bench field (cumulus
    512x512x160, 64 x 64 nadir image at 64 spp: cloudy and clear pixels,
    scores spread over orders of magnitude)."""
    import bench
    torch, m, ctx = env
    spec, _ = bench.make_workload()
    sc = m.Scene.from_spec(ctx, spec, k=torch.from_numpy(spec.k).cuda())
    cd = m.CameraDesc()
    cam = scenes.nadir_camera(spec, 64, 64)
    for i in range(3):
        cd.pos[i], cd.target[i], cd.up[i] = cam.pos[i], cam.target[i], cam.up[i]
    cd.fov_deg, cd.width, cd.height = cam.fov_deg, cam.width, cam.height
    try:
        sums = {}
        for chunk in (1, 8):
            o = m.mcrt_trace_opts_default()
            o.chunk = chunk
            t = m.mcrt_trace_camera(ctx.h, sc.h, cd, 64, 9, o)
            try:
                sums[chunk] = m.mcrt_tally_read_sums(ctx.h, t)
            finally:
                m.mcrt_tally_destroy(t)
        for q in range(2):
            exact, grouped = sums[1][q][:, 0], sums[8][q][:, 0]
            assert exact.max() > 0.0
            bound = 7 * 2.0 ** -24 * exact + 1e-15 * exact.max()
            assert np.all(np.abs(grouped - exact) <= bound), float(np.max(np.abs(grouped - exact) / np.maximum(exact, 1e-300)))
    finally:
        sc.close()
