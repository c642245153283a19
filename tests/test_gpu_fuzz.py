"""Randomised parity with the oracle: the grids and the traversal bit for
bit, then the estimators on random scenes.

Thirty seeded cases, each drawn at random:
- field shape (1 to 40 voxels per axis, so levels are clipped at ragged edges);
- voxel size and aspect; a sparse lognormal extinction of random scale;
- FP32 or BF16 storage;
- the tracked grid (8^L pyramid or 2^L octree), the finest level and tau~.

Every case checks that the GPU's grid levels equal the oracle's bit for bit.
Each of its rays must then give the same leaves and the same t bits as the
oracle's FP32 traversal spec. The rays are random, plus hard ones: starting
exactly on voxel faces, on the ground and top faces, along the axes, and
nearly parallel to a face.

Sixteen more seeded cases draw the scene constants and the options (g,
both single-scattering albedos, clear-sky extinction, ground albedo, sun
position, ratio / delta / decomposition tracking, grid, finest level, tau~,
storage); their flux tallies and image means must agree with the oracle's
within 4 combined SE on the same seeds.
"""
import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu

CASES = 30
TAUS = (0.0, 0.05, 0.5, 1.0, 3.0, 30.0, float("inf"))


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1902_01137_gb300 as m
    from paper_1902_01137_gb300 import build
    build.build()
    ctx = m.Context(0)
    yield m, ctx
    ctx.close()


def _case(i):
    r = np.random.default_rng(7000 + i)
    nx, ny, nz = (int(v) for v in r.integers(1, 41, 3))
    h = float(r.choice([0.025, 0.1, 0.37, 1.0]))
    dx, dy, dz = (float(np.float32(h * a)) for a in (1.0, float(r.choice([1.0, 0.5])), float(r.choice([0.5, 1.0, 2.0]))))
    k = r.lognormal(r.uniform(-3.0, 2.0), 1.5, (nz, ny, nx))
    k[r.uniform(size=k.shape) > r.uniform(0.2, 1.0)] = 0.0
    k = k.astype(np.float32)
    levels = 1
    while 8 ** levels < max(nx, ny, nz):
        levels += 1
    return dict(k=k, dx=dx, dy=dy, dz=dz, levels=levels, bf16=bool(r.integers(0, 2)), grid=int(r.integers(0, 2)),
                finest=int(r.integers(0, 2)), tau=float(r.choice(TAUS)), seed=8000 + i)


def _rays(c, n=40):
    r = np.random.default_rng(c["seed"])
    nz, ny, nx = c["k"].shape
    L = np.array([nx * c["dx"], ny * c["dy"], nz * c["dz"]], dtype=np.float32)
    o = (r.uniform(size=(n, 3)) * L).astype(np.float32)
    v = r.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    d = v.astype(np.float32)
    # starts exactly on interior voxel faces
    for j in range(0, 8):
        a = j % 3
        nn = (nx, ny, nz)[a]
        o[j, a] = np.float32(np.float32(int(r.integers(0, nn + 1))) * np.float32((c["dx"], c["dy"], c["dz"])[a]))
    extra_o, extra_d = [], []
    mid = (L * 0.37).astype(np.float32)
    extra_o += [[mid[0], mid[1], 0.0], [mid[0], mid[1], L[2]]]             # ground and top faces
    extra_d += [[0.0, 0.0, 1.0], [0.0, 0.0, -1.0]]
    for a in range(3):                                                      # along each axis, both ways
        for s in (1.0, -1.0):
            e = [0.0, 0.0, 0.0]
            e[a] = s
            extra_o.append(list(mid))
            extra_d.append(e)
    t = np.array([1.0, 1e-7, 0.3])                                          # nearly parallel to a face
    extra_o.append(list(mid))
    extra_d.append(list((t / np.linalg.norm(t)).astype(np.float32)))
    o = np.concatenate([o, np.array(extra_o, np.float32)])
    d = np.concatenate([d, np.array(extra_d, np.float32)])
    return o, d


@pytest.mark.parametrize("i", range(CASES))
def test_random_case_bit_exact(env, orc, i):
    m, ctx = env
    c = _case(i)
    sc = m.Scene(ctx, c["k"], c["dx"], c["dy"], c["dz"], levels=c["levels"],
                 storage=m.MCRT_STORAGE_BF16 if c["bf16"] else m.MCRT_STORAGE_F32)
    try:
        # the grids
        want = orc.build_pyramid(c["k"], c["levels"], round_up_bf16=c["bf16"])
        for L in range(1, c["levels"] + 1):
            assert np.array_equal(sc.majorants(L).view(np.uint32), want[L - 1].view(np.uint32)), ("pyramid", L)
        if c["grid"] == 1:
            sc.build_octree()
            ol = orc.octree_levels(c["k"].shape[::-1])
            omax, omin = orc.build_octree(c["k"], ol, round_nearest_bf16=c["bf16"])
            for L in range(1, ol + 1):
                gmax, gmin = sc.octree(L)
                assert np.array_equal(gmax.view(np.uint32), omax[L - 1].view(np.uint32)), ("octree", L)
                assert np.array_equal(gmin.view(np.uint32), omin[L - 1].view(np.uint32)), ("octree min", L)
        # the traversal
        osc = orc.Scene(k=c["k"], dx=c["dx"], dy=c["dy"], dz=c["dz"], levels=c["levels"], tau_merge=c["tau"],
                        finest_level=c["finest"], bf16=c["bf16"], grid=c["grid"])
        o, d = _rays(c)
        for j in range(len(o)):
            cg, tg, sg = sc.dda(o[j], d[j], c["tau"], c["finest"], cap=600, grid=c["grid"])
            co, to, so = orc.dda_spec(osc, o[j], d[j], cap=600)
            assert sg == so, (i, j, sg, so, c["k"].shape)
            assert np.array_equal(cg, co), (i, j)
            assert np.array_equal(tg.view(np.uint32), to.view(np.uint32)), (i, j)
    finally:
        sc.close()


# ---------------------------------------------------------------------------
# estimators: random scene constants and options against the oracle
# ---------------------------------------------------------------------------
TALLY_CASES = 16


def _scene_case(i):
    r = np.random.default_rng(9100 + i)
    nx, ny, nz = (int(v) for v in r.integers(8, 33, 3))
    h = float(np.float32(r.choice([0.05, 0.1, 0.2])))
    k = r.lognormal(r.uniform(-1.0, 2.0), 1.2, (nz, ny, nx))
    k[r.uniform(size=k.shape) < r.uniform(0.3, 0.9)] = 0.0
    k_clear = float(r.choice([0.0, 0.01, 0.2]))
    k = (k + k_clear).astype(np.float32)
    levels = 1
    while 8 ** levels < max(nx, ny, nz):
        levels += 1
    return dict(k=k, h=h, levels=levels, k_clear=k_clear, ssa_clear=float(r.uniform(0.5, 1.0)),
                ssa_cloud=float(r.uniform(0.6, 1.0)), g=float(r.uniform(-0.5, 0.95)),
                albedo=float(r.uniform(0.0, 0.9)), zenith=float(r.uniform(0.0, 80.0)),
                azimuth=float(r.uniform(0.0, 360.0)), sun_mode=int(r.integers(0, 3)), grid=int(r.integers(0, 2)),
                finest=int(r.integers(0, 2)), tau=float(r.choice((0.3, 1.0, 5.0))), bf16=bool(r.integers(0, 2)))


@pytest.mark.parametrize("i", range(TALLY_CASES))
def test_random_scene_tallies(env, orc, i):
    m, ctx = env
    c = _scene_case(i)
    sc = m.Scene(ctx, c["k"], c["h"], c["h"], c["h"], k_clear=c["k_clear"], ssa_clear=c["ssa_clear"],
                 ssa_cloud=c["ssa_cloud"], g=c["g"], levels=c["levels"], albedo=c["albedo"],
                 sun_zenith_deg=c["zenith"], sun_azimuth_deg=c["azimuth"],
                 storage=m.MCRT_STORAGE_BF16 if c["bf16"] else m.MCRT_STORAGE_F32)
    try:
        if c["grid"] == 1:
            sc.build_octree()
        kw = dict(tau_merge=c["tau"], finest_level=c["finest"], sun_mode=c["sun_mode"], grid=c["grid"])
        osc = orc.Scene(k=c["k"], dx=c["h"], dy=c["h"], dz=c["h"], levels=c["levels"], k_clear=c["k_clear"],
                        ssa_clear=c["ssa_clear"], ssa_cloud=c["ssa_cloud"], g=c["g"], ground_albedo=c["albedo"],
                        sun_zenith_deg=c["zenith"], sun_azimuth_deg=c["azimuth"], bf16=c["bf16"],
                        tau_merge=c["tau"], finest_level=c["finest"], sun_mode=c["sun_mode"], grid=c["grid"])
        n = 30000
        g = sc.trace_flux(n, seed=100 + i, **kw)
        o, st = orc.trace_flux(osc, n, seed=100 + i)
        assert st[0] == 0
        for q in range(3):
            s = float(np.hypot(g.se[q], o.se[q]))
            assert abs(g.mean[q] - o.mean[q]) <= 4.0 * s + 1e-12, (i, q, g.mean[:3], o.mean[:3], c)
        nz, ny, nx = c["k"].shape
        spec = scenes.SceneSpec("fuzz", c["k"], c["h"], c["h"], c["h"], c["levels"], c["k_clear"], c["ssa_clear"],
                                c["ssa_cloud"], c["g"], c["albedo"], c["zenith"], c["azimuth"])
        cam = scenes.nadir_camera(spec, 12, 10)
        gi = sc.trace_camera(cam, 16, seed=200 + i, **kw)
        oi, _ = orc.trace_camera(osc, orc.Camera(cam.pos, cam.target, cam.up, cam.fov_deg, cam.width, cam.height),
                                 16, seed=200 + i)
        sg = float(np.sqrt(np.sum(gi.se ** 2))) / gi.se.size
        so = float(np.sqrt(np.sum(oi.se ** 2))) / oi.se.size
        assert abs(gi.mean.mean() - oi.mean.mean()) <= 4.0 * np.hypot(sg, so) + 1e-12, (i, gi.mean.mean(),
                                                                                      oi.mean.mean(), c)
    finally:
        sc.close()
