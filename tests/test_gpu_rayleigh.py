"""Rayleigh clear air on the GPU against the oracle (species sampling at
scattering vertices, mixture phase function in the local estimate):
flux and image tallies within 4 combined SE on the same seeds, the direct
part unchanged, the single-scattering closed form, and refusals."""
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


def test_rayleigh_flux_and_image_vs_oracle(m, ctx, orc):
    sp = scenes.blobs_small(0)
    sp.k = sp.k + np.float32(0.04)           # a thicker clear sky (0.05 km^-1) so the air matters
    sp.k_clear = 0.05
    sc = m.Scene.from_spec(ctx, sp)
    try:
        plain = sc.trace_flux(100000, seed=5)
        m.mcrt_scene_set_clear_sky_phase(ctx.h, sc.h, m.MCRT_PHASE_RAYLEIGH)
        g = sc.trace_flux(100000, seed=5)
        o, _ = orc.trace_flux(oscene(orc, sp, clear_phase=1), 100000, seed=5)
        for q in range(3):
            assert close_4se(g.mean[q], g.se[q], o.mean[q], o.se[q]), (q, g.mean, o.mean)
        assert abs(g.mean[2] - o.mean[2]) < 0.25 * o.se[2]
        assert g.mean[0] == pytest.approx(plain.mean[0], rel=1e-6)     # direct part: same paths, same sun rays
        cam = scenes.nadir_camera(sp, 32, 32)
        gi = sc.trace_camera(cam, 64, seed=6)
        oc = orc.Camera(cam.pos, cam.target, cam.up, cam.fov_deg, cam.width, cam.height)
        oi, _ = orc.trace_camera(oscene(orc, sp, clear_phase=1), oc, 64, seed=6)
        blocks = lambda x: x.reshape(4, 8, 4, 8).sum(axis=(1, 3))
        z = np.abs(blocks(gi.mean) - blocks(oi.mean)) / np.hypot(np.sqrt(blocks(gi.se ** 2)),
                                                                 np.sqrt(blocks(oi.se ** 2)))
        assert int((z > 4).sum()) <= 1, z
    finally:
        sc.close()


def test_rayleigh_single_scattering_gpu(m, ctx):
    k, om, th0, thv = 0.8, 0.95, 35.0, 40.0
    sp = scenes.homogeneous(16, 16, 8, 0.1, k, levels=1, g=0.85, ssa_cloud=0.5, ssa_clear=om,
                            sun_zenith_deg=th0, sun_azimuth_deg=0.0, k_clear=k)
    sc = m.Scene.from_spec(ctx, sp)
    try:
        m.mcrt_scene_set_clear_sky_phase(ctx.h, sc.h, m.MCRT_PHASE_RAYLEIGH)
        d = np.array([math.sin(math.radians(thv)), 0.0, -math.cos(math.radians(thv))])
        pos = np.array([0.8, 0.8, 0.8]) - 20.0 * d

        class Cam:
            pass
        cam = Cam()
        cam.pos, cam.target, cam.up = tuple(pos), (0.8, 0.8, 0.8), (0.0, 0.0, 1.0)
        cam.fov_deg, cam.width, cam.height = 1e-3, 1, 1
        r = sc.trace_camera(cam, 400000, seed=7, max_order=1)
        mu0, mu = math.cos(math.radians(th0)), math.cos(math.radians(thv))
        c = float(d @ np.array([math.sin(math.radians(th0)), 0.0, mu0]))
        tau = k * 8 * float(np.float32(0.1))
        want = om * 3 * (1 + c * c) / (16 * math.pi) * mu0 / (mu0 + mu) * (1 - math.exp(-tau * (1 / mu0 + 1 / mu)))
        assert abs(r.mean[0, 0] - want) < 3.0 * r.se[0, 0], (r.mean[0, 0], want, r.se[0, 0])
    finally:
        sc.close()


def test_rayleigh_refusals(m, ctx):
    sp = scenes.blobs_small(0)
    sc = m.Scene.from_spec(ctx, sp)
    try:
        with pytest.raises(m.McrtError) as e:
            m.mcrt_scene_set_clear_sky_phase(ctx.h, sc.h, 7)
        assert e.value.status == m.MCRT_ERR_ARG
        m.mcrt_scene_set_clear_sky_phase(ctx.h, sc.h, m.MCRT_PHASE_RAYLEIGH)
        with pytest.raises(m.McrtError) as e:
            m.trace_batch(ctx, [(sc, 0.0, 30.0, 0.0, 100, 1)])
        assert e.value.status == m.MCRT_ERR_UNSUPPORTED
        prop = m.Proposal(ctx, seed=1)
        try:
            with pytest.raises(m.McrtError) as e:
                sc.trace_flux(100, seed=1, proposal=prop)
            assert e.value.status == m.MCRT_ERR_UNSUPPORTED
        finally:
            prop.close()
    finally:
        sc.close()


def test_rayleigh_colour_bands(m, ctx, orc):
    """Three bands (650, 550, 450 nm) of Rayleigh clear air over a dark
    ground: the sky light reaching the ground grows toward the blue, the
    direct beam shrinks, each band within 4 SE of the oracle."""
    sp = scenes.blobs_small(0)
    sp.ground_albedo = 0.05
    res = []
    for kc in scenes.rayleigh_band_extinction(0.012):
        k = (sp.k - np.float32(sp.k_clear) + np.float32(kc)).astype(np.float32)
        spb = scenes.SceneSpec("band", k, sp.dx, sp.dy, sp.dz, sp.levels, kc, 1.0, sp.ssa_cloud, sp.g,
                               sp.ground_albedo, sp.sun_zenith_deg)
        sc = m.Scene.from_spec(ctx, spb)
        try:
            m.mcrt_scene_set_clear_sky_phase(ctx.h, sc.h, m.MCRT_PHASE_RAYLEIGH)
            g = sc.trace_flux(200000, seed=9)
        finally:
            sc.close()
        o, _ = orc.trace_flux(oscene(orc, spb, clear_phase=1), 100000, seed=9)
        for q in range(3):
            assert close_4se(g.mean[q], g.se[q], o.mean[q], o.se[q]), (kc, q, g.mean, o.mean)
        res.append(g)
    assert res[0].mean[0] > res[1].mean[0] > res[2].mean[0]          # direct: red > green > blue
