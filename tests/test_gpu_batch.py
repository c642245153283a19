"""Batches (many flux problems in one persistent launch) against the oracle.

* Each item against the oracle's flux tracer with that item's gas
  absorption, sun and phase function: T_dir, T_dif, T_tot, dT_tot/dg and
  dT_tot/dalpha within 4 combined standard errors.
* Each item against a single-problem GPU trace with the same seed: path j of
  the item draws what path j of the single trace draws, so the two differ
  only in how FP32 chunk sums are grouped (relative <= 64 * 2^-24 ~ 4e-6).
* Closed form: a pure gas absorber over a black ground gives
  T_dir = exp(-k_gas H / mu0) and T_dif = 0.
* Ragged item sizes (1 path, a chunk and a bit), argument errors, and the
  autotuner's choice changing the speed but not the results.
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


@pytest.fixture(scope="module")
def two_scenes(m, ctx):
    a = scenes.blobs_small(0)
    b = scenes.blobs_small(3)
    b.g = 0.6
    b.ground_albedo = 0.35
    sa, sb = m.Scene.from_spec(ctx, a), m.Scene.from_spec(ctx, b)
    yield (a, sa), (b, sb)
    sa.close()
    sb.close()


def test_batch_items_vs_oracle(m, ctx, orc, two_scenes):
    (a, sa), (b, sb) = two_scenes
    n = 60000
    items = [(sa, 0.0, 30.0, 0.0, n, 11), (sb, 0.05, 60.0, 40.0, n, 12), (sa, 0.6, 75.0, 200.0, n, 13),
             (sb, 0.0, 0.0, 0.0, n, 14)]
    r = m.trace_batch(ctx, items, batch_dalpha=1)
    assert r.mean.shape == (4, 5)
    for i, (s, kg, z, az, npaths, seed) in enumerate(items):
        sp = a if s is sa else b
        o, _ = orc.trace_flux(oscene(orc, sp, k_gas=kg, sun_zenith_deg=z, sun_azimuth_deg=az), npaths, seed=seed)
        for q in range(5):
            assert close_4se(r.mean[i, q], r.se[i, q], o.mean[q], o.se[q]), (i, q, r.mean[i], o.mean)
        assert np.all(r.n[i] == npaths)
        # same random numbers on both sides: far closer than the noise
        assert abs(r.mean[i, 2] - o.mean[2]) < 0.25 * o.se[2] + 1e-12


def test_batch_dg_vs_finite_difference(m, ctx):
    """dT_tot/dg from the score function against a central difference of
    T_tot over fields with g -/+ delta, on common random numbers (same seed;
    the SE of the difference is bounded by the sum of the two SEs).  The
    truncation error delta^2 T'''/6 is far below the noise at delta = 0.03."""
    sp = scenes.blobs_small(0)
    delta, n = 0.03, 400000
    sc = [m.Scene.from_spec(ctx, sp)]
    for g in (sp.g - delta, sp.g + delta):
        sp2 = scenes.blobs_small(0)
        sp2.g = g
        sc.append(m.Scene.from_spec(ctx, sp2))
    try:
        r = m.trace_batch(ctx, [(s, 0.0, 30.0, 0.0, n, 77) for s in sc])
        fd = (r.mean[2, 2] - r.mean[1, 2]) / (2 * delta)
        sfd = (r.se[2, 2] + r.se[1, 2]) / (2 * delta)
        assert abs(r.mean[0, 3] - fd) <= 4 * math.hypot(r.se[0, 3], sfd), (r.mean[0, 3], r.se[0, 3], fd, sfd)
        assert r.se[0, 3] < 0.2 and sfd < 0.2
    finally:
        for s in sc:
            s.close()


def test_batch_dalpha_is_opt_in(m, ctx, two_scenes):
    """Without batch_dalpha the fifth quantity is 0 and the others are the
    same paths' estimates as with it (to FP32 chunk-sum rounding)."""
    (a, sa), _ = two_scenes
    it = [(sa, 0.01, 40.0, 0.0, 30000, 3)]
    r0 = m.trace_batch(ctx, it)
    r1 = m.trace_batch(ctx, it, batch_dalpha=1)
    assert r0.mean[0, 4] == 0.0 and r1.mean[0, 4] != 0.0
    np.testing.assert_allclose(r0.mean[0, :4], r1.mean[0, :4], rtol=4e-6, atol=1e-12)


def test_batch_matches_single_traces(m, ctx, two_scenes):
    (a, sa), (b, sb) = two_scenes
    items = [(sa, 0.0, 20.0, 10.0, 30001, 5), (sb, 0.0, 45.0, 0.0, 1, 6), (sa, 0.0, 20.0, 10.0, 5, 7),
             (sb, 0.0, 70.0, 300.0, 25000, 8)]
    r = m.trace_batch(ctx, items)
    try:
        for i, (s, kg, z, az, npaths, seed) in enumerate(items):
            m.mcrt_scene_set_sun(ctx.h, s.h, z, az)
            single = s.trace_flux(npaths, seed=seed)
            np.testing.assert_allclose(r.mean[i, :3], single.mean, rtol=4e-6, atol=1e-12)
            np.testing.assert_allclose(r.se[i, :3], single.se, rtol=1e-4, atol=1e-12)
    finally:
        m.mcrt_scene_set_sun(ctx.h, sa.h, a.sun_zenith_deg, a.sun_azimuth_deg)
        m.mcrt_scene_set_sun(ctx.h, sb.h, b.sun_zenith_deg, b.sun_azimuth_deg)


def test_batch_gas_closed_form(m, ctx):
    sp = scenes.homogeneous(16, 16, 20, 0.1, 0.0, levels=2, ground_albedo=0.0, sun_zenith_deg=0.0)
    sc = m.Scene.from_spec(ctx, sp)
    try:
        H = 20 * 0.1
        items = [(sc, kg, z, 0.0, 200000, 100 + j) for j, (kg, z) in enumerate([(0.3, 0.0), (0.8, 50.0), (2.0, 70.0)])]
        r = m.trace_batch(ctx, items)
        for i, (_, kg, z, _, n, _) in enumerate(items):
            mu0 = math.cos(math.radians(z))
            want = math.exp(-kg * H / mu0)
            assert abs(r.mean[i, 0] - want) <= 3 * r.se[i, 0] + 1e-12, (i, r.mean[i, 0], want)
            assert r.mean[i, 1] == 0.0 and r.mean[i, 3] == 0.0 and r.mean[i, 4] == 0.0
    finally:
        sc.close()


def test_batch_dalpha_scales_each_order(m, ctx):
    """Pure cloud over a black ground: the order-n estimate carries omega^n,
    so -omega dT/dalpha = T for orders capped at 1 and 2 T(<=2) - T(<=1)
    for the cap 2, on the same paths (FP32 sums: rel 2e-5)."""
    om = 0.9
    sp = scenes.homogeneous(16, 16, 8, 0.1, 1.3, levels=1, g=0.7, ssa_cloud=om, ssa_clear=1.0, sun_zenith_deg=25.0)
    sc = m.Scene.from_spec(ctx, sp)
    try:
        it = [(sc, 0.0, 25.0, 0.0, 50000, 71)]
        one = m.trace_batch(ctx, it, max_order=1, batch_dalpha=1)
        two = m.trace_batch(ctx, it, max_order=2, batch_dalpha=1)
        assert one.mean[0, 1] > 0.01
        assert -om * one.mean[0, 4] == pytest.approx(one.mean[0, 1], rel=2e-5)
        assert -om * two.mean[0, 4] == pytest.approx(2 * two.mean[0, 1] - one.mean[0, 1], rel=2e-5)
    finally:
        sc.close()


def test_batch_bad_arguments(m, ctx, two_scenes):
    (a, sa), _ = two_scenes
    for bad in [[(sa, -1.0, 0.0, 0.0, 10, 1)], [(sa, 0.0, 95.0, 0.0, 10, 1)], [(sa, 0.0, 0.0, 0.0, 0, 1)],
                [(None, 0.0, 0.0, 0.0, 10, 1)]]:
        with pytest.raises(m.McrtError) as e:
            m.trace_batch(ctx, bad)
        assert e.value.status == m.MCRT_ERR_ARG
    with pytest.raises(m.McrtError) as e:
        m.trace_batch(ctx, [])
    assert e.value.status == m.MCRT_ERR_ARG
    bf = m.Scene.from_spec(ctx, a, storage=m.MCRT_STORAGE_BF16)
    try:
        with pytest.raises(m.McrtError) as e:
            m.trace_batch(ctx, [(sa, 0.0, 0.0, 0.0, 10, 1), (bf, 0.0, 0.0, 0.0, 10, 1)])
        assert e.value.status == m.MCRT_ERR_UNSUPPORTED
        r = m.trace_batch(ctx, [(bf, 0.0, 30.0, 0.0, 1000, 1)])      # BF16 alone is fine
        assert np.isfinite(r.mean).all()
    finally:
        bf.close()


def test_autotuner_changes_speed_not_results(m, ctx, two_scenes):
    (a, sa), (b, sb) = two_scenes
    items = [(sa, 0.01, 30.0, 0.0, 20000, 1), (sb, 0.2, 60.0, 0.0, 7000, 2)]
    opts, best = m.mcrt_autotune_batch(ctx.h, items, 0.5, m.mcrt_trace_opts_default())
    assert best > 0.0
    assert opts.chunk in (1, 2, 4, 8) and opts.rare_batch in (4, 8, 12) and opts.block_size in (64, 128)
    r0 = m.trace_batch(ctx, items)
    r1 = m.trace_batch(ctx, items, chunk=opts.chunk, rare_batch=opts.rare_batch, block_size=opts.block_size)
    np.testing.assert_allclose(r0.mean, r1.mean, rtol=4e-6, atol=1e-12)


def test_graph_plan_replays_the_batch(m, ctx, two_scenes):
    (a, sa), (b, sb) = two_scenes
    items = [(sa, 0.02, 30.0, 0.0, 20000, 21), (sb, 0.0, 50.0, 90.0, 9, 22), (sb, 1.5, 10.0, 0.0, 15000, 23)]
    direct = m.trace_batch(ctx, items)
    plan = m.BatchPlan(ctx, items)
    try:
        r1 = plan.run()
        r2 = plan.run()
        np.testing.assert_allclose(r1.mean, direct.mean, rtol=4e-6, atol=1e-12)
        np.testing.assert_allclose(r1.se, direct.se, rtol=1e-4, atol=1e-12)
        np.testing.assert_allclose(r2.mean, r1.mean, rtol=4e-6, atol=1e-12)
        assert r1.kernel_ms > 0.0
        # new seeds: new paths, same expectation
        plan.set_seeds([101, 102, 103])
        r3 = plan.run()
        assert not np.allclose(r3.mean[0, :3], r1.mean[0, :3], rtol=1e-9, atol=0)
        for q in range(5):
            assert close_4se(r3.mean[0, q], r3.se[0, q], r1.mean[0, q], r1.se[0, q])
        other = m.trace_batch(ctx, [(s, kg, z, az, n, 101 + i) for i, (s, kg, z, az, n, _) in enumerate(items)])
        np.testing.assert_allclose(r3.mean, other.mean, rtol=4e-6, atol=1e-12)
        # the plan's tally reads like any other
        import ctypes as C
        h = C.c_void_p()
        assert m.lib().mcrt_batch_plan_tally(plan.h, C.byref(h)) == 0
        mean, se, n = m.mcrt_tally_read(ctx.h, h)
        np.testing.assert_allclose(mean.reshape(3, 5), r3.mean, rtol=1e-12)
        assert list(n.reshape(3, 5)[:, 0]) == [20000, 9, 15000]
    finally:
        plan.close()
    with pytest.raises(m.McrtError) as e:
        m.BatchPlan(ctx, items, deadline_ms=5.0)
    assert e.value.status == m.MCRT_ERR_UNSUPPORTED
