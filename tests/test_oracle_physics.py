"""Oracle pins against what the physics and the mathematics fix.

* Beer's law through homogeneous and layered slabs (Sec. 2.2; Sec. 2.3
  algorithm, whose expectation Eq. 2 is exp(-tau)).
* Heterogeneous voxels along fixed rays: exp(-sum k_v l_v) with the lengths
  from the brute-force face list (ratio and delta tracking unbiased).
* Majorant invariance (Sec. 2.3-2.4: any valid majorant gives the same
  expectation): global, pyramid at several tau~, voxel-exact tracking.
* Black-sky Lambertian ground: radiance rho mu0 / pi with zero variance.
* Single scattering in a homogeneous slab: closed forms (reflected and
  transmitted radiance, order-1 tally only).
* Energy balance of the forward analog estimator, per photon; R + T = 1 for
  a conservative medium over a black ground, forward vs backward.
* Reciprocity: backward local-estimate ground flux = forward analog flux.
* Henyey-Greenstein moments and normalisation; exponential free paths.
"""
import math

import numpy as np
import pytest

import scenes


def _oscene(orc, sp, **kw):
    args = dict(k=sp.k, dx=sp.dx, dy=sp.dy, dz=sp.dz, levels=sp.levels, k_clear=sp.k_clear,
                ssa_clear=sp.ssa_clear, ssa_cloud=sp.ssa_cloud, g=sp.g, ground_albedo=sp.ground_albedo,
                sun_zenith_deg=sp.sun_zenith_deg, sun_azimuth_deg=sp.sun_azimuth_deg)
    args.update(kw)
    return orc.Scene(**args)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_beer_homogeneous_slab(orc, mode):
    # (decomposition: k = 0.75 is a bfloat16 value, so the leaves' minorant
    #  is k itself, and tau < ln 10 keeps the roulette out)
    k, H, th = (1.7 if mode < 2 else 0.75), 16 * float(np.float32(0.1)), 40.0   # 16 voxels of FP32 0.1 km
    sp = scenes.homogeneous(16, 16, 16, 0.1, k, levels=2, sun_zenith_deg=th)
    sc = _oscene(orc, sp, sun_mode=mode)
    T, _ = orc.trace_flux(sc, 40000, seed=5)
    want = math.exp(-k * H / math.cos(math.radians(th)))
    assert abs(T.mean[0] - want) < 3.0 * T.se[0] + 1e-12, (T.mean[0], want, T.se[0])
    if mode == 2:
        # decomposition tracking: the uniform field is its own minorant, so
        # every path gets exp(-tau) exactly (no random draw on the sun ray)
        assert T.mean[0] == pytest.approx(want, rel=1e-12) and T.se[0] < 1e-12


def test_beer_layered_slabs(orc):
    """Layers whose interfaces fall inside level-1 cells (not multiples of 8)."""
    nz = 40
    kz = np.zeros(nz, dtype=np.float32)
    kz[0:3] = 0.5
    kz[3:11] = 2.0
    kz[11:13] = 0.0
    kz[13:29] = 0.25
    kz[29:40] = 1.1
    k = np.broadcast_to(kz[:, None, None], (nz, 16, 16)).astype(np.float32).copy()
    th = 25.0
    sp = scenes.SceneSpec("layers", k, 0.05, 0.05, 0.05, 2, 0.0, 1.0, 1.0, 0.85, 0.0, th)
    for tau, fin, mode in [(1.0, 1, 0), (0.0, 0, 0), (float("inf"), 1, 0), (1.0, 1, 2), (0.0, 0, 2),
                           (float("inf"), 1, 2)]:
        sc = _oscene(orc, sp, tau_merge=tau, finest_level=fin, sun_mode=mode)
        T, _ = orc.trace_flux(sc, 30000, seed=9)
        tau_v = float(np.sum(kz.astype(np.float64) * float(np.float32(0.05))))   # FP32 voxel height
        want = math.exp(-tau_v / math.cos(math.radians(th)))
        assert abs(T.mean[0] - want) < 3.0 * T.se[0] + 1e-12, (tau, mode, T.mean[0], want, T.se[0])
        if mode == 2 and fin == 0:
            # voxel leaves: the control is the voxel, exp(-tau) exactly (roulette aside:
            # tau here is below ln 10, so no path is rouletted)
            assert T.mean[0] == pytest.approx(want, rel=1e-9) and T.se[0] < 1e-12


def _exact_optical_depth(orc, sp, o, d):
    """Brute-force optical depth: voxel-level leaves (tau~ = 0, finest 0)."""
    sc = orc.Scene(k=sp.k, dx=sp.dx, dy=sp.dy, dz=sp.dz, levels=sp.levels, tau_merge=0.0, finest_level=0)
    cells, tio, st = orc.dda_bruteforce(sc, np.asarray(o, np.float64), np.asarray(d, np.float64))
    assert st == 1
    tau = 0.0
    for (lev, ix, iy, iz), (t0, t1) in zip(cells, tio):
        if lev == 0:
            tau += float(sp.k[iz, iy, ix]) * (t1 - t0)
        else:
            assert sp.k[iz * 8 ** lev:(iz + 1) * 8 ** lev, iy * 8 ** lev:(iy + 1) * 8 ** lev,
                         ix * 8 ** lev:(ix + 1) * 8 ** lev].max() == 0.0
    return tau


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_heterogeneous_ray_transmissivity(orc, mode):
    sp = scenes.random_voxels(32, 32, 24, 0.1, 4.0, seed=21, levels=2, sparsity=0.6)
    r = np.random.default_rng(7)
    for j in range(3):
        o = np.array([r.uniform(0, 3.2), r.uniform(0, 3.2), r.uniform(0, 1.0)])
        v = np.array([r.normal(), r.normal(), abs(r.normal()) + 0.3])
        v /= np.linalg.norm(v)
        tau = _exact_optical_depth(orc, sp, o, v)
        sc = orc.Scene(k=sp.k, dx=sp.dx, dy=sp.dy, dz=sp.dz, levels=2, tau_merge=1.0, sun_mode=mode)
        t = orc.transmissivity_many(sc, o, v, seed=1000 + j, n=100000)
        want = math.exp(-tau)
        se = t.std(ddof=1) / math.sqrt(t.size)
        assert abs(t.mean() - want) < 3.0 * se + 1e-12, (j, t.mean(), want, se, tau)
        if mode == 2:
            # the control removes most of the variance ratio tracking has
            r0 = orc.transmissivity_many(orc.Scene(k=sp.k, dx=sp.dx, dy=sp.dy, dz=sp.dz, levels=2, tau_merge=1.0,
                                                   sun_mode=0), o, v, seed=1000 + j, n=100000)
            assert t.var() < r0.var()


def test_majorant_invariance(orc):
    """Same flux tallies whatever valid majorant is used."""
    sp = scenes.blobs_small(0)
    res = []
    for tau, fin in [(0.1, 1), (1.0, 1), (10.0, 1), (float("inf"), 1), (0.0, 0)]:
        sc = _oscene(orc, sp, tau_merge=tau, finest_level=fin)
        T, _ = orc.trace_flux(sc, 40000, seed=3 + int(min(tau, 100)) + 7 * fin)
        res.append(T)
    for i in range(len(res)):
        for j in range(i + 1, len(res)):
            for q in range(3):
                d = abs(res[i].mean[q] - res[j].mean[q])
                s = math.hypot(res[i].se[q], res[j].se[q])
                assert d < 4.0 * s, (i, j, q, d, s)


def test_decomposition_tracking_tallies_match_ratio_tracking(orc):
    """Sun transmissivity by decomposition tracking (minorant control, ratio
    tracking on the residual) gives the same flux expectations as ratio
    tracking, with a smaller variance of the diffuse part."""
    sp = scenes.blobs_small(0)
    a, _ = orc.trace_flux(_oscene(orc, sp, sun_mode=0), 60000, seed=41)
    b, _ = orc.trace_flux(_oscene(orc, sp, sun_mode=2), 60000, seed=42)
    for q in range(3):
        assert abs(a.mean[q] - b.mean[q]) < 4.0 * math.hypot(a.se[q], b.se[q]), (q, a.mean[q], b.mean[q])
    assert b.se[1] < a.se[1]


def test_black_sky_lambertian_ground(orc):
    rho, th = 0.3, 35.0
    sp = scenes.homogeneous(16, 16, 8, 0.1, 0.0, levels=1, ground_albedo=rho, sun_zenith_deg=th)
    sc = _oscene(orc, sp)
    cam = scenes.nadir_camera(sp, 8, 8)
    I, _ = orc.trace_camera(sc, orc.Camera(cam.pos, cam.target, cam.up, cam.fov_deg, 8, 8), 64, seed=2)
    want = rho * math.cos(math.radians(th)) / math.pi
    assert np.max(np.abs(I.mean - want)) <= 1e-12 * want
    assert np.max(I.se) <= 1e-12 * want


def _hg(g, mu):
    return (1 - g * g) / (4 * math.pi * (1 + g * g - 2 * g * mu) ** 1.5)


def test_single_scattering_reflected(orc):
    k, H, g, om, th0 = 2.0, 0.8, 0.7, 0.9, 30.0
    sp = scenes.homogeneous(16, 16, 8, 0.1, k, levels=1, g=g, ssa_cloud=om, ssa_clear=om,
                            sun_zenith_deg=th0, sun_azimuth_deg=0.0)
    sc = _oscene(orc, sp, max_order=1)
    thv = 50.0          # viewing zenith (camera looks down along -d)
    d = np.array([math.sin(math.radians(thv)), 0.0, -math.cos(math.radians(thv))])
    pos = np.array([0.8, 0.8, 0.8]) - 20.0 * d
    cam = orc.Camera(tuple(pos), (0.8, 0.8, 0.8), (0.0, 0.0, 1.0), 1e-3, 1, 1)
    I, _ = orc.trace_camera(sc, cam, 200000, seed=4)
    mu0, mu = math.cos(math.radians(th0)), math.cos(math.radians(thv))
    s = np.array([math.sin(math.radians(th0)), 0.0, mu0])
    tau = k * H
    want = om * _hg(g, float(d @ s)) * mu0 / (mu0 + mu) * (1 - math.exp(-tau * (1 / mu0 + 1 / mu)))
    assert abs(I.mean[0, 0] - want) < 3.0 * I.se[0, 0], (I.mean[0, 0], want, I.se[0, 0])


def test_single_scattering_transmitted(orc):
    """Slab between z = 0.4 and 1.2 km over clear air; camera below looks up."""
    g, om, th0, kk = 0.6, 1.0, 20.0, 1.5
    k = np.zeros((12, 16, 16), dtype=np.float32)
    k[4:12] = kk
    sp = scenes.SceneSpec("slab", k, 0.1, 0.1, 0.1, 1, 0.0, om, om, g, 0.0, th0)
    sc = _oscene(orc, sp, max_order=1)
    thv = 45.0
    d = np.array([math.sin(math.radians(thv)) * math.cos(0.7), math.sin(math.radians(thv)) * math.sin(0.7),
                  math.cos(math.radians(thv))])
    pos = (0.8, 0.8, 0.05)
    tgt = tuple(np.array(pos) + d)
    cam = orc.Camera(pos, tgt, (1.0, 0.0, 0.0), 1e-3, 1, 1)
    I, _ = orc.trace_camera(sc, cam, 200000, seed=6)
    mu0, mu = math.cos(math.radians(th0)), math.cos(math.radians(thv))
    s = np.array([math.sin(math.radians(th0)), 0.0, mu0])
    tau = kk * 0.8
    want = om * _hg(g, float(d @ s)) * mu0 / (mu0 - mu) * (math.exp(-tau / mu0) - math.exp(-tau / mu))
    assert abs(I.mean[0, 0] - want) < 3.0 * I.se[0, 0], (I.mean[0, 0], want, I.se[0, 0])


def test_forward_energy_balance_per_photon(orc):
    sp = scenes.blobs_small(0)
    sc = _oscene(orc, sp)
    assert orc.forward_balance_residual(sc, seed=1, nphotons=3000) < 1e-12


def test_conservative_R_plus_T(orc):
    """omega = 1, black ground: every photon escapes or reaches the ground
    once, so R_forward + T_backward = 1."""
    sp = scenes.blobs_small(0)
    sc = _oscene(orc, sp, ssa_clear=1.0, ssa_cloud=1.0, ground_albedo=0.0)
    F, _ = orc.trace_forward(sc, 60000, seed=8)
    B, _ = orc.trace_flux(sc, 60000, seed=9)
    R = F.mean[0]
    assert F.mean[3] == 0.0 and F.mean[4] == pytest.approx(F.mean[1] + F.mean[2])
    d = abs(R + B.mean[2] - 1.0)
    s = math.hypot(F.se[0], B.se[2])
    assert d < 4.0 * s, (R, B.mean[2], s)


def test_reciprocity_backward_vs_forward(orc):
    sp = scenes.blobs_small(0)
    sc = _oscene(orc, sp)
    F, _ = orc.trace_forward(sc, 80000, seed=10)
    B, _ = orc.trace_flux(sc, 80000, seed=11)
    for qb, qf in [(0, 1), (1, 2)]:
        d = abs(B.mean[qb] - F.mean[qf])
        s = math.hypot(B.se[qb], F.se[qf])
        assert d < 4.0 * s, (qb, B.mean[qb], F.mean[qf], s)


@pytest.mark.parametrize("g", [0.0, 0.3, 0.85, -0.5])
def test_hg_moments_and_normalisation(orc, g):
    from scipy import integrate
    r = np.random.default_rng(12)
    xi = 1.0 - r.uniform(size=200000)           # (0, 1]
    mu = np.array([orc.hg_sample_mu(g, x) for x in xi])
    m1, m2 = mu.mean(), (mu * mu).mean()
    se1 = mu.std() / math.sqrt(mu.size)
    se2 = (mu * mu).std() / math.sqrt(mu.size)
    assert abs(m1 - g) < 3 * se1 + 1e-12
    assert abs(m2 - (1 + 2 * g * g) / 3) < 3 * se2 + 1e-12
    total, _ = integrate.quad(lambda m: 2 * math.pi * orc.hg_pdf(g, m), -1, 1, epsabs=1e-12, points=[1.0])
    assert total == pytest.approx(1.0, abs=1e-8)
    # sampled cosines follow the pdf: compare binned frequencies
    edges = np.linspace(-1, 1, 41)
    h, _ = np.histogram(mu, bins=edges)
    p = np.array([integrate.quad(lambda m: 2 * math.pi * orc.hg_pdf(g, m), a, b)[0]
                  for a, b in zip(edges[:-1], edges[1:])])
    e = p * mu.size
    mask = e > 20
    chi2 = float(((h[mask] - e[mask]) ** 2 / e[mask]).sum())
    assert chi2 < 90.0, chi2


def test_hg_rotation(orc):
    r = np.random.default_rng(13)
    d = r.normal(size=(5000, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    d[0] = (0, 0, 1)
    d[1] = (0, 0, -1)
    xi = 1.0 - r.uniform(size=(5000, 2))
    out = orc.hg_sample_dirs(0.8, d, xi)
    assert np.allclose(np.linalg.norm(out, axis=1), 1.0, atol=1e-12)
    mu = np.array([orc.hg_sample_mu(0.8, x) for x in xi[:, 0]])
    assert np.allclose((out * d).sum(axis=1), mu, atol=1e-9)


def test_free_path_exponential(orc):
    from scipy import stats
    k = 3.0
    sp = scenes.homogeneous(16, 16, 8, 0.1, k, levels=2)
    sc = orc.Scene(k=sp.k, dx=sp.dx, dy=sp.dy, dz=sp.dz, levels=2, tau_merge=1.0)
    a = 0.3
    dist = orc.first_collision_distances(sc, (0.33, 0.71, 0.45), (math.cos(a), math.sin(a), 0.0), seed=3, n=20000)
    assert np.all(dist > 0)
    se = dist.std() / math.sqrt(dist.size)
    assert abs(dist.mean() - 1.0 / k) < 3 * se
    assert stats.kstest(dist, "expon", args=(0, 1.0 / k)).pvalue > 1e-3


def test_dT_dg_score_estimator_matches_finite_differences(orc):
    """d T_dif / d g by the score-function estimator against central
    differences of T_dif at g +- 0.01 with common random numbers."""
    sp = scenes.blobs_small(0)
    n = 150000
    g0, h = 0.85, 0.01
    T0, _ = orc.trace_flux(_oscene(orc, sp, g=g0), n, seed=61)
    Tp, _ = orc.trace_flux(_oscene(orc, sp, g=g0 + h), n, seed=61)
    Tm, _ = orc.trace_flux(_oscene(orc, sp, g=g0 - h), n, seed=61)
    fd = (Tp.mean[1] - Tm.mean[1]) / (2 * h)
    est, se = T0.mean[3], T0.se[3]
    # the central difference of means of correlated estimates: its own noise
    # is bounded by that of the two runs (taken independent, conservative)
    fd_se = math.hypot(Tp.se[1], Tm.se[1]) / (2 * h)
    assert abs(est - fd) < 4 * math.hypot(se, fd_se), (est, fd, se, fd_se)
    # the direct part does not depend on g
    assert Tp.mean[0] == T0.mean[0] == Tm.mean[0]


def test_dT_dg_single_scattering_closed_form(orc):
    """Order-1 ground flux under a homogeneous slab over a black ground:
    T_dif,1 = (pi/mu0) int_{up} L1(mu) mu dOmega with the transmitted single-
    scattering radiance; its g-derivative is the same integral of d p_HG/dg."""
    from scipy import integrate
    kk, H, g, th0 = 0.7, 0.8, 0.6, 30.0
    sp = scenes.homogeneous(16, 16, 8, 0.1, kk, levels=1, g=g, ssa_cloud=1.0, ssa_clear=1.0, sun_zenith_deg=th0)
    T, _ = orc.trace_flux(_oscene(orc, sp, max_order=1), 200000, seed=62)
    mu0 = math.cos(math.radians(th0))
    tau = kk * H

    def L1(mu, phi, dphase):
        s = (math.sin(math.radians(th0)), 0.0, mu0)
        d = (math.sqrt(1 - mu * mu) * math.cos(phi), math.sqrt(1 - mu * mu) * math.sin(phi), mu)   # looking up
        c = d[0] * s[0] + d[1] * s[1] + d[2] * s[2]
        pf = dphase(c)
        if abs(mu - mu0) < 1e-9:
            return pf * tau / mu0 * math.exp(-tau / mu0)
        return pf * mu0 / (mu0 - mu) * (math.exp(-tau / mu0) - math.exp(-tau / mu))

    pHG = lambda c: (1 - g * g) / (4 * math.pi * (1 + g * g - 2 * g * c) ** 1.5)
    # d p_HG / d g written out from the closed form of p_HG
    dpHG = lambda c: pHG(c) * (-2 * g / (1 - g * g) - 1.5 * (2 * g - 2 * c) / (1 + g * g - 2 * g * c))
    # T = (1 / mu0) int_{upper hemisphere} L(mu) mu dOmega  (F0 = 1)
    flux = lambda dp: integrate.dblquad(lambda phi, mu: L1(mu, phi, dp) * mu, 0, 1, 0, 2 * math.pi,
                                        epsabs=1e-9)[0] / mu0
    want_T = flux(pHG)
    want_d = flux(dpHG)
    assert abs(T.mean[1] - want_T) < 3 * T.se[1], (T.mean[1], want_T)
    assert abs(T.mean[3] - want_d) < 3 * T.se[3], (T.mean[3], want_d)


def test_dT_dalpha_scales_each_order_exactly(orc):
    """In a pure cloud (no clear-sky part) over a black ground, the order-n
    estimate carries omega^n, so its derivative with respect to the
    absorptivity alpha = 1 - omega is -n/omega times it.  With orders capped
    at 1 and at 2 on the same seed (the same paths), the sensitivity estimate
    must satisfy -omega dT/dalpha = T(<=1) exactly for the cap 1 and
    2 T(<=2) - T(<=1) for the cap 2 (path by path, so up to FP64 rounding)."""
    om = 0.9
    sp = scenes.homogeneous(16, 16, 8, 0.1, 1.3, levels=1, g=0.7, ssa_cloud=om, ssa_clear=1.0, sun_zenith_deg=25.0)
    one, _ = orc.trace_flux(_oscene(orc, sp, max_order=1), 20000, seed=71)
    two, _ = orc.trace_flux(_oscene(orc, sp, max_order=2), 20000, seed=71)
    assert one.mean[1] > 0.01
    assert -om * one.mean[4] == pytest.approx(one.mean[1], rel=1e-12)
    assert -om * two.mean[4] == pytest.approx(2 * two.mean[1] - one.mean[1], rel=1e-12)


def test_dT_dalpha_matches_finite_differences(orc):
    """Central differences over omega_cloud = 1 - alpha -/+ delta on common
    random numbers (the free paths do not depend on alpha)."""
    sp = scenes.blobs_small(0)
    om, delta, n = 0.95, 0.01, 60000
    mid, _ = orc.trace_flux(_oscene(orc, sp, ssa_cloud=om), n, seed=81)
    lo, _ = orc.trace_flux(_oscene(orc, sp, ssa_cloud=om + delta), n, seed=81)    # alpha - delta
    hi, _ = orc.trace_flux(_oscene(orc, sp, ssa_cloud=om - delta), n, seed=81)    # alpha + delta
    fd = (hi.mean[2] - lo.mean[2]) / (2 * delta)
    sfd = (hi.se[2] + lo.se[2]) / (2 * delta)
    assert fd < 0.0                                       # more absorption, less light
    assert abs(mid.mean[4] - fd) <= 4 * math.hypot(mid.se[4], sfd), (mid.mean[4], mid.se[4], fd, sfd)


def test_rayleigh_sampler_and_normalisation(orc):
    """Rayleigh cosines: E[mu] = 0, E[mu^2] = 2/5, a normalised pdf, binned
    frequencies following it, and the inverse CDF hitting -1, 0, 1."""
    from scipy import integrate
    r = np.random.default_rng(14)
    xi = 1.0 - r.uniform(size=200000)
    mu = np.array([orc.rayleigh_sample_mu(x) for x in xi])
    se1 = mu.std() / math.sqrt(mu.size)
    se2 = (mu * mu).std() / math.sqrt(mu.size)
    assert abs(mu.mean()) < 3 * se1
    assert abs((mu * mu).mean() - 0.4) < 3 * se2
    total, _ = integrate.quad(lambda m: 2 * math.pi * orc.rayleigh_pdf(m), -1, 1)
    assert total == pytest.approx(1.0, abs=1e-12)
    edges = np.linspace(-1, 1, 41)
    h, _ = np.histogram(mu, bins=edges)
    e = np.array([integrate.quad(lambda m: 2 * math.pi * orc.rayleigh_pdf(m), a, b)[0]
                  for a, b in zip(edges[:-1], edges[1:])]) * mu.size
    assert float(((h - e) ** 2 / e).sum()) < 90.0
    assert orc.rayleigh_sample_mu(1.0) == pytest.approx(1.0, abs=1e-12)
    assert orc.rayleigh_sample_mu(0.5) == pytest.approx(0.0, abs=1e-12)
    assert orc.rayleigh_sample_mu(1e-12) == pytest.approx(-1.0, abs=1e-6)


def test_rayleigh_single_scattering_reflected(orc):
    """A clear-air slab with a Rayleigh phase function, first order, seen from
    above: omega p_R(Theta) mu0 / (mu0 + mu) (1 - exp(-tau (1/mu0 + 1/mu)))."""
    k, H, om, th0 = 0.8, 0.8, 0.95, 35.0
    sp = scenes.homogeneous(16, 16, 8, 0.1, k, levels=1, g=0.85, ssa_cloud=0.5, ssa_clear=om,
                            sun_zenith_deg=th0, sun_azimuth_deg=0.0)
    sc = _oscene(orc, sp, max_order=1, k_clear=k, clear_phase=1)      # the whole field is clear air
    thv = 40.0
    d = np.array([math.sin(math.radians(thv)), 0.0, -math.cos(math.radians(thv))])
    pos = np.array([0.8, 0.8, 0.8]) - 20.0 * d
    cam = orc.Camera(tuple(pos), (0.8, 0.8, 0.8), (0.0, 0.0, 1.0), 1e-3, 1, 1)
    I, _ = orc.trace_camera(sc, cam, 200000, seed=6)
    mu0, mu = math.cos(math.radians(th0)), math.cos(math.radians(thv))
    s = np.array([math.sin(math.radians(th0)), 0.0, mu0])
    c = float(d @ s)
    tau = k * 8 * float(np.float32(0.1))
    want = om * 3 * (1 + c * c) / (16 * math.pi) * mu0 / (mu0 + mu) * (1 - math.exp(-tau * (1 / mu0 + 1 / mu)))
    assert abs(I.mean[0, 0] - want) < 3.0 * I.se[0, 0], (I.mean[0, 0], want, I.se[0, 0])
    # and not the HG answer: the phase functions differ a lot at this angle
    hg = om * _hg(0.85, c) * mu0 / (mu0 + mu) * (1 - math.exp(-tau * (1 / mu0 + 1 / mu)))
    assert abs(I.mean[0, 0] - hg) > 10 * I.se[0, 0]


def test_rayleigh_clear_air_changes_diffuse_not_direct(orc):
    """Blobs over clear air: switching the clear air's phase function to
    Rayleigh leaves T_dir unchanged (same paths, same sun rays) and moves
    T_dif; dT/dg with the mixture score still matches finite differences."""
    sp = scenes.blobs_small(0)
    kw = dict(k_clear=0.05)
    a, _ = orc.trace_flux(_oscene(orc, sp, **kw), 40000, seed=91)
    b, _ = orc.trace_flux(_oscene(orc, sp, clear_phase=1, **kw), 40000, seed=91)
    assert a.mean[0] == b.mean[0]
    delta = 0.03
    lo, _ = orc.trace_flux(_oscene(orc, sp, clear_phase=1, g=sp.g - delta, **kw), 40000, seed=91)
    hi, _ = orc.trace_flux(_oscene(orc, sp, clear_phase=1, g=sp.g + delta, **kw), 40000, seed=91)
    fd = (hi.mean[2] - lo.mean[2]) / (2 * delta)
    sfd = (hi.se[2] + lo.se[2]) / (2 * delta)
    assert abs(b.mean[3] - fd) <= 4 * math.hypot(b.se[3], sfd), (b.mean[3], b.se[3], fd, sfd)
