"""Oracle pins for the heightfield ground (an extension of the flat
Lambertian ground; a project addition beside Sec. 1's remark that the
ground's shape matters little for the cloud estimates).

* Ray-surface hits against brute force: every triangle of every periodic
  image intersected in 3D (Moller-Trumbore), the nearest kept.
* Surface height and normal against points built from the triangle's
  corners by barycentric weights and the normal from an edge cross product.
* A flat heightfield at z = 0 reproduces the flat ground.
* No atmosphere: with the sun overhead every path gets T_dir = 1 exactly;
  at any sun the domain mean of the direct irradiance is 1 (all sunlight
  lands somewhere), which pins the 1 / (n_z mu0) normalisation, normals and
  terrain shadows together.
* Black-sky radiance of a tilted facet seen from above, first order:
  rho / pi * (n . s) exactly.
"""
import math

import numpy as np
import pytest

import scenes


def _scene(orc, heights, nx=8, ny=8, nz=8, d=0.1, k=0.0, **kw):
    sp = scenes.homogeneous(nx, ny, nz, d, k)
    a = dict(k=sp.k, dx=d, dy=d, dz=d, levels=1, heights=heights)
    a.update(kw)
    return orc.Scene(**a)


def _triangles(h, hx, hy):
    """All triangles of the periodic surface in one period: (ny, nx, 2, 3, 3)."""
    ny, nx = h.shape
    out = np.zeros((ny, nx, 2, 3, 3))
    for j in range(ny):
        for i in range(nx):
            z00, z10 = h[j, i], h[j, (i + 1) % nx]
            z01, z11 = h[(j + 1) % ny, i], h[(j + 1) % ny, (i + 1) % nx]
            P00 = (i * hx, j * hy, z00)
            P10 = ((i + 1) * hx, j * hy, z10)
            P01 = (i * hx, (j + 1) * hy, z01)
            P11 = ((i + 1) * hx, (j + 1) * hy, z11)
            out[j, i, 0] = (P00, P10, P11)
            out[j, i, 1] = (P00, P11, P01)
    return out


def _brute_hit(tris, Lx, Ly, o, d, images):
    """Nearest t > -1e-12 over every triangle of the images in range."""
    best = (math.inf, None)
    T = tris.reshape(-1, 3, 3)
    ids = [(j, i, t) for j in range(tris.shape[0]) for i in range(tris.shape[1]) for t in range(2)]
    for ox in images[0]:
        for oy in images[1]:
            shift = np.array([ox * Lx, oy * Ly, 0.0])
            v0, v1, v2 = T[:, 0] + shift, T[:, 1] + shift, T[:, 2] + shift
            e1, e2 = v1 - v0, v2 - v0
            pv = np.cross(d, e2)
            det = (e1 * pv).sum(1)
            ok = np.abs(det) > 1e-14
            inv = np.where(ok, 1.0 / np.where(ok, det, 1.0), 0.0)
            tv = o - v0
            u = (tv * pv).sum(1) * inv
            qv = np.cross(tv, e1)
            v = (qv * d).sum(1) * inv
            t = (e2 * qv).sum(1) * inv
            hit = ok & (u >= -1e-12) & (v >= -1e-12) & (u + v <= 1 + 1e-12) & (t >= -1e-12)
            for k in np.nonzero(hit)[0]:
                if t[k] < best[0]:
                    j, i, tri = ids[k]
                    best = (t[k], (i + ox * tris.shape[1], j + oy * tris.shape[0], tri))
    return best


def test_terrain_hit_matches_brute_force(orc):
    r = np.random.default_rng(1)
    nx, ny = 6, 5
    h = r.uniform(0.0, 0.3, (ny, nx)).astype(np.float32)
    S = _scene(orc, h, nx=8, ny=8)
    Lx = Ly = 8 * float(np.float32(0.1))       # the domain is nx voxels of the FP32 voxel size
    hx, hy = Lx / nx, Ly / ny
    tris = _triangles(h.astype(np.float64), hx, hy)
    n_hit = 0
    for k in range(300):
        o = np.array([r.uniform(0, Lx), r.uniform(0, Ly), r.uniform(0.31, 0.8)])
        d = r.normal(size=3)
        d[2] = -abs(d[2]) - 0.05
        d /= np.linalg.norm(d)
        if k % 10 == 0:                  # starts inside the relief layer above the surface
            z, _ = orc.terrain_height(S, o[0], o[1])
            o[2] = z + r.uniform(0.001, 0.05)
            d[2] = r.normal() * 0.3
            d /= np.linalg.norm(d)
        got = orc.terrain_hit(S, o, d)
        tmax = o[2] / -d[2] if d[2] < 0 else (0.3 - o[2]) / d[2] if d[2] > 0 else 10.0
        reach = [int(math.floor(min(o[a], o[a] + tmax * d[a]) / L)) - 1 for a, L in ((0, Lx), (1, Ly))]
        reach_hi = [int(math.floor(max(o[a], o[a] + tmax * d[a]) / L)) + 1 for a, L in ((0, Lx), (1, Ly))]
        tb, idb = _brute_hit(tris, Lx, Ly, o, d, (range(reach[0], reach_hi[0] + 1), range(reach[1], reach_hi[1] + 1)))
        if got is None:
            assert tb == math.inf or tb > 1e3, (k, tb)
            continue
        n_hit += 1
        t, cell, tri = got
        assert t == pytest.approx(tb, rel=1e-9, abs=1e-12), (k, t, tb)
        assert (cell[0], cell[1], tri) == idb, (k, cell, tri, idb)
    assert n_hit > 250


def test_terrain_height_and_normal_from_corners(orc):
    r = np.random.default_rng(2)
    nx, ny = 7, 4
    h = r.uniform(0.0, 0.3, (ny, nx)).astype(np.float32)
    S = _scene(orc, h)
    Lx = Ly = 8 * float(np.float32(0.1))
    tris = _triangles(h.astype(np.float64), Lx / nx, Ly / ny)
    for _ in range(200):
        j, i, t = r.integers(0, ny), r.integers(0, nx), r.integers(0, 2)
        P = tris[j, i, t]
        lam = r.dirichlet([1, 1, 1])
        x, y, z = lam @ P
        got, n = orc.terrain_height(S, x, y)
        assert got == pytest.approx(z, abs=1e-12)
        nn = np.cross(P[1] - P[0], P[2] - P[0])
        nn /= np.linalg.norm(nn)
        if nn[2] < 0:
            nn = -nn
        np.testing.assert_allclose(n, nn, atol=1e-12)


def test_flat_heightfield_is_the_flat_ground(orc):
    sp = scenes.blobs_small(0)
    base = dict(k=sp.k, dx=sp.dx, dy=sp.dy, dz=sp.dz, levels=sp.levels, k_clear=sp.k_clear, ssa_clear=sp.ssa_clear,
                ssa_cloud=sp.ssa_cloud, g=sp.g, ground_albedo=sp.ground_albedo, sun_zenith_deg=sp.sun_zenith_deg)
    n = 20000
    a, _ = orc.trace_flux(orc.Scene(**base), n, seed=3)
    b, _ = orc.trace_flux(orc.Scene(**base, heights=np.zeros((16, 16), np.float32)), n, seed=3)
    for q in range(3):
        assert abs(a.mean[q] - b.mean[q]) <= 4 * math.hypot(a.se[q], b.se[q])
        # same random numbers; the 1e-5 km lift off the surface barely matters
        assert abs(a.mean[q] - b.mean[q]) <= 0.05 * a.se[q] + 1e-12


def _bumpy(n=32, seed=4, relief=0.3):
    r = np.random.default_rng(seed)
    f = np.fft.ifft2(np.fft.fft2(r.normal(size=(n, n))) / (1 + np.add.outer(np.fft.fftfreq(n) ** 2,
                                                                           np.fft.fftfreq(n) ** 2) * 400)).real
    f = (f - f.min()) / (f.max() - f.min()) * relief
    return f.astype(np.float32)


@pytest.mark.parametrize("zenith,azimuth", [(0.0, 0.0), (40.0, 30.0), (70.0, 200.0)])
def test_direct_irradiance_conserves_sunlight(orc, zenith, azimuth):
    h = _bumpy()
    S = _scene(orc, h, nx=16, ny=16, nz=8, d=0.1, ground_albedo=0.0, sun_zenith_deg=zenith, sun_azimuth_deg=azimuth)
    t, _ = orc.trace_flux(S, 200000, seed=5)
    if zenith == 0.0:
        assert t.mean[0] == pytest.approx(1.0, abs=1e-12) and t.se[0] < 1e-12
    else:
        assert abs(t.mean[0] - 1.0) <= 3 * t.se[0], (t.mean[0], t.se[0])
        assert t.se[0] > 1e-4                        # tilt and shadows do vary per path
    assert t.mean[1] == 0.0


def test_black_sky_facet_radiance(orc):
    """A roof-shaped surface (triangle wave along x, slope 0.3), no
    atmosphere, sun in the x-z plane at 20 deg: every first-order pixel
    seeing a facet gets rho / pi * (n . s), with zero variance."""
    nx = 16
    i = np.arange(nx)
    prof = 0.3 * 0.05 * np.minimum(i, nx - i)           # heights of a periodic ridge, hx = 0.05 km
    h = np.tile(prof, (4, 1)).astype(np.float32)
    rho = 0.4
    S = _scene(orc, h, nx=8, ny=8, nz=8, d=0.1, ground_albedo=rho, sun_zenith_deg=20.0, max_order=1)
    sun = np.array(S.sun_dir())
    cam = orc.Camera((0.4, 0.4, 20.0), (0.4, 0.4, 0.0), (0.0, 1.0, 0.0), 2 * math.degrees(math.atan(0.4 / 20.0)), 32, 8)
    img, _ = orc.trace_camera(S, cam, 4, seed=1)
    hx = 8 * float(np.float32(0.1)) / nx
    s_up = (float(h[0, 1]) - float(h[0, 0])) / hx        # slopes of the stored (FP32) heights
    s_dn = (float(h[0, nx // 2 + 1]) - float(h[0, nx // 2])) / hx
    assert s_up == pytest.approx(0.3, rel=1e-6) and s_dn == pytest.approx(-0.3, rel=1e-6)
    n_up = np.array([-s_up, 0, 1]) / math.hypot(s_up, 1)     # facet rising with x
    n_dn = np.array([-s_dn, 0, 1]) / math.hypot(s_dn, 1)
    want_up, want_dn = rho / math.pi * n_up @ sun, rho / math.pi * n_dn @ sun
    m = img.mean
    # pixel columns away from the ridge lines at x = 0 and x = 0.4 km
    x = (np.arange(32) + 0.5) / 32 * 0.8
    left = (x > 0.05) & (x < 0.35)
    right = (x > 0.45) & (x < 0.75)
    # rtol: the FP32 heights make each cell's slope differ from 0.3 by ~1e-7
    np.testing.assert_allclose(m[:, left], want_up, rtol=1e-6)
    np.testing.assert_allclose(m[:, right], want_dn, rtol=1e-6)
    assert np.all(img.se[:, left] < 1e-6 * want_up)
