"""Oracle pins for the paper's octree (Sec. 3.1.1: groups of 2^3 cells are
tested recursively for merging; merged cells keep the min and the max
extinction; Sec. 4.2: merge while the vertical optical depth of the merged
region stays below tau~).

* Every octree level equals the max / min over aligned 2^L voxel blocks
  computed by numpy (pad and reshape), ragged edges included.
* Every leaf the traversal spec enters is the coarsest octree cell whose
  majorant times its height is <= tau~ (block maxima from numpy).
* The FP32 traversal spec over the octree matches the brute-force FP64
  face list.
* Beer's law through layered slabs and the flux tallies are the same over
  the octree as over the 8^L pyramid (any valid majorant: Sec. 2.3-2.4).
"""
import math

import numpy as np
import pytest

import scenes


def _block(k, L, op, fill):
    f = 1 << L
    nz, ny, nx = k.shape
    pz, py, px = -(-nz // f) * f, -(-ny // f) * f, -(-nx // f) * f
    pad = np.full((pz, py, px), fill, dtype=np.float32)
    pad[:nz, :ny, :nx] = k
    return op(pad.reshape(pz // f, f, py // f, f, px // f, f), axis=(1, 3, 5))


@pytest.mark.parametrize("shape", [(32, 64, 64), (13, 9, 17), (20, 24, 72), (1, 5, 3)])
def test_octree_equals_block_max_min(orc, shape):
    r = np.random.default_rng(31)
    k = (r.lognormal(0.0, 2.0, shape) * (r.uniform(size=shape) < 0.4)).astype(np.float32)
    levels = orc.octree_levels(shape[::-1])
    omax, omin = orc.build_octree(k, levels)
    assert omax[-1].size == 1 and omax[-1].item() == k.max() and omin[-1].item() == k.min()
    for L in range(1, levels + 1):
        assert np.array_equal(omax[L - 1], _block(k, L, np.max, 0.0)), L
        assert np.array_equal(omin[L - 1], _block(k, L, np.min, np.inf)), L
    rn = orc.bf16_round_nearest_array(k)
    bmax, bmin = orc.build_octree(k, 2, round_nearest_bf16=True)
    assert np.array_equal(bmax[1], _block(rn, 2, np.max, 0.0))
    assert np.array_equal(bmin[0], _block(rn, 1, np.min, np.inf))


def test_octree_levels_count(orc):
    assert orc.octree_levels((64, 64, 32)) == 6
    assert orc.octree_levels((512, 512, 160)) == 9
    assert orc.octree_levels((72, 64, 40)) == 7
    assert orc.octree_levels((1, 1, 1)) == 1


def _field(seed):
    sp = scenes.random_voxels(72, 64, 40, 0.1, 3.0, seed=seed, sparsity=0.5)
    k = sp.k.copy()
    k[:, :, 32:64] = 0.0       # empty region: coarse leaves
    k[24:, :, :] *= 0.01       # thin upper layer: mid-level leaves
    k[:, 40:44, :] *= 0.2      # a band of mid values: 2- and 4-voxel leaves
    return sp, k


@pytest.mark.parametrize("tau,finest", [(1.0, 0), (0.3, 0), (5.0, 1), (float("inf"), 0)])
def test_octree_leaves_are_coarsest_qualifying(orc, tau, finest):
    sp, k = _field(5)
    sc = orc.Scene(k=k, dx=sp.dx, dy=sp.dy, dz=sp.dz, levels=2, tau_merge=tau, finest_level=finest, grid=1)
    top = orc.octree_levels(k.shape[::-1])
    bmax = {L: _block(k, L, np.max, 0.0) for L in range(1, top + 1)}
    dz = np.float32(sp.dz)

    def ok(L, c):
        return np.float32(bmax[L][c[2], c[1], c[0]]) * np.float32(dz * np.float32(1 << L)) <= np.float32(tau)

    o, d = scenes.random_rays(sp, 80, seed=17)
    seen = set()
    for i in range(len(o)):
        cells, _, _ = orc.dda_spec(sc, o[i], d[i])
        for L, ix, iy, iz in cells:
            L = int(L)
            seen.add(L)
            c = (int(ix), int(iy), int(iz))
            if L == 0:
                assert finest == 0 and not ok(1, (c[0] >> 1, c[1] >> 1, c[2] >> 1))
                continue
            assert L == finest or ok(L, c), (L, c)
            if L < top:
                assert not ok(L + 1, (c[0] >> 1, c[1] >> 1, c[2] >> 1)), (L, c)
    assert len(seen) >= (3 if tau <= 1.0 else 1), seen      # leaves of several sizes were crossed


@pytest.mark.parametrize("tau,finest", [(1.0, 0), (0.3, 0), (5.0, 1), (float("inf"), 1)])
def test_octree_spec_matches_bruteforce(orc, tau, finest):
    sp, k = _field(2)
    sc = orc.Scene(k=k, dx=sp.dx, dy=sp.dy, dz=sp.dz, levels=2, tau_merge=tau, finest_level=finest, grid=1)
    o, d = scenes.random_rays(sp, 200, seed=13)
    checked = 0
    for i in range(len(o)):
        c2, t2, s2 = orc.dda_bruteforce(sc, o[i].astype(np.float64), d[i].astype(np.float64))
        seg = t2[:, 1] - t2[:, 0]
        if len(seg) and seg.min() < 1e-5 * max(1.0, t2[-1, 1]):
            continue
        c1, t1, s1 = orc.dda_spec(sc, o[i], d[i])
        assert s1 == s2, (i, s1, s2)
        assert np.array_equal(c1, c2), i
        np.testing.assert_allclose(t1, t2, rtol=2e-5, atol=2e-5)
        checked += 1
    assert checked > 150


def test_octree_beer_layered_slabs(orc):
    """Layer interfaces at odd voxel heights: the octree's 2^L cells split
    them differently from the pyramid; Beer's law holds over both."""
    nz = 40
    kz = np.zeros(nz, dtype=np.float32)
    kz[0:3] = 0.5
    kz[3:11] = 2.0
    kz[13:29] = 0.25
    kz[29:40] = 1.1
    k = np.broadcast_to(kz[:, None, None], (nz, 16, 16)).astype(np.float32).copy()
    th = 25.0
    sp = scenes.SceneSpec("layers", k, 0.05, 0.05, 0.05, 2, 0.0, 1.0, 1.0, 0.85, 0.0, th)
    tau_v = float(np.sum(kz.astype(np.float64) * float(np.float32(0.05))))
    want = math.exp(-tau_v / math.cos(math.radians(th)))
    for tau, fin, mode in [(1.0, 0, 0), (0.2, 0, 1), (float("inf"), 0, 0), (1.0, 0, 2)]:
        sc = orc.Scene(k=k, dx=sp.dx, dy=sp.dy, dz=sp.dz, levels=2, tau_merge=tau, finest_level=fin,
                       sun_zenith_deg=th, sun_mode=mode, grid=1)
        T, _ = orc.trace_flux(sc, 30000, seed=19)
        assert abs(T.mean[0] - want) < 3.0 * T.se[0] + 1e-12, (tau, mode, T.mean[0], want, T.se[0])


def test_octree_flux_matches_pyramid(orc):
    """Same flux tallies over the octree and the pyramid (independent seeds)."""
    sp = scenes.blobs_small(0)
    base = dict(k=sp.k, dx=sp.dx, dy=sp.dy, dz=sp.dz, levels=sp.levels, k_clear=sp.k_clear, ssa_clear=sp.ssa_clear,
                ssa_cloud=sp.ssa_cloud, g=sp.g, ground_albedo=sp.ground_albedo, sun_zenith_deg=sp.sun_zenith_deg)
    ref, _ = orc.trace_flux(orc.Scene(**base, tau_merge=1.0), 40000, seed=41)
    for tau, seed in [(1.0, 43), (10.0, 47)]:
        T, _ = orc.trace_flux(orc.Scene(**base, tau_merge=tau, grid=1), 40000, seed=seed)
        for q in range(3):
            d = abs(T.mean[q] - ref.mean[q])
            s = math.hypot(T.se[q], ref.se[q])
            assert d < 4.0 * s, (tau, q, d, s)
