"""Oracle pins: Philox4x32-10, uniforms, BF16 rounding, majorant pyramid.

The Philox values are the published known-answer vectors (golden file);
the pyramid is checked against numpy's block max (a different code path)
and against the max invariants of Sec. 3.1.1 (merged voxels store the max).
"""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        w = [int(x, 16) for x in line.split()]
        rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answers(orc):
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, want in rows:
        got = orc.philox4x32_10(ctr, key)[0]
        assert [int(x) for x in got] == want


def test_uniform_range_and_chi2(orc):
    n = 1 << 18
    ctr = np.zeros((n, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(n, dtype=np.uint32)
    ctr[:, 2] = 7
    key = np.tile(np.array([12345, 678], dtype=np.uint32), (n, 1))
    w = orc.philox4x32_10(ctr, key).ravel()
    u = orc.u01(w)
    assert u.min() > 0.0 and u.max() <= 1.0
    # extremes of the mapping are exact
    assert orc.u01(np.uint32(0)) == 2.0 ** -24
    assert orc.u01(np.uint32(0xFFFFFFFF)) == 1.0
    # chi-square on 64 bins (dof 63): 99.99% quantile is about 116
    h, _ = np.histogram(u, bins=64, range=(0.0, 1.0))
    e = u.size / 64.0
    chi2 = float(((h - e) ** 2 / e).sum())
    assert chi2 < 116.0, chi2
    # words are not correlated with their neighbours
    c = np.corrcoef(u[:-1], u[1:])[0, 1]
    assert abs(c) < 5.0 / np.sqrt(u.size)


def test_bf16_rounding(orc):
    torch = pytest.importorskip("torch")
    r = np.random.default_rng(1)
    x = np.concatenate([r.uniform(0, 100, 2000), r.lognormal(0, 4, 2000), [0.0, 1.0, 3.0e-39, 65504.0]])
    x = x.astype(np.float32)
    rn = np.array([orc.bf16_round_nearest(v) for v in x], dtype=np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(rn, ref)
    ru = np.array([orc.bf16_round_up(v) for v in x], dtype=np.float32)
    assert np.all(ru >= x)
    # representable in bf16 and the smallest such value
    assert np.all((ru.view(np.uint32) & 0xFFFF) == 0)
    below = (ru.view(np.uint32) - 0x10000).view(np.float32)
    mask = ru > 0
    assert np.all(below[mask] < x[mask])
    # array version used for BF16 scenes agrees
    assert np.array_equal(orc.bf16_round_nearest_array(x), rn)


def _block_max(a, levels):
    """Reference block max with numpy: pad with zeros to a multiple of 8
    (extinction is >= 0, so padding cannot raise a max) and reduce."""
    out = []
    cur = a
    for _ in range(levels):
        nz, ny, nx = cur.shape
        pz, py, px = -(-nz // 8) * 8, -(-ny // 8) * 8, -(-nx // 8) * 8
        p = np.zeros((pz, py, px), dtype=cur.dtype)
        p[:nz, :ny, :nx] = cur
        cur = p.reshape(pz // 8, 8, py // 8, 8, px // 8, 8).max(axis=(1, 3, 5))
        out.append(cur)
    return out


@pytest.mark.parametrize("shape", [(32, 64, 64), (20, 24, 72), (13, 9, 17), (160, 64, 64)])
def test_pyramid_equals_block_max(orc, shape):
    r = np.random.default_rng(3)
    k = (r.lognormal(0.0, 2.0, shape) * (r.uniform(size=shape) < 0.3)).astype(np.float32)
    levels = 3
    got = orc.build_pyramid(k, levels)
    want = _block_max(k, levels)
    for g, w in zip(got, want):
        assert g.shape == w.shape
        assert np.array_equal(g, w)
    # invariants: every level bounds the finer one, the top holds the global max
    assert got[-1].max() == k.max()
    for l in range(levels):
        fine = k if l == 0 else got[l - 1]
        coarse = got[l]
        up = np.repeat(np.repeat(np.repeat(coarse, 8, 0), 8, 1), 8, 2)[:fine.shape[0], :fine.shape[1], :fine.shape[2]]
        assert np.all(up >= fine)


def test_pyramid_bf16_round_up_bounds_rn_field(orc):
    r = np.random.default_rng(4)
    k = r.lognormal(1.0, 1.5, (24, 32, 40)).astype(np.float32)
    pyr = orc.build_pyramid(k, 2, round_up_bf16=True)
    rn = orc.bf16_round_nearest_array(k)
    up = np.repeat(np.repeat(np.repeat(pyr[0], 8, 0), 8, 1), 8, 2)[:24, :32, :40]
    assert np.all(up >= rn) and np.all(up >= k)
    assert np.all((pyr[0].view(np.uint32) & 0xFFFF) == 0)
    plain = orc.build_pyramid(k, 2)
    want = np.array([orc.bf16_round_up(v) for v in plain[0].ravel()], dtype=np.float32).reshape(plain[0].shape)
    assert np.array_equal(pyr[0], want)


@pytest.mark.parametrize("shape", [(32, 64, 64), (13, 9, 17)])
def test_minorant_pyramid_equals_block_min(orc, shape):
    r = np.random.default_rng(5)
    k = (r.lognormal(0.0, 2.0, shape) * (r.uniform(size=shape) < 0.7)).astype(np.float32)
    got = orc.build_pyramid_min(k, 2)
    # block min over existing children: pad with +inf to whole blocks
    pz, py, px = (-(-s // 8) * 8 for s in shape)
    pad = np.full((pz, py, px), np.inf, dtype=np.float32)
    pad[:shape[0], :shape[1], :shape[2]] = k
    l1 = pad.reshape(pz // 8, 8, py // 8, 8, px // 8, 8).min(axis=(1, 3, 5))
    assert np.array_equal(got[0], l1)
    assert got[1].min() == k.min() and np.all(got[1] <= got[0].min())
    rn = orc.bf16_round_nearest_array(k)
    gb = orc.build_pyramid_min(k, 1, round_nearest_bf16=True)[0]
    padb = np.full((pz, py, px), np.inf, dtype=np.float32)
    padb[:shape[0], :shape[1], :shape[2]] = rn
    assert np.array_equal(gb, padb.reshape(pz // 8, 8, py // 8, 8, px // 8, 8).min(axis=(1, 3, 5)))
    # rounding down to bfloat16 keeps a minorant
    for v in (0.0, 1e-3, 0.3, 45.1, 431.7):
        d = orc.bf16_round_down(v)
        assert d <= v and (np.float32(d).view(np.uint32) & 0xFFFF) == 0
        assert d == 0.0 or orc.bf16_round_up(v) == d or v - d < v * 2.0 ** -7
