"""Randomised bit-exact parity of the grids and the traversal.

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
