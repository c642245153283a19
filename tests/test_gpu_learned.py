"""GPU parity of the learned proposal's network against the FP64 oracle.

* Inference (tensor cores, BF16 operands, FP32 accumulation): raw outputs
  within a bound derived from the arithmetic -- the GPU rounds each layer's
  activations to BF16 (relative error <= 2^-9, taken as 2^-8), the error is
  carried through the layers by |W| and the GELU Lipschitz constant (1.13),
  plus FP32 accumulation slack; the mixture epilogue is checked against the
  oracle's mixture of the same raw outputs.
* Training (FP32): the gradient of the mean KL loss against the oracle's
  FP64 gradient on the same records, and one Adam step.
"""
import math

import numpy as np
import pytest

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
    yield m, ctx
    ctx.close()


def bf16(x):
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).reshape(np.shape(x)).astype(np.float64)


def gelu(x):
    return 0.5 * x * (1 + np.tanh(0.7978845608028654 * (x + 0.044715 * x ** 3)))


def _params(orc, seed):
    p = orc.xavier_init(seed)
    r = np.random.default_rng(seed)
    p[p.size - 40:] = r.normal(size=40) * 0.5
    return p.astype(np.float32).astype(np.float64)


def _features(n, seed):
    r = np.random.default_rng(seed)
    x = np.concatenate([r.uniform(-1, 1, (n, 3)), r.normal(size=(n, 3)), r.uniform(-8, 6, (n, 3))], axis=1)
    x[:, 3:6] /= np.linalg.norm(x[:, 3:6], axis=1, keepdims=True)
    return x.astype(np.float32)


def test_mlp_inference_vs_oracle(env, orc):
    m, ctx = env
    p = _params(orc, 3)
    prop = m.Proposal(ctx, params=p)
    try:
        n = 1000                                   # 7 full 128-row tiles and a ragged tail
        x = _features(n, 4)
        mix, raw = prop.eval(x)
        W1, b1, W2, b2, W3, b3, W4, b4 = orc.mlp_split(p)
        Wb = [bf16(W) for W in (W1, W2, W3, W4)]
        a = bf16(x.astype(np.float64))
        ref = orc.mlp_forward(np.concatenate([Wb[0].ravel(), b1, Wb[1].ravel(), b2, Wb[2].ravel(), b3,
                                              Wb[3].ravel(), b4]), a)
        # error bound through the layers: the propagated error (GELU
        # Lipschitz 1.13), BF16 rounding of each activation (2^-8 relative),
        # and the hardware tanh inside GELU (tanh.approx.f32, relative error
        # below 2^-10.9 of |tanh| <= 1, so at most 0.5 |z| 2^-10.9 in GELU)
        da = np.zeros_like(a)
        h = a
        for W, b in ((Wb[0], b1), (Wb[1], b2), (Wb[2], b3)):
            z = h @ W.T + b
            dz = (np.abs(da) @ np.abs(W).T) + 64 * 2.0 ** -23 * (np.abs(h) @ np.abs(W).T + np.abs(b))
            h = gelu(z)
            da = 1.13 * dz + 2.0 ** -8 * np.abs(h) + 0.5 * np.abs(z) * 2.0 ** -10.9
        bound = np.abs(da) @ np.abs(Wb[3]).T + 64 * 2.0 ** -23 * (np.abs(h) @ np.abs(Wb[3]).T + np.abs(b4))
        err = np.abs(raw - ref)
        assert np.all(err <= bound + 1e-6), (err.max(), (err - bound).max())
        # the epilogue: mixture of the raw outputs
        for i in range(0, n, 97):
            mu, ka, pi = orc.mixture(raw[i].astype(np.float64))
            got = mix[i].reshape(8, 5)
            np.testing.assert_allclose(got[:, :3], mu, rtol=1e-5, atol=1e-6)
            np.testing.assert_allclose(got[:, 3], ka, rtol=1e-5, atol=1e-6)
            np.testing.assert_allclose(got[:, 4], pi, rtol=1e-4, atol=1e-7)
    finally:
        prop.close()


@pytest.mark.parametrize("n", [1, 127, 129, 4097])
def test_mlp_inference_tile_edges(env, orc, n):
    """Row counts around the 128-row tile: every row's raw outputs equal the
    same rows evaluated in a larger batch bit for bit (a row's result does
    not depend on its tile neighbours), and the mixture of each row matches
    the oracle's mixture of its raw outputs."""
    m, ctx = env
    p = _params(orc, 9)
    prop = m.Proposal(ctx, params=p)
    try:
        x = _features(5000, 10)
        mix_all, raw_all = prop.eval(x)
        mix, raw = prop.eval(x[:n])
        np.testing.assert_array_equal(raw, raw_all[:n])
        np.testing.assert_array_equal(mix, mix_all[:n])
        for i in sorted({0, n // 2, n - 1}):
            mu, ka, pi = orc.mixture(raw[i].astype(np.float64))
            got = mix[i].reshape(8, 5)
            np.testing.assert_allclose(got[:, :3], mu, rtol=1e-5, atol=1e-6)
            np.testing.assert_allclose(got[:, 4], pi, rtol=1e-4, atol=1e-7)
    finally:
        prop.close()


def test_mlp_gradient_and_adam_vs_oracle(env, orc):
    m, ctx = env
    p = _params(orc, 5)
    prop = m.Proposal(ctx, params=p, training=m.MCRT_TRAIN_FP32)
    try:
        n = 3000
        x = _features(n, 6)
        r = np.random.default_rng(7)
        d = r.normal(size=(n, 3)); d /= np.linalg.norm(d, axis=1, keepdims=True)
        t = r.exponential(size=n)
        t[::7] = 0.0                               # records that brought nothing back
        loss, g = prop.train_step(x, d.astype(np.float32), t.astype(np.float32), lr=0.0)
        xb = bf16(x.astype(np.float64))            # the network sees BF16 features
        oloss, og = orc.mlp_loss_grad(p, xb, d.astype(np.float32).astype(np.float64),
                                      t.astype(np.float32).astype(np.float64))
        assert loss == pytest.approx(oloss, rel=1e-4)
        scale = np.abs(og).max()
        assert np.abs(g - og).max() <= 2e-4 * scale, (np.abs(g - og).max(), scale)
        # one Adam step
        lr = 1e-3
        loss2, g2 = prop.train_step(x, d.astype(np.float32), t.astype(np.float32), lr=lr)
        newp = prop.params.astype(np.float64)
        pp = p.copy(); mm = np.zeros_like(p); vv = np.zeros_like(p)
        orc.adam_step(pp, mm, vv, g2.astype(np.float64), 1, lr=lr)
        np.testing.assert_allclose(newp, pp, rtol=1e-5, atol=1e-7)
    finally:
        prop.close()


def test_mlp_gradient_on_tensor_cores(env, orc):
    """The tensor-core gradient (BF16 operands and activations, FP32
    accumulation) against the FP64 oracle on the same records.  Each
    product carries BF16 rounding of both operands (relative 2^-8 each,
    taken as 2^-8 combined after the FP32 sums), compounded over the
    three hidden layers, so a few per cent of relative error in each
    parameter block is the expected size: the test asks for a relative L2
    error below 4 % per weight matrix, a cosine above 0.998 overall, and
    the same loss to 1e-3 (the loss uses BF16 activations too)."""
    m, ctx = env
    p = _params(orc, 5)
    prop = m.Proposal(ctx, params=p)            # tensor cores by default
    try:
        n = 3000
        x = _features(n, 6)
        r = np.random.default_rng(7)
        d = r.normal(size=(n, 3)); d /= np.linalg.norm(d, axis=1, keepdims=True)
        t = r.exponential(size=n)
        t[::7] = 0.0
        loss, g = prop.train_step(x, d.astype(np.float32), t.astype(np.float32), lr=0.0)
        xb = bf16(x.astype(np.float64))
        oloss, og = orc.mlp_loss_grad(p, xb, d.astype(np.float32).astype(np.float64),
                                      t.astype(np.float32).astype(np.float64))
        assert loss == pytest.approx(oloss, rel=1e-3)
        offs = [0, 576, 640, 4736, 4800, 8896, 8960, 11520, 11560]
        for a, b in zip(offs[:-1:2], offs[1::2]):
            gg, oo = g[a:b].astype(np.float64), og[a:b]
            assert np.linalg.norm(gg - oo) <= 0.04 * np.linalg.norm(oo), (a, np.linalg.norm(gg - oo) / np.linalg.norm(oo))
        cos = float(g.astype(np.float64) @ og / (np.linalg.norm(g) * np.linalg.norm(og)))
        assert cos > 0.998, cos
    finally:
        prop.close()


# ---------------------------------------------------------------------------
# the learned proposal inside the tracer
# ---------------------------------------------------------------------------
def _oscene(orc, sp, **kw):
    a = dict(k=sp.k, dx=sp.dx, dy=sp.dy, dz=sp.dz, levels=sp.levels, k_clear=sp.k_clear, ssa_clear=sp.ssa_clear,
             ssa_cloud=sp.ssa_cloud, g=sp.g, ground_albedo=sp.ground_albedo, sun_zenith_deg=sp.sun_zenith_deg)
    a.update(kw)
    return orc.Scene(**a)


def _close(a, sa, b, sb):
    return abs(a - b) <= 4.0 * math.hypot(sa, sb)


def test_learned_tracer_unbiased_and_matches_oracle(env, orc):
    """A fixed network (no training): the MIS-weighted estimate equals the
    plain one (GPU and oracle) and the oracle's learned estimate with the same
    parameters, within 4 combined SE, for flux and image tallies."""
    import scenes
    m, ctx = env
    sp = scenes.blobs_small(0)
    p = _params(orc, 21)
    sc = m.Scene.from_spec(ctx, sp)
    prop = m.Proposal(ctx, params=p)
    try:
        n = 100000
        plain = sc.trace_flux(n, seed=41)
        learned = sc.trace_flux(n, seed=42, proposal=prop, batch_paths=30000)
        ol, _ = orc.trace_flux(_oscene(orc, sp, mlp=p), n, seed=42)
        op, _ = orc.trace_flux(_oscene(orc, sp), n, seed=41)
        for q in range(3):
            assert _close(learned.mean[q], learned.se[q], plain.mean[q], plain.se[q]), (q, learned.mean, plain.mean)
            assert _close(learned.mean[q], learned.se[q], ol.mean[q], ol.se[q]), (q, learned.mean, ol.mean)
            assert _close(plain.mean[q], plain.se[q], op.mean[q], op.se[q])
        cam = scenes.nadir_camera(sp, 32, 32)
        a = sc.trace_camera(cam, 64, seed=43)
        b = sc.trace_camera(cam, 64, seed=44, proposal=prop, batch_paths=16384)
        ma, mb = a.mean.mean(), b.mean.mean()
        sa = math.sqrt((a.se ** 2).sum()) / a.se.size
        sb = math.sqrt((b.se ** 2).sum()) / b.se.size
        assert _close(ma, sa, mb, sb), (ma, mb, sa, sb)
        blocks = lambda x: x.reshape(4, 8, 4, 8).sum(axis=(1, 3))
        z = np.abs(blocks(a.mean) - blocks(b.mean)) / np.hypot(np.sqrt(blocks(a.se ** 2)), np.sqrt(blocks(b.se ** 2)))
        assert int((z > 4).sum()) <= 1
    finally:
        prop.close()
        sc.close()


def test_learned_result_independent_of_batches(env, orc):
    """A frozen network's estimate depends only on the path ids: one pixel
    (or one path) per batch, three pixels per batch and the whole image in
    one batch give the same tallies up to the order of the additions.  The
    batches change which paths share a pass and which vertices share a
    network tile, so this also checks that no path is lost or repeated
    between passes and that a row's network output does not depend on the
    rows beside it."""
    import scenes
    m, ctx = env
    sp = scenes.blobs_small(0)
    sc = m.Scene.from_spec(ctx, sp)
    prop = m.Proposal(ctx, params=_params(orc, 23))
    try:
        cam = scenes.nadir_camera(sp, 16, 16)
        kw = dict(seed=61, proposal=prop, n_learned=3, mis_alpha=0.5)
        one = sc.trace_camera(cam, 32, batch_paths=32, **kw)          # a pixel per batch
        three = sc.trace_camera(cam, 32, batch_paths=32 * 3, **kw)    # 3 pixels per batch
        whole = sc.trace_camera(cam, 32, batch_paths=1 << 20, **kw)   # one batch
        assert one.mean.max() > 0.0
        for r in (three, whole):
            np.testing.assert_allclose(r.mean, one.mean, rtol=2e-6, atol=1e-9)
            np.testing.assert_allclose(r.se, one.se, rtol=1e-4, atol=1e-8)
        f1 = sc.trace_flux(4099, seed=62, proposal=prop, batch_paths=1, n_learned=3)
        f4 = sc.trace_flux(4099, seed=62, proposal=prop, batch_paths=1 << 20, n_learned=3)
        np.testing.assert_allclose(f4.mean, f1.mean, rtol=2e-6, atol=1e-9)
    finally:
        prop.close()
        sc.close()


def test_training_gains_where_directions_matter(env):
    """What the trained network gains over the method without it, on a scene
    whose radiance hinges on the scattering direction: a nadir view of a
    homogeneous slab (tau = 2, albedo 1, g = 0.85) over a black ground with
    the sun at 30 deg, scored to order 2.  Most of the second-order radiance
    arrives from near the sun direction, which the forward-peaked HG phase
    function rarely samples from a downward path (a back-scatter), so plain
    sampling has a heavy-tailed, high variance.  A network trained online
    on camera paths of that view (one learned vertex, MIS share 0.5) must
    cut the per-path variance of the image at least 10-fold against plain
    HG sampling and 3-fold against the same untrained network (measured:
    55-fold and 6.5-fold; a hand-set lobe toward the sun cuts it 40- to
    80-fold on the oracle), and the three images must agree in their mean.  Variances are pooled over the 64
    pixels of 2^18 paths each, so they are estimated from 2^24 paths."""
    import scenes
    m, ctx = env
    sp = scenes.homogeneous(16, 16, 10, 0.1, 2.0, levels=1, g=0.85, ssa_cloud=1.0, ssa_clear=1.0,
                            sun_zenith_deg=30.0)
    sc = m.Scene.from_spec(ctx, sp)
    cam = scenes.nadir_camera(sp, 8, 8)
    spp = 1 << 18
    kw = dict(max_order=2)

    def pooled(r):
        return float(r.mean.mean()), float(np.mean(r.se ** 2) * spp), math.sqrt(float(np.mean(r.se ** 2)) / r.se.size)

    trained = m.Proposal(ctx, seed=7)
    untrained = m.Proposal(ctx, seed=7)
    try:
        sc.trace_camera(cam, 1 << 16, seed=1, proposal=trained, learn=1, batch_paths=1 << 18, n_learned=1,
                        mis_alpha=0.5, train_steps=8, learning_rate=3e-3, **kw)
        plain = pooled(sc.trace_camera(cam, spp, seed=2, **kw))
        lt = pooled(sc.trace_camera(cam, spp, seed=3, proposal=trained, learn=0, n_learned=1, mis_alpha=0.5, **kw))
        lu = pooled(sc.trace_camera(cam, spp, seed=4, proposal=untrained, learn=0, n_learned=1, mis_alpha=0.5,
                                    **kw))
        assert lt[1] < plain[1] / 10.0, (lt[1], plain[1])
        assert lt[1] < lu[1] / 3.0, (lt[1], lu[1])
        for other in (plain, lu):
            assert abs(lt[0] - other[0]) <= 4.0 * math.hypot(lt[2], other[2]), (lt[0], other[0])
    finally:
        trained.close()
        untrained.close()
        sc.close()


def test_online_training_changes_network_and_stays_unbiased(env, orc):
    import scenes
    m, ctx = env
    sp = scenes.blobs_small(0)
    sc = m.Scene.from_spec(ctx, sp)
    prop = m.Proposal(ctx, seed=5)
    try:
        p0 = prop.params.copy()
        n = 200000
        learned = sc.trace_flux(n, seed=51, proposal=prop, learn=1, batch_paths=25000, train_steps=4)
        p1 = prop.params
        assert np.abs(p1 - p0).max() > 1e-4            # Adam moved the weights
        assert np.all(np.isfinite(p1))
        plain = sc.trace_flux(n, seed=52)
        for q in range(3):
            assert _close(learned.mean[q], learned.se[q], plain.mean[q], plain.se[q]), (q, learned.mean, plain.mean)
    finally:
        prop.close()
        sc.close()


def test_apply_gradient_matches_oracle_adam(env, orc):
    """Data-parallel building block: a gradient taken with lr = 0 and then
    applied with apply_gradient gives the oracle's Adam step on that same
    gradient.  (Two gradient calls on the same records agree only to FP32
    rounding -- the kernel adds its partial sums with atomics in varying
    order -- which is why every rank applies one averaged copy.)"""
    m, ctx = env
    p = _params(orc, 9)
    a = m.Proposal(ctx, params=p, training=m.MCRT_TRAIN_FP32)
    b = m.Proposal(ctx, params=p, training=m.MCRT_TRAIN_FP32)
    try:
        n = 2000
        x = _features(n, 10)
        r = np.random.default_rng(11)
        d = r.normal(size=(n, 3)); d /= np.linalg.norm(d, axis=1, keepdims=True)
        d = d.astype(np.float32)
        t = r.exponential(size=n).astype(np.float32)
        _, ga = a.train_step(x, d, t, lr=0.0)
        _, gb = b.train_step(x, d, t, lr=0.0)
        np.testing.assert_allclose(ga, gb, rtol=0, atol=1e-6 * np.abs(gb).max())
        b.apply_gradient(gb, lr=1e-3)
        a.apply_gradient(gb, lr=1e-3)
        np.testing.assert_array_equal(a.params, b.params)     # same gradient, same step
        pp = p.copy(); mm = np.zeros_like(p); vv = np.zeros_like(p)
        orc.adam_step(pp, mm, vv, gb.astype(np.float64), 1, lr=1e-3)
        np.testing.assert_allclose(b.params.astype(np.float64), pp, rtol=1e-5, atol=1e-7)
        with pytest.raises(m.McrtError):
            b.apply_gradient(np.full(11560, np.nan, dtype=np.float32))
    finally:
        a.close()
        b.close()


def _vmf_np(mu, kappa, r):
    """vMF directions about unit rows of mu (Wood 1994 inversion)."""
    n = mu.shape[0]
    xi, phi = r.uniform(size=n), 2.0 * np.pi * r.uniform(size=n)
    w = 1.0 + np.log(xi + (1.0 - xi) * np.exp(-2.0 * kappa)) / kappa
    s = np.sqrt(np.maximum(0.0, 1.0 - w * w))
    a = np.where(np.abs(mu[:, 2:3]) < 0.9, np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]]))
    b1 = np.cross(mu, a)
    b1 /= np.linalg.norm(b1, axis=1, keepdims=True)
    b2 = np.cross(mu, b1)
    return w[:, None] * mu + (s * np.cos(phi))[:, None] * b1 + (s * np.sin(phi))[:, None] * b2


def _direction_field_records(n, r, kappa=20.0):
    x = np.concatenate([r.uniform(-1, 1, (n, 3)), r.normal(size=(n, 3)), r.uniform(-8, 6, (n, 3))], axis=1)
    x[:, 3:6] /= np.linalg.norm(x[:, 3:6], axis=1, keepdims=True)
    mu = np.stack([x[:, 0], x[:, 1], np.ones(n)], axis=1)
    mu /= np.linalg.norm(mu, axis=1, keepdims=True)
    return x.astype(np.float32), _vmf_np(mu, kappa, r).astype(np.float32), np.ones(n, np.float32), mu


def test_training_learns_a_known_direction_field(env):
    """What training gains, against a known answer: records whose directions
    follow a vMF lobe (kappa 20) about mu(x) = normalise(x0, x1, 1) with unit
    targets.  The loss is then the cross-entropy of that lobe against the
    network's mixture, minimal (the lobe's entropy, -0.158) when the mixture
    is the lobe itself.  The untrained network sits near the uniform
    density's log(4 pi) = 2.53; 400 Adam steps on the tensor-core gradient
    must bring the held-out loss within 0.15 of the optimum and point the
    mixture's mean direction along mu(x)."""
    m, ctx = env
    kappa = 20.0
    h_opt = math.log(4.0 * math.pi * math.sinh(kappa) / kappa) - kappa * (1.0 / math.tanh(kappa) - 1.0 / kappa)
    prop = m.Proposal(ctx, seed=13)
    try:
        xt, dt, tt, mut = _direction_field_records(4096, np.random.default_rng(99), kappa)
        l0, _ = prop.train_step(xt, dt, tt, lr=0.0)
        r = np.random.default_rng(21)
        for _ in range(400):
            x, d, t, _ = _direction_field_records(4096, r, kappa)
            prop.train_step(x, d, t, lr=3e-3)
        l1, _ = prop.train_step(xt, dt, tt, lr=0.0)
        assert l0 > 2.2, l0
        assert l1 < h_opt + 0.15, (l1, h_opt)
        mix, _ = prop.eval(xt)
        lobes = mix.reshape(-1, 8, 5).astype(np.float64)
        mean_dir = np.sum(lobes[:, :, 4:5] * lobes[:, :, :3], axis=1)
        mean_dir /= np.linalg.norm(mean_dir, axis=1, keepdims=True)
        cos = np.sum(mean_dir * mut, axis=1)
        assert np.mean(cos) > 0.95 and np.quantile(cos, 0.05) > 0.8, (np.mean(cos), np.quantile(cos, 0.05))
    finally:
        prop.close()


# ---------------------------------------------------------------------------
# Online-training records against the oracle's, path by path
# ---------------------------------------------------------------------------
def _pair_records(g, o):
    """Group GPU records (in pass order) and oracle records (in vertex
    order) by path; return (paths with equal counts / all paths, list of
    (gpu index, oracle index) pairs for those paths)."""
    go = {}
    for i, pth in enumerate(g["path"].tolist()):
        go.setdefault(pth, []).append(i)
    oo = {}
    for i, pth in enumerate(o["path"].tolist()):
        oo.setdefault(pth, []).append(i)
    paths = set(go) | set(oo)
    same = [p for p in paths if len(go.get(p, [])) == len(oo.get(p, []))]
    pairs = [(gi, oi) for p in same for gi, oi in zip(go[p], oo[p])]
    return len(same) / max(1, len(paths)), np.array(pairs, dtype=np.int64).reshape(-1, 2)


@pytest.mark.parametrize("sensor", ["camera", "flux"])
def test_training_records_match_oracle(env, orc, sensor):
    """Every learned vertex's record -- features, sampled direction, score
    before it, w * omega, its own estimate and the KL target -- against the
    oracle's records of the same path ids (HG directions, alpha = 1, so the
    paths draw the same numbers on both sides and differ only by FP32
    rounding): features to one BF16 step, directions and weights to FP32
    rounding, targets to a tolerance scaled by the score they are the
    difference of.  The oracle's targets are pinned by the single-scatter
    closed form in the oracle tests."""
    import scenes
    m, ctx = env
    sp = scenes.blobs_small(0)
    p = _params(orc, 31)
    sc = m.Scene.from_spec(ctx, sp)
    prop = m.Proposal(ctx, params=p)
    try:
        osc = _oscene(orc, sp, mlp=p, n_learned=3, mis_alpha=1.0)
        if sensor == "camera":
            cam = scenes.nadir_camera(sp, 32, 32)
            spp = 4
            g = sc.learned_records(cam, spp, seed=71, proposal=prop, n_learned=3, mis_alpha=1.0)
            o, _ = orc.learned_records(osc, orc.Camera(cam.pos, cam.target, cam.up, cam.fov_deg, 32, 32), spp,
                                       seed=71, begin=0, end=32 * 32 * spp)
        else:
            n = 4096
            g = sc.learned_records(None, n, seed=72, proposal=prop, n_learned=3, mis_alpha=1.0)
            o, _ = orc.learned_records(osc, None, 0, seed=72, begin=0, end=n)
        assert g["count"] == len(g["path"]) and len(o) > 1000
        assert abs(len(g["path"]) - len(o)) <= 0.03 * len(o), (len(g["path"]), len(o))
        frac_paths, pairs = _pair_records(g, o)
        assert frac_paths >= 0.97, frac_paths
        gi, oi = pairs[:, 0], pairs[:, 1]
        # features: the oracle's FP64 values rounded to BF16, within one BF16 step
        of = bf16(o["x"][oi].astype(np.float32))
        gf = g["feat"][gi].astype(np.float64)
        step = np.maximum(np.abs(of), 1e-30) * 2.0 ** -7
        feat_ok = np.all(np.abs(gf - of) <= step + 1e-6, axis=1)
        dir_ok = np.all(np.abs(g["dir"][gi] - o["dir"][oi]) <= 2e-4, axis=1)
        w_ok = np.abs(g["w_omega"][gi] - o["w_omega"][oi]) <= 1e-4 * o["w_omega"][oi] + 1e-9
        scale = o["before"][oi] + o["own"][oi] + o["w_omega"][oi] * o["target"][oi]
        b_ok = np.abs(g["before"][gi] - o["before"][oi]) <= 1e-3 * scale + 1e-9
        own_ok = np.abs(g["own"][gi] - o["own"][oi]) <= 1e-3 * np.abs(o["own"][oi]) + 1e-4 * scale + 1e-9
        t_tol = 2e-3 * scale / np.maximum(o["w_omega"][oi], 1e-12) + 1e-3 * o["target"][oi] + 1e-9
        t_ok = np.abs(g["target"][gi] - o["target"][oi]) <= t_tol
        for name, ok in (("feat", feat_ok), ("dir", dir_ok), ("w_omega", w_ok), ("before", b_ok),
                         ("own", own_ok), ("target", t_ok)):
            assert ok.mean() >= 0.97, (name, ok.mean())
        # the targets' sum over all records agrees too (no systematic factor)
        st = float(g["target"].sum()), float(o["target"].sum())
        assert abs(st[0] - st[1]) <= 0.02 * abs(st[1]), st
    finally:
        prop.close()
        sc.close()


def test_training_records_with_network_match_oracle(env, orc):
    """With the network in the mixture (alpha = 0.5) the GPU's BF16 network
    and the oracle's FP64 one sample slightly different directions, so paths
    part after their first learned vertex: the first vertex's features still
    pair up exactly, and the mean KL target of all records agrees within 4
    combined standard errors."""
    import scenes
    m, ctx = env
    sp = scenes.blobs_small(0)
    p = _params(orc, 33)
    sc = m.Scene.from_spec(ctx, sp)
    prop = m.Proposal(ctx, params=p)
    try:
        n = 16384
        g = sc.learned_records(None, n, seed=73, proposal=prop, n_learned=3, mis_alpha=0.5, cap=1 << 17)
        o, _ = orc.learned_records(_oscene(orc, sp, mlp=p, n_learned=3, mis_alpha=0.5), None, 0, seed=73,
                                   begin=0, end=n, cap=1 << 17)
        first_o = o[o["vertex"] == 0]
        gpos = {}
        for i, pth in enumerate(g["path"].tolist()):
            gpos.setdefault(pth, i)          # a path's first record comes from the first pass
        idx = [(gpos[int(pth)], j) for j, pth in enumerate(first_o["path"].tolist()) if int(pth) in gpos]
        assert len(idx) >= 0.97 * len(first_o)
        gi, oi = np.array(idx).T
        of = bf16(first_o["x"][oi].astype(np.float32))
        feat_ok = np.all(np.abs(g["feat"][gi] - of) <= np.maximum(np.abs(of), 1e-30) * 2.0 ** -7 + 1e-6, axis=1)
        assert feat_ok.mean() >= 0.97
        tg, to = g["target"].astype(np.float64), o["target"]
        se = math.hypot(tg.std() / math.sqrt(len(tg)), to.std() / math.sqrt(len(to)))
        assert abs(tg.mean() - to.mean()) <= 4 * se, (tg.mean(), to.mean(), se)
    finally:
        prop.close()
        sc.close()
