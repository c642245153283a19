"""Oracle pins for the learned scattering proposal (no counterpart in the
paper; a project addition): network forward and gradient against torch's
float64 autograd, gradient against central finite differences, vMF
normalisation and moments, one-sample MIS unbiasedness, Adam against
torch.optim.Adam, and the learned tracer against the plain tracer."""
import math

import numpy as np
import pytest

import scenes


def _torch_mlp(torch, params, x):
    W1, b1, W2, b2, W3, b3, W4, b4 = params
    F = torch.nn.functional
    h = F.gelu(x @ W1.T + b1, approximate="tanh")
    h = F.gelu(h @ W2.T + b2, approximate="tanh")
    h = F.gelu(h @ W3.T + b3, approximate="tanh")
    return h @ W4.T + b4


def _torch_loss(torch, raw, dirs, t):
    """-t log q_vMF written with torch primitives (log-sum-exp form)."""
    B = raw.shape[0]
    r = raw.reshape(B, 8, 5)
    mu = r[:, :, :3] / torch.linalg.norm(r[:, :, :3], dim=2, keepdim=True)
    kappa = torch.nn.functional.softplus(r[:, :, 3]) + 1e-3
    logpi = torch.log_softmax(r[:, :, 4], dim=1)
    c = (mu * dirs[:, None, :]).sum(dim=2)
    logf = torch.log(kappa) - math.log(2 * math.pi) - torch.log(-torch.expm1(-2 * kappa)) + kappa * (c - 1)
    logq = torch.logsumexp(logpi + logf, dim=1)
    return (-(t * logq)).sum() / B


def _records(n, seed):
    r = np.random.default_rng(seed)
    x = r.normal(size=(n, 9)) * np.array([0.6, 0.6, 0.6, 0.6, 0.6, 0.6, 2.0, 2.0, 2.0])
    d = r.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    t = r.exponential(size=n)
    return x, d, t


def test_mlp_forward_matches_torch(orc):
    torch = pytest.importorskip("torch")
    p = orc.xavier_init(3)
    p[p.size - 40:] = np.random.default_rng(1).normal(size=40) * 0.1      # non-zero output bias
    x, _, _ = _records(64, 4)
    got = orc.mlp_forward(p, x)
    tp = [torch.tensor(a, dtype=torch.float64) for a in orc.mlp_split(p)]
    want = _torch_mlp(torch, tp, torch.tensor(x)).numpy()
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)


def test_mlp_gradient_matches_torch_autograd(orc):
    torch = pytest.importorskip("torch")
    p = orc.xavier_init(5)
    x, d, t = _records(48, 6)
    loss, g = orc.mlp_loss_grad(p, x, d, t)
    tp = [torch.tensor(a, dtype=torch.float64, requires_grad=True) for a in orc.mlp_split(p)]
    raw = _torch_mlp(torch, tp, torch.tensor(x))
    L = _torch_loss(torch, raw, torch.tensor(d), torch.tensor(t))
    L.backward()
    want = np.concatenate([a.grad.numpy().ravel() for a in tp])
    assert loss == pytest.approx(L.item(), rel=1e-12)
    np.testing.assert_allclose(g, want, rtol=1e-9, atol=1e-12)


def test_mlp_gradient_matches_finite_differences(orc):
    p = orc.xavier_init(7)
    x, d, t = _records(16, 8)
    _, g = orc.mlp_loss_grad(p, x, d, t)
    r = np.random.default_rng(9)
    idx = np.concatenate([r.choice(p.size, 40, replace=False), [0, 575, 640, 11519, 11559]])
    h = 1e-6
    for i in idx:
        pp = p.copy(); pp[i] += h
        pm = p.copy(); pm[i] -= h
        fd = (orc.mlp_loss_grad(pp, x, d, t)[0] - orc.mlp_loss_grad(pm, x, d, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])


@pytest.mark.parametrize("kappa", [0.05, 1.0, 12.0, 300.0])
def test_vmf_normalisation_and_mean(orc, kappa):
    from scipy import integrate
    mu = np.array([0.3, -0.5, 0.8]); mu /= np.linalg.norm(mu)
    # density depends on c = mu.x only: integral over the sphere = 2 pi int f(c) dc
    ortho = np.cross(mu, [1.0, 0.0, 0.0]); ortho /= np.linalg.norm(ortho)

    def f(c):
        x = c * mu + math.sqrt(max(0.0, 1 - c * c)) * ortho
        return orc.vmf_pdf(mu, kappa, x)
    total, _ = integrate.quad(lambda c: 2 * math.pi * f(c), -1, 1, points=[1 - 1e-3, 1 - 1e-2], limit=200)
    assert total == pytest.approx(1.0, rel=1e-7)
    r = np.random.default_rng(int(kappa * 10))
    xi = 1.0 - r.uniform(size=(40000, 2))
    c = np.array([orc.vmf_sample(mu, kappa, a, b) @ mu for a, b in xi])
    want = 1.0 / math.tanh(kappa) - 1.0 / kappa
    se = c.std() / math.sqrt(c.size)
    assert abs(c.mean() - want) < 3 * se + 1e-12


def test_mis_sampling_is_unbiased(orc):
    """E_q[(p_HG / q) h] = E_HG[h] for the defensive mixture, whatever the
    network outputs are."""
    r = np.random.default_rng(11)
    raw = r.normal(size=40) * 1.5
    g, alpha = 0.85, 0.5
    d = np.array([0.2, -0.3, -0.93]); d /= np.linalg.norm(d)
    s = np.array([0.5, 0.0, 0.866])
    h = lambda w: (w @ s) ** 2 + 0.3 * w[2]
    n = 60000
    u = 1.0 - r.uniform(size=(n, 4))
    est = np.array([f * h(w) for w, f, _, _ in (orc.mis_sample(raw, g, alpha, d, ui) for ui in u)])
    xi = 1.0 - r.uniform(size=(n, 2))
    ref = np.array([h(w) for w in orc.hg_sample_dirs(g, np.tile(d, (n, 1)), xi)])
    dd = abs(est.mean() - ref.mean())
    assert dd < 4 * math.hypot(est.std() / math.sqrt(n), ref.std() / math.sqrt(n))
    # the returned q is the mixture density of the returned direction
    w, f, q, ph = orc.mis_sample(raw, g, alpha, d, u[0])
    assert q == pytest.approx(alpha * ph + (1 - alpha) * orc.mixture_pdf(raw, w), rel=1e-12)
    assert f == pytest.approx(ph / q, rel=1e-12)


def test_adam_matches_torch(orc):
    torch = pytest.importorskip("torch")
    r = np.random.default_rng(12)
    p = r.normal(size=50)
    m = np.zeros(50); v = np.zeros(50)
    tp = torch.tensor(p.copy(), requires_grad=True)
    opt = torch.optim.Adam([tp], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    for step in range(1, 6):
        g = r.normal(size=50)
        orc.adam_step(p, m, v, g, step)
        opt.zero_grad()
        tp.grad = torch.tensor(g)
        opt.step()
    np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_learned_tracer_unbiased(orc):
    """Any network gives the same expectation as plain HG sampling."""
    sp = scenes.blobs_small(0)
    base = dict(k=sp.k, dx=sp.dx, dy=sp.dy, dz=sp.dz, levels=sp.levels, k_clear=sp.k_clear,
                ssa_clear=sp.ssa_clear, ssa_cloud=sp.ssa_cloud, g=sp.g, ground_albedo=sp.ground_albedo,
                sun_zenith_deg=sp.sun_zenith_deg)
    p = orc.xavier_init(21)
    p[-40:] = np.random.default_rng(2).normal(size=40)
    plain, _ = orc.trace_flux(orc.Scene(**base), 80000, seed=31)
    learned, _ = orc.trace_flux(orc.Scene(**base, mlp=p), 80000, seed=32)
    for q in range(3):
        d = abs(plain.mean[q] - learned.mean[q])
        assert d < 4 * math.hypot(plain.se[q], learned.se[q]), (q, plain.mean[q], learned.mean[q])
    cam = scenes.nadir_camera(sp, 16, 16)
    oc = orc.Camera(cam.pos, cam.target, cam.up, cam.fov_deg, 16, 16)
    a, _ = orc.trace_camera(orc.Scene(**base), oc, 256, seed=33)
    b, _ = orc.trace_camera(orc.Scene(**base, mlp=p), oc, 256, seed=34)
    ma, mb = a.mean.mean(), b.mean.mean()
    sa, sb = math.sqrt((a.se ** 2).sum()) / a.se.size, math.sqrt((b.se ** 2).sum()) / b.se.size
    assert abs(ma - mb) < 4 * math.hypot(sa, sb)


# ---------------------------------------------------------------------------
# Online-training records and their KL targets
# ---------------------------------------------------------------------------
def _hg(g, mu):
    return (1 - g * g) / (4 * math.pi * (1 + g * g - 2 * g * mu) ** 1.5)


def _slab_record_expectation(orc, recs, k, H, om, g, s, alpha, params):
    """E[target | vertex height z, incoming d, sampled w] for the first
    learned vertex of a path in a homogeneous slab (extinction k, height H,
    albedo om, black ground) when only two orders are scored: the next
    vertex's estimate over w * omega, i.e. p_HG(d.w) / q_mix(w) times the
    single-scattered radiance arriving from w,
        om p_HG(w.s) k exp(-k (H - z) / mu0) (1 - exp(-a t_max)) / a,
    a = k (1 - w_z / mu0), t_max the distance to the slab's top or bottom
    along w (a bottom exit meets the black ground and scores nothing)."""
    mu0 = s[2]
    z = (recs["x"][:, 2] + 1.0) * 0.5 * H
    d = recs["x"][:, 3:6]
    w = recs["dir"]
    wz = w[:, 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        tmax = np.where(wz > 0, (H - z) / wz, np.where(wz < 0, z / -wz, np.inf))
    a = k * (1.0 - wz / mu0)
    integ = np.where(np.abs(a) > 1e-12, -np.expm1(-a * tmax) / np.where(np.abs(a) > 1e-12, a, 1.0), tmax)
    L1 = om * _hg(g, w @ s) * k * np.exp(-k * (H - z) / mu0) * integ
    phg = _hg(g, np.einsum("ij,ij->i", d, w))
    if alpha >= 1.0:
        return L1
    raw = orc.mlp_forward(params, recs["x"])
    qv = np.array([orc.mixture_pdf(raw[i], w[i]) for i in range(len(w))])
    return phg / (alpha * phg + (1 - alpha) * qv) * L1


@pytest.mark.parametrize("alpha", [1.0, 0.5])
def test_record_targets_match_single_scatter_radiance(orc, alpha):
    """The records' targets are the radiance the sampled direction brought
    back, weighted by p_HG / q_mix: in a homogeneous slab scored to order 2
    their mean matches the closed form of the single-scattered radiance
    arriving along each record's direction, and a second learned vertex,
    after which nothing is scored, has target 0 exactly."""
    k, H, om, g, th0 = 1.0, 1.0, 0.9, 0.7, 30.0
    sp = scenes.homogeneous(16, 16, 10, 0.1, k, levels=1, g=g, ssa_cloud=om, ssa_clear=om,
                            sun_zenith_deg=th0)
    p = orc.xavier_init(11)
    p[-40:] = np.random.default_rng(12).normal(size=40) * 0.5
    sc = orc.Scene(k=sp.k, dx=sp.dx, dy=sp.dy, dz=sp.dz, levels=sp.levels, k_clear=0.0, ssa_clear=om,
                   ssa_cloud=om, g=g, ground_albedo=0.0, sun_zenith_deg=th0, max_order=2, mlp=p, n_learned=2,
                   mis_alpha=alpha)
    recs, scores = orc.learned_records(sc, None, 0, seed=5, begin=0, end=60000, cap=1 << 18)
    first = recs[recs["vertex"] == 0]
    second = recs[recs["vertex"] == 1]
    assert len(first) > 20000 and len(second) > 5000
    # before the first vertex nothing has been scored; after the second, nothing is
    assert np.all(first["before"] == 0.0)
    # (target 0 up to the rounding of score - before - own in FP64)
    assert np.all(np.abs(second["target"] * second["w_omega"]) <= 1e-14 * (second["before"] + second["own"]))
    mu0 = math.cos(math.radians(th0))
    s = np.array([math.sin(math.radians(th0)), 0.0, mu0])
    want = _slab_record_expectation(orc, first, k, H, om, g, s, alpha, p)
    r = first["target"] - want
    se = r.std() / math.sqrt(len(r))
    assert abs(r.mean()) < 4 * se, (r.mean(), se, first["target"].mean(), want.mean())
    for sel in (first["dir"][:, 2] > 0, first["dir"][:, 2] < 0):
        rs = r[sel]
        assert abs(rs.mean()) < 4 * rs.std() / math.sqrt(len(rs))
    # the record's pieces add up to the path's score (before + own + w omega target)
    idx = first["path"].astype(np.int64)
    total = first["before"] + first["own"] + first["w_omega"] * first["target"]
    np.testing.assert_allclose(total, scores[idx], rtol=1e-12, atol=1e-15)
