"""Checkpoint and resume on the GPU: a segmented camera run stopped and
resumed from its file equals the uninterrupted run (to the order of the
FP64 atomic adds inside a segment); a network restored with its Adam state
continues training bit for bit."""
import numpy as np
import pytest

import scenes

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


def test_segmented_camera_run_resumes(env, tmp_path):
    m, ctx = env
    from paper_1902_01137_gb300.checkpoint import Accumulator
    sp = scenes.blobs_small(0)
    sc = m.Scene.from_spec(ctx, sp)
    cam = scenes.nadir_camera(sp, 24, 16)
    try:
        def run(acc, k):
            for _ in range(k):
                t = m.mcrt_trace_camera(ctx.h, sc.h, _desc(m, cam), 8, acc.next_seed(), m.mcrt_trace_opts_default())
                try:
                    s1, s2 = m.mcrt_tally_read_sums(ctx.h, t)
                finally:
                    m.mcrt_tally_destroy(t)
                acc.add(s1.reshape(16, 24), s2.reshape(16, 24), 8.0)
        full = Accumulator((16, 24), seed=5)
        run(full, 4)
        part = Accumulator((16, 24), seed=5)
        run(part, 2)
        path = str(tmp_path / "cam.ckpt")
        part.save(path)
        resumed = Accumulator.load(path)
        run(resumed, 2)
        np.testing.assert_allclose(resumed.s1, full.s1, rtol=1e-12, atol=0)
        np.testing.assert_allclose(resumed.s2, full.s2, rtol=1e-12, atol=0)
        assert np.array_equal(resumed.n, full.n) and float(full.n[0, 0]) == 32.0
    finally:
        sc.close()


def _desc(m, cam):
    cd = m.CameraDesc()
    for i in range(3):
        cd.pos[i], cd.target[i], cd.up[i] = cam.pos[i], cam.target[i], cam.up[i]
    cd.fov_deg, cd.width, cd.height = cam.fov_deg, cam.width, cam.height
    return cd


def test_network_checkpoint_continues_training_exactly(env, orc, tmp_path):
    m, ctx = env
    from paper_1902_01137_gb300.checkpoint import Accumulator
    p0 = orc.xavier_init(3).astype(np.float32)
    r = np.random.default_rng(17)
    grads = [(r.normal(size=11560) * 1e-2).astype(np.float32) for _ in range(6)]
    a = m.Proposal(ctx, params=p0)
    b = m.Proposal(ctx, params=p0)
    c = m.Proposal(ctx)
    try:
        for g in grads:
            a.apply_gradient(g, lr=2e-3)
        for g in grads[:3]:
            b.apply_gradient(g, lr=2e-3)
        acc = Accumulator((1,), seed=9)
        path = str(tmp_path / "net.ckpt")
        acc.save(path, proposal=b)
        Accumulator.load(path, proposal=c)              # a fresh network takes the saved state
        mm, vv, st = c.adam_state
        assert st == 3 and np.all(vv >= 0)
        for g in grads[3:]:
            c.apply_gradient(g, lr=2e-3)
        np.testing.assert_array_equal(c.params, a.params)
        with pytest.raises(m.McrtError):
            c.adam_state = (mm, -np.ones_like(vv), 3)   # a negative second moment is refused
    finally:
        a.close()
        b.close()
        c.close()
