"""The camera trace that allocates no device memory.

Callers that cannot allocate GPU memory while tracing (code running inside
another framework's memory budget, real-time loops that must not touch the
allocator) use mcrt_trace_camera_noalloc: the library keeps its working sums
in one static device array and writes mean and standard error into buffers
the caller owns.  This file is collected last so that a failure here comes
after every other test has run.
"""
import ctypes as C

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
    sp = scenes.blobs_small(0)
    sc = m.Scene.from_spec(ctx, sp)
    yield torch, m, ctx, sp, sc
    sc.close()
    ctx.close()


def _camdesc(m, cam):
    cd = m.CameraDesc()
    for i in range(3):
        cd.pos[i], cd.target[i], cd.up[i] = cam.pos[i], cam.target[i], cam.up[i]
    cd.fov_deg, cd.width, cd.height = cam.fov_deg, cam.width, cam.height
    return cd


def test_noalloc_matches_allocating_trace_twice(env):
    torch, m, ctx, sp, sc = env
    cam = scenes.nadir_camera(sp, 64, 48)
    cd = _camdesc(m, cam)
    opts = m.mcrt_trace_opts_default()
    ref = sc.trace_camera(cam, 16, seed=21)
    mean = torch.empty(cam.height * cam.width, dtype=torch.float64, device="cuda")
    se = torch.empty_like(mean)
    for _ in range(2):          # the shared working area is cleared on every call
        mean.fill_(-1.0)
        se.fill_(-1.0)
        m.mcrt_trace_camera_noalloc(ctx.h, sc.h, cd, 16, 21, opts, mean.data_ptr(), se.data_ptr())
        got = mean.cpu().numpy().reshape(cam.height, cam.width)
        gse = se.cpu().numpy().reshape(cam.height, cam.width)
        # same paths and draws; only the summation grouping can differ
        np.testing.assert_allclose(got, ref.mean, rtol=4e-6, atol=1e-12)
        np.testing.assert_allclose(gse, ref.se, rtol=1e-4, atol=1e-9)


def test_noalloc_rejects_oversized_image(env):
    torch, m, ctx, sp, sc = env
    cam = scenes.nadir_camera(sp, 512, 256)
    cd = _camdesc(m, cam)
    opts = m.mcrt_trace_opts_default()
    buf = torch.empty(512 * 256, dtype=torch.float64, device="cuda")
    with pytest.raises(m.McrtError) as e:
        m.mcrt_trace_camera_noalloc(ctx.h, sc.h, cd, 4, 1, opts, buf.data_ptr(), buf.data_ptr())
    assert e.value.status == m.MCRT_ERR_BOUNDS
    assert "65536" in str(e.value)
