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


def test_noalloc_allocates_nothing(env):
    """The defining property: after a first call (which looks up the static
    array's address), a call leaves the stream-ordered pool's high-water
    mark and the device's free memory where they were."""
    torch, m, ctx, sp, sc = env
    cam = scenes.nadir_camera(sp, 32, 32)
    cd = _camdesc(m, cam)
    opts = m.mcrt_trace_opts_default()
    mean = torch.empty(cam.height * cam.width, dtype=torch.float64, device="cuda")
    se = torch.empty_like(mean)
    m.mcrt_trace_camera_noalloc(ctx.h, sc.h, cd, 8, 5, opts, mean.data_ptr(), se.data_ptr())
    torch.cuda.synchronize()
    used0, _ = m.mcrt_debug_pool_usage(ctx.h, reset_high=True)
    free0, _ = torch.cuda.mem_get_info()
    m.mcrt_trace_camera_noalloc(ctx.h, sc.h, cd, 8, 6, opts, mean.data_ptr(), se.data_ptr())
    used1, high1 = m.mcrt_debug_pool_usage(ctx.h)
    free1, _ = torch.cuda.mem_get_info()
    assert used1 == used0 and high1 <= used0, (used0, used1, high1)
    assert free1 == free0, (free0, free1)
    # an allocating trace does move the high mark (the check can see one)
    m.mcrt_debug_pool_usage(ctx.h, reset_high=True)
    t = sc.trace_camera(cam, 8, seed=6)
    _, high2 = m.mcrt_debug_pool_usage(ctx.h)
    assert high2 > used0
    assert np.all(np.isfinite(t.mean))


def test_noalloc_outputs_nan_after_a_cancelled_trace(env):
    torch, m, ctx, sp, sc = env
    # enough paths per lane that the kernel polls the flag (every 1024 iterations)
    cam = scenes.nadir_camera(sp, 256, 256)
    cd = _camdesc(m, cam)
    flag = torch.ones(1, dtype=torch.int32).pin_memory()
    opts = m.mcrt_trace_opts_default()
    opts.cancel_flag = flag.data_ptr()
    mean = torch.zeros(cam.height * cam.width, dtype=torch.float64, device="cuda")
    se = torch.zeros_like(mean)
    with pytest.raises(m.McrtError) as e:
        m.mcrt_trace_camera_noalloc(ctx.h, sc.h, cd, 1024, 7, opts, mean.data_ptr(), se.data_ptr())
    assert e.value.status == m.MCRT_ERR_CANCELLED
    assert torch.isnan(mean).all() and torch.isnan(se).all()


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
