"""GPU: the wavefront schedule of the camera trace (SoA queues of flights and
vertices, one kernel per stage and round) against the persistent kernel and
the CPU oracle.

Both schedules draw every random number at the same Philox counter and take
the same FP32 steps, so every path scores the same value bit for bit; the
persistent kernel with one path per claim adds each path's x and x^2 to the
FP64 sums as the wavefront does, so the images agree up to the order of the
FP64 additions (relative 1e-10 is far above that and far below any change of
a single path's score).
"""
import numpy as np
import pytest

import scenes
from parity_util import image_parity, ocam, oscene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1902_01137_gb300 as mod
    from paper_1902_01137_gb300 import build
    build.build()
    return mod


@pytest.fixture(scope="module")
def ctx(m):
    c = m.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def blobs(m, ctx):
    sp = scenes.blobs_small(0)
    sc = m.Scene.from_spec(ctx, sp)
    sc.build_octree()
    yield sp, sc
    sc.close()


def same_image(a, b):
    np.testing.assert_allclose(a.mean, b.mean, rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(a.se, b.se, rtol=1e-6, atol=1e-14)


# 48 x 40 pixels: not a multiple of the 8 x 8 claim-order tiles
@pytest.mark.parametrize("opts", [
    {},
    {"sun_mode": 1},                                    # delta tracking of the sun rays
    {"max_order": 2},                                   # order cut
    {"tau_merge": 0.0},                                 # voxels as leaves everywhere
    {"tau_merge": float("inf")},                        # one global majorant
    {"grid": 1, "finest_level": 1},                     # the paper's octree
    {"pixel_order": 1},                                 # raster claims
    {"wavefront_slots": 777},                           # a ragged pool: many rounds
    {"wavefront_slots": 1 << 26},                       # more slots than paths
])
def test_wavefront_equals_persistent(m, blobs, opts):
    sp, sc = blobs
    cam = scenes.nadir_camera(sp, 48, 40)
    popts = {k: v for k, v in opts.items() if k != "wavefront_slots"}
    ref = sc.trace_camera(cam, 16, seed=21, chunk=1, **popts)
    wf = sc.trace_camera(cam, 16, seed=21, schedule=m.MCRT_SCHEDULE_WAVEFRONT, **opts)
    same_image(wf, ref)
    assert np.all(wf.n == 16)


def test_wavefront_bf16_storage(m, ctx):
    sp = scenes.blobs_small(1)
    sc = m.Scene.from_spec(ctx, sp, storage=m.MCRT_STORAGE_BF16)
    try:
        cam = scenes.nadir_camera(sp, 40, 32)
        ref = sc.trace_camera(cam, 8, seed=5, chunk=1)
        wf = sc.trace_camera(cam, 8, seed=5, schedule=m.MCRT_SCHEDULE_WAVEFRONT, wavefront_slots=4096)
        same_image(wf, ref)
    finally:
        sc.close()


def test_wavefront_one_pixel_one_path(m, blobs):
    sp, sc = blobs
    cam = scenes.nadir_camera(sp, 1, 1)
    ref = sc.trace_camera(cam, 1, seed=3, chunk=1)
    wf = sc.trace_camera(cam, 1, seed=3, schedule=m.MCRT_SCHEDULE_WAVEFRONT)
    same_image(wf, ref)


def test_wavefront_vs_oracle(m, orc, blobs):
    sp, sc = blobs
    cam = scenes.nadir_camera(sp, 64, 64)
    g = sc.trace_camera(cam, 16, seed=0, schedule=m.MCRT_SCHEDULE_WAVEFRONT)
    o, _ = orc.trace_camera(oscene(orc, sp), ocam(orc, cam), 16, seed=0)
    ok, info = image_parity(g.mean, g.se, o.mean, o.se, 16)
    assert ok, info
    rel = np.abs(g.mean - o.mean) / np.maximum(np.abs(o.mean), 1e-3)
    assert np.median(rel) < 1e-3, np.median(rel)


def test_wavefront_arguments(m, ctx, blobs):
    sp, sc = blobs
    cam = scenes.nadir_camera(sp, 8, 8)
    bad = [({"schedule": 2}, m.MCRT_ERR_ARG),
           ({"schedule": 1, "wavefront_slots": -1}, m.MCRT_ERR_ARG),
           ({"schedule": 1, "wavefront_slots": (1 << 26) + 1}, m.MCRT_ERR_ARG),
           ({"schedule": 1, "count_events": 1}, m.MCRT_ERR_UNSUPPORTED),
           ({"schedule": 1, "sun_mode": 2}, m.MCRT_ERR_UNSUPPORTED),
           ({"schedule": 1, "shard_count": 2, "shard_index": 0}, m.MCRT_ERR_UNSUPPORTED),
           ({"schedule": 1, "deadline_ms": 1000.0}, m.MCRT_ERR_UNSUPPORTED)]
    for kw, status in bad:
        with pytest.raises(m.McrtError) as e:
            sc.trace_camera(cam, 4, seed=1, **kw)
        assert e.value.status == status, kw
    with pytest.raises(m.McrtError) as e:
        sc.trace_flux(1000, seed=1, schedule=1)
    assert e.value.status == m.MCRT_ERR_UNSUPPORTED
