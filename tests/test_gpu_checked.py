"""The bounds-checked build (-DMCRT_CHECKED) run over every trace kernel
variant on small cases: camera and flux, FP32 and BF16, pyramid and
octree, ratio / delta / decomposition tracking, Rayleigh clear air, a
heightfield, batches, event counting, the learned proposal and the
no-allocation entry point.  No voxel, leaf-map, tally or heightfield index
may fall outside its array (violations are counted on the device, never
followed).  This stands in for compute-sanitizer, closed on this pool."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

_CHILD = r'''
import json, sys
sys.path.insert(0, {root!r})
import numpy as np, torch, scenes
import paper_1902_01137_gb300 as m
ctx = m.Context(0)
out = {{}}
sp = scenes.blobs_small(0)
cam = scenes.nadir_camera(sp, 21, 13)
for storage in (m.MCRT_STORAGE_F32, m.MCRT_STORAGE_BF16):
    sc = m.Scene.from_spec(ctx, sp, storage=storage)
    sc.build_octree()
    for grid, fin in ((m.MCRT_GRID_PYRAMID, 0), (m.MCRT_GRID_PYRAMID, 1), (m.MCRT_GRID_OCTREE, 0),
                      (m.MCRT_GRID_OCTREE, 1)):
        for tau in (0.0, 1.0, float("inf")):
            if fin == 1 and tau == 0.0:
                continue
            kw = dict(grid=grid, finest_level=fin, tau_merge=tau)
            sc.trace_camera(cam, 4, seed=1, **kw)
            for mode in (0, 1, 2):
                sc.trace_flux(3000, seed=2, sun_mode=mode, **kw)
            sc.trace_flux(2000, seed=3, count_events=1, **kw)
    m.mcrt_scene_set_clear_sky_phase(ctx.h, sc.h, m.MCRT_PHASE_RAYLEIGH)
    sc.trace_flux(3000, seed=4)
    sc.trace_camera(cam, 4, seed=5, grid=m.MCRT_GRID_OCTREE)
    m.mcrt_scene_set_clear_sky_phase(ctx.h, sc.h, m.MCRT_PHASE_HG)
    m.trace_batch(ctx, [(sc, 0.0, 20.0, 0.0, 3000, 6), (sc, 0.05, 70.0, 90.0, 1000, 7)], batch_dalpha=1)
    m.trace_batch(ctx, [(sc, 0.0, 20.0, 0.0, 3000, 6)], grid=m.MCRT_GRID_OCTREE, finest_level=1)
    prop = m.Proposal(ctx, seed=3)
    sc.trace_flux(6000, seed=8, proposal=prop, learn=1, batch_paths=2000)
    sc.trace_camera(cam, 8, seed=9, proposal=prop, batch_paths=1024)
    prop.close()
    sc.set_heightfield(scenes.heightfield(128, 0.3, seed=1)[:96, :], sp.ground_albedo)
    for grid in (m.MCRT_GRID_PYRAMID, m.MCRT_GRID_OCTREE):
        sc.trace_flux(3000, seed=10, grid=grid)
        sc.trace_camera(cam, 4, seed=11, grid=grid)
    sc.close()
chk, n, code = m.mcrt_debug_bounds_violations(ctx.h)
out.update(checked=chk, violations=n, first_code=code)
print("RESULT " + json.dumps(out))
'''


def test_checked_build_finds_no_out_of_range_index(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_01137_gb300 import build
    lib = build.build(checked=True)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "child.py"
    script.write_text(_CHILD.format(root=root))
    env = dict(os.environ, MCRT_LIBRARY=lib)
    r = subprocess.run([sys.executable, str(script)], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [l for l in r.stdout.splitlines() if l.startswith("RESULT ")][-1]
    res = json.loads(line[7:])
    assert res["checked"] is True, res
    assert res["violations"] == 0, res


def test_normal_build_reports_unchecked():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1902_01137_gb300 as m
    from paper_1902_01137_gb300 import build
    build.build()
    with m.Context(0) as ctx:
        assert m.mcrt_debug_bounds_violations(ctx.h) == (False, 0, 0)
