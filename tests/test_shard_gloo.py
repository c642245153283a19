"""Multi-process path sharding on CPU (world size 2, gloo).

Each rank traces a contiguous path-id range (the CPU oracle stands in for
a rank's GPU on this machine) and the per-rank FP64 sums are reduced in
rank order.  The reduced sums equal one process's sums to FP64 rounding,
are bit-identical on both ranks and from run to run, and independent
replicas (distinct seeds) combine to an estimate consistent with a single
run.  The max-over-ranks step time is the largest rank's.
"""
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _scene():
    import oracle
    import scenes
    sp = scenes.blobs_small(0)
    return oracle.Scene(k=sp.k, dx=sp.dx, dy=sp.dy, dz=sp.dz, levels=sp.levels, k_clear=sp.k_clear,
                        ssa_clear=sp.ssa_clear, ssa_cloud=sp.ssa_cloud, g=sp.g, ground_albedo=sp.ground_albedo,
                        sun_zenith_deg=sp.sun_zenith_deg)


def _worker(rank, world, port, total, out_dir):
    import torch.distributed as dist
    import oracle
    from paper_1902_01137_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        S = _scene()
        b, e = shard.shard_range(total, rank, world, align=1024)
        t, _ = oracle.trace_flux(S, e - b, seed=5, begin=b, nthreads=2)
        r1 = shard.reduce_sums([t.s1, t.s2, t.n[:1]])
        r2 = shard.reduce_sums([t.s1, t.s2, t.n[:1]])
        # independent replicas: own seed, own paths
        rt, _ = oracle.trace_flux(S, 4096, seed=shard.replica_seed(77, rank), nthreads=2)
        rep = shard.reduce_sums([rt.s1, rt.s2, rt.n[:1]])
        mx = shard.max_over_ranks(10.0 + rank)
        np.savez(os.path.join(out_dir, "r%d.npz" % rank), s1=r1[0], s2=r1[1], n=r1[2], s1b=r2[0], s2b=r2[1],
                 rs1=rep[0], rs2=rep[1], rn=rep[2], mx=mx, b=b, e=e)
    finally:
        dist.destroy_process_group()


def _image_worker(rank, world, port, out_dir):
    """One image split by pixels over the ranks (the bench's multi-GPU step),
    the CPU oracle tracing each rank's shard, combined by shard.combine_image."""
    import torch.distributed as dist
    import oracle
    import scenes
    from paper_1902_01137_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        S = _scene()
        sp = scenes.blobs_small(0)
        cam = scenes.nadir_camera(sp, 12, 10)
        oc = oracle.Camera(cam.pos, cam.target, cam.up, cam.fov_deg, 12, 10)
        px = shard.image_shard_pixels(120, rank, world)
        t, _ = oracle.trace_camera(S, oc, 8, seed=9, pixels=px, nthreads=2)
        s1, s2, mean, se = shard.combine_image(t.s1.ravel(), t.s2.ravel(), 8)
        np.savez(os.path.join(out_dir, "img%d.npz" % rank), s1=s1, s2=s2, mean=mean, se=se, px=px)
    finally:
        dist.destroy_process_group()


def _records(n, seed):
    r = np.random.default_rng(seed)
    x = np.concatenate([r.uniform(-1, 1, (n, 3)), r.normal(size=(n, 3)), r.uniform(-8, 6, (n, 3))], axis=1)
    d = r.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return x, d, r.exponential(size=n)


def _dp_worker(rank, world, port, out_dir):
    """Data-parallel training step of the proposal network: each rank takes
    the gradient of its own records (the oracle's FP64 gradient stands in
    for the GPU kernel here), the ranks average them by record count, and
    each applies the same Adam step."""
    import torch.distributed as dist
    import oracle
    from paper_1902_01137_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        x, d, t = _records(1200, 3)
        lo, hi = (0, 700) if rank == 0 else (700, 1200)       # uneven shares
        p = oracle.xavier_init(5)
        _, g = oracle.mlp_loss_grad(p, x[lo:hi], d[lo:hi], t[lo:hi])
        avg = shard.average_gradient(g, hi - lo)
        pp, m, v = p.copy(), np.zeros_like(p), np.zeros_like(p)
        oracle.adam_step(pp, m, v, avg.astype(np.float64), 1, lr=1e-3)
        np.savez(os.path.join(out_dir, "dp%d.npz" % rank), avg=avg, params=pp)
    finally:
        dist.destroy_process_group()


def test_shard_ranges_cover_and_align():
    from paper_1902_01137_gb300 import shard
    for total in (0, 1, 1023, 1024, 5000, 10 ** 6 + 7):
        for world in (1, 2, 3, 8):
            rs = [shard.shard_range(total, r, world, align=64) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == total
            for (b0, e0), (b1, e1) in zip(rs, rs[1:]):
                assert e0 == b1 and b0 <= e0 and e0 % 64 == 0
    assert len({shard.replica_seed(1, r) for r in range(64)}) == 64
    with pytest.raises(ValueError):
        shard.shard_range(10, 2, 2)


def test_two_ranks_gloo_match_one_process(tmp_path):
    import torch.multiprocessing as mp
    import oracle
    from paper_1902_01137_gb300 import shard
    total = 6000
    port = 29500 + (os.getpid() % 1000)
    mp.start_processes(_worker, args=(2, port, total, str(tmp_path)), nprocs=2, start_method="spawn")
    a = np.load(tmp_path / "r0.npz")
    b = np.load(tmp_path / "r1.npz")
    for k in ("s1", "s2", "n", "rs1", "rs2", "rn", "mx"):
        assert np.array_equal(a[k], b[k]), k                   # identical result on both ranks
    assert np.array_equal(a["s1"], a["s1b"]) and np.array_equal(a["s2"], a["s2b"])   # deterministic
    one, _ = oracle.trace_flux(_scene(), total, seed=5, nthreads=2)
    np.testing.assert_allclose(a["s1"], one.s1, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(a["s2"], one.s2, rtol=1e-12, atol=1e-12)
    assert float(a["n"][0]) == total
    assert float(a["mx"]) == 11.0                               # max over ranks
    assert (int(a["b"]), int(a["e"]), int(b["b"]), int(b["e"])) == (0, 3072, 3072, total)
    # replicas combine to a consistent estimate
    m, se = shard.mean_se(a["rs1"], a["rs2"], a["rn"][0])
    for q in range(3):
        assert abs(m[q] - one.mean[q]) <= 4 * math.hypot(se[q], one.se[q])


def test_image_split_over_two_ranks_equals_one_process(tmp_path):
    """A 2-rank pixel split of one image, combined in rank order, gives the
    one-process image's sums bit for bit (each pixel's sums come from one
    rank, the other adds exact zeros), on both ranks."""
    import torch.multiprocessing as mp
    import oracle
    import scenes
    port = 30600 + (os.getpid() % 1000)
    mp.start_processes(_image_worker, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn")
    a = np.load(tmp_path / "img0.npz")
    b = np.load(tmp_path / "img1.npz")
    for k in ("s1", "s2", "mean", "se"):
        assert np.array_equal(a[k], b[k]), k
    assert sorted(np.concatenate([a["px"], b["px"]]).tolist()) == list(range(120))
    sp = scenes.blobs_small(0)
    cam = scenes.nadir_camera(sp, 12, 10)
    one, _ = oracle.trace_camera(_scene(), oracle.Camera(cam.pos, cam.target, cam.up, cam.fov_deg, 12, 10), 8,
                                 seed=9, nthreads=2)
    assert np.array_equal(a["s1"], one.s1.ravel()) and np.array_equal(a["s2"], one.s2.ravel())
    np.testing.assert_array_equal(a["mean"], one.mean.ravel())
    assert a["mean"].max() > 0.0


def test_data_parallel_training_step_gloo(tmp_path):
    """Two ranks with 700 and 500 records: the count-weighted gradient
    average equals the gradient of the mean loss over all 1,200 records,
    and both ranks end the Adam step with identical parameters."""
    import torch.multiprocessing as mp
    import oracle
    port = 30500 + (os.getpid() % 1000)
    mp.start_processes(_dp_worker, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn")
    a = np.load(tmp_path / "dp0.npz")
    b = np.load(tmp_path / "dp1.npz")
    assert np.array_equal(a["avg"], b["avg"]) and np.array_equal(a["params"], b["params"])
    x, d, t = _records(1200, 3)
    _, g_all = oracle.mlp_loss_grad(oracle.xavier_init(5), x, d, t)
    scale = np.abs(g_all).max()
    np.testing.assert_allclose(a["avg"], g_all, rtol=1e-6, atol=1e-7 * scale)


_DYING = r'''
import os, sys, time, json
from datetime import timedelta
sys.path.insert(0, {root!r})
import numpy as np
import torch.distributed as dist
from paper_1902_01137_gb300 import shard
rank = int(sys.argv[1])
os.environ["MASTER_ADDR"] = "127.0.0.1"
os.environ["MASTER_PORT"] = {port!r}
dist.init_process_group("gloo", rank=rank, world_size=2, timeout=timedelta(seconds=4))
shard.reduce_sums([np.ones(3)])                # one step together
if rank == 1:
    os._exit(0)                                # this rank leaves between steps
t0 = time.time()
try:
    shard.reduce_sums([np.ones(3)])
    out = "returned"
except Exception as e:                         # the survivor learns of it
    out = "raised " + type(e).__name__
with open({res!r}, "w") as f:
    json.dump({{"result": out, "seconds": time.time() - t0}}, f)
os._exit(0)
'''


def test_rank_leaving_is_detected_not_hung(tmp_path):
    """A rank that exits between steps: the other rank's next reduction
    ends with an error within the process group's timeout (4 s here)."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    port = str(31500 + (os.getpid() % 1000))
    res = str(tmp_path / "survivor.json")
    script = tmp_path / "dying.py"
    script.write_text(_DYING.format(root=root, port=port, res=res))
    procs = [subprocess.Popen([sys.executable, str(script), str(r)]) for r in (0, 1)]
    try:
        for p in procs:
            p.wait(timeout=90)
    finally:
        for p in procs:
            if p.poll() is None:
                p.kill()                                 # our own child, by handle
    with open(res) as f:
        out = json.load(f)
    assert out["result"].startswith("raised"), out
    assert out["seconds"] < 60, out
