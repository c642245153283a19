"""Checkpoint and resume of segmented runs (CPU: the oracle traces each
segment).  A run stopped after any segment and resumed from its
checkpoint file ends with exactly the sums of the uninterrupted run; the
file is replaced atomically; distinct segments draw distinct seeds."""
import os

import numpy as np
import pytest

import scenes


def _scene(orc):
    sp = scenes.blobs_small(0)
    return orc.Scene(k=sp.k, dx=sp.dx, dy=sp.dy, dz=sp.dz, levels=sp.levels, k_clear=sp.k_clear,
                     ssa_clear=sp.ssa_clear, ssa_cloud=sp.ssa_cloud, g=sp.g, ground_albedo=sp.ground_albedo,
                     sun_zenith_deg=sp.sun_zenith_deg)


def _segment(orc, S, acc, n=3000):
    t, _ = orc.trace_flux(S, n, seed=acc.next_seed(), nthreads=2)
    acc.add(t.s1[:3], t.s2[:3], t.n[:3])


def test_resumed_run_equals_uninterrupted(orc, tmp_path):
    from paper_1902_01137_gb300.checkpoint import Accumulator
    S = _scene(orc)
    full = Accumulator((3,), seed=41)
    for _ in range(6):
        _segment(orc, S, full)
    part = Accumulator((3,), seed=41)
    for _ in range(3):
        _segment(orc, S, part)
    path = str(tmp_path / "run.ckpt")
    part.save(path)
    assert not os.path.exists(path + ".tmp")
    del part
    resumed = Accumulator.load(path)
    assert resumed.next_segment == 3 and resumed.seed == 41
    for _ in range(3):
        _segment(orc, S, resumed)
    assert np.array_equal(resumed.s1, full.s1) and np.array_equal(resumed.s2, full.s2)
    assert np.array_equal(resumed.n, full.n) and float(full.n[0]) == 18000
    m, se = resumed.mean_se()
    assert np.all(np.isfinite(m)) and np.all(se > 0)
    with pytest.raises(ValueError):
        Accumulator.load(path, proposal=object())          # no network state in this file


def test_segment_seeds_are_distinct():
    from paper_1902_01137_gb300.checkpoint import segment_seed
    seeds = {segment_seed(s, k) for s in (0, 1, 2 ** 63) for k in range(1000)}
    assert len(seeds) == 3000
    assert all(0 <= v < 2 ** 64 for v in seeds)
