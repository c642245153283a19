"""How much could any guide of the first scattering direction lower the
variance?  An oracle-side bound for the learned proposal (a project addition
with no counterpart in the paper), used to read the GPU's measured figure of
merit.  TEST INFRASTRUCTURE: it runs the CPU oracle only.

A path's score is S = E + F: E the estimates up to and including the first
volume vertex (not affected by how the next direction is drawn) and F what
the path scores after that vertex.  Drawing that direction from q = p_HG r
instead of p_HG (r >= 0, E_pHG[r] = 1) makes the score E + F / r, with

    Var_r = E[E^2] + 2 E[E F] + E[F^2 / r] - mean^2        (expectations under p_HG).

Over a partition of the vertex's context (position block x incoming-direction
bin) and of the outgoing direction into bins, the r that minimises Var_r
among functions constant on each (context, bin) cell is
r = sqrt(m2) / sum_b P_b sqrt(m2_b), with m2 the mean of F^2 in the cell and
P_b the HG probability of bin b (its frequency among the HG-drawn
directions).  It is fitted on half the paths and evaluated on the other
half (and, as an optimistic figure, on the same paths it was fitted on); with
the defensive share alpha of the tracer's MIS (r -> alpha + (1 - alpha) r) a
bin the fit never saw keeps a finite variance.  The result
is the relative-variance ratio plain / best guide for the ground flux T_dif
and for the pixels of a 64 x 64 nadir image (mean pixel relative variance),
on paths traced with HG sampling (mis_alpha = 1, so the network is never
used).

    python -m oracle.guide_bound [--paths N] [--field cumulus|blobs]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _dbin(d, nz, nphi):
    """Equal-area direction bin: cos theta x azimuth."""
    cz = np.clip(((d[:, 2] + 1) * 0.5 * nz).astype(int), 0, nz - 1)
    ph = np.clip(((np.arctan2(d[:, 1], d[:, 0]) + math.pi) / (2 * math.pi) * nphi).astype(int), 0, nphi - 1)
    return cz * nphi + ph


def _bins(recs, pos_blocks, in_bins, dir_bins):
    """Context index (position block x incoming-direction bin) and outgoing
    direction bin of each record."""
    x = recs["x"]
    px = np.clip(((x[:, 0] + 1) * 0.5 * pos_blocks).astype(int), 0, pos_blocks - 1)
    py = np.clip(((x[:, 1] + 1) * 0.5 * pos_blocks).astype(int), 0, pos_blocks - 1)
    ni = in_bins[0] * in_bins[1]
    ctx = (px * pos_blocks + py) * ni + _dbin(x[:, 3:6], *in_bins)
    return ctx, _dbin(recs["dir"], *dir_bins), pos_blocks * pos_blocks * ni, dir_bins[0] * dir_bins[1]


def bound(recs, scores, spp=None, pos_blocks=4, in_bins=(2, 4), dir_bins=(8, 16), alpha=0.0, seed=0,
          in_sample=False):
    """Relative-variance ratio plain / best piecewise-constant guide of the
    first learned vertex's direction (fit on one half of the paths,
    evaluated on the other).  scores: every path's score, indexed by path
    id; spp: paths per pixel of an image (the ratio is then of the mean
    pixel relative variance over pixels brighter than 1e-3 of the maximum),
    None for a single tally."""
    n = len(scores)
    first = recs[recs["vertex"] == 0]
    pid = first["path"].astype(np.int64)
    F = first["w_omega"] * first["target"]                  # score after the vertex
    E = first["before"] + first["own"]
    ctx, b, nctx, nb = _bins(first, pos_blocks, in_bins, dir_bins)
    cell = ctx * nb + b
    half = np.random.default_rng(seed).random(n) < 0.5        # path id -> fit half
    if in_sample:                                            # fit and evaluate on all paths (optimistic)
        half[:] = True
    fit = half[pid]
    ev = fit if in_sample else ~fit
    ncell = nctx * nb
    cnt = np.bincount(cell[fit], minlength=ncell).astype(float)
    m2 = np.bincount(cell[fit], weights=F[fit] ** 2, minlength=ncell) / np.maximum(cnt, 1.0)
    cctx = np.arange(ncell) // nb
    cnt_ctx = np.bincount(ctx[fit], minlength=ncell // nb).astype(float)
    P = cnt / np.maximum(cnt_ctx[cctx], 1.0)                  # HG frequency of each bin in its context
    root = np.sqrt(m2)
    norm = np.bincount(cctx, weights=P * root, minlength=ncell // nb)[cctx]
    r = np.where(norm > 0, root / np.where(norm > 0, norm, 1.0), 1.0)
    r = alpha + (1.0 - alpha) * r
    # second moments per evaluated path: plain S^2; guided E^2 + 2 E F + F^2 / r
    # where the path has a first vertex, S^2 otherwise
    S = np.asarray(scores, dtype=np.float64)
    g2 = S * S
    rr = r[cell[ev]]
    with np.errstate(divide="ignore", invalid="ignore"):
        term = E[ev] ** 2 + 2 * E[ev] * F[ev] + np.where(rr > 0, F[ev] ** 2 / rr, np.where(F[ev] > 0, np.inf, 0.0))
    g2[pid[ev]] = term
    evp = half if in_sample else ~half
    grp = (np.arange(n) // spp) if spp else np.zeros(n, np.int64)
    ng = int(grp.max()) + 1
    k = np.bincount(grp[evp], minlength=ng).astype(float)
    mu = np.bincount(grp[evp], weights=S[evp], minlength=ng) / np.maximum(k, 1.0)
    v_plain = np.bincount(grp[evp], weights=S[evp] ** 2, minlength=ng) / np.maximum(k, 1.0) - mu ** 2
    v_guided = np.bincount(grp[evp], weights=g2[evp], minlength=ng) / np.maximum(k, 1.0) - mu ** 2
    ok = (mu > 1e-3 * mu.max()) & (k > 1)
    rv_plain = float(np.mean(v_plain[ok] / mu[ok] ** 2))
    rv_guided = float(np.mean(v_guided[ok] / mu[ok] ** 2))
    return {"rel_var_plain": rv_plain, "rel_var_guided": rv_guided,
            "gain": rv_plain / rv_guided if rv_guided > 0 else float("inf"),
            "records": int(len(first)), "paths": int(n), "alpha": alpha, "in_sample": in_sample,
            "bins": {"position_blocks": pos_blocks, "incoming_direction_bins": list(in_bins),
                     "direction_bins": list(dir_bins)}}


def main(argv=None):
    import oracle
    import scenes
    from scenes.configs import CUMULUS
    ap = argparse.ArgumentParser()
    ap.add_argument("--paths", type=int, default=200000)
    ap.add_argument("--field", default="cumulus", choices=["cumulus", "blobs"])
    args = ap.parse_args(argv)
    sp = CUMULUS.scene() if args.field == "cumulus" else scenes.blobs_small(0)
    p = oracle.xavier_init(1)                                 # never used: mis_alpha = 1
    S = oracle.Scene(k=sp.k, dx=sp.dx, dy=sp.dy, dz=sp.dz, levels=sp.levels, k_clear=sp.k_clear,
                     ssa_clear=sp.ssa_clear, ssa_cloud=sp.ssa_cloud, g=sp.g, ground_albedo=sp.ground_albedo,
                     sun_zenith_deg=sp.sun_zenith_deg, mlp=p, n_learned=1, mis_alpha=1.0)
    out = {"field": args.field, "sun_zenith_deg": sp.sun_zenith_deg}
    n = args.paths
    recs, scores = oracle.learned_records(S, None, 0, seed=11, begin=0, end=n, cap=4 * n)
    out["flux_T_dif"] = {"held_out": {a: bound(recs, scores, alpha=a) for a in (0.0, 0.25, 0.5)},
                         "in_sample": bound(recs, scores, alpha=0.0, in_sample=True)}
    cam = scenes.nadir_camera(sp, 64, 64)
    spp = max(1, n // (64 * 64))
    oc = oracle.Camera(cam.pos, cam.target, cam.up, cam.fov_deg, 64, 64)
    recs, scores = oracle.learned_records(S, oc, spp, seed=12, begin=0, end=64 * 64 * spp, cap=4 * n)
    out["image_64px"] = {"held_out": {a: bound(recs, scores, spp=spp, alpha=a) for a in (0.0, 0.25, 0.5)},
                         "in_sample": bound(recs, scores, spp=spp, alpha=0.0, in_sample=True)}
    print(json.dumps(out, indent=1, default=str))
    return out


if __name__ == "__main__":
    main()
