"""Helpers shared by the GPU parity tests: the oracle's scene and camera
from a scene spec, and the statistical comparisons."""
import math

import numpy as np


def oscene(orc, sp, **kw):
    a = dict(k=sp.k, dx=sp.dx, dy=sp.dy, dz=sp.dz, levels=sp.levels, k_clear=sp.k_clear, ssa_clear=sp.ssa_clear,
             ssa_cloud=sp.ssa_cloud, g=sp.g, ground_albedo=sp.ground_albedo, sun_zenith_deg=sp.sun_zenith_deg,
             sun_azimuth_deg=sp.sun_azimuth_deg)
    a.update(kw)
    return orc.Scene(**a)


def ocam(orc, cam):
    return orc.Camera(cam.pos, cam.target, cam.up, cam.fov_deg, cam.width, cam.height)


def close_4se(a, sa, b, sb):
    return abs(a - b) <= 4.0 * math.hypot(sa, sb) + 1e-12


def _block(a, b=8):
    h, w = a.shape
    return a.reshape(h // b, b, w // b, b).sum(axis=(1, 3))


def image_parity(g_mean, g_se, o_mean, o_se, spp):
    """Block sums (8x8 pixels) and the image mean within 4 combined SE; at most
    max(1, 3x the normal expectation) violating blocks."""
    gm, om = _block(g_mean), _block(o_mean)
    gs, os_ = np.sqrt(_block(g_se ** 2)), np.sqrt(_block(o_se ** 2))
    z = np.abs(gm - om) / np.maximum(np.hypot(gs, os_), 1e-300)
    nb = z.size
    allowed = max(1, int(3 * nb * 6.33e-5))
    bad = int(np.sum(z > 4.0))
    mg, mo = g_mean.mean(), o_mean.mean()
    sg = math.sqrt(np.sum(g_se ** 2)) / g_mean.size
    so = math.sqrt(np.sum(o_se ** 2)) / o_mean.size
    return bad <= allowed and close_4se(mg, sg, mo, so), (bad, allowed, mg, mo, sg, so)
