"""Seeded synthetic scene generators (inputs only).

These build the extinction fields, optical constants, sun and camera poses
of the workloads.  They hold none of the method's arithmetic (no majorants,
no traversal, no estimator), so both the CUDA path and the CPU oracle may
read their output.  Random draws use numpy's Philox bit generator with an
explicit seed.

The paper's LES fields (Meso-NH congestus, BOMEX, ARMCu, FIRE; Sec. 4.3 and
App. B) are not available, so seeded fields with the same shapes, voxel
sizes and value ranges stand in for them:

* ``blobs_small``: 64x64x32 voxels of 100 m, three Gaussian blobs (peak
  50 km^-1, horizontal sigma 0.4-0.8 km, vertical sigma 0.3 km, centre
  height 1-2 km) over a uniform clear sky of 0.01 km^-1.
* ``cumulus``: 512x512x160 voxels of 25 m (12.8 x 12.8 x 4 km) shaped like
  a shallow-cumulus LES: 20 % cover from a band-limited Gaussian field with
  a k^-5/3 one-dimensional spectrum thresholded at its 80th percentile,
  cloud base 0.8 km, tops up to 2.8 km, log-normal liquid water content
  (median 0.3 g m^-3, sigma_ln 0.6) and extinction 1.5 LWC / (rho_w r_eff)
  with r_eff = 10 um, plus the clear sky.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class SceneSpec:
    """Field plus the constants a trace needs (units: km, km^-1)."""
    name: str
    k: np.ndarray            # [z][y][x] float32 total extinction
    dx: float
    dy: float
    dz: float
    levels: int              # majorant levels above the voxels
    k_clear: float
    ssa_clear: float
    ssa_cloud: float
    g: float
    ground_albedo: float
    sun_zenith_deg: float
    sun_azimuth_deg: float = 0.0

    @property
    def shape_xyz(self):
        nz, ny, nx = self.k.shape
        return nx, ny, nz

    @property
    def extent(self):
        nx, ny, nz = self.shape_xyz
        return (np.float32(nx) * np.float32(self.dx), np.float32(ny) * np.float32(self.dy),
                np.float32(nz) * np.float32(self.dz))


@dataclass
class CameraSpec:
    pos: tuple
    target: tuple
    up: tuple
    fov_deg: float
    width: int
    height: int


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(seed))


def nadir_camera(spec: SceneSpec, width: int, height: int, height_above_top: float = 10.0) -> CameraSpec:
    """Pinhole camera above the domain centre looking straight down; the
    field of view makes the image footprint at the ground the domain width."""
    Lx, Ly, Lz = (float(v) for v in spec.extent)
    z = Lz + height_above_top
    fov = 2.0 * math.degrees(math.atan((0.5 * Lx) / z))
    return CameraSpec(pos=(0.5 * Lx, 0.5 * Ly, z), target=(0.5 * Lx, 0.5 * Ly, 0.0), up=(0.0, 1.0, 0.0),
                      fov_deg=fov, width=width, height=height)


def blobs_small(seed: int = 0) -> SceneSpec:
    """64x64x32 voxels of 100 m: three Gaussian blobs over clear sky."""
    nx, ny, nz = 64, 64, 32
    dx = dy = dz = 0.1
    Lx, Ly = nx * dx, ny * dy
    r = _rng(seed)
    cx = r.uniform(0.0, Lx, 3)
    cy = r.uniform(0.0, Ly, 3)
    cz = r.uniform(1.0, 2.0, 3)
    sh = r.uniform(0.4, 0.8, 3)
    sz = 0.3
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dy
    z = (np.arange(nz) + 0.5) * dz
    k = np.full((nz, ny, nx), 0.01, dtype=np.float64)
    for b in range(3):
        ddx = x - cx[b]
        ddx -= Lx * np.round(ddx / Lx)          # periodic minimum image
        ddy = y - cy[b]
        ddy -= Ly * np.round(ddy / Ly)
        ddz = z - cz[b]
        h2 = (ddx[None, None, :] ** 2 + ddy[None, :, None] ** 2) / (2.0 * sh[b] ** 2)
        v2 = ddz[:, None, None] ** 2 / (2.0 * sz ** 2)
        k += 50.0 * np.exp(-(h2 + v2))
    return SceneSpec(name="blobs-64x64x32-100m", k=k.astype(np.float32), dx=dx, dy=dy, dz=dz, levels=2,
                     k_clear=0.01, ssa_clear=0.9, ssa_cloud=1.0, g=0.85, ground_albedo=0.2,
                     sun_zenith_deg=30.0)


def _band_limited_2d(n: int, L: float, kmax: int, slope_psd: float, r: np.random.Generator) -> np.ndarray:
    """Periodic Gaussian field on an n x n grid whose Fourier coefficients are
    fixed for |k| <= kmax (cycles per domain) and zero above, so that every
    resolution samples the same continuous field."""
    ks = np.arange(-kmax, kmax + 1)
    KX, KY = np.meshgrid(ks, ks, indexing="xy")
    kk = np.sqrt(KX.astype(np.float64) ** 2 + KY ** 2)
    amp = np.where(kk > 0, np.power(np.maximum(kk, 1e-12), slope_psd / 2.0), 0.0)
    c = (r.standard_normal(KX.shape) + 1j * r.standard_normal(KX.shape)) * amp
    F = np.zeros((n, n), dtype=np.complex128)
    F[KY % n, KX % n] = c
    f = np.fft.ifft2(F).real * (n * n)
    f = (f - f.mean()) / f.std()
    return f


def _band_limited_3d(nx: int, ny: int, nz: int, kxy: int, kz: int, r: np.random.Generator) -> np.ndarray:
    """Unit-variance periodic 3D Gaussian field with a k^-11/3 spectrum,
    band-limited to |kx|,|ky| <= kxy and |kz| <= kz (cycles per domain)."""
    kxs = np.arange(-kxy, kxy + 1)
    kzs = np.arange(-kz, kz + 1)
    KZ, KY, KX = np.meshgrid(kzs, kxs, kxs, indexing="ij")
    kk = np.sqrt(KX.astype(np.float64) ** 2 + KY ** 2 + (KZ * 3.2) ** 2)
    amp = np.where(kk > 0, np.power(np.maximum(kk, 1e-12), -11.0 / 6.0), 0.0)
    c = (r.standard_normal(KX.shape) + 1j * r.standard_normal(KX.shape)) * amp
    F = np.zeros((nz, ny, nx), dtype=np.complex64)
    F[KZ % nz, KY % ny, KX % nx] = c.astype(np.complex64)
    f = np.fft.ifftn(F).real.astype(np.float64)
    f = (f - f.mean()) / f.std()
    return f.astype(np.float32)


def _band_limited_3d_coeffs(nx: int, ny: int, nz: int, kxy: int, kz: int, r: np.random.Generator):
    kxs = np.arange(-kxy, kxy + 1)
    kzs = np.arange(-kz, kz + 1)
    KZ, KY, KX = np.meshgrid(kzs, kxs, kxs, indexing="ij")
    kk = np.sqrt(KX.astype(np.float64) ** 2 + KY ** 2 + (KZ * 3.2) ** 2)
    amp = np.where(kk > 0, np.power(np.maximum(kk, 1e-12), -11.0 / 6.0), 0.0)
    c = (r.standard_normal(KX.shape) + 1j * r.standard_normal(KX.shape)) * amp
    return KZ % nz, KY % ny, KX % nx, c.astype(np.complex64)


def _band_limited_3d(nx: int, ny: int, nz: int, kxy: int, kz: int, r: np.random.Generator) -> np.ndarray:
    """Unit-variance periodic 3D Gaussian field with a k^-11/3 spectrum,
    band-limited to |kx|,|ky| <= kxy and |kz| <= kz (cycles per domain)."""
    iz, iy, ix, c = _band_limited_3d_coeffs(nx, ny, nz, kxy, kz, r)
    F = np.zeros((nz, ny, nx), dtype=np.complex64)
    F[iz, iy, ix] = c
    f = np.fft.ifftn(F).real.astype(np.float64)
    f = (f - f.mean()) / f.std()
    return f.astype(np.float32)


def cumulus(nx: int = 512, ny: int = 512, nz: int = 160, seed: int = 0, cover: float = 0.20,
            k_clear: float = 0.01, device=None) -> SceneSpec:
    """Shallow-cumulus-like field over a 12.8 x 12.8 x 4 km domain.

    With ``device`` (a torch CUDA device) the 3D part is transformed and the
    field assembled on that device and ``k`` is a device tensor: the same
    random draws, but FFT rounding differs from numpy's, so such a field is
    for timing only (parity cases use the host form)."""
    Lx, Lz = 12.8, 4.0
    dx = Lx / nx
    dz = Lz / nz
    r = _rng(seed)
    f = _band_limited_2d(nx, Lx, 48, -8.0 / 3.0, r)           # 2D PSD ~ k^-8/3
    thr = np.quantile(f, 1.0 - cover)
    fmax = f.max()
    base = 0.8
    top = np.where(f > thr, base + 2.0 * (f - thr) / (fmax - thr), base)   # [y][x]
    zc = (np.arange(nz) + 0.5) * dz
    rho_w = 1.0e6                                           # g m^-3
    r_eff = 10e-6                                           # m
    kfac = 1.5 / (rho_w * r_eff) * 1000.0                   # LWC [g m^-3] -> extinction [km^-1]
    if device is None:
        incloud = (zc[:, None, None] >= base) & (zc[:, None, None] < top[None, :, :])
        g3 = _band_limited_3d(nx, ny, nz, 24, 6, r).astype(np.float64)
        # log-normal LWC with median 0.3 g m^-3 and sigma_ln 0.6 over the cloudy voxels
        zc_ = g3[incloud]
        g3 = (g3 - np.median(zc_)) / zc_.std()
        lwc = 0.3 * np.exp(0.6 * g3)                        # g m^-3
        k = (np.where(incloud, kfac * lwc, 0.0) + k_clear).astype(np.float32)
    else:
        import torch
        iz, iy, ix, c = _band_limited_3d_coeffs(nx, ny, nz, 24, 6, r)
        F = torch.zeros((nz, ny, nx), dtype=torch.complex64, device=device)
        F[torch.from_numpy(iz).to(device), torch.from_numpy(iy).to(device), torch.from_numpy(ix).to(device)] = \
            torch.from_numpy(c).to(device)
        g3 = torch.fft.ifftn(F).real
        del F
        g3 = (g3 - g3.mean()) / g3.std()
        zt = torch.from_numpy(zc).to(device=device, dtype=torch.float32)
        tt = torch.from_numpy(top).to(device=device, dtype=torch.float32)
        incloud = (zt[:, None, None] >= base) & (zt[:, None, None] < tt[None, :, :])
        zc_ = g3[incloud]
        g3 = (g3 - zc_.median()) / zc_.std()
        k = torch.where(incloud, kfac * 0.3 * torch.exp(0.6 * g3), torch.zeros((), device=device)) + k_clear
        k = k.to(torch.float32).contiguous()
    return SceneSpec(name="cumulus-%dx%dx%d" % (nx, ny, nz), k=k, dx=dx, dy=dx, dz=dz,
                     levels=3, k_clear=k_clear, ssa_clear=0.9, ssa_cloud=0.999, g=0.86, ground_albedo=0.1,
                     sun_zenith_deg=60.0)


@dataclass
class BatchInstance:
    """One field of a batch with its sun and spectral bands."""
    nx: int
    nz: int
    field_seed: int
    sun_zenith_deg: float
    sun_azimuth_deg: float
    k_gas: list              # one gas absorption [km^-1] per band
    npaths: int              # paths of the instance, split over its bands


BATCH_SIZES = ((64, 32), (128, 40), (256, 80), (512, 160), (1024, 160))


def batch_instances(seed: int = 0, n: int = 96, max_nx: int = 1024, paths_lo: float = 1e5,
                    paths_hi: float = 1e7) -> list:
    """Many flux problems of uneven sizes: field sizes drawn uniformly from
    64^2x32 ... 1024^2x160 (cumulus statistics over the same 12.8 km domain),
    1-16 spectral bands per field with log-normal gas absorption (median
    1e-3 km^-1, sigma_ln 2), sun zenith uniform in [0, 75] deg, azimuth
    uniform, and a log-uniform path count in [paths_lo, paths_hi] per field."""
    r = _rng(seed)
    sizes = [s for s in BATCH_SIZES if s[0] <= max_nx]
    out = []
    for i in range(n):
        nx, nz = sizes[int(r.integers(0, len(sizes)))]
        nb = int(r.integers(1, 17))
        kg = list(np.exp(np.log(1e-3) + 2.0 * r.standard_normal(nb)))
        out.append(BatchInstance(nx=nx, nz=nz, field_seed=1000 + i, sun_zenith_deg=float(r.uniform(0.0, 75.0)),
                                 sun_azimuth_deg=float(r.uniform(0.0, 360.0)), k_gas=[float(v) for v in kg],
                                 npaths=int(round(math.exp(r.uniform(math.log(paths_lo), math.log(paths_hi)))))))
    return out


def batch_items(instances, scene_of) -> list:
    """Flattens instances into (scene, k_gas, zenith, azimuth, npaths, seed)
    items, one per band; ``scene_of(i)`` gives instance i's scene."""
    items = []
    for i, b in enumerate(instances):
        nb = len(b.k_gas)
        per = max(1, b.npaths // nb)
        for j, kg in enumerate(b.k_gas):
            items.append((scene_of(i), kg, b.sun_zenith_deg, b.sun_azimuth_deg, per, (i << 8) | j))
    return items


def heightfield(n: int = 4096, relief: float = 0.3, seed: int = 0, psd_slope: float = -3.2) -> np.ndarray:
    """Periodic fractal terrain: n x n heights [km] from a Gaussian field
    with a 2D power spectrum ~ k^psd_slope, rescaled to [0, relief]."""
    r = _rng(seed)
    kx = np.fft.fftfreq(n) * n
    kk = np.sqrt(kx[None, :] ** 2 + kx[:, None] ** 2)
    amp = np.where(kk > 0, np.power(np.maximum(kk, 1e-12), psd_slope / 2.0), 0.0)
    c = (r.standard_normal((n, n)) + 1j * r.standard_normal((n, n))) * amp
    f = np.fft.ifft2(c).real
    f = (f - f.min()) / (f.max() - f.min()) * relief
    return f.astype(np.float32)


# Colour bands (nm) for three-band renders: one band per eye cone class
# stands in for the paper's CIE responsivity integration (Sec. 4.1), whose
# spectra and k-distribution data are not available here.
RGB_BANDS_NM = (650.0, 550.0, 450.0)


def rayleigh_band_extinction(k_ref: float, lam_ref_nm: float = 550.0, bands_nm=RGB_BANDS_NM) -> list:
    """Clear-air (molecular) extinction per band, scaled as lambda^-4 from
    k_ref at lam_ref_nm."""
    return [k_ref * (lam_ref_nm / lam) ** 4 for lam in bands_nm]


def homogeneous(nx: int, ny: int, nz: int, d: float, k: float, **kw) -> SceneSpec:
    """Uniform field (pins: Beer's law, single scattering)."""
    levels = kw.pop("levels", 1)
    f = np.full((nz, ny, nx), k, dtype=np.float32)
    base = dict(k_clear=0.0, ssa_clear=1.0, ssa_cloud=1.0, g=0.85, ground_albedo=0.0, sun_zenith_deg=0.0)
    base.update(kw)
    return SceneSpec(name="homogeneous", k=f, dx=d, dy=d, dz=d, levels=levels, **base)


def random_voxels(nx: int, ny: int, nz: int, d: float, kmax: float, seed: int, levels: int = 1,
                  sparsity: float = 0.5, **kw) -> SceneSpec:
    """Independent random voxel values, a fraction of them zero."""
    r = _rng(seed)
    f = r.uniform(0.0, kmax, (nz, ny, nx))
    f[r.uniform(size=f.shape) < sparsity] = 0.0
    base = dict(k_clear=0.0, ssa_clear=1.0, ssa_cloud=1.0, g=0.85, ground_albedo=0.0, sun_zenith_deg=0.0)
    base.update(kw)
    return SceneSpec(name="random", k=f.astype(np.float32), dx=d, dy=d, dz=d, levels=levels, **base)


def random_rays(spec: SceneSpec, n: int, seed: int):
    """Origins inside the domain and unit directions (float32)."""
    r = _rng(seed)
    Lx, Ly, Lz = (float(v) for v in spec.extent)
    o = np.stack([r.uniform(0, Lx, n), r.uniform(0, Ly, n), r.uniform(0, Lz, n)], axis=1).astype(np.float32)
    v = r.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return o, v.astype(np.float32)
