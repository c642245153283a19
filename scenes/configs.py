"""The five benchmark workloads as data: every constant of a workload in
one place, with its seed.  The scene generators in this package build the
fields; bench.py and the tests read sizes, sample counts and options from
here.

PLAIN_SMALL       plain method on the blob field: a 64 x 64 image and ground flux.
CUMULUS           plain method on the LES-like cumulus: the bench image.
REFINEMENT_SWEEP  five resolutions of the cumulus over a heightfield, FP32 and BF16.
BATCHING          96 uneven flux problems in one launch.
LEARNED_PROPOSAL  the learned scattering proposal on the cumulus field.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import scenes


@dataclass(frozen=True)
class ImageConfig:
    width: int
    height: int
    spp: int
    seed: int = 0


@dataclass(frozen=True)
class PlainSmall:
    """64x64x32 voxels of 100 m, three Gaussian blobs (peak 50 km^-1)
    over clear sky 0.01 km^-1; albedo 1 in cloud, 0.9 in clear sky; HG
    g 0.85; Lambertian ground 0.2; sun zenith 30 deg; 2-level pyramid."""
    field_seed: int = 0
    image: ImageConfig = ImageConfig(64, 64, 16)
    flux_paths: int = 100_000
    seed: int = 0

    def scene(self):
        return scenes.blobs_small(self.field_seed)


@dataclass(frozen=True)
class Cumulus:
    """512x512x160 voxels of 25 m (20 % cover, spectral slope -5/3,
    base 800 m, log-normal LWC median 0.3 g/m^3, r_eff 10 um); albedo 0.999
    in cloud; HG g 0.86; ground 0.1; sun zenith 60 deg; 3-level pyramid;
    a 1024 x 1024 nadir image at 64 paths per pixel."""
    nx: int = 512
    nz: int = 160
    field_seed: int = 0
    image: ImageConfig = ImageConfig(1024, 1024, 64)

    def scene(self, device=None):
        return scenes.cumulus(self.nx, self.nx, self.nz, seed=self.field_seed, device=device)

    def camera(self, spec):
        return scenes.nadir_camera(spec, self.image.width, self.image.height)


@dataclass(frozen=True)
class RefinementSweep:
    """The cumulus statistics at five resolutions of the same 12.8 km
    domain, over a 4096 x 4096 fractal heightfield (0-300 m relief), 1e8
    flux paths per point, FP32 and BF16 storage, sun zenith 60 deg."""
    sizes: tuple = ((128, 40), (256, 80), (512, 160), (1024, 320), (2048, 640))
    heightfield_n: int = 4096
    relief_km: float = 0.3
    heightfield_seed: int = 0
    paths: int = 100_000_000
    sun_zenith_deg: float = 60.0

    def heightfield(self):
        return scenes.heightfield(self.heightfield_n, self.relief_km, seed=self.heightfield_seed)


@dataclass(frozen=True)
class Batching:
    """96 instances, fields from 64^2x32 to 1024^2x160, 1-16 bands with
    log-normal gas absorption (median 1e-3 km^-1, sigma_ln 2), sun zenith
    uniform in [0, 75] deg, 1e5-1e7 paths each; tallies T_dir, T_dif and
    dT/dg; launch shapes from the autotuner."""
    instances: int = 96
    seed: int = 0
    paths_lo: float = 1e5
    paths_hi: float = 1e7

    def instance_list(self):
        return scenes.batch_instances(self.seed, n=self.instances, paths_lo=self.paths_lo, paths_hi=self.paths_hi)


@dataclass(frozen=True)
class LearnedProposal:
    """The cumulus field; MLP 9 -> 64 -> 64 -> 64 -> 40 (GELU), an 8-lobe vMF
    mixture MIS-mixed with HG at alpha 0.5; online Adam (lr 1e-3, 2^20
    vertices per step); 1/(variance x time) for the ground flux and a
    512 x 512 image at sun zenith 60 deg, against plain HG."""
    field: Cumulus = field(default_factory=Cumulus)
    mis_alpha: float = 0.5
    learning_rate: float = 1e-3
    vertices_per_step: int = 1 << 20
    image: ImageConfig = ImageConfig(512, 512, 16)
    flux_paths: int = 1 << 24


PLAIN_SMALL = PlainSmall()
CUMULUS = Cumulus()
REFINEMENT_SWEEP = RefinementSweep()
BATCHING = Batching()
LEARNED_PROPOSAL = LearnedProposal()
