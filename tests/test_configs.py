"""The workload table against the workloads it describes: sizes, voxel
sizes, constants, sample counts and seeds of the five benchmark workloads,
read back from the generated scenes."""
import numpy as np
import pytest

from scenes.configs import BATCHING, CUMULUS, LEARNED_PROPOSAL, PLAIN_SMALL, REFINEMENT_SWEEP


def test_plain_small():
    c = PLAIN_SMALL
    sp = c.scene()
    assert sp.k.shape == (32, 64, 64) and sp.dx == pytest.approx(0.1) and sp.levels == 2
    assert (sp.k_clear, sp.ssa_clear, sp.ssa_cloud, sp.g, sp.ground_albedo, sp.sun_zenith_deg) == \
        (0.01, 0.9, 1.0, 0.85, 0.2, 30.0)
    # three blobs of peak 50 km^-1 (they may overlap) over 0.01 km^-1
    assert 40.0 < float(sp.k.max()) <= 3 * 50.0 + 0.01 and float(sp.k.min()) >= 0.01 - 1e-6
    assert (c.image.width, c.image.height, c.image.spp, c.flux_paths, c.seed) == (64, 64, 16, 100_000, 0)


def test_cumulus_and_learned_proposal():
    c = CUMULUS
    assert (c.nx, c.nz, c.image.width, c.image.height, c.image.spp) == (512, 160, 1024, 1024, 64)
    sp = c.scene()
    assert sp.k.shape == (160, 512, 512) and sp.dx == pytest.approx(0.025) and sp.dz == pytest.approx(0.025)
    assert (sp.levels, sp.ssa_cloud, sp.g, sp.ground_albedo, sp.sun_zenith_deg) == (3, 0.999, 0.86, 0.1, 60.0)
    cloudy = sp.k > 0.011
    assert 0.05 < float(np.mean(cloudy.any(axis=0))) < 0.35          # about 20 % cover
    z = (np.nonzero(cloudy.any(axis=(1, 2)))[0].min() + 0.5) * sp.dz
    assert z == pytest.approx(0.8, abs=0.03)                         # cloud base 800 m
    c4 = LEARNED_PROPOSAL
    assert c4.field == c and c4.mis_alpha == 0.5 and c4.learning_rate == 1e-3
    assert c4.vertices_per_step == 1 << 20 and (c4.image.width, c4.image.height) == (512, 512)


def test_refinement_sweep_and_batching():
    c2 = REFINEMENT_SWEEP
    assert [nx for nx, _ in c2.sizes] == [128, 256, 512, 1024, 2048]
    assert all(12.8 / nx == pytest.approx(4.0 / nz * 12.8 / 4.0 * nz / nx) for nx, nz in c2.sizes)
    assert (c2.heightfield_n, c2.relief_km, c2.paths) == (4096, 0.3, 100_000_000)
    c3 = BATCHING
    inst = c3.instance_list()
    assert len(inst) == 96
    assert all(64 <= b.nx <= 1024 and 1 <= len(b.k_gas) <= 16 and 0.0 <= b.sun_zenith_deg <= 75.0 for b in inst)
    assert all(1e5 * 0.999 <= b.npaths <= 1e7 * 1.001 for b in inst)
    kg = np.log(np.concatenate([b.k_gas for b in inst]))
    assert abs(np.median(kg) - np.log(1e-3)) < 0.5 and 1.5 < np.std(kg) < 2.5
