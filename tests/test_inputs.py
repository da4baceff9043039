"""Seeded workload generators: sizes, structure and determinism (CPU only)."""
import numpy as np
import pytest

from paper_1603_05143_gb300 import inputs as I


def _periodic_min_dist(p, box):
    from scipy.spatial import cKDTree
    d, _ = cKDTree(p, boxsize=box).query(p, k=2)
    return d[:, 1].min()


def test_mixed_phase_exact_count_species_and_repeatable():
    f = I.config_mixed_phase(n_target=1 << 14)
    g = I.config_mixed_phase(n_target=1 << 14)
    assert f.n == 1 << 14 and f.positions.dtype == np.float32
    assert np.array_equal(f.positions, g.positions) and np.array_equal(f.species, g.species)
    assert f.species.dtype == np.int8 and set(np.unique(f.species)) <= {0, 1}
    L = np.diag(f.cell)
    assert np.all(f.positions >= 0) and np.all(f.positions < L)
    # the only minority species are the Au of the L1_2 slab (third fifth along x)
    x = f.positions[f.species == 1, 0] / (L[0] / 5)
    assert np.all((x > 1.9) & (x < 3.1))


def test_mixed_phase_noise_free_slabs_are_seam_free_and_liquid_spaced():
    """Without noise: each crystal slab is an exact lattice across the periodic
    y and z boundaries (all its interior atoms see the ideal nearest-neighbour
    distance), and liquid points keep the 2.0 A minimum distance."""
    f = I.config_mixed_phase(n_target=1 << 15, sigma=0.0)
    L = np.diag(f.cell)
    t = L[0] / 5
    from scipy.spatial import cKDTree
    tree = cKDTree(f.positions.astype(np.float64), boxsize=L)
    nn = {0: I.A_BCC_FE * np.sqrt(3) / 2, 1: I.A_FCC_CU / np.sqrt(2), 2: I.A_L12 / np.sqrt(2), 3: I.A_SC}
    for s, d0 in nn.items():
        x = f.positions[:, 0]
        inner = (x > s * t + 4) & (x < (s + 1) * t - 4)
        d, _ = tree.query(f.positions[inner].astype(np.float64), k=2)
        # lattice constant rescaled to fit Ly: within 3 % at this size
        assert np.allclose(d[:, 1], d[:, 1].mean(), rtol=0, atol=1e-4), s
        assert abs(d[:, 1].mean() / d0 - 1) < 0.03, s
    liq = f.positions[f.positions[:, 0] > 4 * t + 0.5].astype(np.float64)
    assert _periodic_min_dist(liq, [1e9, L[1], L[2]]) >= 2.0 - 1e-4
    assert 0.045 < f.meta["liquid_density"] < 0.065


def test_rsa_liquid_reaches_target_and_spacing():
    rng = I.rng_for(3)
    p = I._rsa_liquid(rng, (0.0, 30.0), 30.0, 1500, 2.0, 0.01)
    assert len(p) == 1500
    assert _periodic_min_dist(p, [1e9, 30.0, 30.0]) >= 2.0 - 1e-9


@pytest.mark.parametrize("n", [1 << 14])
def test_polycrystal_count_and_range(n):
    f = I.config_polycrystal(n_target=n)
    L = np.diag(f.cell)
    assert abs(f.n - n) <= 0.02 * n
    assert np.all(f.positions >= 0) and np.all(f.positions < L)
