"""Pins of the oracle's derived quantities (CPU only): von Mises strain (Sec. 8),
Rodrigues-Frank vectors of fundamental-zone orientations (Sec. 7) and the
per-structure RMSD histogram (Sec. 5.1)."""
import math

import numpy as np

import oracle as O
from paper_1603_05143_gb300 import inputs as I


def test_von_mises_closed_forms():
    assert O.von_mises(np.eye(3)) == 0
    assert abs(O.von_mises(2.7 * np.eye(3))) < 1e-12          # hydrostatic: no shear
    for e in (1e-3, 0.02, 0.1):
        P = np.diag([1 + e, 1 - e, 1.0])                      # pure shear
        assert abs(O.von_mises(P) - math.sqrt(3) * e) < 1e-12
    assert O.von_mises(np.zeros((3, 3))) == 0


def test_von_mises_component_form_and_rotation_invariance():
    """Equals the component form sqrt(((P11-P22)^2 + (P22-P33)^2 + (P33-P11)^2)/2
    + 3 (P12^2 + P23^2 + P31^2)) for symmetric P, and is invariant under rotation."""
    rng = I.rng_for(11)
    for _ in range(50):
        A = rng.normal(0, 0.05, (3, 3))
        P = np.eye(3) + 0.5 * (A + A.T)
        comp = math.sqrt(0.5 * ((P[0, 0] - P[1, 1]) ** 2 + (P[1, 1] - P[2, 2]) ** 2 + (P[2, 2] - P[0, 0]) ** 2)
                         + 3 * (P[0, 1] ** 2 + P[1, 2] ** 2 + P[2, 0] ** 2))
        assert abs(O.von_mises(P) - comp) < 1e-12
        R = I.random_rotation(rng)
        assert abs(O.von_mises(R @ P @ R.T) - comp) < 1e-12
    stack = np.stack([np.eye(3), np.diag([1.1, 0.9, 1.0])])
    assert np.allclose(O.von_mises(stack), [0.0, math.sqrt(3) * 0.1])


def test_rodrigues_axis_angle():
    rng = I.rng_for(12)
    for _ in range(20):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        th = rng.uniform(0, 3)
        q = np.concatenate([[math.cos(th / 2)], n * math.sin(th / 2)])
        assert np.allclose(O.rodrigues(q), n * math.tan(th / 2), atol=1e-12)


def test_rodrigues_of_cubic_fundamental_zone_lies_in_truncated_octahedron():
    """The oracle's fundamental-zone orientations of randomly rotated cubic
    lattices (FCC, BCC, SC) map into the cubic fundamental zone of
    Rodrigues-Frank space, the truncated octahedron |r_i| <= sqrt(2) - 1,
    |r_1| + |r_2| + |r_3| <= 1."""
    rng = I.rng_for(13)
    for kind, a, S in (("fcc", I.A_FCC_CU, O.FCC), ("bcc", I.A_BCC_FE, O.BCC), ("sc", I.A_SC, O.SC)):
        for _ in range(12):
            f = I.crystal(kind, a, 4, rotation=I.random_rotation(rng), dtype=np.float64)
            r = O.classify_frame(f, atoms=np.arange(3))
            assert np.all(r["structure"] == S)
            rf = O.rodrigues(r["quat"])
            assert np.all(np.abs(rf) <= math.sqrt(2) - 1 + 1e-9)
            assert np.all(np.abs(rf).sum(axis=1) <= 1 + 1e-9)


def test_rmsd_histogram_counts():
    rng = I.rng_for(14)
    n = 5000
    structure = rng.integers(0, 6, n).astype(np.int8)
    rmsd = rng.uniform(0, 0.3, n).astype(np.float32)
    rmsd[structure == 0] = np.inf
    nbins, rmax = 20, 0.25
    # keep values off the bin edges so numpy's own binning must agree
    edges = np.arange(nbins + 1) * (rmax / nbins)
    keep = np.min(np.abs(rmsd[:, None] - edges[None, :]), axis=1) > 1e-4
    structure, rmsd = structure[keep], rmsd[keep]
    h = O.rmsd_histogram(structure, rmsd, nbins, rmax)
    for S in range(1, 6):
        v = rmsd[structure == S]
        ref, _ = np.histogram(v[v < rmax], bins=nbins, range=(0, rmax))
        assert np.array_equal(h[S - 1, :nbins], ref)
        assert h[S - 1, nbins] == np.sum(v >= rmax)
    assert h.sum() == np.sum(structure > 0)
