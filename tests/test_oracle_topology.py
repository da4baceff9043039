"""Pins of the oracle's topological neighbour ordering (Sec. 3, Eq. 5), CPU only.

Voronoi face areas are checked against closed forms of the cells of the cubic
lattices, against the cell volume (sum of area x distance / 6 equals the volume
per atom) and against qhull's Voronoi diagram (scipy) on random point sets; the
ordering against its definition."""
import itertools
import math

import numpy as np
import pytest

import oracle as O
from paper_1603_05143_gb300 import inputs as I


def _shell(kind, a):
    pts = np.array([p for p in itertools.product(range(-2, 3), repeat=3) if any(p)], float)
    if kind == "fcc":
        pts = pts[(pts.sum(1) % 2 == 0)] * a / 2
    elif kind == "bcc":
        half = np.array([p for p in itertools.product((-1.5, -0.5, 0.5, 1.5), repeat=3)], float)
        pts = np.vstack([pts * a, half * a])
    else:
        pts = pts * a
    d = np.linalg.norm(pts, axis=1)
    order = np.argsort(d, kind="stable")
    return pts[order[:18]]


def test_fcc_cell_is_the_rhombic_dodecahedron():
    a = I.A_FCC_CU
    v = _shell("fcc", a)
    ar = O.voronoi_areas(v)
    assert np.allclose(ar[:12], a * a * math.sqrt(2) / 8, rtol=1e-12)
    assert np.all(ar[12:] < 1e-9 * a * a)              # second shell touches at vertices only
    vol = np.sum(ar * np.linalg.norm(v, axis=1)) / 6
    assert abs(vol - a ** 3 / 4) < 1e-9


def test_bcc_cell_is_the_truncated_octahedron():
    a = I.A_BCC_FE
    v = _shell("bcc", a)
    ar = O.voronoi_areas(v)
    d = np.linalg.norm(v, axis=1)
    hexa = ar[np.isclose(d, a * math.sqrt(3) / 2)]
    sq = ar[np.isclose(d, a)]
    assert len(hexa) == 8 and len(sq) == 6
    assert np.allclose(hexa, 3 * math.sqrt(3) * a * a / 16, rtol=1e-12)
    assert np.allclose(sq, a * a / 8, rtol=1e-12)
    assert np.all(ar[~np.isclose(d, a) & ~np.isclose(d, a * math.sqrt(3) / 2)] < 1e-9)
    assert abs(np.sum(ar * d) / 6 - a ** 3 / 2) < 1e-9


def test_sc_cell_is_the_cube():
    a = I.A_SC
    v = _shell("sc", a)
    ar = O.voronoi_areas(v)
    d = np.linalg.norm(v, axis=1)
    assert np.allclose(ar[np.isclose(d, a)], a * a, rtol=1e-12)
    assert np.all(ar[~np.isclose(d, a)] < 1e-9)


def test_areas_match_qhull_voronoi():
    scipy_spatial = pytest.importorskip("scipy.spatial")
    rng = I.rng_for(31)
    for trial in range(20):
        v = _shell(("fcc", "bcc")[trial % 2], 3.0) + rng.normal(0, 0.25, (18, 3))
        ar = O.voronoi_areas(v)
        vor = scipy_spatial.Voronoi(np.vstack([np.zeros(3), v]))
        ref = np.zeros(18)
        for (p, q), rv in zip(vor.ridge_points, vor.ridge_vertices):
            if 0 not in (p, q):
                continue
            assert -1 not in rv                          # the centre's cell is bounded
            poly = vor.vertices[rv]
            other = p + q - 1
            n = v[other] / np.linalg.norm(v[other])
            c = poly.mean(0)
            ang = np.arctan2(np.cross(poly[0] - c, poly - c) @ n, (poly - c) @ (poly[0] - c))
            poly = poly[np.argsort(ang)]
            ref[other] = 0.5 * abs(np.dot(np.sum(np.cross(poly, np.roll(poly, -1, 0)), axis=0), n))
        assert np.allclose(ar, ref, rtol=1e-9, atol=1e-9)


def test_perfect_lattice_order_is_euclidean():
    """Equal areas tie, and ties fall back to the distance order."""
    for kind, a in (("fcc", I.A_FCC_CU), ("bcc", I.A_BCC_FE), ("sc", I.A_SC)):
        f = I.crystal(kind, a, 5, rotation=I.random_rotation(I.rng_for(3)), dtype=np.float64)
        F = O.Frame(f.positions, f.cell, f.pbc)
        for atom in (0, 7, 33):
            ids, imgs, areas = F.topo_knn(atom)
            e_ids, e_imgs = F.knn(atom, 14)[:2]
            assert np.array_equal(ids, e_ids) and np.array_equal(imgs, e_imgs)


def test_order_follows_areas_then_distance():
    rng = I.rng_for(32)
    f = I.crystal("fcc", I.A_FCC_CU, 5, sigma=0.2, seed=4, dtype=np.float64)
    F = O.Frame(f.positions, f.cell, f.pbc)
    for atom in rng.choice(f.n, 30, replace=False):
        ids, imgs, areas = F.topo_knn(int(atom))
        e_ids, e_imgs, _, d2 = F.knn(int(atom), 18)
        rank = {(int(j), tuple(n)): r for r, (j, n) in enumerate(zip(e_ids, e_imgs))}
        r = [rank[(int(j), tuple(n))] for j, n in zip(ids, imgs)]
        a = areas[r]
        band = 1e-3 * np.mean(d2)
        for x, y, rx, ry in zip(a[:-1], a[1:], r[:-1], r[1:]):
            assert x >= y - band                        # areas descend (up to the tie band)
            if x == y:
                assert rx < ry                          # exact ties: nearer first
        # every atom left out has a face no larger than the last one kept
        rest = sorted(set(range(len(e_ids))) - set(r))
        assert all(areas[k] <= a[-1] + band for k in rest)


def test_topological_ordering_finds_more_fcc_when_hot():
    """Sec. 5.2: with large thermal displacements distance ordering loses fcc
    atoms that the area ordering keeps."""
    f = I.crystal("fcc", I.A_FCC_CU, 5, sigma=0.28, seed=8, dtype=np.float64)
    e = O.classify_frame(f)
    t = O.classify_frame(f, ordering="topological")
    ne, nt = np.sum(e["structure"] == O.FCC), np.sum(t["structure"] == O.FCC)
    assert nt > ne
