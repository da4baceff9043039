"""Pins for the oracle's geometric pieces: predicates, hulls, Weinberg codes.

Each test checks the oracle against something other than itself: exact rational
arithmetic, qhull (scipy), Euler's formula, symmetry counts the paper states.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_facts.json")))


# ------------------------------------------------------------- SoS predicate
def _perturbed_orient_sign(pts, prio, eps_bits=20):
    """Sign of det[b-a; c-a; d-a] for points perturbed by eps^(2^(3(r-1)+c)),
    eps = 2^-eps_bits, evaluated exactly with Python integers (all entries are
    scaled by a common power of two so no fractions appear)."""
    bmax = max(3 * (r - 1) + 2 for r in prio)
    D = 1 << (eps_bits * (1 << bmax))
    M = []
    for p, r in zip(pts, prio):
        row = [int(p[c]) * D + (1 << (eps_bits * ((1 << bmax) - (1 << (3 * (r - 1) + c)))))
               for c in range(3)]
        M.append(row)
    a, b, c, d = M
    u = [b[i] - a[i] for i in range(3)]
    v = [c[i] - a[i] for i in range(3)]
    w = [d[i] - a[i] for i in range(3)]
    det = (u[0] * (v[1] * w[2] - v[2] * w[1]) - u[1] * (v[0] * w[2] - v[2] * w[0])
           + u[2] * (v[0] * w[1] - v[1] * w[0]))
    return (det > 0) - (det < 0)


def test_sos_matches_exact_symbolic_perturbation():
    """Simulation of Simplicity (Sec. 4 coplanar facets, reading R7) equals the
    sign of an explicitly perturbed determinant with a concrete tiny epsilon."""
    rng = np.random.default_rng(7)
    cases = [
        ([0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0]),      # coplanar square
        ([0, 0, 0], [1, 0, 0], [2, 0, 0], [0, 1, 0]),      # collinear triple
        ([1, 1, 1], [1, 1, 1], [0, 1, 0], [2, 0, 1]),      # coincident points
        ([0, 0, 0], [0, 0, 0], [0, 0, 0], [0, 0, 0]),      # all equal
        ([0, 0, 1], [1, 0, 1], [0, 1, 1], [2, -1, 1]),
    ]
    for _ in range(300):
        cases.append(tuple(rng.integers(-2, 3, 3) for _ in range(4)))
    n_zero = 0
    for pts in cases:
        for prio in itertools.permutations(range(1, 6), 4):
            if rng.random() > 0.08:
                continue
            got = O.orient(*pts, prio=prio)
            assert got in (-1, 1)
            exact = O.orient_exact(*pts)
            if exact == 0:
                n_zero += 1
            assert got == _perturbed_orient_sign(pts, prio), (pts, prio)
    assert n_zero > 50


def test_sos_antisymmetric():
    rng = np.random.default_rng(3)
    for _ in range(200):
        pts = [rng.integers(-1, 2, 3) for _ in range(4)]
        prio = list(rng.permutation(np.arange(1, 15))[:4])
        s = O.orient(*pts, prio=prio)
        s2 = O.orient(pts[1], pts[0], pts[2], pts[3], prio=[prio[1], prio[0], prio[2], prio[3]])
        assert s == -s2


# ---------------------------------------------------------------------- hulls
def _check_closed_triangulated_sphere(f, k):
    f = np.asarray(f)
    assert len(f) == 2 * k - 4                      # Euler: F = 2V - 4
    directed = set()
    for a, b, c in f:
        for e in ((a, b), (b, c), (c, a)):
            assert e not in directed
            directed.add(e)
    for (a, b) in directed:
        assert (b, a) in directed                   # each edge in two facets, opposite ways
    assert len(directed) // 2 == 3 * k - 6          # E = 3V - 6
    assert set(f.ravel().tolist()) == set(range(k))


def test_hull_matches_qhull_on_generic_points():
    from scipy.spatial import ConvexHull
    rng = np.random.default_rng(11)
    for k in (6, 12, 14):
        for _ in range(20):
            p = rng.normal(size=(k, 3))
            p /= np.linalg.norm(p, axis=1, keepdims=True)
            q = np.round(p * 2 ** 18).astype(np.int64)
            f = O.hull(q)
            assert f is not None
            _check_closed_triangulated_sphere(f, k)
            ref = ConvexHull(q.astype(float))
            assert {tuple(sorted(t)) for t in f.tolist()} == {tuple(sorted(t)) for t in ref.simplices.tolist()}
            c = q.mean(0)
            for a, b, cc in f:
                n = np.cross(q[b] - q[a], q[cc] - q[a]).astype(float)
                assert n @ (q[a] - c) > 0                   # counter-clockwise seen from outside


@pytest.mark.parametrize("name", ["cube", "cuboctahedron", "rhombic_dodecahedron", "octahedron",
                                  "hexagonal_prism"])
def test_hull_degenerate_shapes_triangulate(name):
    if name == "cube":
        q = np.array(list(itertools.product((-1, 1), repeat=3)))
    elif name == "cuboctahedron":
        q = np.array([p for p in itertools.product((-1, 0, 1), repeat=3) if sum(map(abs, p)) == 2])
    elif name == "rhombic_dodecahedron":
        q = np.array(list(itertools.product((-1, 1), repeat=3))
                     + [(2, 0, 0), (-2, 0, 0), (0, 2, 0), (0, -2, 0), (0, 0, 2), (0, 0, -2)])
    elif name == "octahedron":
        q = np.array([(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)])
    else:   # hexagonal prism: two coplanar hexagon faces
        q = np.array([(2, 0, 1), (1, 2, 1), (-1, 2, 1), (-2, 0, 1), (-1, -2, 1), (1, -2, 1),
                      (2, 0, -1), (1, 2, -1), (-1, 2, -1), (-2, 0, -1), (-1, -2, -1), (1, -2, -1)])
    rng = np.random.default_rng(0)
    for _ in range(5):
        perm = rng.permutation(len(q))
        f = O.hull(q[perm].astype(np.int64))
        assert f is not None
        _check_closed_triangulated_sphere(f, len(q))


def test_hull_rejects_interior_point():
    q = np.array([(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
                  (0, 0, 0)], np.int64) * 4
    assert O.hull(q) is None


# --------------------------------------------------------------- Weinberg
def _codes_all_starts(nv, f):
    f = np.asarray(f)
    out = []
    for a, b, c in f:
        for u, v in ((a, b), (b, c), (c, a)):
            code, _ = O.weinberg(nv, f, int(u), int(v))
            out.append(bytes(code.tolist()))
    return out


def test_weinberg_code_length_and_template_automorphisms():
    """Walk covers every edge twice (2E + 1 labels); the SC and ICO graphs have
    24 and 60 orientation-preserving automorphisms (Appendix A)."""
    for S, name in enumerate(O.TEMPLATES):
        k = O.K_OF[S]
        tris = O.triangulations(S)
        for t in tris[:: max(1, len(tris) // 16)]:
            f = t - 1
            _check_closed_triangulated_sphere(f, k)
            codes = _codes_all_starts(k, f)
            assert all(len(c) == 2 * (3 * k - 6) + 1 for c in codes)
    for name in ("SC", "ICO"):
        S = O.TEMPLATES.index(name)
        f = O.triangulations(S)[0] - 1
        codes = _codes_all_starts(O.K_OF[S], f)
        assert codes.count(codes[0]) == GOLDEN["graph_automorphisms"][name]


def _automorphisms(f):
    """All graph automorphisms of a triangulation (networkx VF2), split into those
    that keep the facet orientation and those that reverse it."""
    nx = pytest.importorskip("networkx")
    from networkx.algorithms.isomorphism import GraphMatcher
    G = nx.Graph()
    tri = {tuple(t) for t in np.asarray(f).tolist()}
    cyc = set()
    for a, b, c in tri:
        G.add_edges_from([(a, b), (b, c), (c, a)])
        cyc |= {(a, b, c), (b, c, a), (c, a, b)}
    keep = rev = 0
    for m in GraphMatcher(G, G).isomorphisms_iter():
        img = [(m[a], m[b], m[c]) for a, b, c in tri]
        if all(t in cyc for t in img):
            keep += 1
        elif all((t[0], t[2], t[1]) in cyc for t in img):
            rev += 1
    return keep, rev


def test_weinberg_codes_decide_oriented_isomorphism():
    """Codes are invariant under relabelling and proper rotation; a mirror image
    gives the same code set exactly when an orientation-reversing automorphism
    exists; |Aut+| equals the number of starts sharing a code (Sec. 4)."""
    rng = np.random.default_rng(5)
    seen_chiral = seen_achiral = 0
    for _ in range(12):
        p = rng.normal(size=(12, 3))
        q = np.round(p / np.linalg.norm(p, axis=1, keepdims=True) * 2 ** 16).astype(np.int64)
        f = O.hull(q)
        codes = _codes_all_starts(12, f)
        base = sorted(codes)
        q2 = q[rng.permutation(12)]                  # relabel
        rot = q2[:, [1, 2, 0]]                       # proper rotation (cyclic axis swap)
        assert sorted(_codes_all_starts(12, O.hull(rot))) == base
        mirror = q2 * np.array([-1, 1, 1])
        same = sorted(_codes_all_starts(12, O.hull(mirror))) == base
        keep, rev = _automorphisms(f)
        assert codes.count(codes[0]) == keep
        assert same == (rev > 0)
        seen_chiral += not same
        seen_achiral += same
    assert seen_chiral and seen_achiral


# ------------------------------------------------------- templates / tables
def test_template_counts_match_paper():
    for S, name in enumerate(O.TEMPLATES):
        assert O.K_OF[S] == GOLDEN["neighbours_required"][name]
        assert O.lib().ptmo_n_triangulations(S) == GOLDEN["triangulations"][name]
        perms, quats = O.group(S)
        assert len(perms) == GOLDEN["symmetry_orders"][name]


def test_template_geometry_independently_typed():
    """Template shells compared as point sets with an independent construction."""
    r2 = math.sqrt(2)
    phi = (1 + math.sqrt(5)) / 2
    raw = {
        "SC": [p for p in itertools.product((-1, 0, 1), repeat=3) if sum(map(abs, p)) == 1],
        "FCC": [np.array(p) / r2 for p in itertools.product((-1, 0, 1), repeat=3) if sum(map(abs, p)) == 2],
        "ICO": [np.roll([0, a, b * phi], s) for a in (-1, 1) for b in (-1, 1) for s in range(3)],
        "BCC": [np.array(p) * 0.5 for p in itertools.product((-1, 1), repeat=3)]
               + [p for p in itertools.product((-1, 0, 1), repeat=3) if sum(map(abs, p)) == 1],
    }
    for name, pts in raw.items():
        pts = np.array(pts, float)
        pts = np.vstack([np.zeros(3), pts])
        pts = (pts - pts.mean(0)) / np.mean(np.linalg.norm(pts - pts.mean(0), axis=1))
        w = O.template(O.TEMPLATES.index(name))
        assert np.allclose(w[0], 0)
        d = np.linalg.norm(w[:, None, :] - pts[None, :, :], axis=2)
        assert np.all(d.min(1) < 1e-12) and np.all(d.min(0) < 1e-12), name
    # hcp: every neighbour at distance 1 (raw), 6 in the basal plane, eclipsed triangles
    w = O.template(2)
    l = np.mean(np.linalg.norm(w, axis=1))
    raw = w / np.linalg.norm(w[1])
    assert np.allclose(np.linalg.norm(raw[1:], axis=1), 1)
    assert np.sum(np.abs(raw[1:, 2]) < 1e-12) == 6
    up = raw[raw[:, 2] > 1e-6]
    dn = raw[raw[:, 2] < -1e-6]
    assert np.allclose(np.sort(up[:, :2], 0), np.sort(dn[:, :2], 0))
    # nearest-neighbour distances within the shell equal the shell radius (close packing)
    dd = np.linalg.norm(raw[1:, None] - raw[None, 1:], axis=2)
    assert np.allclose(np.sort(dd, 1)[:, 1], 1)
    for S in range(5):
        w = O.template(S)
        assert np.allclose(w.mean(0), 0, atol=1e-14)
        assert abs(np.mean(np.linalg.norm(w, axis=1)) - 1) < 1e-14   # Eq. 4


def test_rotation_groups_are_symmetries():
    for S in range(5):
        w = O.template(S)
        perms, quats = O.group(S)
        for p, q in zip(perms, quats):
            a, b, c, d = q
            R = np.array([[1 - 2 * (c * c + d * d), 2 * (b * c - a * d), 2 * (b * d + a * c)],
                          [2 * (b * c + a * d), 1 - 2 * (b * b + d * d), 2 * (c * d - a * b)],
                          [2 * (b * d - a * c), 2 * (c * d + a * b), 1 - 2 * (b * b + c * c)]])
            assert np.allclose(w @ R.T, w[p], atol=1e-12)


def test_template_graph_collisions():
    """FCC and HCP triangulations share graphs, and both reach the ICO graph (Sec. 4)."""
    codes = {}
    for name in ("FCC", "HCP", "ICO"):
        S = O.TEMPLATES.index(name)
        s = set()
        for t in O.triangulations(S):
            s.update(_codes_all_starts(12, t - 1))
        codes[name] = s
    assert codes["FCC"] & codes["HCP"]
    assert codes["FCC"] & codes["ICO"]
    assert codes["HCP"] & codes["ICO"]
