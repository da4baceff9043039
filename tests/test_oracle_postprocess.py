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


# -------------------------------------------------- quantisation for the hulls
def test_quantise_power_of_two_grid_half_even_and_bound():
    """q = round-half-even(dr * 2^(19 - e)) with 2^(e-1) <= max |dr| < 2^e:
    restated with Python's frexp and round (which rounds half to even) on
    crafted values: exact powers of two as the maximum, values exactly half a
    grid step off, negative halves, and random vectors (|q| < 2^19, the largest
    component at least 2^18)."""
    def ref(dr):
        mx = float(np.max(np.abs(dr)))
        e = math.frexp(mx)[1]
        return np.array([round(v * 2.0 ** (19 - e)) for v in dr.ravel()], np.int64).reshape(dr.shape), e

    step = 2.0 ** (2 - 19)                              # grid when the maximum is in [2, 4)
    crafted = [
        np.array([[2.0, 0.0, 0.0], [-1.0, 0.5, 0.25]]),                 # maximum exactly 2^1 -> e = 2
        np.array([[3.9, 0.5 * step, 1.5 * step], [2.5 * step, -0.5 * step, -1.5 * step]]),
        np.array([[-3.0, 7.5 * step, -7.5 * step], [1.0 + 0.5 * step, 1.0 + 1.5 * step, 0.0]]),
        np.array([[0.75, 0.375, -0.1875]]),                              # maximum below 1 -> e = 0
        np.array([[1e-3, -2e-3, 3e-3]]),
    ]
    rng = np.random.default_rng(31)
    crafted += [rng.normal(0, rng.uniform(0.5, 8), (14, 3)) for _ in range(40)]
    for dr in crafted:
        q, e = O.quantise(dr)
        qr, er = ref(dr)
        assert e == er
        assert np.array_equal(q, qr), (dr, q, qr)
        assert np.max(np.abs(q)) < 2 ** 19 and np.max(np.abs(q)) >= 2 ** 18
    q, e = O.quantise(crafted[1])
    assert q[0, 1] == 0 and q[0, 2] == 2 and q[1, 0] == 2 and q[1, 1] == 0 and q[1, 2] == -2   # halves to even


# ------------------------------------ fundamental zones of HCP and ICO (Sec. 7)
def _axis_quat(n, theta):
    n = np.asarray(n, float) / np.linalg.norm(n)
    return np.concatenate([[math.cos(theta / 2)], n * math.sin(theta / 2)])


def _qmul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def _hcp_group():
    """D3 in the template frame: rotations by 0, 120, 240 degrees about c (z)
    and half turns about the basal axes at 30, 90 and 150 degrees (the basal
    hexagon has a vertex on x; the upper and lower triangles sit at 30, 150
    and 270 degrees)."""
    g = [_axis_quat([0, 0, 1], t) for t in (0.0, 2 * math.pi / 3, 4 * math.pi / 3)]
    g += [_axis_quat([math.cos(p), math.sin(p), 0], math.pi) for p in np.radians([30, 90, 150])]
    return np.array(g)


def _ico_group():
    """The 60 rotations of the icosahedron with vertices at the cyclic
    permutations of (0, +-1, +-phi): turns by k 72 degrees about the 6 vertex
    axes, by 120 and 240 degrees about the 10 face axes, half turns about the
    15 edge axes, and the identity."""
    phi = (1 + math.sqrt(5)) / 2
    V = []
    for s1 in (1, -1):
        for s2 in (1, -1):
            V += [(0, s1, s2 * phi), (s1, s2 * phi, 0), (s2 * phi, 0, s1)]
    V = np.array(V)
    edge = 2.0

    def axes(points):
        out = []
        for p in points:
            p = p / np.linalg.norm(p)
            if not any(abs(abs(np.dot(p, o)) - 1) < 1e-9 for o in out):
                out.append(p)
        return out
    pairs = [(i, j) for i in range(12) for j in range(i + 1, 12) if abs(np.linalg.norm(V[i] - V[j]) - edge) < 1e-9]
    tris = [(i, j, k) for i, j in pairs for k in range(j + 1, 12)
            if abs(np.linalg.norm(V[i] - V[k]) - edge) < 1e-9 and abs(np.linalg.norm(V[j] - V[k]) - edge) < 1e-9]
    five, three, two = axes(V), axes([V[i] + V[j] + V[k] for i, j, k in tris]), axes([V[i] + V[j] for i, j in pairs])
    assert (len(five), len(three), len(two)) == (6, 10, 15)
    g = [np.array([1.0, 0, 0, 0])]
    g += [_axis_quat(a, 2 * math.pi * k / 5) for a in five for k in range(1, 5)]
    g += [_axis_quat(a, 2 * math.pi * k / 3) for a in three for k in (1, 2)]
    g += [_axis_quat(a, math.pi) for a in two]
    return np.array(g)


def _check_zone(q, G, q_applied=None):
    """q (w >= 0) has the largest |w| over its orbit {q g : g in G}; if given,
    the applied rotation is in that orbit."""
    assert q[0] >= 0
    ws = [abs(_qmul(q, g)[0]) for g in G]
    assert abs(q[0] - max(ws)) < 1e-9, (q, max(ws))
    if q_applied is not None:
        d = min(1 - abs(np.dot(_qmul(q, g), q_applied)) for g in G)
        assert d < 1e-9, d


def test_fundamental_zone_hcp_and_ico_against_independent_groups():
    """Randomly rotated perfect HCP lattices and icosahedral clusters: the
    oracle reports the member of the orientation's orbit under the template's
    rotation group with the largest |w| (the smallest rotation angle), the
    groups typed here from the geometry (D3 of order 6, the icosahedral group
    of order 60).  For the icosahedron, whose template frame is that of the
    generated cluster, the applied rotation must also lie in the orbit."""
    G_hcp, G_ico = _hcp_group(), _ico_group()
    assert len(G_hcp) == 6 and len(G_ico) == 60
    rng = I.rng_for(41)
    for _ in range(10):
        f = I.crystal("hcp", I.A_HCP, (4, 3, 3), rotation=I.random_rotation(rng), dtype=np.float64)
        r = O.classify_frame(f, atoms=np.arange(4))
        assert np.all(r["structure"] == O.HCP)
        for q in r["quat"]:
            _check_zone(q, G_hcp)
    clusters, applied = [], []
    for _ in range(10):
        R = I.random_rotation(rng)
        clusters.append(I.ico_cluster(rotation=R))
        applied.append(R)
    fr = I.isolated_clusters(clusters)
    r = O.classify_frame(fr, atoms=np.arange(0, 13 * len(clusters), 13))
    assert np.all(r["structure"] == O.ICO)
    from scipy.spatial.transform import Rotation
    for q, R in zip(r["quat"], applied):
        x, y, z, w = Rotation.from_matrix(R).as_quat()
        _check_zone(q, G_ico, np.array([w, x, y, z]))
