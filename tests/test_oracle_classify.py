"""Pins for the oracle's metric pieces and the whole per-atom classification.

References used here instead of the oracle itself: scipy's cKDTree and an
explicit image sum (neighbours), numpy SVD (Kabsch with scale, polar
decomposition), brute force over all 720 correspondences (k = 6), and lattices
whose structure, orientation, scale, strain and alloy label are known exactly.
"""
import itertools
import math

import numpy as np
import pytest

import oracle as O
from paper_1603_05143_gb300 import inputs as I


def _kabsch_scaled_r2(v, w):
    """min over s, proper Q of mean |s v' - Q w'|^2 via SVD (Eq. 3)."""
    vp = v - v.mean(0)
    wp = w - w.mean(0)
    H = wp.T @ vp
    U, S, Vt = np.linalg.svd(H)
    d = np.sign(np.linalg.det(U @ Vt))
    lam = S[0] + S[1] + d * S[2]
    return (np.sum(wp * wp) - lam * lam / np.sum(vp * vp)) / len(v)


def _qmat(q):
    a, b, c, d = q
    return np.array([[1 - 2 * (c * c + d * d), 2 * (b * c - a * d), 2 * (b * d + a * c)],
                     [2 * (b * c + a * d), 1 - 2 * (b * b + d * d), 2 * (c * d - a * b)],
                     [2 * (b * d - a * c), 2 * (c * d + a * b), 1 - 2 * (b * b + c * c)]])


def test_superpose_matches_kabsch_svd():
    rng = np.random.default_rng(1)
    for N in (7, 13, 15):
        for _ in range(50):
            v = rng.normal(size=(N, 3))
            w = rng.normal(size=(N, 3))
            r2, q, s, lam = O.superpose(v, w)
            assert abs(r2 - _kabsch_scaled_r2(v, w)) < 1e-12
            assert abs(np.linalg.norm(q) - 1) < 1e-14


def test_superpose_recovers_rotation_and_scale():
    rng = np.random.default_rng(2)
    for S in range(5):
        w = O.template(S)
        R = I.random_rotation(rng)
        s0 = rng.uniform(0.2, 5)
        v = (w @ R.T) / s0 + rng.normal(size=3)
        r2, q, s, lam = O.superpose(v, w)
        assert r2 < 1e-26
        assert abs(s - s0) < 1e-12 * s0
        assert np.allclose(_qmat(q), R, atol=1e-12)


def test_polar_matches_svd():
    rng = np.random.default_rng(4)
    for _ in range(100):
        A = np.eye(3) + 0.2 * rng.normal(size=(3, 3))
        if rng.random() < 0.2:
            A[:, 0] *= -1                       # det < 0: U must still be a rotation
        P, U = O.polar(A)
        X, S, Yt = np.linalg.svd(A)
        if np.linalg.det(X @ Yt) < 0:
            S[-1] = -S[-1]
            Yt[-1] = -Yt[-1]
        assert np.allclose(P, X @ np.diag(S) @ X.T, atol=1e-12)
        assert np.allclose(P, P.T, atol=1e-14)
        assert np.allclose(P @ U, A, atol=1e-12)
        assert abs(np.linalg.det(U) - 1) < 1e-12


# ------------------------------------------------------------------ neighbours
def _brute_knn(x, H, i, k, reach=3, pbc=(True, True, True)):
    """The k nearest images of atom i by an explicit sum over images in
    [-reach, reach]^3, in FP64 (float32 positions widened first, which is
    exact), one IEEE operation at a time; ties by (atom id, image)."""
    x = np.asarray(x, np.float64)
    rows = []
    rng_ = [range(-reach, reach + 1) if p else range(1) for p in pbc]
    for n in itertools.product(*rng_):
        s = (n[0] * H[0] + n[1] * H[1]) + n[2] * H[2]
        d = (x - x[i]) + s
        d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
        for j in range(len(x)):
            if j == i and n == (0, 0, 0):
                continue
            rows.append((d2[j], j, n, d[j]))
    rows.sort(key=lambda r: r[:3])
    return rows[:k]


def test_knn_matches_kdtree_orthorhombic():
    from scipy.spatial import cKDTree
    f = I.crystal("fcc", 3.615, (5, 6, 7), sigma=0.2, seed=9)
    F = O.Frame(f.positions, f.cell)
    L = np.diag(f.cell)
    tree = cKDTree(np.mod(f.positions, L), boxsize=L)
    rng = np.random.default_rng(0)
    for i in rng.choice(f.n, 60, replace=False):
        ids, imgs, dr, d2 = F.knn(int(i))
        dist, idx = tree.query(np.mod(f.positions[i], L), k=15)
        assert np.allclose(np.sqrt(d2), dist[1:], atol=1e-12)
        assert set(ids.tolist()) == set(idx[1:].tolist())


def test_knn_triclinic_and_tiny_box_against_image_sum():
    """Explicit sum over images in [-3, 3]^3; ties resolved by (id, image)."""
    rng = np.random.default_rng(3)
    R = I.random_rotation(rng)
    E = np.eye(3) + 0.1 * rng.normal(size=(3, 3))
    for reps in ((2, 2, 2), (3, 2, 2), (4, 4, 4)):
        f = I.crystal("bcc", 2.8665, reps, sigma=0.05, seed=2, rotation=R, deform=E)
        F = O.Frame(f.positions, f.cell)
        for i in range(0, f.n, max(1, f.n // 12)):
            rows = _brute_knn(f.positions, f.cell, i, 14)
            ids, imgs, dr, d2 = F.knn(i)
            assert [r[1] for r in rows] == ids.tolist()
            assert [tuple(r[2]) for r in rows] == [tuple(t) for t in imgs.tolist()]
            assert np.array_equal(np.array([r[0] for r in rows]), d2)
            assert np.array_equal(np.array([r[3] for r in rows]), dr)


def test_knn_float32_input_ordered_in_fp64():
    """Float32 positions: the order is that of the FP64 distances between the
    given points (Sec. 3 orders by distance; widening float32 is exact)."""
    rng = np.random.default_rng(8)
    f = I.crystal("fcc", 3.615, 4, sigma=0.1, seed=8, dtype=np.float32,
                  rotation=I.random_rotation(rng), deform=np.eye(3) + 0.03 * rng.normal(size=(3, 3)))
    F = O.Frame(f.positions, f.cell)
    for i in (0, 17, 100, 255):
        rows = _brute_knn(f.positions, f.cell, i, 14, reach=1)
        ids, imgs, dr, d2 = F.knn(i)
        assert [r[1] for r in rows] == ids.tolist()
        assert [tuple(r[2]) for r in rows] == [tuple(t) for t in imgs.tolist()]
        assert np.array_equal(np.array([r[0] for r in rows]), d2)
        assert np.array_equal(np.array([r[3] for r in rows]), dr)


def _f32_order(x, H, i, cand):
    """Order of the candidate (j, image) pairs when the same contract runs in
    float32 operations (the mistake the next test must catch)."""
    x32 = np.asarray(x, np.float32)
    keys = []
    for j, n in cand:
        s = ((n[0] * H[0] + n[1] * H[1]) + n[2] * H[2]).astype(np.float32)
        d = (x32[j] - x32[i]) + s
        keys.append(((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2], j, tuple(n)))
    return [k[1:] for k in sorted(keys)]


def test_knn_near_ties_follow_fp64_not_float32():
    """A perfect (sigma = 0) rotated float32 fcc lattice: mirror-image
    neighbours sit at distances that differ only by the float32 rounding of the
    positions, less than the float32 rounding of d^2 itself, and the six second
    shell neighbours straddle the 14th/15th boundary.  The oracle must follow
    the FP64 brute force on every sampled atom, and the case must really
    separate the precisions: a float32 contract orders them differently and
    even picks a different set of 14."""
    rng = np.random.default_rng(21)
    f = I.crystal("fcc", 3.615, 3, sigma=0.0, seed=5, dtype=np.float32, rotation=I.random_rotation(rng))
    x = f.positions
    F = O.Frame(x, f.cell)
    order_differs = set_differs = 0
    for i in range(0, len(x), 3):
        rows = _brute_knn(x, f.cell, i, 14, reach=1)
        ids, imgs, dr, d2 = F.knn(i)
        assert [r[1] for r in rows] == ids.tolist()
        assert [tuple(r[2]) for r in rows] == [tuple(t) for t in imgs.tolist()]
        assert np.array_equal(np.array([r[0] for r in rows]), d2)
        fp64 = [(r[1], tuple(r[2])) for r in rows]
        more = _brute_knn(x, f.cell, i, 24, reach=1)
        f32 = _f32_order(x, f.cell, i, [(r[1], r[2]) for r in more])[:14]
        order_differs += f32 != fp64
        set_differs += set(f32) != set(fp64)
    assert order_differs >= 20 and set_differs >= 10, (order_differs, set_differs)


# ------------------------------------------------------ whole classification
def _misorientation(qa, qb, S):
    """Smallest rotation angle between orientations qa and qb modulo the group of
    structure S (1..5)."""
    _, G = O.group(S - 1)
    Ra, Rb = _qmat(qa), _qmat(qb)
    best = 10.0
    for g in G:
        M = Ra.T @ Rb @ _qmat(g)
        # |M - I|_F = 2 sqrt(2) sin(theta / 2): accurate for small angles
        x = np.linalg.norm(M - np.eye(3)) / (2 * math.sqrt(2))
        best = min(best, 2 * math.asin(min(1.0, x)))
    return best


def _rot_to_quat(R):
    w = math.sqrt(max(0.0, 1 + R[0, 0] + R[1, 1] + R[2, 2])) / 2
    if w > 1e-3:
        return np.array([w, (R[2, 1] - R[1, 2]) / (4 * w), (R[0, 2] - R[2, 0]) / (4 * w),
                         (R[1, 0] - R[0, 1]) / (4 * w)])
    ev, V = np.linalg.eigh(np.array([
        [R[0, 0] + R[1, 1] + R[2, 2], R[2, 1] - R[1, 2], R[0, 2] - R[2, 0], R[1, 0] - R[0, 1]],
        [R[2, 1] - R[1, 2], R[0, 0] - R[1, 1] - R[2, 2], R[0, 1] + R[1, 0], R[0, 2] + R[2, 0]],
        [R[0, 2] - R[2, 0], R[0, 1] + R[1, 0], R[1, 1] - R[0, 0] - R[2, 2], R[1, 2] + R[2, 1]],
        [R[1, 0] - R[0, 1], R[0, 2] + R[2, 0], R[1, 2] + R[2, 1], R[2, 2] - R[0, 0] - R[1, 1]]]) / 3)
    return V[:, -1]


# raw lattice orientation relative to the template of each structure
LATTICES = [("sc", I.A_SC, O.SC), ("fcc", I.A_FCC_CU, O.FCC), ("bcc", I.A_BCC_FE, O.BCC),
            ("hcp", I.A_HCP, O.HCP)]


@pytest.mark.parametrize("kind,a,S", LATTICES)
def test_perfect_rotated_lattice(kind, a, S):
    """Perfect lattice, any rotation: RMSD 0, structure S, applied rotation
    recovered modulo the template group, analytic scale, strain identity."""
    rng = np.random.default_rng(S)
    R = I.random_rotation(rng)
    reps = (4, 3, 3) if kind == "hcp" else 4
    f = I.crystal(kind, a, reps, rotation=R, dtype=np.float64)
    atoms = rng.choice(f.n, 24, replace=False)
    r = O.classify_frame(f, atoms=atoms, species=None)
    assert np.all(r["structure"] == S)
    assert np.all(r["rmsd"] < 1e-10)
    qR = _rot_to_quat(R)
    # hcp: the two sublattices see shells rotated by 60 degrees about c, which is
    # not in the 6-element group of the template
    c60 = np.array([[0.5, -math.sqrt(3) / 2, 0], [math.sqrt(3) / 2, 0.5, 0], [0, 0, 1]])
    alt = _rot_to_quat(R @ c60) if kind == "hcp" else qR
    n_alt = 0
    for q in r["quat"]:
        m0, m1 = _misorientation(q, qR, S), _misorientation(q, alt, S)
        assert min(m0, m1) < 1e-8
        n_alt += m0 >= 1e-8
    if kind == "hcp":
        assert 0 < n_alt < len(atoms)
    F = O.Frame(f.positions, f.cell)
    for t, i in enumerate(atoms[:4]):
        ids, imgs, dr, d2 = F.knn(int(i), O.K_OF[S - 1])
        v = np.vstack([np.zeros(3), dr])
        s_exact = len(v) / np.sum(np.linalg.norm(v - v.mean(0), axis=1))
        assert abs(r["scale"][t] - s_exact) < 1e-12
    for P in r["strain"]:
        assert np.allclose(P, np.eye(3), atol=1e-10)


def test_icosahedral_cluster_centre():
    rng = np.random.default_rng(12)
    clusters = [I.ico_cluster(2.556, rotation=I.random_rotation(rng)) for _ in range(8)]
    f = I.isolated_clusters(clusters, spacing=40.0)
    r = O.classify_frame(f, atoms=np.arange(0, f.n, 13), species=None)
    assert np.all(r["structure"] == O.ICO)
    assert np.all(r["rmsd"] < 1e-10)


def test_small_noise_sc_matches_brute_force_over_all_permutations():
    """k = 6: the best topologically admissible correspondence is the best of all
    6! correspondences (Kabsch with scale) for a mildly perturbed SC shell."""
    rng = np.random.default_rng(21)
    w = O.template(O.SC - 1)
    for trial in range(6):
        f = I.crystal("sc", I.A_SC, 4, sigma=0.04, seed=trial, rotation=I.random_rotation(rng))
        i = int(rng.integers(f.n))
        r = O.classify_frame(f, atoms=[i], species=None, mask=1)
        F = O.Frame(f.positions, f.cell)
        ids, imgs, dr, d2 = F.knn(i, 6)
        v = np.vstack([np.zeros(3), dr])
        best = min(_kabsch_scaled_r2(v[[0] + [1 + p for p in perm]], w)
                   for perm in itertools.permutations(range(6)))
        assert r["structure"][0] == O.SC
        assert abs(r["rmsd"][0] ** 2 - best) < 1e-12


def test_affine_strain_recovered():
    """Eq. 6-7: a crystal deformed by F = V R gives P / det(P)^(1/3) = V / det(V)^(1/3)."""
    rng = np.random.default_rng(8)
    for kind, a, S in LATTICES:
        E = rng.uniform(-0.05, 0.05, (3, 3))
        V = np.eye(3) + 0.5 * (E + E.T)
        R = I.random_rotation(rng)
        reps = (4, 3, 3) if kind == "hcp" else 4
        f = I.crystal(kind, a, reps, rotation=R, deform=V)
        r = O.classify_frame(f, atoms=np.arange(0, f.n, 7), species=None)
        assert np.all(r["structure"] == S)
        Vn = V / np.cbrt(np.linalg.det(V))
        for P in r["strain"]:
            assert np.allclose(P / np.cbrt(np.linalg.det(P)), Vn, atol=1e-10)


@pytest.mark.parametrize("kind,expect", [
    ("fcc", {0: O.ALLOY_PURE}),
    ("l10", {0: O.ALLOY_L10, 1: O.ALLOY_L10}),
    ("l12", {0: O.ALLOY_L12_MAJ, 1: O.ALLOY_L12_MIN}),
    ("bcc", {0: O.ALLOY_PURE}),
    ("b2", {0: O.ALLOY_B2, 1: O.ALLOY_B2}),
])
def test_alloy_labels(kind, expect):
    """Table 3 (FCC) and the A2/B2 rules of Sec. 6 on perfect ordered lattices."""
    rng = np.random.default_rng(5)
    a = I.A_L12 if kind in ("l10", "l12") else (I.A_FCC_CU if kind == "fcc" else I.A_BCC_FE)
    f = I.crystal(kind, a, 4, sigma=0.02, seed=3, rotation=I.random_rotation(rng))
    r = O.classify_frame(f)
    for sp, lab in expect.items():
        sel = f.species == sp
        assert np.all(r["alloy"][sel] == lab), (kind, sp, np.unique(r["alloy"][sel]))
    r2 = O.classify_frame(f, species=None)
    assert np.all(r2["alloy"] == O.ALLOY_NONE)


def test_rmsd_max_cutoff_and_unmatched_outputs():
    f = I.crystal("fcc", I.A_FCC_CU, 4, sigma=0.1, seed=1)
    r = O.classify_frame(f, atoms=np.arange(40), species=None)
    assert np.all(r["structure"] == O.FCC)
    cut = float(np.median(r["rmsd"]))
    r2 = O.classify_frame(f, atoms=np.arange(40), species=None, rmsd_max=cut)
    assert np.array_equal(r2["structure"] == O.FCC, r["rmsd"] <= cut)
    un = r2["structure"] == O.NONE
    assert np.all(np.isinf(r2["rmsd"][un]))
    assert np.all(r2["quat"][un] == [1, 0, 0, 0])
    assert np.all(r2["corr"][un] == -1)
    assert np.all(r2["strain"][un] == 0)


def test_correspondence_is_canonical_orbit_minimum():
    """Reported correspondence (R12) is the same for the same environment under
    any rotation of the sample; and maps each neighbour to its matching slot."""
    f = I.crystal("fcc", I.A_FCC_CU, 4, sigma=0.05, seed=4)
    r = O.classify_frame(f, atoms=np.arange(10), species=None)
    rng = np.random.default_rng(0)
    R = I.random_rotation(rng)
    g = I.Frame(f.positions @ R.T, f.cell @ R.T, f.pbc, None)
    r2 = O.classify_frame(g, atoms=np.arange(10), species=None)
    assert np.array_equal(r["corr"], r2["corr"])
    assert np.all(r["corr"][:, 0] == np.arange(10))
    assert np.all(r["corr"][:, 13:] == -1)
