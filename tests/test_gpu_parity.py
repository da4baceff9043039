"""CUDA path vs the oracle, element by element, through the C ABI (GPU only)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1603_05143_gb300 import inputs as I
from parity import compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ptm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_05143_gb300 import PTM
    p = PTM(0)
    yield p
    p.close()


def run_gpu(ptm, frame, mask=31, rmsd_max=math.inf, species="frame"):
    import torch
    sp = frame.species if isinstance(species, str) else species
    pos = torch.from_numpy(np.ascontiguousarray(frame.positions)).cuda()
    spt = None if sp is None else torch.from_numpy(np.ascontiguousarray(sp, np.int8)).cuda()
    out = ptm.classify(pos, frame.cell, frame.pbc, species=spt, mask=mask, rmsd_max=rmsd_max)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    return res


def check(ptm, frame, atoms=None, mask=31, rmsd_max=math.inf, species="frame"):
    g = run_gpu(ptm, frame, mask, rmsd_max, species)
    sp = frame.species if isinstance(species, str) else species
    F = O.Frame(frame.positions, frame.cell, frame.pbc)
    ref = F.classify(atoms, species=sp, mask=mask, rmsd_max=rmsd_max)
    st = compare(g, ref, atoms)
    assert ptm.stats()["internal"] == 0
    return st, g, ref


def test_fcc4000_float64_full(ptm):
    """4000-atom fcc Cu, sigma 0.10 A, float64 positions: every atom."""
    f = I.config_fcc_small()
    st, g, ref = check(ptm, f)
    assert st["matched"] >= 0.99 * f.n


@pytest.mark.parametrize("kind,a,reps,dtype", [
    ("fcc", I.A_FCC_CU, 5, np.float32), ("bcc", I.A_BCC_FE, 6, np.float32),
    ("hcp", I.A_HCP, (6, 4, 4), np.float32), ("sc", I.A_SC, 6, np.float64),
    ("fcc", I.A_FCC_CU, 5, np.float64), ("bcc", I.A_BCC_FE, 5, np.float64)])
@pytest.mark.parametrize("sigma", [0.0, 0.05, 0.2])
def test_lattices(ptm, kind, a, reps, dtype, sigma):
    R = I.random_rotation(I.rng_for(int(sigma * 100) + 7))
    f = I.crystal(kind, a, reps, sigma=sigma, seed=3, rotation=R, dtype=dtype)
    check(ptm, f)


def test_unrotated_perfect_lattices_exact_ties(ptm):
    """Axis-aligned perfect lattices: coplanar facets everywhere (SoS), tied
    distances; the 14th neighbour falls inside a tied shell for fcc and hcp
    (2 of the 6 second neighbours), so the kNN must order ties by atom id."""
    for kind, a, reps in (("fcc", I.A_FCC_CU, 4), ("bcc", I.A_BCC_FE, 4), ("sc", I.A_SC, 4),
                          ("hcp", I.A_HCP, (6, 4, 4))):
        for dtype in (np.float32, np.float64):
            check(ptm, I.crystal(kind, a, reps, dtype=dtype))


@pytest.mark.parametrize("kind", ["l10", "l12", "b2"])
def test_alloys(ptm, kind):
    a = I.A_BCC_FE if kind == "b2" else I.A_L12
    f = I.crystal(kind, a, 5, sigma=0.05, seed=2, rotation=I.random_rotation(I.rng_for(4)), dtype=np.float32)
    st, g, ref = check(ptm, f)
    assert np.all(g["alloy"] > 0)


def test_strained_triclinic_frames(ptm):
    """Frames shaped like the batched workload: triclinic cells, strain, noise."""
    frames = I.config_batch(seed=99, n_frames=6, n_min=300, n_max=3000)
    for f in frames:
        check(ptm, f)


def test_icosahedral_clusters_and_nonperiodic(ptm):
    rng = I.rng_for(5)
    cl = [I.ico_cluster(2.556, rotation=I.random_rotation(rng), sigma=0.02, seed=i) for i in range(10)]
    f = I.isolated_clusters(cl, spacing=12.0)
    check(ptm, f)
    g = I.Frame(f.positions, f.cell, (False, False, False), None, "nonperiodic")
    check(ptm, g)


def test_tiny_box_own_images(ptm):
    """2x2x2 cells: an atom's own periodic images are among its neighbours."""
    for kind, a in (("bcc", I.A_BCC_FE), ("fcc", I.A_FCC_CU), ("sc", I.A_SC)):
        check(ptm, I.crystal(kind, a, 2, sigma=0.05, seed=1, dtype=np.float64))
        check(ptm, I.crystal(kind, a, (1, 2, 3), sigma=0.05, seed=1, dtype=np.float32))


def test_atoms_outside_cell(ptm):
    """Unwrapped positions (atoms up to two cells away) give the same answer."""
    f = I.crystal("fcc", I.A_FCC_CU, 4, sigma=0.1, seed=5, dtype=np.float64)
    rng = I.rng_for(8)
    shift = rng.integers(-2, 3, (f.n, 3)) @ f.cell
    g = I.Frame(f.positions + shift, f.cell, f.pbc, None, "unwrapped")
    st, g1, _ = check(ptm, g)
    g0 = run_gpu(ptm, f)
    assert np.array_equal(g0["structure"], g1["structure"])


def test_atoms_outside_cell_float32(ptm):
    """Unwrapped float32 positions take the general neighbour search, whose
    FP32 filter must keep every candidate the FP64 order can pick."""
    f = I.crystal("bcc", I.A_BCC_FE, 4, sigma=0.0, dtype=np.float64, rotation=I.random_rotation(I.rng_for(12)))
    rng = I.rng_for(9)
    shift = rng.integers(-2, 3, (f.n, 3)) @ f.cell
    g = I.Frame((f.positions + shift).astype(np.float32), f.cell, f.pbc, None, "unwrapped32")
    check(ptm, g)
    assert ptm.stats()["knn_fp64"] == f.n


@pytest.mark.parametrize("kind,a,reps", [("fcc", I.A_FCC_CU, 3), ("fcc", I.A_FCC_CU, 6), ("bcc", I.A_BCC_FE, 5),
                                         ("hcp", I.A_HCP, (5, 3, 3)), ("sc", I.A_SC, 5), ("l12", I.A_L12, 4)])
@pytest.mark.parametrize("sigma", [0.0, 1e-6])
def test_float32_near_ties_follow_fp64(ptm, kind, a, reps, sigma):
    """Perfect (or 1e-6 A noise) rotated float32 lattices: mirror-image
    neighbours differ in distance only by the float32 rounding of the
    positions, less than the float32 rounding of d^2, so the FP32 order is not
    the FP64 order of the oracle (which also decides the SoS priorities and the
    reported correspondence); every atom must still match it exactly."""
    f = I.crystal(kind, a, reps, sigma=sigma, seed=4, dtype=np.float32, rotation=I.random_rotation(I.rng_for(31)))
    check(ptm, f)
    assert ptm.stats()["knn_fp64"] > 0


@pytest.mark.parametrize("sigma", [0.0, 1e-7])
def test_float32_near_ties_across_a_long_periodic_side(ptm, sigma):
    """An fcc slab across the x = 0 side of a 1000 A box: neighbours reached
    through the periodic image carry a 1000 A shift, whose float32 rounding
    moves d^2 by about as much as the gaps between mirror-image neighbours, so
    the FP32 error bound must account for the shift."""
    c = I.crystal("fcc", I.A_FCC_CU, (8, 4, 4), sigma=sigma, seed=6, dtype=np.float64, wrap=False)
    pos = c.positions - np.array([4 * I.A_FCC_CU, 0.0, 0.0])
    cell = np.diag([1000.0, 4 * I.A_FCC_CU, 4 * I.A_FCC_CU])
    pos[:, 0] = np.mod(pos[:, 0], 1000.0)
    f = I.Frame(pos.astype(np.float32), cell, (True, True, True), None, "slab")
    st, g, ref = check(ptm, f)
    assert st["matched"] > f.n // 2


@pytest.mark.parametrize("mask", [1, 2, 4, 8, 16, 6, 14, 30, 17])
def test_template_masks(ptm, mask):
    f = I.crystal("fcc", I.A_FCC_CU, 4, sigma=0.25, seed=3, dtype=np.float32)
    check(ptm, f, mask=mask)


def test_rmsd_max_cut(ptm):
    f = I.crystal("fcc", I.A_FCC_CU, 4, sigma=0.12, seed=3, dtype=np.float64)
    g = run_gpu(ptm, f)
    cut = float(np.median(g["rmsd"])) + 1e-4        # away from any atom's value
    check(ptm, f, rmsd_max=cut)


def test_polycrystal_small_full(ptm):
    """65536-atom periodic polycrystal with stacking faults, float32: every atom."""
    f = I.config_polycrystal(n_target=1 << 16)
    st, g, ref = check(ptm, f)
    counts = np.bincount(g["structure"], minlength=6)
    # 16 grains in a 92 A box: about 45% of the atoms sit near a grain boundary
    assert counts[2] > 0.5 * f.n and counts[3] > 0


def test_polycrystal_full_size_sampled(ptm):
    """The 1,048,576-atom polycrystal in the launch configuration of bench.py;
    a seeded sample of atoms is checked against the oracle one by one."""
    f = I.config_polycrystal()
    atoms = np.sort(I.rng_for(77).choice(f.n, 3000, replace=False))
    st, g, ref = check(ptm, f, atoms=atoms)
    assert st["matched"] > 0.9 * len(atoms)


def test_mixed_phase_small_full(ptm):
    """65536-atom mixed-phase frame (bcc / fcc / L1_2 with antisites / sc /
    liquid with icosahedral seeds), int8 species, sigma 0.20 A: every atom."""
    f = I.config_mixed_phase(n_target=1 << 16)
    st, g, ref = check(ptm, f)
    counts = np.bincount(g["structure"], minlength=6)
    assert counts[5] > 0.1 * f.n and counts[2] > 0.2 * f.n and counts[1] > 0.1 * f.n
    assert np.any(g["alloy"] >= 3)      # L1_2 sites found


def test_mixed_phase_full_size_sampled(ptm):
    """The 4,194,304-atom mixed-phase frame; a seeded sample of atoms (liquid
    included) is checked against the oracle one by one."""
    f = I.config_mixed_phase()
    atoms = np.sort(I.rng_for(78).choice(f.n, 3000, replace=False))
    st, g, ref = check(ptm, f, atoms=atoms)
    assert st["matched"] > 0.5 * len(atoms)


def test_host_entry_point_matches_device(ptm):
    f = I.crystal("l12", I.A_L12, 5, sigma=0.1, seed=9, dtype=np.float32)
    d = run_gpu(ptm, f)
    h = ptm.classify_host(f.positions, f.cell, f.pbc, species=f.species)
    for k in d:
        assert np.array_equal(d[k], h[k]), k


def test_repeatable_and_stream_ordered(ptm):
    import torch
    f = I.crystal("bcc", I.A_BCC_FE, 8, sigma=0.15, seed=4, dtype=np.float32)
    a = run_gpu(ptm, f)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        pos = torch.from_numpy(f.positions).cuda()
        sp = torch.from_numpy(f.species).cuda()
        outs = [ptm.classify(pos, f.cell, species=sp) for _ in range(3)]
    s.synchronize()
    for o in outs:
        for k in a:
            assert np.array_equal(a[k], o[k].cpu().numpy()), k


# --------------------------------------------------------------- FP64 form
@pytest.fixture(scope="module")
def ptm64():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_05143_gb300 import PTM
    p = PTM(0, precision="fp64")
    yield p
    p.close()


@pytest.mark.parametrize("case", ["fcc4000", "l12", "bcc_b2_strained", "hcp", "ico", "polycrystal"])
def test_fp64_form_matches_oracle(ptm64, case):
    """The one-frame-per-launch FP64 form meets the same parity bar."""
    rng = I.rng_for(31)
    if case == "fcc4000":
        f = I.config_fcc_small()
    elif case == "l12":
        f = I.crystal("l12", I.A_L12, 5, sigma=0.08, seed=4, rotation=I.random_rotation(rng), dtype=np.float32)
    elif case == "bcc_b2_strained":
        E = np.eye(3) + np.array([[0.03, 0.01, 0], [0.01, -0.02, 0.02], [0, 0.02, 0.01]])
        f = I.crystal("b2", I.A_BCC_FE, 6, sigma=0.0, rotation=I.random_rotation(rng), deform=E, dtype=np.float32)
    elif case == "hcp":
        f = I.crystal("hcp", I.A_HCP, (6, 4, 4), sigma=0.1, seed=5, dtype=np.float32)
    elif case == "ico":
        cl = [I.ico_cluster(2.556, rotation=I.random_rotation(rng), sigma=0.05, seed=i) for i in range(20)]
        f = I.isolated_clusters(cl, dtype=np.float32)
    else:
        f = I.config_polycrystal(n_target=1 << 14)
    st, g, ref = check(ptm64, f)
    assert st["matched"] > 0


def test_fp64_form_agrees_with_fp32_form(ptm, ptm64):
    f = I.config_mixed_phase(n_target=1 << 15)
    a = run_gpu(ptm, f)
    b = run_gpu(ptm64, f)
    for k in ("structure", "alloy", "correspondence"):
        assert np.array_equal(a[k], b[k]), k
    m = a["structure"] > 0
    assert np.abs(a["rmsd"][m] - b["rmsd"][m]).max() < 1e-5
