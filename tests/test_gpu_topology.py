"""Topological neighbour ordering (Sec. 3, Eq. 5) on the GPU against the oracle
(GPU only): same parity bar as the Euclidean path."""
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


def run(ptm, f, ordering="topological", mask=31):
    import torch
    sp = None if f.species is None else torch.from_numpy(np.ascontiguousarray(f.species, np.int8)).cuda()
    out = ptm.classify(torch.from_numpy(np.ascontiguousarray(f.positions)).cuda(), f.cell, f.pbc, species=sp,
                       mask=mask, ordering=ordering)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def check(ptm, f, atoms=None, mask=31):
    g = run(ptm, f, mask=mask)
    F = O.Frame(f.positions, f.cell, f.pbc)
    ref = F.classify(atoms, species=f.species, mask=mask, ordering="topological")
    st = compare(g, ref, atoms)
    s = ptm.stats()
    assert s["internal"] == 0
    return st, g, ref, s


@pytest.mark.parametrize("kind,a,reps", [("fcc", I.A_FCC_CU, 5), ("bcc", I.A_BCC_FE, 6), ("sc", I.A_SC, 6),
                                         ("hcp", I.A_HCP, (6, 4, 4)), ("l12", I.A_L12, 5)])
def test_perfect_lattices_match_euclidean_and_oracle(ptm, kind, a, reps):
    f = I.crystal(kind, a, reps, rotation=I.random_rotation(I.rng_for(5)), dtype=np.float32)
    st, g, ref, s = check(ptm, f)
    e = run(ptm, f, ordering="euclidean")
    for k in ("structure", "correspondence", "alloy"):
        assert np.array_equal(g[k], e[k]), k
    assert st["matched"] == f.n


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_unrotated_perfect_lattices_exact_ties(ptm, dtype):
    """Axis-aligned lattices: the 18 nearest hold whole shells of equal
    distances (bcc: 4 of the 12 third neighbours), ordered by atom id."""
    for kind, a in (("fcc", I.A_FCC_CU), ("bcc", I.A_BCC_FE), ("sc", I.A_SC)):
        f = I.crystal(kind, a, 4, dtype=dtype)
        st, g, ref, s = check(ptm, f)
        assert st["matched"] == f.n


@pytest.mark.parametrize("sigma,dtype", [(0.1, np.float32), (0.2, np.float64), (0.28, np.float32)])
def test_noisy_fcc_full(ptm, sigma, dtype):
    f = I.crystal("fcc", I.A_FCC_CU, 6, sigma=sigma, seed=8, rotation=I.random_rotation(I.rng_for(6)), dtype=dtype)
    st, g, ref, s = check(ptm, f)
    e = run(ptm, f, ordering="euclidean")
    if sigma >= 0.2:                 # Sec. 5.2: the area order keeps more fcc atoms when hot
        assert np.sum(g["structure"] == 2) > np.sum(e["structure"] == 2)


def test_polycrystal_and_mixed_phase_full(ptm):
    for f in (I.config_polycrystal(n_target=1 << 14), I.config_mixed_phase(n_target=1 << 14)):
        check(ptm, f)


def test_strained_triclinic_and_masks(ptm):
    fr = I.config_batch(seed=7, n_frames=4, n_min=2000, n_max=6000)
    for f in fr:
        check(ptm, f)
    f = I.config_mixed_phase(n_target=1 << 12)
    for m in (1, 2, 16, 6):
        check(ptm, f, mask=m)


def test_clusters_and_small_boxes(ptm):
    rng = I.rng_for(9)
    cl = [I.ico_cluster(2.556, rotation=I.random_rotation(rng), sigma=0.05, seed=i) for i in range(12)]
    f = I.isolated_clusters(cl, dtype=np.float32)
    check(ptm, f)
    f = I.crystal("bcc", I.A_BCC_FE, 2, sigma=0.05, seed=3, dtype=np.float32)     # atoms see own images
    check(ptm, f)


def _band_edge_strain(target=1e-3 + 1e-5):
    """Uniaxial strain of a perfect fcc lattice for which the gap between its
    two first-shell face areas is `target` x the mean squared distance (the
    gap grows monotonically with the strain), by bisection on the oracle's
    areas."""
    def gap(eps):
        f = I.crystal("fcc", I.A_FCC_CU, 3, deform=np.diag([1.0, 1.0, 1.0 + eps]), dtype=np.float64)
        F = O.Frame(f.positions, f.cell, f.pbc)
        ids, imgs, dr, d2 = F.knn(0, O.TOPO_N)
        v = np.asarray(dr, float).reshape(-1, 3)
        a = np.sort(O.voronoi_areas(v))[::-1]
        g = a[:-1] - a[1:]
        return g[g > 1e-9 * a[0]][0] / np.mean(np.sum(v * v, 1))
    lo, hi = 0.5e-3, 2e-3
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if gap(mid) < target else (lo, mid)
    return 0.5 * (lo + hi)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_band_edge_lattice_every_atom_decided_in_fp64(ptm, dtype):
    """A strained fcc lattice whose two first-shell face areas differ by the
    band plus half the guard: every atom has a gap at the band edge, so every
    atom goes to the FP64 pass, and the three quarters past the records the
    FP32 pass keeps find their neighbours again and recompute every face."""
    eps = _band_edge_strain()
    f = I.crystal("fcc", I.A_FCC_CU, 10, deform=np.diag([1.0, 1.0, 1.0 + eps]), dtype=dtype)
    atoms = np.sort(I.rng_for(81).choice(f.n, 400, replace=False))     # equivalent atoms: a sample
    st, g, ref, s = check(ptm, f, atoms=atoms)
    assert s["topo_fp64"] == f.n
    assert st["matched"] == len(atoms) and np.all(g["structure"] == 2)


def test_host_entry_and_noalloc_rejection(ptm):
    import ctypes as C
    from paper_1603_05143_gb300.binding import _frame, ptm_outputs, PTM_F32
    f = I.config_mixed_phase(n_target=1 << 13)
    d = run(ptm, f)
    h = ptm.classify_host(f.positions, f.cell, f.pbc, species=f.species, ordering="topological")
    for k in d:
        assert np.array_equal(d[k], h[k]), k
    # the allocation-free entry has no room for the ordering buffers
    fr = _frame(f.n, f.positions.ctypes.data, PTM_F32, None, f.cell, f.pbc, 31, math.inf, "topological")
    assert ptm.lib.ptm_classify_frame_noalloc(C.byref(fr), C.byref(ptm_outputs()), None) == 1


def test_batch_mixing_orderings_matches_single_frames(ptm):
    """A batch whose frames ask for either order gives each frame the results of
    a single-frame call with its order (the frames' ordering buffers are
    segments of one batch buffer)."""
    import torch
    frames = I.config_batch(seed=12, n_frames=6, n_min=1500, n_max=9000)
    frames.append(I.config_mixed_phase(n_target=1 << 13))
    orders = ["topological" if i % 2 == 0 else "euclidean" for i in range(len(frames))]
    dev = [{"positions": torch.from_numpy(f.positions).cuda(), "species": torch.from_numpy(f.species).cuda(),
            "cell": f.cell, "pbc": f.pbc, "ordering": o} for f, o in zip(frames, orders)]
    b = ptm.batch(dev)
    b.run()
    torch.cuda.synchronize()
    for f, o, out in zip(frames, orders, b.outputs):
        single = run(ptm, f, ordering=o)
        for k in single:
            assert np.array_equal(out[k].cpu().numpy(), single[k]), (f.name, o, k)
    b.close()


def test_server_serves_topological_frames(ptm):
    from paper_1603_05143_gb300 import Server
    frames = I.config_batch(seed=13, n_frames=5, n_min=1000, n_max=6000)
    srv = Server(ptm, streams=2)
    tickets = [srv.submit(f.positions, f.cell, f.pbc, species=f.species, ordering="topological") for f in frames]
    for f, t in zip(frames, tickets):
        out = srv.wait(t, 60000)
        single = run(ptm, f)
        for k in single:
            assert np.array_equal(out[k], single[k]), (f.name, k)
        srv.release(t)
    srv.close()


def test_topological_full_size_sampled(ptm):
    """The 2^20-atom polycrystal: a seeded sample checked one by one."""
    f = I.config_polycrystal()
    f.species = None
    atoms = np.sort(I.rng_for(79).choice(f.n, 2000, replace=False))
    st, g, ref, s = check(ptm, f, atoms=atoms)
    assert st["matched"] > 0.9 * len(atoms)
