"""Derived outputs (Sec. 7, 8, 5.1) on the GPU against the oracle (GPU only).

Tolerances: von Mises strain is sqrt(3/2) times the Frobenius norm of the
deviator of P, so its error is at most sqrt(3/2) * 3 * (strain tolerance 1e-5)
= 3.7e-5; the Rodrigues-Frank vector is compared where the two orientations
pick the same fundamental-zone representative (quaternions within 1e-4)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1603_05143_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL_VM = math.sqrt(1.5) * 3 * 1e-5


@pytest.fixture(scope="module")
def ptm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_05143_gb300 import PTM
    p = PTM(0)
    yield p
    p.close()


def _frames():
    rng = I.rng_for(21)
    E = np.eye(3) + np.array([[0.02, 0.01, 0.0], [0.01, -0.03, 0.015], [0.0, 0.015, 0.01]])
    return [I.crystal("fcc", I.A_FCC_CU, 5, sigma=0.05, seed=2, rotation=I.random_rotation(rng), deform=E,
                      dtype=np.float32),
            I.crystal("bcc", I.A_BCC_FE, 6, sigma=0.0, rotation=I.random_rotation(rng), deform=E, dtype=np.float32),
            I.config_mixed_phase(n_target=1 << 14)]


def _classify(ptm, f, outputs):
    import torch
    out = ptm.classify(torch.from_numpy(f.positions).cuda(), f.cell, f.pbc,
                       species=None if f.species is None else torch.from_numpy(f.species).cuda(), outputs=outputs)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def test_von_mises_and_rodrigues_against_oracle(ptm):
    from paper_1603_05143_gb300.binding import OUTPUT_FIELDS
    for f in _frames():
        g = _classify(ptm, f, OUTPUT_FIELDS)
        ref = O.classify_frame(f)
        m = ref["structure"] > 0
        assert np.array_equal(g["structure"], ref["structure"])
        vm_ref = O.von_mises(ref["strain"])
        assert np.abs(g["von_mises"][m] - vm_ref[m]).max() <= TOL_VM
        # the kernel's value is the definition applied to its own P
        assert np.abs(g["von_mises"][m] - O.von_mises(g["strain"][m])).max() < 2e-6
        rf_own = O.rodrigues(g["quat"][m])
        assert np.allclose(g["rodrigues"][m], rf_own, rtol=1e-5, atol=1e-6)
        same = np.abs(g["quat"][m].astype(np.float64) - ref["quat"][m]).max(axis=1) < 1e-4
        assert same.mean() > 0.95
        rf_ref = O.rodrigues(ref["quat"][m][same])
        assert np.abs(g["rodrigues"][m][same] - rf_ref).max() < 1e-3
        assert np.all(g["von_mises"][~m] == 0) and np.all(g["rodrigues"][~m] == 0)


def test_derived_outputs_optional_and_consistent_across_entry_points(ptm):
    from paper_1603_05143_gb300.binding import OUTPUT_FIELDS, OUTPUT_NAMES
    f = _frames()[2]
    a = _classify(ptm, f, OUTPUT_FIELDS)
    b = _classify(ptm, f, OUTPUT_NAMES)
    for k in OUTPUT_NAMES:
        assert np.array_equal(a[k], b[k]), k
    h = ptm.classify_host(f.positions, f.cell, f.pbc, species=f.species, outputs=OUTPUT_FIELDS)
    for k in OUTPUT_FIELDS:
        assert np.array_equal(a[k], h[k]), k
    # only von Mises requested: computed without the strain output
    c = _classify(ptm, f, ("structure", "von_mises"))
    assert np.array_equal(c["von_mises"], a["von_mises"])


def test_rmsd_histogram_matches_definition(ptm):
    import torch
    f = I.config_mixed_phase(n_target=1 << 16)
    out = ptm.classify(torch.from_numpy(f.positions).cuda(), f.cell, f.pbc,
                       species=torch.from_numpy(f.species).cuda())
    for nbins, rmax in ((100, 0.5), (7, 0.1234), (2048, 1.0), (1, 0.05)):
        h = ptm.rmsd_histogram(out["structure"], out["rmsd"], nbins, rmax).cpu().numpy()
        ref = O.rmsd_histogram(out["structure"].cpu().numpy(), out["rmsd"].cpu().numpy(), nbins, rmax)
        assert np.array_equal(h, ref), (nbins, rmax)
    assert h.sum() == int((out["structure"] > 0).sum())
    from paper_1603_05143_gb300 import PTMError
    with pytest.raises(PTMError):
        ptm.rmsd_histogram(out["structure"], out["rmsd"], 0, 0.5)
    with pytest.raises(PTMError):
        ptm.rmsd_histogram(out["structure"], out["rmsd"], 10, float("inf"))


def test_derived_outputs_in_a_batch(ptm):
    import torch
    from paper_1603_05143_gb300.binding import OUTPUT_FIELDS
    frames = _frames()
    dev = [{"positions": torch.from_numpy(f.positions).cuda(),
            "species": None if f.species is None else torch.from_numpy(f.species).cuda(),
            "cell": f.cell, "pbc": f.pbc} for f in frames]
    b = ptm.batch(dev, outputs=OUTPUT_FIELDS)
    b.run()
    torch.cuda.synchronize()
    for f, o in zip(frames, b.outputs):
        single = _classify(ptm, f, OUTPUT_FIELDS)
        for k in OUTPUT_FIELDS:
            assert np.array_equal(o[k].cpu().numpy(), single[k]), k
    b.close()
