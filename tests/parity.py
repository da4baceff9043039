"""Shared comparison of the CUDA path against the oracle.

Tolerances: structure, correspondence and alloy bit-exact; RMSD within 1e-5
(template units, where the mean neighbour distance is 1); scale within 1e-5
relative; orientation within 1e-4 rad modulo the template's rotation group;
strain components within 1e-5.
"""
import math

import numpy as np

import oracle as O

TOL_RMSD = 1e-5
TOL_SCALE = 1e-5
TOL_ANGLE = 1e-4
TOL_STRAIN = 1e-5


def qmat(q):
    a, b, c, d = [float(x) for x in q]
    return np.array([[1 - 2 * (c * c + d * d), 2 * (b * c - a * d), 2 * (b * d + a * c)],
                     [2 * (b * c + a * d), 1 - 2 * (b * b + d * d), 2 * (c * d - a * b)],
                     [2 * (b * d - a * c), 2 * (c * d + a * b), 1 - 2 * (b * b + c * c)]])


_groups = {}


def misorientation(qa, qb, structure):
    """Smallest angle between two orientations modulo the template group."""
    if structure not in _groups:
        _groups[structure] = [qmat(g) for g in O.group(structure - 1)[1]]
    Ra, Rb = qmat(qa), qmat(qb)
    best = 10.0
    for G in _groups[structure]:
        x = np.linalg.norm(Ra.T @ Rb @ G - np.eye(3)) / (2 * math.sqrt(2))
        best = min(best, 2 * math.asin(min(1.0, x)))
    return best


def compare(gpu: dict, ref: dict, atoms=None, check_orientation=True):
    """Assert parity of GPU outputs (numpy, full frame) with oracle outputs for
    `atoms` (oracle arrays are indexed by list position).  Returns error stats."""
    atoms = np.arange(len(ref["structure"])) if atoms is None else np.asarray(atoms)
    gs = gpu["structure"][atoms]
    bad = np.nonzero(gs != ref["structure"])[0]
    assert len(bad) == 0, f"structure mismatch at {atoms[bad[:10]]}: gpu {gs[bad[:10]]} oracle {ref['structure'][bad[:10]]}"
    gc = gpu["correspondence"][atoms]
    badc = np.nonzero(np.any(gc != ref["corr"], axis=1))[0]
    assert len(badc) == 0, f"correspondence mismatch at {atoms[badc[:5]]}: {gc[badc[:2]]} vs {ref['corr'][badc[:2]]}"
    ga = gpu["alloy"][atoms]
    assert np.array_equal(ga, ref["alloy"]), "alloy mismatch"
    m = ref["structure"] > 0
    stats = {"atoms": int(len(atoms)), "matched": int(m.sum())}
    if m.any():
        er = np.abs(gpu["rmsd"][atoms][m].astype(np.float64) - ref["rmsd"][m])
        es = np.abs(gpu["scale"][atoms][m] / ref["scale"][m] - 1)
        et = np.abs(gpu["strain"][atoms][m].astype(np.float64) - ref["strain"][m]).max(axis=(1, 2))
        stats.update(rmsd=float(er.max()), scale=float(es.max()), strain=float(et.max()))
        assert er.max() <= TOL_RMSD, f"rmsd error {er.max():.3g}"
        assert es.max() <= TOL_SCALE, f"scale error {es.max():.3g}"
        assert et.max() <= TOL_STRAIN, f"strain error {et.max():.3g}"
        if check_orientation:
            idx = np.nonzero(m)[0]
            pick = idx if len(idx) <= 400 else idx[np.linspace(0, len(idx) - 1, 400).astype(int)]
            ang = max(misorientation(gpu["quat"][atoms[i]], ref["quat"][i], int(ref["structure"][i])) for i in pick)
            stats["angle"] = ang
            assert ang <= TOL_ANGLE, f"misorientation {ang:.3g}"
    un = ~m
    if un.any():
        assert np.all(np.isinf(gpu["rmsd"][atoms][un]))
        assert np.all(gpu["correspondence"][atoms][un] == -1)
        assert np.all(gpu["quat"][atoms][un] == np.array([1, 0, 0, 0], np.float32))
        assert np.all(gpu["strain"][atoms][un] == 0)
    return stats
