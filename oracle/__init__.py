"""Python handle on the plain FP64 CPU oracle (``ptm_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use this module.  The library that serves users
(``paper_1603_05143_gb300``) never imports it, and it imports nothing from that
library.

Threads: ctypes releases the GIL during foreign calls, so ``classify`` splits
its atom list over a thread pool; a frame handle is read-only once built.
"""
from __future__ import annotations

import concurrent.futures as cf
import ctypes as C
import os
import pathlib
import subprocess

import numpy as np

HERE = pathlib.Path(__file__).resolve().parent
LIB = HERE / "_build" / "libptm_oracle.so"
SRC = HERE / "ptm_oracle.c"

TEMPLATES = ("SC", "FCC", "HCP", "ICO", "BCC")
K_OF = (6, 12, 12, 12, 14)
NONE, SC, FCC, HCP, ICO, BCC = range(6)
ALLOY_NONE, ALLOY_PURE, ALLOY_L10, ALLOY_L12_MAJ, ALLOY_L12_MIN, ALLOY_B2 = range(6)
ALL_TEMPLATES = 0x1F
ORDERINGS = {"euclidean": 0, "topological": 1}
TOPO_N = 18

_lib = None


def build(force: bool = False) -> pathlib.Path:
    """Compile the oracle with gcc (-ffp-contract=off keeps the distance contract)."""
    LIB.parent.mkdir(exist_ok=True)
    if force or not LIB.exists() or LIB.stat().st_mtime < SRC.stat().st_mtime:
        tmp = LIB.with_suffix(f".{os.getpid()}.tmp")
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", str(tmp), str(SRC), "-lm"])
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(str(LIB))
        P = C.c_void_p
        L.ptmo_init.restype = C.c_int
        L.ptmo_template.argtypes = [C.c_int, P, P]
        L.ptmo_group.argtypes = [C.c_int, P, P]
        L.ptmo_n_triangulations.argtypes = [C.c_int]
        L.ptmo_triangulation.argtypes = [C.c_int, C.c_int, P]
        L.ptmo_orient.argtypes = [P, P, P, P, P]
        L.ptmo_orient_exact.argtypes = [P, P, P, P]
        L.ptmo_hull.argtypes = [P, C.c_int, P]
        L.ptmo_weinberg.argtypes = [C.c_int, C.c_int, P, C.c_int, C.c_int, P, P]
        L.ptmo_superpose.argtypes = [C.c_int, P, P, P, P, P]
        L.ptmo_superpose.restype = C.c_double
        L.ptmo_polar.argtypes = [P, P, P]
        L.ptmo_polar.restype = None
        L.ptmo_frame_new.argtypes = [P, C.c_int, C.c_int64, P, P]
        L.ptmo_frame_new.restype = P
        L.ptmo_frame_free.argtypes = [P]
        L.ptmo_frame_free.restype = None
        L.ptmo_knn.argtypes = [P, C.c_int64, C.c_int, P, P, P, P]
        L.ptmo_quantise.argtypes = [C.c_int, P, P]
        L.ptmo_classify.argtypes = [P, P, C.c_uint32, C.c_double, C.c_int, P, C.c_int64] + [P] * 9
        L.ptmo_voronoi_areas.argtypes = [C.c_int, P, P]
        L.ptmo_topo_knn.argtypes = [P, C.c_int64, P, P, P]
        rc = L.ptmo_init()
        if rc:
            raise RuntimeError(f"oracle template construction failed ({rc})")
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


# ------------------------------------------------------------------ pieces
def template(S: int) -> np.ndarray:
    """Normalised template (k+1 x 3), slot 0 = centre (Eq. 4)."""
    w = np.zeros((15, 3))
    k = C.c_int()
    lib().ptmo_template(S, _p(w), C.byref(k))
    return w[: k.value + 1].copy()


def group(S: int):
    """Rotation group of template S: (permutations |G| x (k+1), quaternions |G| x 4)."""
    k = K_OF[S]
    perms = np.zeros((60, k + 1), np.int32)
    quats = np.zeros((60, 4))
    g = lib().ptmo_group(S, _p(perms), _p(quats))
    return perms[:g].copy(), quats[:g].copy()


def triangulations(S: int) -> np.ndarray:
    n = lib().ptmo_n_triangulations(S)
    k = K_OF[S]
    out = np.zeros((n, 2 * k - 4, 3), np.int32)
    for t in range(n):
        lib().ptmo_triangulation(S, t, _p(out[t]))
    return out


def orient(a, b, c, d, prio=(1, 2, 3, 4)) -> int:
    arrs = [np.ascontiguousarray(x, np.int64) for x in (a, b, c, d)]
    pr = np.ascontiguousarray(prio, np.int32)
    return lib().ptmo_orient(*[_p(x) for x in arrs], _p(pr))


def orient_exact(a, b, c, d) -> int:
    arrs = [np.ascontiguousarray(x, np.int64) for x in (a, b, c, d)]
    return lib().ptmo_orient_exact(*[_p(x) for x in arrs])


def hull(q: np.ndarray):
    """Brute-force SoS hull of k integer points: facets (ccw from outside) or None."""
    q = np.ascontiguousarray(q, np.int64)
    f = np.zeros((40, 3), np.int32)
    nf = lib().ptmo_hull(_p(q), len(q), _p(f))
    return None if nf < 0 else f[:nf].copy()


def weinberg(nv: int, facets: np.ndarray, u: int, v: int):
    facets = np.ascontiguousarray(facets, np.int32)
    code = np.zeros(80, np.uint8)
    lab = np.zeros(16, np.uint8)
    n = lib().ptmo_weinberg(nv, len(facets), _p(facets), u, v, _p(code), _p(lab))
    if n < 0:
        raise ValueError("not a directed edge")
    return code[:n].copy(), lab[:nv].copy()


def superpose(v: np.ndarray, w: np.ndarray):
    """(RMSD^2, quaternion (w,x,y,z), scale, lambda) for paired rows, Eq. 3."""
    v = np.ascontiguousarray(v, np.float64)
    w = np.ascontiguousarray(w, np.float64)
    q = np.zeros(4)
    s = C.c_double()
    lam = C.c_double()
    r2 = lib().ptmo_superpose(len(v), _p(v), _p(w), _p(q), C.byref(s), C.byref(lam))
    return r2, q, s.value, lam.value


def polar(A: np.ndarray):
    A = np.ascontiguousarray(A, np.float64)
    P = np.zeros((3, 3))
    U = np.zeros((3, 3))
    lib().ptmo_polar(_p(A), _p(P), _p(U))
    return P, U


def quantise(drc: np.ndarray):
    drc = np.ascontiguousarray(drc, np.float64)
    q = np.zeros(drc.shape, np.int64)
    e = lib().ptmo_quantise(len(drc), _p(drc), _p(q))
    return q, e


# ------------------------------------------------------------------ frames
class Frame:
    """Oracle view of one frame (keeps the position array alive)."""

    def __init__(self, positions, cell, pbc=(True, True, True)):
        pos = np.ascontiguousarray(positions)
        if pos.dtype not in (np.float32, np.float64):
            pos = pos.astype(np.float64)
        self.pos = pos
        self.cell = np.ascontiguousarray(cell, np.float64)
        self.pbc = np.ascontiguousarray([bool(x) for x in pbc], np.uint8)
        self.n = len(pos)
        self.h = lib().ptmo_frame_new(_p(self.pos), int(pos.dtype == np.float64), self.n,
                                      _p(self.cell), _p(self.pbc))

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.ptmo_frame_free(self.h)
            self.h = None

    def knn(self, atom: int, k: int = 14):
        """The k nearest periodic images of ``atom`` in the oracle's order (FP64
        squared distance, then atom id, then image): ids, images (k x 3), FP64
        contract vectors (k x 3) and squared distances."""
        ids = np.zeros(k, np.int32)
        imgs = np.zeros((k, 3), np.int32)
        dr = np.zeros((k, 3))
        d2 = np.zeros(k)
        m = lib().ptmo_knn(self.h, atom, k, _p(ids), _p(imgs), _p(dr), _p(d2))
        return ids[:m], imgs[:m], dr[:m], d2[:m]

    def topo_knn(self, atom: int):
        """Ids, images (k x 3) of the first min(14, m) neighbours in topological
        order, and the Voronoi face areas of the 18 nearest by Euclidean rank."""
        ids = np.zeros(14, np.int32)
        imgs = np.zeros((14, 3), np.int32)
        areas = np.zeros(TOPO_N)
        k = lib().ptmo_topo_knn(self.h, atom, _p(ids), _p(imgs), _p(areas))
        return ids[:k], imgs[:k], areas

    def classify(self, atoms=None, species=None, mask=ALL_TEMPLATES, rmsd_max=np.inf,
                 threads: int | None = None, chunk: int = 64, ordering: str = "euclidean"):
        """ordering "euclidean" (14 nearest) or "topological" (Eq. 5: the 18
        nearest reordered by Voronoi face area, first 14 kept)."""
        atoms = np.arange(self.n, dtype=np.int64) if atoms is None else np.ascontiguousarray(atoms, np.int64)
        m = len(atoms)
        sp = None if species is None else np.ascontiguousarray(species, np.int8)
        out = {
            "structure": np.zeros(m, np.int8), "alloy": np.zeros(m, np.int8),
            "rmsd": np.zeros(m), "scale": np.zeros(m), "quat": np.zeros((m, 4)),
            "strain": np.zeros((m, 3, 3)), "corr": np.zeros((m, 15), np.int32),
            "nbrs": np.zeros((m, 14), np.int32), "ncand": np.zeros(m, np.int32),
        }
        keys = ("structure", "alloy", "rmsd", "scale", "quat", "strain", "corr", "nbrs", "ncand")

        def run(lo, hi):
            ptrs = [out[k][lo:hi].ctypes.data_as(C.c_void_p) for k in keys]
            rc = lib().ptmo_classify(self.h, _p(sp), mask, rmsd_max, ORDERINGS[ordering],
                                     atoms[lo:hi].ctypes.data_as(C.c_void_p), hi - lo, *ptrs)
            if rc:
                raise RuntimeError(f"oracle classify failed ({rc})")

        threads = threads or os.cpu_count() or 1
        if threads <= 1 or m <= chunk:
            run(0, m)
        else:
            with cf.ThreadPoolExecutor(threads) as ex:
                list(ex.map(lambda lo: run(lo, min(m, lo + chunk)), range(0, m, chunk)))
        return out


def classify_frame(frame, atoms=None, mask=ALL_TEMPLATES, rmsd_max=np.inf, threads=None,
                   species="frame", ordering="euclidean"):
    """Classify atoms of an ``inputs.Frame``-like object (positions, cell, pbc, species)."""
    sp = frame.species if isinstance(species, str) and species == "frame" else species
    F = Frame(frame.positions, frame.cell, frame.pbc)
    return F.classify(atoms, species=sp, mask=mask, rmsd_max=rmsd_max, threads=threads, ordering=ordering)


# ------------------------------------------------------------ post-processing
# Plain definitions of the derived per-atom quantities; each reads the oracle's
# own outputs.

def von_mises(P: np.ndarray) -> np.ndarray:
    """Von Mises shear strain of the elastic strain matrix P (Sec. 8):
    sqrt(3/2 sum_ij P_ij^2 - 1/2 (sum_k P_kk)^2), for one (3, 3) matrix or a
    stack (..., 3, 3).  Unmatched atoms (P = 0) give 0."""
    P = np.asarray(P, np.float64)
    s = 1.5 * np.sum(P * P, axis=(-2, -1)) - 0.5 * np.trace(P, axis1=-2, axis2=-1) ** 2
    return np.sqrt(np.maximum(s, 0.0))


def rodrigues(q: np.ndarray) -> np.ndarray:
    """Rodrigues-Frank vector (x, y, z) / w of an orientation quaternion
    (w, x, y, z) with w > 0 (Sec. 7: the fundamental-zone orientation projected
    into Rodrigues-Frank space); (..., 4) -> (..., 3)."""
    q = np.asarray(q, np.float64)
    return q[..., 1:] / q[..., :1]


def rmsd_histogram(structure: np.ndarray, rmsd: np.ndarray, nbins: int, rmsd_max: float) -> np.ndarray:
    """Counts of matched atoms per structure (rows SC, FCC, HCP, ICO, BCC) and
    RMSD bin (Sec. 5.1: the histogram from which RMSD_max is chosen).  The
    paper fixes no binning; the rule here: the bin width factor nbins / rmsd_max
    is rounded to float32 once, each float32 RMSD is multiplied by it in one
    rounded float32 product, and bin b holds the atoms whose product p has
    b <= p < b + 1 (so the decision is taken in the precision of the stored
    RMSD); column nbins counts the atoms at or beyond rmsd_max, and unmatched
    atoms (infinite RMSD) are not counted."""
    structure = np.asarray(structure)
    r = np.asarray(rmsd, np.float32)
    scale = np.float32(nbins / rmsd_max)
    out = np.zeros((5, nbins + 1), np.int64)
    for S in range(1, 6):
        v = r[(structure == S) & np.isfinite(r)]
        b = np.floor((v * scale).astype(np.float32)).astype(np.int64)
        out[S - 1] = np.bincount(np.minimum(b, nbins), minlength=nbins + 1)
    return out


def voronoi_areas(v: np.ndarray) -> np.ndarray:
    """Face areas of the Voronoi cell of the origin among the points v (m x 3):
    the bisector plane of each point clipped by the others (Sec. 3, Eq. 5)."""
    v = np.ascontiguousarray(v, np.float64)
    a = np.zeros(len(v))
    if lib().ptmo_voronoi_areas(len(v), _p(v), _p(a)):
        raise ValueError("1 to 64 points")
    return a
