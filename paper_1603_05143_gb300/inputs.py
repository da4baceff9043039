"""Seeded synthetic frames shaped like the PTM paper's workloads.

This module only builds inputs (positions, periodic cells, species).  It holds
none of the structure-identification arithmetic, so both the CUDA path and the
CPU oracle may be fed from it.

Every generator draws from ``numpy.random.Generator(PCG64(seed))``.  The lattices
are the five structures of Table 1 (sc, fcc, hcp, bcc, plus icosahedral clusters)
and the ordered alloys of Sec. 6 (L1_0, L1_2, B2).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

A_FCC_CU = 3.615      # Angstrom
A_BCC_FE = 2.8665
A_L12 = 3.75
A_SC = 2.5
A_HCP = 2.556         # nearest-neighbour distance, ideal c/a


@dataclasses.dataclass
class Frame:
    """One periodic frame: positions (n x 3), cell rows = cell vectors."""
    positions: np.ndarray
    cell: np.ndarray                 # (3, 3) float64, rows are the cell vectors
    pbc: tuple = (True, True, True)
    species: np.ndarray | None = None   # int8 per atom, or None
    name: str = ""
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.positions.shape[0])


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation (Shoemake's subgroup algorithm, unit quaternion)."""
    u1, u2, u3 = rng.random(3)
    q = np.array([math.sqrt(1 - u1) * math.sin(2 * math.pi * u2),
                  math.sqrt(1 - u1) * math.cos(2 * math.pi * u2),
                  math.sqrt(u1) * math.sin(2 * math.pi * u3),
                  math.sqrt(u1) * math.cos(2 * math.pi * u3)])
    w, x, y, z = q[3], q[0], q[1], q[2]
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


# ---------------------------------------------------------------- unit cells
def unit_cell(kind: str, a: float):
    """(cell rows, fractional basis, species per basis site) of a conventional cell."""
    if kind == "sc":
        return np.eye(3) * a, np.zeros((1, 3)), np.zeros(1, np.int8)
    if kind in ("fcc", "l12", "l10"):
        basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
        if kind == "l12":      # Cu3Au: Au (1) at the corner, Cu (0) on the faces
            sp = np.array([1, 0, 0, 0], np.int8)
        elif kind == "l10":    # CuAu: alternate (001) layers
            sp = np.array([0, 0, 1, 1], np.int8)
        else:
            sp = np.zeros(4, np.int8)
        return np.eye(3) * a, basis, sp
    if kind in ("bcc", "b2"):
        basis = np.array([[0, 0, 0], [0.5, 0.5, 0.5]])
        sp = np.array([0, 1], np.int8) if kind == "b2" else np.zeros(2, np.int8)
        return np.eye(3) * a, basis, sp
    if kind == "hcp":          # orthohexagonal cell, 4 atoms, ideal c/a
        c = a * math.sqrt(8.0 / 3.0)
        cell = np.diag([a, a * math.sqrt(3.0), c])
        basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 1.0 / 6.0, 0.5], [0, 2.0 / 3.0, 0.5]])
        return cell, basis, np.zeros(4, np.int8)
    raise ValueError(kind)


def crystal(kind: str, a: float, reps, *, sigma: float = 0.0, seed: int = 0,
            rotation: np.ndarray | None = None, deform: np.ndarray | None = None,
            dtype=np.float64, wrap: bool = True, name: str = "") -> Frame:
    """Periodic supercell of ``reps`` conventional cells.

    ``rotation`` and ``deform`` (3x3) act on both positions and cell vectors, so
    the crystal stays periodic (the cell becomes triclinic).  Gaussian noise of
    standard deviation ``sigma`` is added per component.
    """
    rng = rng_for(seed)
    cell0, basis, sp0 = unit_cell(kind, a)
    reps = np.broadcast_to(np.asarray(reps, int), (3,))
    grid = np.stack(np.meshgrid(*[np.arange(r) for r in reps], indexing="ij"), -1).reshape(-1, 3)
    frac = (grid[:, None, :] + basis[None, :, :]).reshape(-1, 3)
    pos = frac @ cell0
    species = np.tile(sp0, len(grid))
    cell = cell0 * reps[:, None]
    lin = np.eye(3)
    if rotation is not None:
        lin = rotation @ lin
    if deform is not None:
        lin = deform @ lin
    pos = pos @ lin.T
    cell = cell @ lin.T
    if sigma > 0:
        pos = pos + rng.normal(0.0, sigma, pos.shape)
    if wrap:
        pos = wrap_positions(pos, cell)
    return Frame(pos.astype(dtype), cell.astype(np.float64), (True, True, True), species,
                 name or kind, {"kind": kind, "a": a, "reps": reps.tolist(), "sigma": sigma})


def wrap_positions(pos: np.ndarray, cell: np.ndarray) -> np.ndarray:
    """Map positions into the parallelepiped spanned by the cell rows."""
    f = pos @ np.linalg.inv(cell)
    f = f - np.floor(f)
    f[f >= 1.0] = 0.0
    return f @ cell


def ico_cluster(r: float = 2.556, *, rotation=None, sigma=0.0, seed=0) -> np.ndarray:
    """Centre plus the 12 vertices of a regular icosahedron at distance r."""
    phi = (1 + math.sqrt(5)) / 2
    v = []
    for s1 in (1, -1):
        for s2 in (1, -1):
            v += [(0, s1, s2 * phi), (s1, s2 * phi, 0), (s2 * phi, 0, s1)]
    v = np.array(v, float)
    v *= r / np.linalg.norm(v[0])
    pts = np.vstack([np.zeros(3), v])
    if rotation is not None:
        pts = pts @ rotation.T
    if sigma > 0:
        pts = pts + rng_for(seed).normal(0, sigma, pts.shape)
    return pts


def isolated_clusters(clusters, spacing: float = 30.0, dtype=np.float64) -> Frame:
    """Place point clusters on a coarse grid inside one large periodic box."""
    m = len(clusters)
    side = int(math.ceil(m ** (1 / 3)))
    pos = []
    for i, c in enumerate(clusters):
        g = np.array([i % side, (i // side) % side, i // (side * side)], float)
        pos.append(c + (g + 0.5) * spacing)
    cell = np.eye(3) * spacing * side
    return Frame(np.vstack(pos).astype(dtype), cell, (True, True, True), None, "clusters")


# ------------------------------------------------------------ workload configs
def config_fcc_small(seed: int = 1603) -> Frame:
    """4000-atom fcc Cu, 10^3 cells, sigma 0.10 A, float64 positions."""
    f = crystal("fcc", A_FCC_CU, 10, sigma=0.10, seed=seed, dtype=np.float64, name="fcc4000")
    return f


def config_polycrystal(seed: int = 5143, n_target: int = 1 << 20, n_grains: int = 16,
                       n_faults: int = 4, sigma: float = 0.15) -> Frame:
    """Periodic Voronoi polycrystal of fcc Cu with stacking-fault slabs.

    The box is the fcc-density cube for ``n_target`` atoms (L = 231.36 A for 2^20).
    Each grain fills the part of the box closest (minimum image) to its centre
    with its own randomly rotated lattice; atoms closer than 1.5 A across grain
    boundaries are thinned; the count is trimmed (or, rarely, padded with random
    points) to exactly ``n_target``.  In ``n_faults`` grains all atoms above a
    {111} plane through the grain centre are shifted by a/6<112>, which leaves
    two hcp planes at the fault.
    """
    rng = rng_for(seed)
    a = A_FCC_CU
    L = (n_target / 4.0) ** (1.0 / 3.0) * a
    cell = np.eye(3) * L
    centres = rng.random((n_grains, 3)) * L
    rots = [random_rotation(rng) for _ in range(n_grains)]
    fault_grains = set(rng.choice(n_grains, size=min(n_faults, n_grains), replace=False).tolist())
    # radius of each grain's cell from a coarse ownership grid
    g = (np.arange(40) + 0.5) / 40 * L
    grid = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    dg = np.stack([_min_image_dist2(grid, c, L) for c in centres], 1)
    own = dg.argmin(1)
    rg = np.array([math.sqrt(dg[own == i, i].max()) if np.any(own == i) else 0.0
                   for i in range(n_grains)]) + 2 * L / 40 + 2 * a
    cell0, basis, _ = unit_cell("fcc", a)
    pieces = []
    for gi in range(n_grains):
        m = int(math.ceil(rg[gi] / a)) + 1
        ijk = np.stack(np.meshgrid(*[np.arange(-m, m + 1)] * 3, indexing="ij"), -1).reshape(-1, 3)
        p = ((ijk[:, None, :] + basis[None]).reshape(-1, 3)) @ cell0
        p = p[np.einsum("ij,ij->i", p, p) <= rg[gi] ** 2]
        if gi in fault_grains:
            nrm = np.array([1.0, 1.0, 1.0]) / math.sqrt(3)
            p[p @ nrm > a / (4 * math.sqrt(3))] += a / 6.0 * np.array([1.0, 1.0, -2.0])
        off = p @ rots[gi].T
        off = off[np.all(np.abs(off) < L / 2, axis=1)]          # minimal image only
        q = off + centres[gi]
        d_own = np.einsum("ij,ij->i", off, off)
        keep = np.ones(len(q), bool)
        for gj in range(n_grains):
            if gj != gi:
                keep &= d_own < _min_image_dist2(q, centres[gj], L)
        pieces.append(np.mod(q[keep], L))
    pos = np.vstack(pieces)
    pos = _thin_close_pairs(pos, L, 1.5, rng)
    n = len(pos)
    if n > n_target:
        pos = pos[np.sort(rng.choice(n, n_target, replace=False))]
    elif n < n_target:
        extra = rng.random((n_target - n, 3)) * L
        pos = np.vstack([pos, extra])
    pos = pos + rng.normal(0.0, sigma, pos.shape)
    pos = np.mod(pos, L)
    pos[pos >= L] = 0.0
    return Frame(pos.astype(np.float32), cell, (True, True, True), None, "polycrystal",
                 {"L": L, "grains": n_grains, "faults": sorted(fault_grains), "raw_count": n,
                  "padded": max(0, n_target - n)})


def _min_image_dist2(p, c, L):
    d = p - c
    d -= L * np.round(d / L)
    return np.einsum("ij,ij->i", d, d)


def _thin_close_pairs(pos, L, dmin, rng):
    """Drop one atom of every pair closer than dmin (periodic cube), grid accelerated."""
    n = len(pos)
    nb = max(1, int(L // dmin))
    w = L / nb
    cidx = np.minimum((pos // w).astype(np.int64), nb - 1)
    key = (cidx[:, 0] * nb + cidx[:, 1]) * nb + cidx[:, 2]
    order = np.argsort(key, kind="stable")
    skey = key[order]
    starts = np.searchsorted(skey, np.arange(nb ** 3))
    ends = np.searchsorted(skey, np.arange(nb ** 3), side="right")
    removed = np.zeros(n, bool)
    prio = rng.permutation(n)
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dz in (-1, 0, 1):
                nc = (cidx + [dx, dy, dz]) % nb
                nkey = (nc[:, 0] * nb + nc[:, 1]) * nb + nc[:, 2]
                # pairs (i, j in neighbouring cell): vectorise over the max occupancy
                occ = ends[nkey] - starts[nkey]
                for t in range(int(occ.max()) if n else 0):
                    has = occ > t
                    ii = np.nonzero(has)[0]
                    jj = order[starts[nkey[ii]] + t]
                    ok = jj != ii
                    ii, jj = ii[ok], jj[ok]
                    d = pos[jj] - pos[ii]
                    d -= L * np.round(d / L)
                    close = np.einsum("ij,ij->i", d, d) < dmin * dmin
                    ii, jj = ii[close], jj[close]
                    lose = np.where(prio[ii] > prio[jj], ii, jj)
                    removed[lose] = True
    return pos[~removed]


LIQUID_DENSITY = 0.058   # A^-3: ~70 % of fcc Cu, reachable by bounded random sequential addition


def config_mixed_phase(seed: int = 13, n_target: int = 1 << 22, sigma: float = 0.20,
                       antisite: float = 0.10, ico_fraction: float = 0.01) -> Frame:
    """Five equal slabs along x: bcc Fe, fcc Cu, L1_2 Cu3Au (int8 species, 10 %
    antisites), sc, and a liquid: random sequential addition with a 2.0 A
    minimum distance, seeded with 13-atom Mackay icosahedra (1 % of the liquid
    atoms).  fcc density is ~93 % of the RSA jamming limit for 2.0 A, which
    uniform proposals approach only slowly, so the box is sized for a liquid
    near LIQUID_DENSITY.  Each crystal's lattice constant is rescaled (by well
    under 1 % at 2^22 atoms) to a whole number of cells across Ly, so the
    periodic y and z boundaries leave no seam; the liquid takes exactly the
    atoms that remain to n_target."""
    rng = rng_for(seed)
    phases = [("bcc", A_BCC_FE), ("fcc", A_FCC_CU), ("l12", A_L12), ("sc", A_SC)]
    rho = [len(unit_cell(k, a)[1]) / a ** 3 for k, a in phases] + [LIQUID_DENSITY]
    ly = (n_target / (sum(rho) * 0.4)) ** (1.0 / 3.0)
    lx = 2.0 * ly
    t = lx / 5.0
    pieces, species = [], []
    for si, (kind, a0) in enumerate(phases):
        ncell = max(1, int(round(ly / a0)))
        a = ly / ncell
        cell0, basis, sp0 = unit_cell(kind, a)
        nx = int(math.ceil(t / a))
        g = np.stack(np.meshgrid(np.arange(nx), np.arange(ncell), np.arange(ncell), indexing="ij"), -1).reshape(-1, 3)
        p = ((g[:, None, :] + basis[None]).reshape(-1, 3)) @ cell0
        sp = np.tile(sp0, len(g)).astype(np.int8)
        keep = p[:, 0] < t
        p, sp = p[keep], sp[keep]
        p[:, 0] += si * t
        if kind == "l12":
            flip = rng.random(len(sp)) < antisite
            sp = np.where(flip, 1 - sp, sp).astype(np.int8)
        pieces.append(p)
        species.append(sp)
    n_liq = n_target - sum(len(p) for p in pieces)
    liq = _rsa_liquid(rng, (4 * t, 5 * t), ly, n_liq, 2.0, ico_fraction)
    if len(liq) < n_liq:
        raise RuntimeError(f"liquid short of atoms: {len(liq)} < {n_liq}")
    pieces.append(liq)
    species.append(np.zeros(len(liq), np.int8))
    pos = np.vstack(pieces)
    pos = pos + rng.normal(0.0, sigma, pos.shape)
    cell = np.diag([lx, ly, ly])
    pos = wrap_positions(pos, cell)
    return Frame(pos.astype(np.float32), cell, (True, True, True), np.concatenate(species), "mixed_phase",
                 {"Lx": lx, "Ly": ly, "liquid_atoms": len(liq),
                  "liquid_density": len(liq) / (t * ly * ly)})


def _rsa_liquid(rng, xr, ly, n_target, dmin, ico_fraction, max_rounds=60, batch=None):
    """Random sequential addition of points at least dmin apart in the slab
    x in [xr), periodic in y and z, seeded with 13-atom Mackay icosahedra
    (centre + 12 at 2.556 A).  Proposals come in vectorised rounds: each round
    rejects points too close to the accepted set (KD tree) and resolves clashes
    inside the round in proposal order.  Close to the RSA jamming density the
    acceptance rate falls, so the rounds are capped and the count reached is
    returned."""
    from scipy.spatial import cKDTree
    x0, x1 = xr
    box = np.array([x1 - x0, ly, ly])
    pts = np.zeros((0, 3))
    n_ico = int(ico_fraction * n_target / 13)
    if n_ico:
        cs = np.column_stack([rng.uniform(3, box[0] - 3, n_ico), rng.uniform(0, ly, n_ico), rng.uniform(0, ly, n_ico)])
        cl = np.vstack([ico_cluster(2.556, rotation=random_rotation(rng)) + c for c in cs])
        cl[:, 1:] %= ly
        keep = np.ones(n_ico, bool)
        tree = cKDTree(cs, boxsize=[1e9, ly, ly])
        for i, j in sorted(tree.query_pairs(2.556 * 2 + dmin)):
            if keep[i]:
                keep[j] = False
        pts = cl.reshape(n_ico, 13, 3)[keep].reshape(-1, 3)
    batch = batch or max(4096, n_target // 8)
    rate = 1.0    # acceptance rate of the previous round sizes the next one
    for _ in range(max_rounds):
        need = n_target - len(pts)
        if need <= 0:
            break
        m = int(min(max(batch, 2.0 * need / max(rate, 1e-3)), 8 * n_target + 4096))
        cand = rng.random((m, 3)) * box
        if len(pts):
            tree = cKDTree(pts, boxsize=[1e9, ly, ly])
            dist, _ = tree.query(cand, k=1, distance_upper_bound=dmin)
            cand = cand[~np.isfinite(dist)]
        if len(cand) > 1:
            ok = np.ones(len(cand), bool)
            for i, j in sorted(cKDTree(cand, boxsize=[1e9, ly, ly]).query_pairs(dmin)):
                if ok[i] and ok[j]:
                    ok[j] = False
            cand = cand[ok]
        rate = max(len(cand), 1) / m
        pts = np.vstack([pts, cand[:need]])
    out = pts.copy()
    out[:, 0] += x0
    return out


_BATCH_KINDS = [("fcc", A_FCC_CU), ("hcp", A_HCP), ("bcc", A_BCC_FE), ("l10", A_L12),
                ("l12", A_L12), ("sc", A_SC)]


def _lattice_frame(rng, kind, a, target, fi, sigma_max, strain_max):
    """A random rotation, symmetric affine strain (|E_ij| <= strain_max) and
    noise (uniform in [0, sigma_max], zero for one frame in ten) applied to a
    lattice of about `target` atoms."""
    cell0, basis, _ = unit_cell(kind, a)
    per = len(basis)
    side = max(3, int(round((target / per) ** (1 / 3))))
    reps = np.array([side, side, side])
    if kind == "hcp":   # orthohexagonal cell is elongated in y
        reps = np.array([side, max(3, int(round(side / math.sqrt(3)))), max(3, int(round(side * 0.61)))])
    R = random_rotation(rng)
    E = rng.uniform(-strain_max, strain_max, (3, 3))
    E = 0.5 * (E + E.T)
    sig = float(rng.uniform(0.0, sigma_max))
    if rng.random() < 0.1:
        sig = 0.0
    seed_f = int(rng.integers(1 << 31))
    f = crystal(kind, a, reps, sigma=sig, seed=seed_f, rotation=R, deform=np.eye(3) + E,
                dtype=np.float32, name=f"{kind}{fi}")
    f.meta.update({"E": E.tolist(), "R": R.tolist()})
    return f


def config_batch(seed: int = 256, n_frames: int = 256, n_min: float = 1e3, n_max: float = 1e6,
                 sigma_max: float = 0.25, strain_max: float = 0.05):
    """Uneven frames of random lattices, orientations, noise and affine strain;
    sizes log-uniform in [n_min, n_max]."""
    rng = rng_for(seed)
    frames = []
    for fi in range(n_frames):
        kind, a = _BATCH_KINDS[int(rng.integers(len(_BATCH_KINDS)))]
        target = math.exp(rng.uniform(math.log(n_min), math.log(n_max)))
        frames.append(_lattice_frame(rng, kind, a, target, fi, sigma_max, strain_max))
    return frames


def tile_frame(f: Frame, reps) -> Frame:
    """Periodic repeat of a frame reps[0] x reps[1] x reps[2] times."""
    reps = np.asarray(reps, int)
    g = np.stack(np.meshgrid(*[np.arange(r) for r in reps], indexing="ij"), -1).reshape(-1, 3)
    shift = g @ f.cell
    pos = (f.positions[None, :, :].astype(np.float64) + shift[:, None, :]).reshape(-1, 3)
    sp = None if f.species is None else np.tile(f.species, len(g))
    return Frame(pos.astype(f.positions.dtype), f.cell * reps[:, None], f.pbc, sp, f.name, dict(f.meta, reps=reps.tolist()))


_SERVE_TILES = [(1, 1, 1), (2, 1, 1), (2, 2, 1), (3, 2, 1), (2, 2, 2), (3, 2, 2), (5, 3, 1)]


def config_serve_pool(seed: int = 4096, n_sizes: int = 16, n_min: float = 1e4, n_max: float = 1.6e7,
                      strain_max: float = 0.05, tile_atoms: int = 1 << 20):
    """Frames for a serving workload: mixed-phase frames (bcc / fcc / L1_2 /
    sc / liquid slabs, sigma 0.20 A) whose sizes are log-spaced over
    [n_min, n_max], so a frame drawn uniformly from the pool has a log-uniform
    size.  Frames up to tile_atoms are generated at their size; larger ones
    are periodic tilings of one tile_atoms frame.  Each then gets a random
    rotation and a symmetric affine strain with |E_ij| <= strain_max (cell and
    positions alike, so the frame stays periodic and becomes triclinic)."""
    rng = rng_for(seed)
    base = None
    frames = []
    for fi, target in enumerate(np.geomspace(n_min, n_max, n_sizes)):
        if target <= 1.25 * tile_atoms:
            f = config_mixed_phase(seed=seed + 1 + fi, n_target=int(round(target)))
        else:
            if base is None:
                base = config_mixed_phase(seed=seed, n_target=tile_atoms)
            reps = min(_SERVE_TILES, key=lambda r: abs(math.log(np.prod(r) * tile_atoms / target)))
            f = tile_frame(base, reps)
        R = random_rotation(rng)
        E = rng.uniform(-strain_max, strain_max, (3, 3))
        E = 0.5 * (E + E.T)
        lin = (np.eye(3) + E) @ R
        pos = wrap_positions(f.positions.astype(np.float64) @ lin.T, f.cell @ lin.T)
        frames.append(Frame(pos.astype(np.float32), f.cell @ lin.T, f.pbc, f.species, f"mixed{fi}",
                            dict(f.meta, E=E.tolist(), R=R.tolist())))
    return frames


def poisson_arrivals(rng, n: int, rate_hz: float, pool_size: int):
    """n request times (seconds from 0) of a Poisson process of rate rate_hz,
    each with a pool index drawn uniformly."""
    t = np.cumsum(rng.exponential(1.0 / rate_hz, n))
    return t - t[0], rng.integers(pool_size, size=n)


def describe(frame: Frame) -> str:
    return f"{frame.name}: n={frame.n} dtype={frame.positions.dtype} cell={np.round(frame.cell, 3).tolist()}"
