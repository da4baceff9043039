"""Template tables for the CUDA kernels, generated at build time.

For each reference template of Table 1 this module builds, from geometry alone:

* the normalised template (barycentre at the origin, mean distance 1 over the
  centre and its k neighbours, Eq. 4);
* its proper rotation group (orders 24, 24, 6, 60, 24; Sec. 4);
* every triangulation of its hull: the hull faces are found with qhull and each
  square or rhombus face is split along either diagonal (2^6 for FCC and HCP,
  2^12 for BCC; Sec. 4);
* the canonical form of each triangulation's planar graph and, per canonical
  code, the symmetry-inequivalent correspondences "canonical label -> template
  slot" (Appendix A: equivalent correspondences give equal RMSD).

Canonical form (one embedding, orientation-preserving; Sec. 4): every directed
edge u->v gets the key (deg u, deg v, deg w1, deg w2, deg a1, deg b1, deg a2,
deg b2), where (u, v, w1) and (v, u, w2) are the two facets on the edge and
a1, b1, a2, b2 the third vertices of the facets across their outer edges
(v, w1), (w1, u), (u, w2), (w2, v); among the edges with the largest key
(compared in that order) are the start edges.  A Weinberg walk from a start
edge gives a code and a first-visit labelling; the key is invariant under
orientation-preserving isomorphisms, so the codes from the start edges of two
embedded graphs are the same set exactly when such an isomorphism exists, and
a code determines the graph.  The tables therefore list, per template
triangulation, the code of every start edge (starts related by an automorphism
share one), and the kernels need one walk per hull (the paper's canonical form
takes the smallest code over all starts; one lookup among all start codes is
the same isomorphism test).

Weinberg walk (counter-clockwise rotation seen from outside): at a new vertex
leave by the edge after the arrival edge; at an old vertex reached along an edge
never walked before, walk straight back; otherwise leave by the first unused
edge after the arrival edge.  The code is the sequence of first-visit labels.

The emitted C header is included by the CUDA sources.
"""
from __future__ import annotations

import itertools
import math
import pathlib

import numpy as np

TEMPLATE_NAMES = ("SC", "FCC", "HCP", "ICO", "BCC")
K = (6, 12, 12, 12, 14)
NIB_WORDS = 9           # labels 3..73 of the longest code, four bits each (labels 1, 2 are fixed)
HASH_MUL = 0x100000001B3
HASH_INIT = 0xCBF29CE484222325
MASK64 = (1 << 64) - 1


# ------------------------------------------------------------ template shells
def _shell(name: str) -> np.ndarray:
    """Neighbour positions (k x 3) of each reference template, fixed slot order."""
    if name == "SC":
        return np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float)
    if name == "FCC":
        rows = [(1, 1, 0), (1, -1, 0), (-1, 1, 0), (-1, -1, 0), (1, 0, 1), (1, 0, -1),
                (-1, 0, 1), (-1, 0, -1), (0, 1, 1), (0, 1, -1), (0, -1, 1), (0, -1, -1)]
        return np.array(rows, float) / math.sqrt(2.0)
    if name == "HCP":
        ring = [(math.cos(t * math.pi / 3), math.sin(t * math.pi / 3), 0.0) for t in range(6)]
        r, h = 1 / math.sqrt(3), math.sqrt(2 / 3)
        tri = [(r * math.cos(a), r * math.sin(a)) for a in (math.pi / 6, 5 * math.pi / 6, 1.5 * math.pi)]
        up = [(x, y, h) for x, y in tri]
        dn = [(x, y, -h) for x, y in tri]
        return np.array(ring + up + dn, float)
    if name == "ICO":
        g = (1 + math.sqrt(5)) / 2
        rows = []
        for a in (1, -1):
            for b in (1, -1):
                rows += [(0, a, b * g), (a, b * g, 0), (b * g, 0, a)]
        return np.array(rows, float)
    if name == "BCC":
        cube = [(sx * .5, sy * .5, sz * .5) for sx in (1, -1) for sy in (1, -1) for sz in (1, -1)]
        axes = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
        return np.array(cube + axes, float)
    raise KeyError(name)


def normalised_template(name: str) -> np.ndarray:
    """(k+1) x 3: centre at slot 0, barycentre removed, mean distance 1 (Eq. 4)."""
    p = np.vstack([np.zeros(3), _shell(name)])
    p = p - p.mean(axis=0)
    return p / np.linalg.norm(p, axis=1).mean()


# ---------------------------------------------------------------- rotations
def rotation_group(w: np.ndarray):
    """Proper rotations mapping the shell (slots 1..k) onto itself.

    Every rotation is pinned down by the images of two independent shell points;
    candidates come from the orthogonal Procrustes fit of those pairs."""
    pts = w[1:]
    k = len(pts)
    i0 = 0
    i1 = next(j for j in range(1, k) if np.linalg.norm(np.cross(pts[0], pts[j])) > 1e-6)
    perms, mats = [], []
    for a in range(k):
        for b in range(k):
            if a == b:
                continue
            src = np.stack([pts[i0], pts[i1], np.cross(pts[i0], pts[i1])])
            dst = np.stack([pts[a], pts[b], np.cross(pts[a], pts[b])])
            u, _, vt = np.linalg.svd(dst.T @ src)
            R = u @ vt
            if np.linalg.det(R) < 0:
                continue
            img = pts @ R.T
            d = np.linalg.norm(img[:, None, :] - pts[None, :, :], axis=2)
            j = d.argmin(axis=1)
            if d[np.arange(k), j].max() > 1e-9 or len(set(j.tolist())) != k:
                continue
            perm = (0,) + tuple(int(x) + 1 for x in j)
            if perm not in perms:
                perms.append(perm)
                mats.append(R)
    return perms, mats


def rot_to_quat(R: np.ndarray) -> np.ndarray:
    """Unit quaternion (w, x, y, z), w >= 0, from the eigenvector of the 4x4
    symmetric matrix whose largest eigenvalue belongs to R."""
    m = np.array([
        [R[0, 0] + R[1, 1] + R[2, 2], R[2, 1] - R[1, 2], R[0, 2] - R[2, 0], R[1, 0] - R[0, 1]],
        [R[2, 1] - R[1, 2], R[0, 0] - R[1, 1] - R[2, 2], R[0, 1] + R[1, 0], R[0, 2] + R[2, 0]],
        [R[0, 2] - R[2, 0], R[0, 1] + R[1, 0], R[1, 1] - R[0, 0] - R[2, 2], R[1, 2] + R[2, 1]],
        [R[1, 0] - R[0, 1], R[0, 2] + R[2, 0], R[1, 2] + R[2, 1], R[2, 2] - R[0, 0] - R[1, 1]]])
    vals, vecs = np.linalg.eigh(m)
    q = vecs[:, -1]
    return q if q[0] >= 0 else -q


# ------------------------------------------------------------ triangulations
def hull_faces(w: np.ndarray):
    """Faces of the template hull as counter-clockwise (from outside) slot lists,
    merging coplanar qhull triangles."""
    from scipy.spatial import ConvexHull
    pts = w[1:]
    hull = ConvexHull(pts)
    groups: dict = {}
    for simplex, eq in zip(hull.simplices, hull.equations):
        key = tuple(np.round(eq, 6))
        groups.setdefault(key, set()).update(int(s) for s in simplex)
    faces = []
    for eq, verts in groups.items():
        n = np.array(eq[:3])
        vs = sorted(verts)
        c = pts[vs].mean(axis=0)
        e1 = pts[vs[0]] - c
        e2 = np.cross(n, e1)
        ang = [math.atan2((pts[v] - c) @ e2, (pts[v] - c) @ e1) for v in vs]
        order = [v + 1 for _, v in sorted(zip(ang, vs))]
        faces.append(order)
    faces.sort()
    return faces


def triangulations(w: np.ndarray):
    """All triangulations: each 4-gon face gets one of its two diagonals."""
    faces = hull_faces(w)
    quads = [f for f in faces if len(f) == 4]
    tris = [tuple(f) for f in faces if len(f) == 3]
    assert all(len(f) in (3, 4) for f in faces)
    out = []
    for choice in itertools.product((0, 1), repeat=len(quads)):
        t = list(tris)
        for (a, b, c, d), ch in zip(quads, choice):
            t += [(a, b, c), (a, c, d)] if ch == 0 else [(b, c, d), (b, d, a)]
        out.append(t)
    return out


# ----------------------------------------------------- canonical form (GPU)
def _third(facets):
    th = {}
    for a, b, c in facets:
        th[(a, b)] = c
        th[(b, c)] = a
        th[(c, a)] = b
    return th


def weinberg(facets, u, v):
    """Weinberg code and first-visit labelling from the directed edge u -> v."""
    th = _third(facets)
    lab = {u: 1}
    code = [1]
    used = {(u, v)}
    fresh = v not in lab
    if fresh:
        lab[v] = len(lab) + 1
    code.append(lab[v])
    while True:
        if fresh:
            w = th[(v, u)]
        elif (v, u) not in used:
            w = u
        else:
            w = None
            x = th[(v, u)]
            while x != u:
                if (v, x) not in used:
                    w = x
                    break
                x = th[(v, x)]
            if w is None:
                break
        used.add((v, w))
        u, v = v, w
        fresh = v not in lab
        if fresh:
            lab[v] = len(lab) + 1
        code.append(lab[v])
    return tuple(code), lab


def edge_key(deg, th, a, b):
    z, w = th[(a, b)], th[(b, a)]
    return (deg[a], deg[b], deg[z], deg[w],
            deg[th[(z, b)]], deg[th[(a, z)]], deg[th[(w, a)]], deg[th[(b, w)]])


def start_codes(facets):
    """Weinberg code -> first-visit labellings, over every start edge with the
    largest key (definition in the module docstring).  The kernels walk from one
    such start, whichever comes first in their facet list, so the tables hold
    the code of each of them; starts related by an automorphism give the same
    code."""
    deg: dict = {}
    for f in facets:
        for x in f:
            deg[x] = deg.get(x, 0) + 1
    th = _third(facets)
    starts = [(a, b) for f in facets for a, b in ((f[0], f[1]), (f[1], f[2]), (f[2], f[0]))]
    top = max(edge_key(deg, th, a, b) for a, b in starts)
    out: dict = {}
    for a, b in starts:
        if edge_key(deg, th, a, b) == top:
            code, lab = weinberg(facets, a, b)
            out.setdefault(code, []).append(lab)
    return out


def pack_code(code) -> list:
    """Labels 3.. of a code as nibbles (every walk starts with labels 1, 2)."""
    assert code[0] == 1 and code[1] == 2
    words = [0] * NIB_WORDS
    for s, x in enumerate(code[2:]):
        words[s // 8] |= (x & 15) << (4 * (s % 8))
    return words


def code_hash(words) -> int:
    h = HASH_INIT
    for x in words:
        h = ((h ^ x) * HASH_MUL) & MASK64
    return h


# ------------------------------------------------------------ SoS term order
def sos_terms():
    """Terms of det[[p_r + eps_r, 1]] (rows sorted by increasing priority, row r
    coordinate c perturbed by eps^(2^(3r + c))) in increasing order of their
    exponent, which is the same for every increasing priority assignment.

    Each term: (kept-row mask, kept-column mask over x, y, z, 1, sign), with
    sign = (-1)^(sum rows + sum cols) * sign of the row -> column bijection."""
    terms = []
    for assign in itertools.product((-1, 0, 1, 2), repeat=4):
        cols = [c for c in assign if c >= 0]
        if len(cols) != len(set(cols)):
            continue
        mask = sum(1 << (3 * r + c) for r, c in enumerate(assign) if c >= 0)
        rows_in = [r for r, c in enumerate(assign) if c >= 0]
        cols_of = [assign[r] for r in rows_in]
        inv = sum(1 for i in range(len(cols_of)) for j in range(i + 1, len(cols_of)) if cols_of[i] > cols_of[j])
        sign = (-1) ** (sum(rows_in) + sum(cols_of) + inv)
        keep_r = sum(1 << r for r in range(4) if r not in rows_in)
        keep_c = sum(1 << c for c in range(4) if c not in cols_of)
        terms.append((mask, keep_r, keep_c, sign))
    terms.sort()
    assert terms[0][0] == 0
    return [(kr, kc, s) for _, kr, kc, s in terms[1:]]


# ------------------------------------------------------------------- tables
def build():
    tpl, groups, quats = [], [], []
    entries: dict = {}          # code -> list of (template, sigma tuple)
    stats = {}
    for S, name in enumerate(TEMPLATE_NAMES):
        w = normalised_template(name)
        k = K[S]
        perms, mats = rotation_group(w)
        tpl.append(w)
        groups.append(perms)
        quats.append([rot_to_quat(R) for R in mats])
        tris = triangulations(w)
        raw = {}
        for t in tris:
            for code, labs in start_codes(t).items():
                for lab in labs:
                    sigma = [0] * (k + 1)            # walk label -> slot
                    for slot, L in lab.items():
                        sigma[L] = slot
                    raw.setdefault(code, set()).add(tuple(sigma[1:]))
        ncand = 0
        for code, sigmas in raw.items():
            reps = set()
            for sg in sigmas:
                orbit = [tuple(g[s] for s in sg) for g in perms]
                reps.add(min(orbit))
            entries.setdefault(code, []).extend((S, r) for r in sorted(reps))
            ncand += len(reps)
        stats[name] = {"k": k, "group": len(perms), "triangulations": len(tris), "codes": len(raw),
                       "candidates": ncand}
    return tpl, groups, quats, entries, stats


def emit_header(path: pathlib.Path) -> dict:
    tpl, groups, quats, entries, stats = build()
    codes = sorted(entries)
    nslots = 1
    while nslots < 2 * len(codes):
        nslots *= 2
    slots = [None] * nslots
    cand = []
    for code in codes:
        words = pack_code(code)
        h = code_hash(words)
        first = len(cand)
        for S, sg in entries[code]:
            v = S << 60
            for L, slot in enumerate(sg):
                v |= slot << (4 * L)
            cand.append(v)
        e = (h, words, (len(code) - 1) // 6 + 2, first, len(cand) - first)
        pos = h & (nslots - 1)
        while slots[pos] is not None:
            pos = (pos + 1) & (nslots - 1)
        slots[pos] = e
    lines = ["/* Generated by paper_1603_05143_gb300/tables.py -- do not edit. */",
             "#pragma once", "#include <stdint.h>",
             "/* storage qualifiers: constant memory for uniform reads, global for tables */",
             "#ifndef PTM_TBL_CONST", "#define PTM_TBL_CONST static const", "#endif",
             "#ifndef PTM_TBL_GLOBAL", "#define PTM_TBL_GLOBAL static const", "#endif",
             "#ifndef PTM_TBL_ALIGN16", "#define PTM_TBL_ALIGN16", "#endif", ""]
    lines.append(f"#define PTM_TBL_NSLOTS {nslots}")
    lines.append(f"#define PTM_TBL_NCAND {len(cand)}")
    lines.append(f"#define PTM_HASH_INIT 0x{HASH_INIT:016x}ULL")
    lines.append(f"#define PTM_HASH_MUL 0x{HASH_MUL:016x}ULL")
    goff = np.cumsum([0] + [len(g) for g in groups]).tolist()
    lines.append(f"#define PTM_GROUP_TOTAL {goff[-1]}")
    lines.append("")
    lines.append("/* normalised templates (x, y, z, .), slot 0 = centre (its .w holds sum |w|^2); Eq. 4 */")
    lines.append("PTM_TBL_GLOBAL float ptm_tpl[5][15][4] PTM_TBL_ALIGN16 = {")
    for w in tpl:
        gw = float(np.sum(w * w))
        # the strain fit uses pinv = V^T / (G_w / 3): every template has an isotropic
        # second moment (cubic, icosahedral and ideal hcp shells)
        assert np.allclose(w.T @ w, gw / 3 * np.eye(3), atol=1e-12)
        rows = [f"{{{x:.9e}f, {y:.9e}f, {z:.9e}f, {(gw if i == 0 else 0.0):.9e}f}}"
                for i, (x, y, z) in enumerate(w)]
        rows += ["{0.f, 0.f, 0.f, 0.f}"] * (15 - len(w))
        lines.append("  {" + ", ".join(rows) + "},")
    lines.append("};")
    lines.append("PTM_TBL_CONST double ptm_tpl64[5][15][3] = {")
    for w in tpl:
        rows = [f"{{{x:.17e}, {y:.17e}, {z:.17e}}}" for x, y, z in w]
        rows += ["{0., 0., 0.}"] * (15 - len(w))
        lines.append("  {" + ", ".join(rows) + "},")
    lines.append("};")
    lines.append("PTM_TBL_CONST int ptm_group_off[6] = {" + ", ".join(map(str, goff)) + "};")
    lines.append("/* rotation g maps slot s to slot perm[g][s] */")
    lines.append("PTM_TBL_CONST uint8_t ptm_group_perm[PTM_GROUP_TOTAL][16] = {")
    for perms in groups:
        for p in perms:
            lines.append("  {" + ", ".join(map(str, list(p) + [0] * (16 - len(p)))) + "},")
    lines.append("};")
    lines.append("PTM_TBL_CONST float ptm_group_quat[PTM_GROUP_TOTAL][4] = {")
    for qs in quats:
        for q in qs:
            lines.append("  {" + ", ".join(f"{x:.9e}f" for x in q) + "},")
    lines.append("};")
    lines.append(f"typedef struct {{ uint64_t hash; uint32_t code[{NIB_WORDS}]; uint16_t nv, first, count, pad; }} ptm_tbl_entry;")
    lines.append("PTM_TBL_GLOBAL ptm_tbl_entry ptm_tbl[PTM_TBL_NSLOTS] = {")
    for e in slots:
        if e is None:
            lines.append("  {0ULL, {0}, 0, 0, 0, 0},")
        else:
            h, words, nv, first, count = e
            lines.append(f"  {{0x{h:016x}ULL, {{{', '.join(f'0x{x:08x}u' for x in words)}}}, {nv}, {first}, {count}, 0}},")
    lines.append("};")
    lines.append("/* candidate: bits 60-62 template, nibble L-1 = slot of canonical label L */")
    lines.append("PTM_TBL_GLOBAL uint64_t ptm_cand[PTM_TBL_NCAND] = {")
    for i in range(0, len(cand), 4):
        lines.append("  " + ", ".join(f"0x{x:016x}ULL" for x in cand[i:i + 4]) + ",")
    lines.append("};")
    terms = sos_terms()
    lines.append(f"#define PTM_SOS_NTERMS {len(terms)}")
    lines.append("/* SoS expansion terms in order: kept rows | kept cols << 4 | (sign < 0) << 8 */")
    lines.append("PTM_TBL_CONST uint16_t ptm_sos_terms[PTM_SOS_NTERMS] = {")
    lines.append("  " + ", ".join(str(kr | (kc << 4) | ((s < 0) << 8)) for kr, kc, s in terms))
    lines.append("};")
    path.write_text("\n".join(lines) + "\n")
    return stats


if __name__ == "__main__":
    import sys
    st = emit_header(pathlib.Path(sys.argv[1] if len(sys.argv) > 1 else "ptm_tables_gen.h"))
    for k, v in st.items():
        print(k, v)
