"""Template tables of the kernels (CPU only): a Weinberg walk from any start
edge with the largest edge key finds its template, with the true
correspondence among the listed candidates (Sec. 4, App. A)."""
import numpy as np

from paper_1603_05143_gb300 import tables as T


def _key_max_codes(facets):
    """(code, labelling) of the walk from every start edge with the largest key."""
    deg: dict = {}
    for f in facets:
        for x in f:
            deg[x] = deg.get(x, 0) + 1
    th = T._third(facets)
    starts = [(a, b) for f in facets for a, b in ((f[0], f[1]), (f[1], f[2]), (f[2], f[0]))]
    top = max(T.edge_key(deg, th, a, b) for a, b in starts)
    return [T.weinberg(facets, a, b) for a, b in starts if T.edge_key(deg, th, a, b) == top]


def test_walk_from_any_key_maximal_start_finds_the_template():
    """Relabel the vertices of template triangulations at random: every start
    edge of largest key gives a code the tables hold, the same codes as before
    relabelling (the key and the walk depend on the embedded graph only), and
    the relabelling's own correspondence (up to the template's rotations) is
    one of the listed candidates."""
    tpl, groups, quats, entries, stats = T.build()
    rng = np.random.default_rng(17)
    for S, name in enumerate(T.TEMPLATE_NAMES):
        k = T.K[S]
        tris = T.triangulations(T.normalised_template(name))
        for t in tris:                                      # every triangulation (4096 for BCC)
            relabel = rng.permutation(k) + 1                 # new name of slot s: relabel[s - 1]
            slot_of = {int(relabel[s - 1]): s for s in range(1, k + 1)}
            facets = [tuple(int(relabel[x - 1]) for x in f) for f in t]
            walks = _key_max_codes(facets)
            if rng.random() < 0.05:
                assert {c for c, _ in walks} == {c for c, _ in _key_max_codes(t)}
            for code, lab in walks:
                assert code in entries, name
                reps = {r for S2, r in entries[code] if S2 == S}
                truth = [0] * (k + 1)                         # walk label -> true slot
                for v, L in lab.items():
                    truth[L] = slot_of[v]
                assert min(tuple(g[s] for s in truth[1:]) for g in groups[S]) in reps, name


def test_table_sizes():
    """Triangulation counts of Sec. 4 (1, 64, 64, 1, 4096) and rotation group
    orders (24, 24, 6, 60, 24); every template graph has at least one code."""
    *_, stats = T.build()
    assert [stats[n]["triangulations"] for n in T.TEMPLATE_NAMES] == [1, 64, 64, 1, 4096]
    assert [stats[n]["group"] for n in T.TEMPLATE_NAMES] == [24, 24, 6, 60, 24]
    assert all(stats[n]["codes"] >= 1 and stats[n]["candidates"] >= stats[n]["codes"] for n in T.TEMPLATE_NAMES)
