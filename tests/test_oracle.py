"""Pins for the CPU oracle (runs without a GPU).

The oracle is checked against things other than itself:
* closed forms on complete, complete-bipartite, star, path and cycle graphs;
* O1 brute force (the definition of Section 2.1) on every labelled graph with
  5 vertices and on random graphs with up to 12 vertices;
* a pure-Python listing by definition on tiny graphs (set equality of matches);
* O3 decomposition identities (Section 5.4 counting-only pruning generalised,
  and the edge-induced -> vertex-induced 4-motif inversion) on mid-size graphs;
* invariants: relabelling, thread count, task-range additivity, the sum of
  induced 4-motifs = number of connected 4-vertex subsets;
* for any pattern (O1b: injective homomorphisms / |Aut(P)|): group orders of
  dihedral, star, bipartite and prism patterns, closed forms on complete,
  cycle, complete-bipartite, star and Petersen graphs, the O1 definition on
  random graphs and the O2 plans on a mid-size graph.
"""
import itertools
import math

import numpy as np
import pytest

import graphgen as gg
import oracle as O

C = math.comb
SMALL_PATTERNS = ["triangle", "4-clique", "5-clique", "diamond", "4-cycle", "tailed-triangle",
                  "3-star", "4-path", "wedge"]


# ------------------------------------------------------------ closed forms

@pytest.mark.parametrize("n", [3, 4, 5, 6, 7, 9])
def test_complete_graph_closed_forms(n):
    g = gg.complete(n)
    exp_edge = {"triangle": C(n, 3), "4-clique": C(n, 4), "5-clique": C(n, 5),
                "4-cycle": 3 * C(n, 4), "diamond": 6 * C(n, 4), "tailed-triangle": 12 * C(n, 4),
                "3-star": 4 * C(n, 4), "4-path": 12 * C(n, 4), "wedge": 3 * C(n, 3)}
    for p, e in exp_edge.items():
        assert O.count(g, p) == e, p
        ind = e if "clique" in p or p == "triangle" else 0
        assert O.count(g, p, induced=True) == ind, p
        if n <= 7:
            assert O.brute_named(g, p, False) == e, p
            assert O.brute_named(g, p, True) == ind, p
    for k in (6, 7, 8):
        assert O.count(g, f"{k}-clique") == C(n, k)


@pytest.mark.parametrize("a,b", [(2, 2), (2, 3), (3, 4), (4, 6), (5, 5)])
def test_complete_bipartite_closed_forms(a, b):
    g = gg.complete_bipartite(a, b)
    for ind in (False, True):
        assert O.count(g, "4-cycle", induced=ind) == C(a, 2) * C(b, 2)
        assert O.count(g, "triangle", induced=ind) == 0
        assert O.count(g, "diamond", induced=ind) == 0
        assert O.count(g, "tailed-triangle", induced=ind) == 0
        assert O.count(g, "3-star", induced=ind) == a * C(b, 3) + b * C(a, 3)
        assert O.count(g, "wedge", induced=ind) == a * C(b, 2) + b * C(a, 2)
    assert O.count(g, "4-path") == a * b * (a - 1) * (b - 1)
    assert O.count(g, "4-path", induced=True) == 0  # x1 ~ y2 closes every path


@pytest.mark.parametrize("leaves", [1, 2, 3, 5, 8])
def test_star_closed_forms(leaves):
    g = gg.star(leaves)
    for ind in (False, True):
        assert O.count(g, "3-star", induced=ind) == C(leaves, 3)
        assert O.count(g, "wedge", induced=ind) == C(leaves, 2)
        assert O.count(g, "triangle", induced=ind) == 0
        assert O.count(g, "4-path", induced=ind) == 0


@pytest.mark.parametrize("n", [2, 3, 4, 5, 9])
def test_path_closed_forms(n):
    g = gg.path(n)
    for ind in (False, True):
        assert O.count(g, "4-path", induced=ind) == max(0, n - 3)
        assert O.count(g, "wedge", induced=ind) == max(0, n - 2)
        assert O.count(g, "3-star", induced=ind) == 0


@pytest.mark.parametrize("n", [3, 4, 5, 6, 11])
def test_cycle_closed_forms(n):
    g = gg.cycle(n)
    assert O.count(g, "4-cycle") == (1 if n == 4 else 0)
    assert O.count(g, "triangle") == (1 if n == 3 else 0)
    if n >= 5:
        assert O.count(g, "4-path") == n
        assert O.count(g, "4-path", induced=True) == n
    if n == 4:
        assert O.count(g, "4-path") == 4
        assert O.count(g, "4-path", induced=True) == 0


def test_empty_and_edgeless_graphs():
    for g in (gg.empty(0), gg.empty(1), gg.empty(7)):
        for p in SMALL_PATTERNS:
            assert O.count(g, p) == 0
            assert O.num_tasks(g, p) == 0


# ------------------------------------------------------ O2 vs O1 brute force

def _all_graphs(n):
    pairs = list(itertools.combinations(range(n), 2))
    for mask in range(1 << len(pairs)):
        yield gg.from_edges(n, [pairs[i] for i in range(len(pairs)) if mask >> i & 1])


def test_matcher_equals_definition_on_every_5_vertex_graph():
    mism = []
    for idx, g in enumerate(_all_graphs(5)):
        for p in ["triangle", "4-clique", "5-clique", "diamond", "4-cycle", "tailed-triangle",
                  "3-star", "4-path", "wedge"]:
            for ind in (False, True):
                a, b = O.count(g, p, induced=ind), O.brute_named(g, p, ind)
                if a != b:
                    mism.append((idx, p, ind, a, b))
    assert not mism, mism[:10]


@pytest.mark.parametrize("n,p,seed", [(6, 0.5, 1), (7, 0.6, 2), (8, 0.5, 3), (9, 0.4, 4),
                                      (10, 0.5, 5), (10, 0.8, 6), (11, 0.3, 7), (12, 0.2, 8),
                                      (12, 0.5, 9), (12, 0.8, 10)])
def test_matcher_equals_definition_random(n, p, seed):
    g = gg.gnp_graph(n, p, seed)
    for pat in SMALL_PATTERNS:
        for ind in (False, True):
            if pat == "5-clique" and n > 10:
                continue
            assert O.count(g, pat, induced=ind) == O.brute_named(g, pat, ind), (pat, ind)


def test_brute_force_automorphism_identity():
    """Edge-induced count = injective homomorphisms / |Aut(P)| (independent form)."""
    aut = {"triangle": 6, "4-clique": 24, "diamond": 4, "4-cycle": 8, "tailed-triangle": 2,
           "3-star": 6, "4-path": 2, "wedge": 2}
    g = gg.gnp_graph(8, 0.5, 11)
    adj = [set() for _ in range(g.n)]
    for u in range(g.n):
        for v in g.nbrs[g.offsets[u]:g.offsets[u + 1]]:
            adj[u].add(int(v))
    for pat, a in aut.items():
        _, k, edges = O.PATTERNS[pat]
        inj = sum(1 for m in itertools.permutations(range(g.n), k)
                  if all(m[y] in adj[m[x]] for x, y in edges))
        assert inj % a == 0
        assert O.count(g, pat) == inj // a, pat


# ------------------------------------------------------ listing by definition

def _py_list(g, pat, induced):
    """Pure-Python listing by definition: canonical forms of all matches."""
    _, k, edges = O.PATTERNS[pat]
    adj = [set(int(v) for v in g.nbrs[g.offsets[u]:g.offsets[u + 1]]) for u in range(g.n)]
    found = set()
    for m in itertools.permutations(range(g.n), k):
        if not all(m[y] in adj[m[x]] for x, y in edges):
            continue
        if induced:
            eset = {frozenset(e) for e in edges}
            if any(m[j] in adj[m[i]] for i in range(k) for j in range(i + 1, k)
                   if frozenset((i, j)) not in eset):
                continue
        found.add(O.canonical(m, edges))
    return found


@pytest.mark.parametrize("seed", [21, 22, 23])
def test_listing_matches_definition(seed):
    g = gg.gnp_graph(8, 0.55, seed)
    for pat in SMALL_PATTERNS:
        _, k, edges = O.PATTERNS[pat]
        for ind in (False, True):
            arr, total = O.list_matches(g, pat, ind)
            assert total == len(arr) == O.count(g, pat, ind)
            mine = {O.canonical(m, edges) for m in arr}
            assert len(mine) == total, "duplicate match listed"
            assert mine == _py_list(g, pat, ind), (pat, ind)


def test_listing_capacity_and_ranges():
    g = gg.gnp_graph(30, 0.3, 5)
    arr, total = O.list_matches(g, "diamond", False, cap=7)
    assert len(arr) == 7 and total == O.count(g, "diamond")
    nt = O.num_tasks(g, "diamond")
    parts = [O.list_matches(g, "diamond", False, lo, min(lo + 9, nt))[1] for lo in range(0, nt, 9)]
    assert sum(parts) == total


# ------------------------------------------------------ O3 identities vs O2

@pytest.mark.parametrize("name", ["er", "rmat", "chunglu"])
def test_identities_equal_matcher(name):
    if name == "er":
        g = gg.er_graph(300, 2400, 7)
    elif name == "rmat":
        g = gg.rmat_graph(9, 8, 7)
    else:
        g = gg.chung_lu_graph(600, 6000, 7, wmax=120.0, i0=3.0)
    ids = O.identities(g)
    assert ids["triangle"] == O.count(g, "triangle")
    assert ids["wedge_e"] == O.count(g, "wedge")
    assert ids["3-star_e"] == O.count(g, "3-star")
    assert ids["4-path_e"] == O.count(g, "4-path")
    assert ids["tailed-triangle_e"] == O.count(g, "tailed-triangle")
    assert ids["diamond_e"] == O.count(g, "diamond")
    assert ids["4-cycle_e"] == O.count(g, "4-cycle")
    assert ids["wedge_v"] == O.count(g, "wedge", induced=True)
    assert O.motif_counts(g, 4, method="identities") == O.motif_counts(g, 4, method="enumerate")
    assert O.motif_counts(g, 3, method="identities") == O.motif_counts(g, 3, method="enumerate")


@pytest.mark.parametrize("n,p,seed", [(9, 0.5, 31), (12, 0.3, 32), (14, 0.35, 33), (20, 0.2, 34)])
def test_induced_motif_sum_is_connected_subsets(n, p, seed):
    g = gg.gnp_graph(n, p, seed)
    assert sum(O.motif_counts(g, 4)) == O.connected_subsets(g, 4)
    assert sum(O.motif_counts(g, 3)) == O.connected_subsets(g, 3)


# ------------------------------------------------------------- invariants

def test_relabelling_invariance():
    g = gg.rmat_graph(8, 8, 3)
    h = gg.permute(g, 99)
    assert gg.csr_checksum(g) != gg.csr_checksum(h)
    for pat in SMALL_PATTERNS:
        for ind in (False, True):
            assert O.count(g, pat, ind) == O.count(h, pat, ind), (pat, ind)


def test_thread_count_and_task_ranges():
    g = gg.rmat_graph(10, 8, 4)
    for pat in ["4-clique", "diamond", "4-cycle", "tailed-triangle"]:
        full = O.count(g, pat)
        assert O.count(g, pat, nthreads=4) == full
        nt = O.num_tasks(g, pat)
        cuts = sorted({0, nt, *np.random.default_rng(1).integers(0, nt, 5).tolist()})
        assert sum(O.count(g, pat, False, a, b) for a, b in zip(cuts, cuts[1:])) == full


def test_task_list_sizes():
    g = gg.er_graph(500, 3000, 3)
    assert O.num_tasks(g, "diamond") == g.m          # v1 > v2: one per undirected edge
    assert O.num_tasks(g, "tailed-triangle") == 2 * g.m  # both directions
    assert O.num_tasks(g, "triangle") == g.m         # one arc per edge in the DAG


def test_generator_shapes_and_determinism():
    g = gg.workload("er-10k")
    assert g.n == 10_000 and g.m == 80_000
    d = g.degrees()
    assert d.sum() == 160_000
    # simple graph: sorted rows, no loops, both directions
    for u in range(0, g.n, 997):
        row = g.nbrs[g.offsets[u]:g.offsets[u + 1]]
        assert np.all(np.diff(row.astype(np.int64)) > 0) and u not in row
        for v in row[:5]:
            r2 = g.nbrs[g.offsets[v]:g.offsets[v + 1]]
            assert u in r2
    assert gg.csr_checksum(gg.workload("er-10k")) == gg.csr_checksum(g)


# ------------------------------------------- any pattern: O1b (injhom / |Aut|)

# patterns beyond the plan families, as (k, edges)
EXTRA_PATTERNS = {
    "5-cycle": (5, [(0, 1), (1, 2), (2, 3), (3, 4), (4, 0)]),
    "5-path": (5, [(0, 1), (1, 2), (2, 3), (3, 4)]),
    "4-star": (5, [(0, 1), (0, 2), (0, 3), (0, 4)]),
    "house": (5, [(0, 1), (1, 2), (2, 3), (3, 0), (0, 4), (1, 4)]),
    "bull": (5, [(0, 1), (1, 2), (2, 0), (0, 3), (1, 4)]),
    "K2,3": (5, [(0, 2), (0, 3), (0, 4), (1, 2), (1, 3), (1, 4)]),
    "gem": (5, [(0, 1), (0, 2), (0, 3), (0, 4), (1, 2), (2, 3), (3, 4)]),
    "prism": (6, [(0, 1), (1, 2), (2, 0), (3, 4), (4, 5), (5, 3), (0, 3), (1, 4), (2, 5)]),
    "K3,3": (6, [(a, b) for a in range(3) for b in range(3, 6)]),
    "6-cycle": (6, [(i, (i + 1) % 6) for i in range(6)]),
}


def test_automorphism_group_orders():
    # the plan families (table of |Aut| used by the oracle's definition)
    want = {"triangle": 6, "wedge": 2, "4-clique": 24, "diamond": 4, "4-cycle": 8,
            "tailed-triangle": 2, "3-star": 6, "4-path": 2, "5-clique": 120}
    for name, a in want.items():
        _, k, e = O.PATTERNS[name]
        assert O.automorphisms(k, e) == a, name
    # dihedral, star, bipartite and product groups
    want = {"5-cycle": 10, "5-path": 2, "4-star": 24, "house": 2, "bull": 2, "K2,3": 12,
            "gem": 2, "prism": 12, "K3,3": 72, "6-cycle": 12}
    for name, a in want.items():
        k, e = EXTRA_PATTERNS[name]
        assert O.automorphisms(k, e) == a, name


@pytest.mark.parametrize("n", [6, 7, 9])
def test_any_pattern_on_complete_graphs(n):
    # in K_n every injective map is an embedding: n!/(n-k)! / |Aut(P)| edge-induced
    # matches; vertex-induced, only complete patterns occur
    for name, (k, e) in EXTRA_PATTERNS.items():
        if k > n:
            continue
        falling = math.factorial(n) // math.factorial(n - k)
        assert O.count_any(gg.complete(n), k, e, False) == falling // O.automorphisms(k, e), name
        assert O.count_any(gg.complete(n), k, e, True) == 0, name
    assert O.count_any(gg.complete(n), 5, O.PATTERNS["5-clique"][2], True) == C(n, 5)


def test_any_pattern_closed_forms():
    # cycles and paths in a cycle graph C_m: m copies of each path shorter than m,
    # one m-cycle
    for m in (7, 9, 12):
        g = gg.cycle(m)
        assert O.count_any(g, 5, EXTRA_PATTERNS["5-path"][1], False) == m
        assert O.count_any(g, 5, EXTRA_PATTERNS["5-path"][1], True) == m
        assert O.count_any(g, 5, EXTRA_PATTERNS["5-cycle"][1], False) == 0
    assert O.count_any(gg.cycle(5), 5, EXTRA_PATTERNS["5-cycle"][1], True) == 1
    # K_{a,b}: no odd cycle; 6-cycles = C(a,3) C(b,3) * 3! * 3! / (2 * 6) ... counted
    # as ordered alternations: C(a,3) C(b,3) * 6; K2,3 copies = C(a,2) C(b,3) + C(a,3) C(b,2)
    for a, b in ((3, 4), (4, 5), (5, 5)):
        g = gg.complete_bipartite(a, b)
        assert O.count_any(g, 5, EXTRA_PATTERNS["5-cycle"][1], False) == 0
        assert O.count_any(g, 6, EXTRA_PATTERNS["6-cycle"][1], False) == C(a, 3) * C(b, 3) * 6
        assert O.count_any(g, 5, EXTRA_PATTERNS["K2,3"][1], True) == C(a, 2) * C(b, 3) + C(a, 3) * C(b, 2)
        assert O.count_any(g, 6, EXTRA_PATTERNS["K3,3"][1], True) == C(a, 3) * C(b, 3)
    # the Petersen graph: 12 five-cycles, 10 six-cycles, no 4-cycle, 15 edges
    outer = [(i, (i + 1) % 5) for i in range(5)]
    inner = [(5 + i, 5 + (i + 2) % 5) for i in range(5)]
    spokes = [(i, i + 5) for i in range(5)]
    pet = gg.from_edges(10, outer + inner + spokes)
    assert O.count_any(pet, 5, EXTRA_PATTERNS["5-cycle"][1], False) == 12
    assert O.count_any(pet, 6, EXTRA_PATTERNS["6-cycle"][1], False) == 10
    assert O.count_any(pet, 4, O.PATTERNS["4-cycle"][2], False) == 0
    # a star K_{1,m}: C(m, 4) four-stars, both modes
    assert O.count_any(gg.star(9), 5, EXTRA_PATTERNS["4-star"][1], False) == C(9, 4)
    assert O.count_any(gg.star(9), 5, EXTRA_PATTERNS["4-star"][1], True) == C(9, 4)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_any_pattern_equals_definition(seed):
    # O1b against the O1 definition (k-subsets x edge subsets x isomorphism)
    g = gg.gnp_graph(11, 0.5, 100 + seed)
    for name, (k, e) in EXTRA_PATTERNS.items():
        if k == 6 and seed > 1:
            continue
        for induced in (False, True):
            assert O.count_any(g, k, e, induced) == O.brute(g, k, e, induced), (name, induced)


def test_any_pattern_equals_plan_families():
    # O1b against the O2 nested-loop plans, mid-size graph, thread count invariant
    g = gg.gnp_graph(70, 0.25, 8)
    for name in SMALL_PATTERNS:
        _, k, e = O.PATTERNS[name]
        for induced in (False, True):
            want = O.count(g, name, induced=induced, nthreads=4)
            assert O.count_any(g, k, e, induced, nthreads=4) == want, (name, induced)
    k, e = EXTRA_PATTERNS["house"]
    assert O.count_any(g, k, e, True, nthreads=1) == O.count_any(g, k, e, True, nthreads=4)
