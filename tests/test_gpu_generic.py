"""GPU parity of the generic interpreter (any connected pattern of 3..8
vertices) with the oracle's injective-homomorphism count, bit-exactly; forced
generic plans of the named families against their hand-written plans; listings
checked as valid, distinct and complete; task ranges additive."""
import numpy as np
import pytest

import graphgen as gg
import oracle as O
import paper_2112_09761_gb300 as G

from test_oracle import EXTRA_PATTERNS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    G.build()


def _petersen():
    outer = [(i, (i + 1) % 5) for i in range(5)]
    inner = [(5 + i, 5 + (i + 2) % 5) for i in range(5)]
    return gg.from_edges(10, outer + inner + [(i, i + 5) for i in range(5)])


# the oracle enumerates every embedding (no symmetry breaking), so the graphs
# for arbitrary patterns stay small; the named families also run on larger ones
GRAPHS = {
    "K8": lambda: gg.complete(8),
    "K_4_5": lambda: gg.complete_bipartite(4, 5),
    "petersen": _petersen,
    "gnp40": lambda: gg.gnp_graph(40, 0.3, 7),
    "gnp200": lambda: gg.gnp_graph(200, 0.06, 7),
    "rmat8": lambda: gg.rmat_graph(8, 6, 11),
}
LARGER = {
    "rmat9": lambda: gg.rmat_graph(9, 8, 11),
    "chunglu": lambda: gg.chung_lu_graph(3000, 20_000, 5, wmax=300.0, i0=2.0),
}
CUBE = (8, [(a, b) for a in range(8) for b in range(a + 1, 8) if bin(a ^ b).count("1") == 1])


@pytest.mark.parametrize("gname", list(GRAPHS))
@pytest.mark.parametrize("induced", [False, True])
def test_generic_patterns_equal_oracle(gname, induced):
    g = GRAPHS[gname]()
    with G.Graph.from_csr(g) as h:
        for name, (k, edges) in EXTRA_PATTERNS.items():
            if k == 6 and gname == "rmat8":
                continue  # oracle time
            pat = G.pattern_from_edges(k, edges)
            want = O.count_any(g, k, edges, induced, nthreads=8)
            assert h.count(pat, induced=induced) == want, (gname, name, induced)


def test_eight_vertex_patterns():
    for g in (gg.complete(9), gg.gnp_graph(16, 0.6, 3)):
        with G.Graph.from_csr(g) as h:
            for k, edges in (CUBE, (8, [(i, (i + 1) % 8) for i in range(8)])):
                for induced in (False, True):
                    pat = G.pattern_from_edges(k, edges)
                    assert h.count(pat, induced=induced) == O.count_any(g, k, edges, induced, 8)


@pytest.mark.parametrize("gname", ["gnp40", "rmat9", "chunglu"])
def test_forced_generic_equals_named_plans(gname):
    g = {**GRAPHS, **LARGER}[gname]()
    with G.Graph.from_csr(g) as h:
        for name in ["triangle", "wedge", "diamond", "4-cycle", "tailed-triangle", "3-star",
                     "4-path", "4-clique", "5-clique"]:
            for induced in (False, True):
                if "clique" in name or name == "triangle":
                    if induced:
                        continue
                want = h.count(name, induced=induced)
                got = h.count(name, induced=induced, opts={"generic_plan": 1})
                assert got == want == O.count(g, name, induced=induced, nthreads=8), (name, induced)
                d = G.gpm_plan_describe(h.plan(name, induced, opts={"generic_plan": 1}))
                assert d.startswith("family: generic")


def _adj(g):
    return {(int(u), int(v)) for u in range(g.n) for v in g.nbrs[g.offsets[u]:g.offsets[u + 1]]}


@pytest.mark.parametrize("name", ["5-cycle", "house", "bull", "K2,3", "prism"])
@pytest.mark.parametrize("induced", [False, True])
def test_generic_listing_valid_distinct_complete(name, induced):
    g = GRAPHS["gnp40"]()
    k, edges = EXTRA_PATTERNS[name]
    adj = _adj(g)
    want = O.count_any(g, k, edges, induced, nthreads=8)
    with G.Graph.from_csr(g) as h:
        out, total, trunc = h.list(G.pattern_from_edges(k, edges), induced=induced,
                                   capacity=want + 10)
    assert not trunc and total == want == len(out)
    arr = out.cpu().numpy().astype(np.int64)
    seen = set()
    for m in arr:
        assert len(set(m.tolist())) == k                     # distinct vertices
        for a, b in edges:                                   # entry i = pattern vertex i
            assert (int(m[a]), int(m[b])) in adj
        if induced:
            pe = {(a, b) for a, b in edges} | {(b, a) for a, b in edges}
            for a in range(k):
                for b in range(a + 1, k):
                    if (a, b) not in pe:
                        assert (int(m[a]), int(m[b])) not in adj
        seen.add(O.canonical(m, edges))
    assert len(seen) == want                                 # no subgraph twice


def test_generic_task_ranges_add_up():
    g = LARGER["rmat9"]()
    k, edges = EXTRA_PATTERNS["house"]
    with G.Graph.from_csr(g) as h:
        p = h.plan(G.pattern_from_edges(k, edges), False)
        nt = G.gpm_plan_info(p)["n_tasks"]
        rng = np.random.default_rng(5)
        cuts = sorted({0, nt, *rng.integers(0, nt, 7).tolist()})
        parts = [G.gpm_count_range(p, a, b) for a, b in zip(cuts, cuts[1:])]
        assert sum(parts) == G.gpm_count(p) == O.count_any(g, k, edges, False, 8)


def test_generic_degenerate_graphs():
    # no edges, fewer vertices than the pattern, trees, a graph equal to the pattern
    cases = [gg.empty(5), gg.empty(3), gg.path(4), gg.star(6), gg.complete(5), gg.cycle(5)]
    for g in cases:
        with G.Graph.from_csr(g) as h:
            for name in ("5-cycle", "house", "4-star", "5-path"):
                k, edges = EXTRA_PATTERNS[name]
                pat = G.pattern_from_edges(k, edges)
                for induced in (False, True):
                    want = O.count_any(g, k, edges, induced) if g.n >= k else 0
                    assert h.count(pat, induced=induced) == want, (g.n, name, induced)
                    assert h.count(pat, induced=induced, opts={"vertex_parallel": 1}) == want
