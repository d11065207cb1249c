"""Vertex parallelism (Section 5.1, opts.vertex_parallel): root tasks are
vertices, no task list is built; counts and listings equal the edge-parallel
plans and the oracle, and vertex ranges add up to the count."""
import numpy as np
import pytest

import graphgen as gg
import oracle as O
import paper_2112_09761_gb300 as G

from test_oracle import EXTRA_PATTERNS

pytestmark = pytest.mark.gpu

VP = {"vertex_parallel": 1}
NAMED = ["triangle", "4-clique", "5-clique", "diamond", "4-cycle", "tailed-triangle", "3-star",
         "4-path", "wedge"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    G.build()


@pytest.mark.parametrize("gname", ["gnp60", "rmat11", "chunglu"])
def test_vertex_parallel_counts(gname):
    g = {"gnp60": lambda: gg.gnp_graph(60, 0.45, 3),
         "rmat11": lambda: gg.rmat_graph(11, 12, 6),
         "chunglu": lambda: gg.chung_lu_graph(5000, 40_000, 9, wmax=600.0, i0=2.0)}[gname]()
    with G.Graph.from_csr(g) as h:
        for name in NAMED:
            for induced in (False, True):
                if induced and ("clique" in name or name == "triangle"):
                    continue
                want = O.count(g, name, induced=induced, nthreads=8)
                assert h.count(name, induced=induced, opts=VP) == want, (name, induced)
                p = h.plan(name, induced, opts=VP)
                assert G.gpm_plan_info(p)["n_tasks"] == g.n
                assert "local graph search" not in G.gpm_plan_describe(p)
        if gname == "gnp60":
            for pname in ("house", "5-cycle", "bull"):
                k, edges = EXTRA_PATTERNS[pname]
                pat = G.pattern_from_edges(k, edges)
                for induced in (False, True):
                    assert h.count(pat, induced=induced, opts=VP) == \
                        O.count_any(g, k, edges, induced, 8), (pname, induced)


def test_vertex_parallel_listing_and_ranges():
    g = gg.rmat_graph(8, 8, 4)
    with G.Graph.from_csr(g) as h:
        for name in ("diamond", "4-cycle", "tailed-triangle", "4-clique"):
            want_arr, want_total = O.list_matches(g, name, False, cap=2_000_000)
            assert want_total <= 2_000_000  # the oracle's listing is complete
            out, total, trunc = h.list(name, capacity=want_total + 10, opts=VP)
            assert not trunc and total == want_total == len(out)
            lib_edges = G.gpm_pattern_named(name).edge_list()
            _, _, or_edges = O.PATTERNS[name]
            got = {O.canonical(m, lib_edges) for m in out.cpu().numpy().astype(np.int64)}
            assert got == {O.canonical(m, or_edges) for m in np.asarray(want_arr, dtype=np.int64)}
        p = h.plan("diamond", opts=VP)
        rng = np.random.default_rng(3)
        cuts = sorted({0, g.n, *rng.integers(0, g.n, 9).tolist()})
        parts = [G.gpm_count_range(p, a, b) for a, b in zip(cuts, cuts[1:])]
        assert sum(parts) == G.gpm_count(p) == O.count(g, "diamond")
