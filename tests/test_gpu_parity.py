"""GPU parity: every count and listing of the CUDA path equals the CPU oracle's,
bit-exactly (uint64 counts; listings as sets of canonical matches).

Graphs span several warp chunks, ragged list tails (lengths not multiples of
32), hub lists longer than the 512-entry shared-memory buffers (HBM buffer
path), skewed and balanced intersections (binary-search and merge variants),
and the degenerate cases (empty graph, isolated vertices, no matches).
"""
import math

import numpy as np
import pytest

import graphgen as gg
import oracle as O
import paper_2112_09761_gb300 as G

pytestmark = pytest.mark.gpu

PATTERNS = ["triangle", "4-clique", "5-clique", "diamond", "4-cycle", "tailed-triangle",
            "3-star", "4-path", "wedge"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a GPU"
    G.build()
    G.lib()


def _graphs():
    return {
        "K7": gg.complete(7),
        "K_5_6": gg.complete_bipartite(5, 6),
        "star40": gg.star(40),
        "gnp60": gg.gnp_graph(60, 0.45, 3),
        "er3k": gg.er_graph(3000, 24_000, 5),
        "rmat11": gg.rmat_graph(11, 12, 6),
        "chunglu8k": gg.chung_lu_graph(8000, 64_000, 7, wmax=1500.0, i0=2.0),
    }


GRAPHS = _graphs()


@pytest.mark.parametrize("gname", list(GRAPHS))
@pytest.mark.parametrize("induced", [False, True])
def test_count_parity(gname, induced):
    g = GRAPHS[gname]
    with G.Graph.from_csr(g) as h:
        for pat in PATTERNS:
            if pat == "5-clique" and gname in ("chunglu8k",) and induced:
                continue
            want = O.count(g, pat, induced=induced, nthreads=4)
            got = h.count(pat, induced=induced)
            assert got == want, (gname, pat, induced, got, want)


@pytest.mark.parametrize("opts", [
    {"bsearch_ratio": 1},                 # binary search for every intersection
    {"bsearch_ratio": 1 << 30},           # chunked merge for every intersection
    {"chunk": 1, "warps_per_block": 1},   # one warp per CTA, one task per grab
    {"chunk": 97, "warps_per_block": 3, "blocks_per_sm": 1},
    {"no_count_only": 1},                 # enumerate instead of counting-only forms
    {"no_lgs": 1},                        # cliques on sorted sets only
])
def test_count_parity_launch_variants(opts):
    g = GRAPHS["rmat11"]
    with G.Graph.from_csr(g) as h:
        for pat in PATTERNS:
            for induced in (False, True):
                want = O.count(g, pat, induced=induced, nthreads=4)
                assert h.count(pat, induced=induced, opts=opts) == want, (pat, induced, opts)


def test_hub_buffers_in_hbm():
    """A 600-vertex clique: out-degrees up to 599 exceed the 512-entry shared
    buffers, so the DFS buffers live in the per-warp HBM slices; the local
    graph search covers its warp (<= 64), 256 and 1024 out-degree classes."""
    n = 600
    g = gg.complete(n)
    with G.Graph.from_csr(g) as h:
        assert h.count("triangle") == math.comb(n, 3)
        assert h.count("4-clique") == math.comb(n, 4)
        assert h.count("4-clique", opts={"no_lgs": 1}) == math.comb(n, 4)
        assert h.count("5-clique") == math.comb(n, 5)
        assert h.info()["max_out_degree"] == n - 1
        assert h.count("diamond") == 6 * math.comb(n, 4)
        assert h.count("diamond", induced=True) == 0
        assert h.count("4-cycle") == 3 * math.comb(n, 4)
        assert h.count("tailed-triangle") == 12 * math.comb(n, 4)


def test_lgs_heavy_roots_fall_back():
    """Roots with more than 1024 out-neighbours are counted on sorted sets."""
    n = 1040
    with G.Graph.from_csr(gg.complete(n)) as h:
        assert h.count("4-clique") == math.comb(n, 4)
        p = h.plan("4-clique")
        nt = G.gpm_plan_info(p)["n_tasks"]
        # ranges cut through heavy and light roots alike
        cuts = [0, 7, 1100, 20_000, 300_000, nt]
        parts = [G.gpm_count_range(p, a, b) for a, b in zip(cuts, cuts[1:])]
        assert sum(parts) == math.comb(n, 4)


@pytest.mark.parametrize("k", [4, 5, 6])
def test_lgs_equals_sorted_sets(k):
    g = gg.rmat_graph(14, 16, 9)
    with G.Graph.from_csr(g) as h:
        a = h.count(f"{k}-clique")
        b = h.count(f"{k}-clique", opts={"no_lgs": 1})
        assert a == b
        if k <= 5:
            assert a == O.count(g, f"{k}-clique", nthreads=8)


def test_lgs_task_ranges():
    g = gg.rmat_graph(13, 16, 4)
    rng = np.random.default_rng(8)
    with G.Graph.from_csr(g) as h:
        for k in (4, 5):
            p = h.plan(f"{k}-clique")
            nt = G.gpm_plan_info(p)["n_tasks"]
            for _ in range(5):
                a = int(rng.integers(0, nt))
                b = int(min(nt, a + rng.integers(1, 5000)))
                assert G.gpm_count_range(p, a, b) == O.count(g, f"{k}-clique", False, a, b)


def test_closed_forms():
    with G.Graph.from_csr(gg.complete_bipartite(40, 70)) as h:
        c4 = math.comb(40, 2) * math.comb(70, 2)
        assert h.count("4-cycle") == c4 and h.count("4-cycle", induced=True) == c4
        assert h.count("triangle") == 0
        assert h.count("4-path", induced=True) == 0
    with G.Graph.from_csr(gg.star(300)) as h:
        assert h.count("3-star") == math.comb(300, 3) == h.count("3-star", induced=True)
        assert h.count("wedge") == math.comb(300, 2)
    with G.Graph.from_csr(gg.path(1000)) as h:
        assert h.count("4-path") == 997 and h.count("4-path", induced=True) == 997
    with G.Graph.from_csr(gg.cycle(1001)) as h:
        assert h.count("4-cycle") == 0 and h.count("4-path") == 1001


def test_empty_and_isolated():
    for g in (gg.empty(0), gg.empty(5), gg.from_edges(10, [(2, 7)])):
        with G.Graph.from_csr(g) as h:
            for pat in PATTERNS:
                for ind in (False, True):
                    assert h.count(pat, induced=ind) == 0


def test_task_ranges_partition_the_count():
    g = GRAPHS["er3k"]
    rng = np.random.default_rng(3)
    with G.Graph.from_csr(g) as h:
        for pat in ["triangle", "4-clique", "diamond", "4-cycle", "tailed-triangle", "3-star"]:
            p = h.plan(pat)
            nt = G.gpm_plan_info(p)["n_tasks"]
            assert nt == O.num_tasks(g, pat)
            cuts = sorted({0, nt, *rng.integers(0, nt, 6).tolist()})
            parts = []
            for a, b in zip(cuts, cuts[1:]):
                got = G.gpm_count_range(p, a, b)
                assert got == O.count(g, pat, False, a, b), (pat, a, b)
                parts.append(got)
            assert sum(parts) == G.gpm_count(p) == O.count(g, pat)


def _canon_set(arr, edges):
    return {O.canonical(m, edges) for m in np.asarray(arr, dtype=np.int64)}


@pytest.mark.parametrize("gname", ["K7", "gnp60", "rmat11"])
@pytest.mark.parametrize("induced", [False, True])
def test_listing_parity(gname, induced):
    g = GRAPHS[gname]
    with G.Graph.from_csr(g) as h:
        for pat in ["triangle", "4-clique", "5-clique", "diamond", "4-cycle", "tailed-triangle",
                    "3-star", "4-path", "wedge"]:
            want_arr, want_total = O.list_matches(g, pat, induced, cap=4_000_000)
            if want_total > 4_000_000:
                continue
            out, total, trunc = h.list(pat, induced=induced, capacity=want_total + 10)
            assert not trunc and total == want_total == len(out), (pat, induced)
            lib_edges = G.gpm_pattern_named(pat).edge_list()
            _, _, or_edges = O.PATTERNS[pat]
            got = _canon_set(out.cpu().numpy().astype(np.uint32), lib_edges)
            assert len(got) == total, "duplicate match listed"
            assert got == _canon_set(want_arr, or_edges), (gname, pat, induced)


def test_listing_truncation():
    g = GRAPHS["gnp60"]
    with G.Graph.from_csr(g) as h:
        total = h.count("diamond")
        out, n_total, trunc = h.list("diamond", capacity=100)
        assert trunc and n_total == total and len(out) == 100
        # the written prefix consists of valid, distinct matches
        edges = G.gpm_pattern_named("diamond").edge_list()
        adj = set()
        for u in range(g.n):
            for v in g.nbrs[g.offsets[u]:g.offsets[u + 1]]:
                adj.add((u, int(v)))
        arr = out.cpu().numpy()
        assert len({O.canonical(m, edges) for m in arr}) == 100
        for m in arr:
            for a, b in edges:
                assert (int(m[a]), int(m[b])) in adj


def test_pattern_given_by_edges_is_identified():
    g = GRAPHS["gnp60"]
    with G.Graph.from_csr(g) as h:
        # a diamond written with another vertex numbering
        p = G.pattern_from_edges(4, [(2, 3), (3, 0), (0, 2), (1, 0), (1, 2)])
        assert G.gpm_count(h.plan(p)) == O.count(g, "diamond")
        # a 4-cycle
        p = G.pattern_from_edges(4, [(0, 2), (2, 1), (1, 3), (3, 0)])
        assert G.gpm_count(h.plan(p, induced=True)) == O.count(g, "4-cycle", induced=True)
        # a pattern outside the named families goes to the generic interpreter
        c5 = [(0, 1), (1, 2), (2, 3), (3, 4), (4, 0)]
        p = h.plan(G.pattern_from_edges(5, c5))
        assert G.gpm_plan_describe(p).startswith("family: generic")
        assert G.gpm_count(p) == O.count_any(g, 5, c5, False, 8)
        # a disconnected one is refused
        with pytest.raises(G.GpmError) as e:
            G.gpm_plan(h.handle, G.pattern_from_edges(4, [(0, 1), (2, 3)]))
        assert e.value.name == "GPM_E_UNSUPPORTED_PATTERN"


def test_validation_errors():
    ok = gg.complete(4)
    bad_cases = {
        "GPM_E_UNSORTED": (ok.offsets, np.array([2, 1, 3, 0, 2, 3, 0, 1, 3, 0, 1, 2], np.uint32)),
        "GPM_E_SELF_LOOP": (ok.offsets, np.array([0, 2, 3, 0, 2, 3, 0, 1, 3, 0, 1, 2], np.uint32)),
        "GPM_E_DUPLICATE": (ok.offsets, np.array([1, 1, 3, 0, 2, 3, 0, 1, 3, 0, 1, 2], np.uint32)),
        "GPM_E_RANGE": (ok.offsets, np.array([1, 2, 9, 0, 2, 3, 0, 1, 3, 0, 1, 2], np.uint32)),
    }
    for name, (off, nbr) in bad_cases.items():
        with pytest.raises(G.GpmError) as e:
            G.gpm_load_csr(off, nbr)
        assert e.value.name == name
    # asymmetric: 0 -> 1 without 1 -> 0
    with pytest.raises(G.GpmError) as e:
        G.gpm_load_csr(np.array([0, 1, 1], np.int64), np.array([1], np.uint32))
    assert e.value.name == "GPM_E_ASYMMETRIC"
    with pytest.raises(G.GpmError) as e:
        G.gpm_load_csr(np.array([0, 2, 1], np.int64), np.array([1, 0], np.uint32))
    assert e.value.name == "GPM_E_RANGE"


def test_int32_offsets_and_device_pointers():
    import torch
    g = GRAPHS["er3k"]
    want = O.count(g, "triangle")
    h = G.gpm_load_csr(g.offsets.astype(np.int32), g.nbrs)
    try:
        assert G.gpm_count(G.gpm_plan(h, "triangle")) == want
    finally:
        G.gpm_graph_free(h)
    off_d = torch.from_numpy(g.offsets).cuda()
    nbr_d = torch.from_numpy(g.nbrs.view(np.int32)).cuda()
    for flags in (0, G.GPM_BORROW):
        h = G.gpm_load_csr(off_d, nbr_d, g.n, flags=flags)
        try:
            assert G.gpm_count(G.gpm_plan(h, "triangle")) == want
        finally:
            G.gpm_graph_free(h)
    h = G.gpm_load_csr(off_d.to(torch.int32), nbr_d, g.n)
    try:
        assert G.gpm_count(G.gpm_plan(h, "triangle")) == want
    finally:
        G.gpm_graph_free(h)


def test_relabelling_invariance_on_gpu():
    g = GRAPHS["rmat11"]
    hperm = gg.permute(g, 5)
    with G.Graph.from_csr(g) as a, G.Graph.from_csr(hperm) as b:
        for pat in ["4-clique", "diamond", "4-cycle"]:
            assert a.count(pat) == b.count(pat)
