"""Renaming the data graph by degree order (GPM_RELABEL, Section 4.2
preprocessing): the renamed CSR equals the permutation computed here with
numpy, counts do not change, and listed matches come back in the caller's IDs."""
import numpy as np
import pytest

import graphgen as gg
import oracle as O
import paper_2112_09761_gb300 as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    G.build()


def renamed(g):
    """New vertex i = the vertex of rank i in ascending (degree, id) order."""
    deg = np.diff(g.offsets).astype(np.int64)
    ids = np.arange(g.n, dtype=np.int64)
    perm = np.lexsort((ids, deg))             # last key is primary
    newid = np.empty(g.n, dtype=np.int64)
    newid[perm] = ids
    off = np.zeros(g.n + 1, dtype=np.int64)
    off[1:] = np.cumsum(deg[perm])
    nbr = np.empty(int(off[-1]), dtype=np.uint32)
    for i, v in enumerate(perm):
        row = newid[g.nbrs[g.offsets[v]:g.offsets[v + 1]]]
        nbr[off[i]:off[i + 1]] = np.sort(row)
    return off, nbr, perm.astype(np.uint32)


# sizes around the 2048-key tile of the sort: nnz of 2048, 4096 and 4160,
# n of 2049 and 3000, and multi-stage sorts (R-MAT, scale 12)
CASES = {
    "cycle1024": lambda: gg.cycle(1024),
    "path2049": lambda: gg.path(2049),
    "K65": lambda: gg.complete(65),
    "star3000": lambda: gg.star(3000),
    "empty5": lambda: gg.empty(5),
    "gnp200": lambda: gg.gnp_graph(200, 0.1, 5),
    "rmat12": lambda: gg.rmat_graph(12, 16, 8),
    "er5000": lambda: gg.er_graph(5000, 40_000, 13),
}


@pytest.mark.parametrize("name", list(CASES))
def test_renamed_csr_matches_numpy(name):
    g = CASES[name]()
    off, nbr, perm = renamed(g)
    with G.Graph.from_csr(g, flags=G.GPM_RELABEL) as h:
        o2, n2, p2 = G.gpm_graph_export(h.handle)
    assert np.array_equal(o2, off)
    assert np.array_equal(n2, nbr)
    assert np.array_equal(p2, perm)
    # without renaming the export is the input and the identity
    with G.Graph.from_csr(g) as h:
        o3, n3, p3 = G.gpm_graph_export(h.handle)
    assert np.array_equal(o3, g.offsets) and np.array_equal(n3, g.nbrs)
    assert np.array_equal(p3, np.arange(g.n, dtype=np.uint32))


@pytest.mark.parametrize("name", ["gnp200", "rmat12", "er5000"])
def test_counts_invariant(name):
    g = CASES[name]()
    with G.Graph.from_csr(g) as h0, G.Graph.from_csr(g, flags=G.GPM_RELABEL) as h1:
        for pat in O.PATTERNS:
            for induced in (False, True):
                if pat.endswith("clique") or pat == "triangle":
                    if induced:
                        continue
                want = O.count(g, pat, induced=induced, nthreads=8)
                assert h0.count(pat, induced=induced) == want, (pat, induced)
                assert h1.count(pat, induced=induced) == want, (pat, induced)
        for k in (3, 4):
            assert G.gpm_motif_count(h1.handle, k) == G.gpm_motif_count(h0.handle, k)


@pytest.mark.parametrize("pat", ["triangle", "4-clique", "diamond", "4-cycle", "tailed-triangle"])
@pytest.mark.parametrize("induced", [False, True])
def test_listing_in_caller_ids(pat, induced):
    g = gg.gnp_graph(120, 0.12, 21)
    want_arr, want_total = O.list_matches(g, pat, induced)
    _, _, or_edges = O.PATTERNS[pat]
    want = {O.canonical(m, or_edges) for m in np.asarray(want_arr, dtype=np.int64)}
    lib_edges = G.gpm_pattern_named(pat).edge_list()
    with G.Graph.from_csr(g, flags=G.GPM_RELABEL) as h:
        out, total, trunc = h.list(pat, induced=induced, capacity=want_total + 10)
        assert not trunc and total == want_total == len(out)
        got = {O.canonical(m, lib_edges) for m in out.cpu().numpy().astype(np.int64)}
        assert got == want
        # truncated listings are translated too
        if want_total > 3:
            out, total, trunc = h.list(pat, induced=induced, capacity=3)
            assert trunc and total == want_total
            assert {O.canonical(m, lib_edges) for m in out.cpu().numpy().astype(np.int64)} <= want
