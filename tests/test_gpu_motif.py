"""GPU parity of motif counting (gpm_motif_count) and of batched counting
(gpm_batch_create / gpm_batch_count) with the CPU oracle, bit-exactly."""
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


SMALL = {
    "K7": lambda: gg.complete(7),
    "K_5_6": lambda: gg.complete_bipartite(5, 6),
    "star40": lambda: gg.star(40),
    "path9": lambda: gg.path(9),
    "gnp60": lambda: gg.gnp_graph(60, 0.45, 3),
    "rmat11": lambda: gg.rmat_graph(11, 12, 6),
}


@pytest.mark.parametrize("name", list(SMALL))
@pytest.mark.parametrize("k", [3, 4])
def test_motif_count_equals_enumeration(name, k):
    g = SMALL[name]()
    with G.Graph.from_csr(g) as h:
        got = G.gpm_motif_count(h.handle, k)
    assert got == O.motif_counts(g, k, nthreads=4, method="enumerate")


@pytest.mark.parametrize("name", ["er", "rmat", "chunglu"])
def test_motif_count_medium(name):
    if name == "er":
        g = gg.er_graph(20_000, 200_000, 9)
    elif name == "rmat":
        g = gg.rmat_graph(15, 16, 9)
    else:
        g = gg.chung_lu_graph(30_000, 300_000, 9, wmax=4000.0, i0=2.0)
    with G.Graph.from_csr(g) as h:
        for k in (3, 4):
            assert G.gpm_motif_count(h.handle, k) == O.motif_counts(g, k, nthreads=8,
                                                                    method="identities")
        # edge-induced 4-motif counts of the per-pattern plans agree with the
        # decomposition used by the motif kernels (different kernels)
        assert h.count("4-cycle") == O.identities(g, 8)["4-cycle_e"]


def _batch_graphs(n, seed0=100):
    gs = []
    rng = np.random.default_rng(seed0)
    for i in range(n):
        nv = int(rng.integers(50, 3000))
        d = float(rng.uniform(2, 24))
        if i % 2 == 0:
            gs.append(gg.er_graph(nv, max(1, int(nv * d / 2)), seed0 + i))
        else:
            scale = max(1, int(np.ceil(np.log2(nv))))
            gs.append(gg.rmat_graph(scale, 0, seed0 + i, n=nv, ndraws=int(nv * d / 2)))
    gs.append(gg.empty(3))            # no edges at all
    gs.append(gg.complete(9))
    return gs


@pytest.mark.parametrize("k", [3, 4])
def test_batch_equals_single_and_oracle(k):
    gs = _batch_graphs(40)
    hs = [G.Graph.from_csr(g) for g in gs]
    try:
        b = G.gpm_batch_create([h.handle for h in hs], k)
        try:
            info = G.gpm_batch_info(b)
            assert info["chunk"] in (4, 32) and info["bsearch_ratio"] in (4, 16)
            res = G.gpm_batch_count(b)
            res2 = G.gpm_batch_count(b)  # the captured graph replays identically
            assert np.array_equal(res, res2)
        finally:
            G.gpm_batch_free(b)
        for g, h, row in zip(gs, hs, res):
            single = G.gpm_motif_count(h.handle, k)
            assert list(map(int, row)) == single
            assert single == O.motif_counts(g, k, nthreads=4, method="identities")
        # forced configurations give the same answer
        for opts in ({"chunk": 1, "bsearch_ratio": 1, "warps_per_block": 2},
                     {"chunk": 64, "bsearch_ratio": 1 << 30, "warps_per_block": 8},
                     {"chunk": 16, "bsearch_ratio": 8, "warps_per_block": 8, "no_lgs": 1}):
            b = G.gpm_batch_create([h.handle for h in hs], k, opts)
            try:
                assert np.array_equal(G.gpm_batch_count(b), res)
            finally:
                G.gpm_batch_free(b)
    finally:
        for h in hs:
            h.close()


def test_batch_lgs_all_classes_closed_form():
    """A batch whose complete graph K_1100 has roots in every out-degree class
    of the local graph search (the DAG of K_n has out-degrees 0 .. n-1), heavy
    roots (out-degree > 1024) and arcs whose arc-level local graph exceeds
    1024 members.  The vertex-induced 4-motifs of K_n are C(n, 4) 4-cliques
    and nothing else; the other graphs must agree with the oracle and the
    sorted-set path."""
    from math import comb
    gs = [gg.complete(1100), gg.er_graph(3000, 30_000, 41), gg.complete(9), gg.empty(5),
          gg.rmat_graph(12, 16, 42), gg.complete(300), gg.complete_bipartite(40, 700)]
    hs = [G.Graph.from_csr(g) for g in gs]
    try:
        res = {}
        for no_lgs in (0, 1):
            b = G.gpm_batch_create([h.handle for h in hs], 4,
                                   {"chunk": 16, "bsearch_ratio": 8, "warps_per_block": 8,
                                    "no_lgs": no_lgs})
            try:
                res[no_lgs] = G.gpm_batch_count(b)
            finally:
                G.gpm_batch_free(b)
        assert np.array_equal(res[0], res[1])
        assert list(map(int, res[0][0])) == [0, 0, 0, 0, 0, comb(1100, 4)]
        assert list(map(int, res[0][5])) == [0, 0, 0, 0, 0, comb(300, 4)]
        for i in (1, 2, 3, 4, 6):
            assert list(map(int, res[0][i])) == O.motif_counts(gs[i], 4, nthreads=8,
                                                               method="identities")
    finally:
        for h in hs:
            h.close()
