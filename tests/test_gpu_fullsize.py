"""Parity at the full workload sizes, in the launch configuration bench.py times.

* Every full count with a stored oracle value (tests/golden/workloads.json,
  written by tests/golden/make_goldens.py from oracle/ alone) is compared
  bit-exactly.
* Counts without a stored value (5-clique on R-MAT 22) and every plan's DFS
  are compared on sampled root-task ranges that the oracle counts live: random
  ranges plus the ranges of the heaviest roots.
* The CSR checksum confirms that this host generated the same graph as the
  host that wrote the goldens.
"""
import json
import os

import numpy as np
import pytest

import graphgen as gg
import oracle as O
import paper_2112_09761_gb300 as G

pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "workloads.json")))
THREADS = os.cpu_count() or 1


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    G.build()


@pytest.fixture(scope="module")
def rmat22():
    g = gg.workload("rmat22")
    h = G.Graph.from_csr(g)
    yield g, h
    h.close()


@pytest.fixture(scope="module")
def chunglu():
    g = gg.workload("chunglu-1m")
    h = G.Graph.from_csr(g)
    yield g, h
    h.close()


def _ranges(nt, rng, k=6, span=2000, extra=()):
    rs = [(int(a), int(min(nt, a + span))) for a in rng.integers(0, max(1, nt - span), k)]
    return rs + [r for r in extra if r[0] < r[1]]


def test_er10k_triangles():
    g = gg.workload("er-10k")
    gold = GOLD["er-10k"]
    assert gg.csr_checksum(g) == gold["checksum"]
    with G.Graph.from_csr(g) as h:
        assert h.count("triangle") == gold["counts"]["triangle"] == O.count(g, "triangle")
        # the stated input format: int32 offsets
        hh = G.gpm_load_csr(g.offsets.astype(np.int32), g.nbrs)
        try:
            assert G.gpm_count(G.gpm_plan(hh, "triangle")) == gold["counts"]["triangle"]
        finally:
            G.gpm_graph_free(hh)


def test_rmat22_full_counts(rmat22):
    g, h = rmat22
    gold = GOLD["rmat22"]
    assert gg.csr_checksum(g) == gold["checksum"]
    assert h.count("triangle") == gold["counts"]["triangle"]
    assert h.count("4-clique") == gold["counts"]["4-clique"]
    # the sorted-set path agrees with the local graph search at full size
    assert h.count("4-clique", opts={"no_lgs": 1}) == gold["counts"]["4-clique"]


@pytest.mark.parametrize("pattern", ["4-clique", "5-clique"])
def test_rmat22_sampled_ranges(rmat22, pattern):
    g, h = rmat22
    p = h.plan(pattern)
    nt = G.gpm_plan_info(p)["n_tasks"]
    info = h.info()
    # heaviest roots: arcs of the vertices with the largest out-degrees
    deg = np.diff(g.offsets)
    rng = np.random.default_rng(22)
    src = np.repeat(np.arange(g.n), deg)
    up = (deg[src] < deg[g.nbrs]) | ((deg[src] == deg[g.nbrs]) & (src < g.nbrs))
    outdeg = np.bincount(src[up], minlength=g.n)
    assert outdeg.max() == info["max_out_degree"]
    doff = np.concatenate([[0], np.cumsum(outdeg)])
    heavy = np.argsort(outdeg)[-3:]
    extra = [(int(doff[v]), int(doff[v] + min(outdeg[v], 300))) for v in heavy]
    ranges = _ranges(nt, rng, extra=extra)
    want, _ = O.count_ranges(g, pattern, ranges, nthreads=THREADS, per_range=True)
    got = [G.gpm_count_range(p, a, b) for a, b in ranges]
    assert got == want


def test_chunglu_full_counts(chunglu):
    g, h = chunglu
    gold = GOLD["chunglu-1m"]
    assert gg.csr_checksum(g) == gold["checksum"]
    for pat in ["triangle", "diamond", "4-cycle", "tailed-triangle", "3-star", "4-path", "wedge"]:
        assert h.count(pat) == gold["counts"][pat], pat


@pytest.mark.parametrize("pattern", ["diamond", "4-cycle", "tailed-triangle"])
def test_chunglu_sampled_ranges(chunglu, pattern):
    g, h = chunglu
    p = h.plan(pattern)
    nt = G.gpm_plan_info(p)["n_tasks"]
    rng = np.random.default_rng(3)
    span = 300 if pattern == "4-cycle" else 2000
    deg = np.diff(g.offsets)
    hub = int(np.argmax(deg))
    # the hub's own root tasks: for the v1 > v2 task list, its last (heaviest)
    # lower neighbours; for the directed task list, its first entries
    if pattern == "tailed-triangle":
        extra = [(int(g.offsets[hub]), int(g.offsets[hub] + 64))]
    else:
        src = np.repeat(np.arange(g.n, dtype=np.int64), deg)
        lower = np.bincount(src[g.nbrs < src], minlength=g.n)
        loff = np.concatenate([[0], np.cumsum(lower)])
        hi_t = int(loff[hub] + lower[hub])
        extra = [(max(int(loff[hub]), hi_t - 8), hi_t)]
    ranges = _ranges(nt, rng, k=4, span=span, extra=extra)
    want, _ = O.count_ranges(g, pattern, ranges, nthreads=THREADS, per_range=True)
    got = [G.gpm_count_range(p, a, b) for a, b in ranges]
    assert got == want
