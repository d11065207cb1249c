"""Randomised GPU parity: many seeded graphs of mixed shapes and sizes, every
pattern in both induced modes, random launch options and random task ranges,
each count compared bit-exactly with the CPU oracle."""
import numpy as np
import pytest

import graphgen as gg
import oracle as O
import paper_2112_09761_gb300 as G

pytestmark = pytest.mark.gpu

PATTERNS = ["triangle", "4-clique", "5-clique", "6-clique", "diamond", "4-cycle",
            "tailed-triangle", "3-star", "4-path", "wedge"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    G.build()


def _graph(rng, i):
    kind = i % 4
    if kind == 0:
        n = int(rng.integers(20, 400))
        return gg.gnp_graph(n, float(rng.uniform(0.02, 0.3)), 500 + i)
    if kind == 1:
        n = int(rng.integers(100, 5000))
        return gg.er_graph(n, int(n * rng.uniform(1, 12)), 500 + i)
    if kind == 2:
        s = int(rng.integers(6, 12))
        return gg.rmat_graph(s, int(rng.integers(4, 20)), 500 + i)
    n = int(rng.integers(200, 4000))
    return gg.chung_lu_graph(n, int(n * rng.uniform(2, 10)), 500 + i,
                             wmax=float(rng.uniform(20, n / 4)), i0=float(rng.uniform(1, 10)))


@pytest.mark.parametrize("i", range(48))
def test_fuzz(i):
    rng = np.random.default_rng(1000 + i)
    g = _graph(rng, i)
    opts = {}
    if rng.random() < 0.5:
        opts["bsearch_ratio"] = int(rng.choice([1, 2, 8, 64, 1 << 20]))
    if rng.random() < 0.3:
        opts["chunk"] = int(rng.integers(1, 200))
    if rng.random() < 0.3:
        opts["warps_per_block"] = int(rng.integers(1, 9))
    if rng.random() < 0.2:
        opts["no_lgs"] = 1
    if rng.random() < 0.2:
        opts["no_count_only"] = 1
    with G.Graph.from_csr(g) as h:
        for pat in PATTERNS:
            for ind in (False, True):
                if pat == "6-clique" and ind:
                    continue
                want = O.count(g, pat, induced=ind, nthreads=4)
                got = h.count(pat, induced=ind, opts=opts or None)
                assert got == want, (g.name, pat, ind, opts, got, want)
        # one random task range per pattern
        for pat in ("4-clique", "diamond", "4-cycle", "tailed-triangle"):
            p = h.plan(pat, opts=opts or None)
            nt = G.gpm_plan_info(p)["n_tasks"]
            if nt == 0:
                continue
            a = int(rng.integers(0, nt))
            b = int(rng.integers(a, nt + 1))
            assert G.gpm_count_range(p, a, b) == O.count(g, pat, False, a, b), (g.name, pat, a, b)
        # motif counts
        for k in (3, 4):
            assert G.gpm_motif_count(h.handle, k) == O.motif_counts(g, k, nthreads=4,
                                                                    method="identities")
