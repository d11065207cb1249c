"""The query server: every result served in a mix of concurrent queries equals
the same query run alone (bit-exact), queries overlap on the device, and the
memory budget serialises them when it is tight."""
import numpy as np
import pytest

import graphgen as gg
import paper_2112_09761_gb300 as G

pytestmark = pytest.mark.gpu

PATTERNS = ["triangle", "4-clique", "5-clique", "4-cycle", "diamond", "tailed-triangle"]


@pytest.fixture(scope="module")
def graphs():
    import torch
    assert torch.cuda.is_available()
    G.build()
    gs = [gg.rmat_graph(13, 16, 31), gg.er_graph(3000, 24_000, 32),
          gg.chung_lu_graph(8000, 64_000, 33, wmax=1500.0, i0=2.0)]
    hs = [G.Graph.from_csr(g) for g in gs]
    alone = {(i, p, ind): h.count(p, induced=ind)
             for i, h in enumerate(hs) for p in PATTERNS for ind in (False, True)}
    yield hs, alone
    for h in hs:
        h.close()


def _run_mix(srv, hs, alone, rng, repeat=2):
    keys = [k for k in alone for _ in range(repeat)]
    rng.shuffle(keys)
    tickets = [(G.gpm_server_submit(srv, hs[i].handle, p, ind), (i, p, ind)) for i, p, ind in keys]
    lat = []
    for t, key in tickets:
        c, l = G.gpm_server_wait(srv, t, 300.0)
        assert c == alone[key], key
        assert l > 0
        lat.append(l)
    return lat


def test_mix_equals_alone(graphs):
    hs, alone = graphs
    srv = G.gpm_server_create(8 << 30, 8)
    try:
        lat = _run_mix(srv, hs, alone, np.random.default_rng(1))
        st = G.gpm_server_stats(srv)
        assert st["completed"] == len(lat) and st["pending"] == 0
        assert st["peak_inflight"] >= 2       # queries overlapped
        assert st["bytes_in_use"] == 0
        # a done query can be polled again
        t = G.gpm_server_submit(srv, hs[0].handle, "triangle")
        c, _ = G.gpm_server_wait(srv, t)
        assert G.gpm_server_poll(srv, t)[:2] == (True, c)
    finally:
        G.gpm_server_free(srv)


def test_tight_budget_serialises(graphs):
    hs, alone = graphs
    srv = G.gpm_server_create(1, 8)  # every query exceeds it: one at a time
    try:
        _run_mix(srv, hs, alone, np.random.default_rng(2), repeat=1)
        assert G.gpm_server_stats(srv)["peak_inflight"] == 1
    finally:
        G.gpm_server_free(srv)


def test_errors(graphs):
    hs, _ = graphs
    srv = G.gpm_server_create(1 << 30, 2)
    try:
        with pytest.raises(G.GpmError) as e:
            G.gpm_server_poll(srv, 12345)
        assert e.value.name == "GPM_E_INVALID_ARG"
        bad = G.pattern_from_edges(4, [(0, 1), (2, 3)])  # disconnected: no plan
        t = G.gpm_server_submit(srv, hs[0].handle, bad)
        with pytest.raises(G.GpmError) as e:
            G.gpm_server_wait(srv, t, 30.0)
        assert e.value.name == "GPM_E_UNSUPPORTED_PATTERN"
    finally:
        G.gpm_server_free(srv)
