"""The pattern analyzer of the generic plans (Section 4.2), host side only: no
GPU.  Its symmetry orders are checked against the paper's diamond example and
against the oracle's automorphism counts: along a stabiliser chain, the orbit
sizes multiply to |Aut(P)|, and position s's orbit is s plus the positions
it is constrained to exceed."""
import itertools
import math
import re

import pytest

import oracle as O
import paper_2112_09761_gb300 as G

from test_oracle import EXTRA_PATTERNS

NAMED = ["triangle", "wedge", "4-clique", "5-clique", "6-clique", "diamond", "4-cycle",
         "tailed-triangle", "3-star", "4-path"]


def _all_patterns():
    out = {name: (O.PATTERNS[name][1], O.PATTERNS[name][2]) for name in NAMED}
    out.update(EXTRA_PATTERNS)
    out["cube"] = (8, [(a, b) for a in range(8) for b in range(a + 1, 8)
                       if bin(a ^ b).count("1") == 1])
    out["8-cycle"] = (8, [(i, (i + 1) % 8) for i in range(8)])
    return out


def _parse(text):
    order = [int(x) for x in re.search(r"order: ([u0-9 ]+);", text).group(1).replace("u", "").split()]
    sym = re.search(r"symmetry: ([^;]+);", text).group(1).strip()
    cons = [] if sym == "none" else [tuple(map(int, c.replace("v", "").split(">")))
                                     for c in sym.split()]
    lower = "tasks: pairs v0>v1" in text
    return order, cons, lower


def test_diamond_symmetry_order_is_the_papers():
    # Section 2.2: with the chord matched first, v1 > v2 and v3 > v4
    text = G.gpm_pattern_describe("diamond", generic=True, n=10**6, nnz=3 * 10**7)
    order, cons, lower = _parse(text)
    assert set(order[:2]) == {0, 1}                 # the chord (degree-3 vertices) first
    assert sorted(cons) == [(0, 1), (2, 3)]
    assert lower                                     # Section 7.2 (2) edgelist reduction


@pytest.mark.parametrize("name", sorted(_all_patterns()))
@pytest.mark.parametrize("induced", [False, True])
def test_stabiliser_chain_orbits_multiply_to_aut(name, induced):
    k, edges = _all_patterns()[name]
    p = G.pattern_from_edges(k, edges)
    text = G.gpm_pattern_describe(p, induced=induced, n=50_000, nnz=1_000_000, generic=True)
    order, cons, lower = _parse(text)
    assert sorted(order) == list(range(k))
    adj = {(a, b) for a, b in edges} | {(b, a) for a, b in edges}
    # a valid matching order: a root edge, then each vertex joined to an earlier one
    assert (order[0], order[1]) in adj
    for t in range(2, k):
        assert any((order[t], order[s]) in adj for s in range(t))
    # constraints run from an earlier to a later position
    assert all(s < t for s, t in cons)
    orbit = [1] * k
    for s, _ in cons:
        orbit[s] += 1
    assert math.prod(orbit) == O.automorphisms(k, edges)
    assert lower == ((0, 1) in cons)
    assert ("vertex-induced" in text) == induced


def test_constraints_break_every_symmetry_exactly_once():
    # brute force on the house pattern: among the |Aut| relabellings of one
    # embedding, exactly one satisfies the symmetry order
    k, edges = EXTRA_PATTERNS["house"]
    text = G.gpm_pattern_describe(G.pattern_from_edges(k, edges), generic=True, n=1000, nnz=8000)
    order, cons, _ = _parse(text)
    adj = {(a, b) for a, b in edges} | {(b, a) for a, b in edges}
    auts = [p for p in itertools.permutations(range(k))
            if all((p[a], p[b]) in adj for a, b in edges)]
    ids = [17, 3, 42, 8, 25]                          # an embedding: pattern vertex -> data ID
    ok = 0
    for g in auts:
        img = [ids[g[u]] for u in range(k)]           # the same subgraph, relabelled
        pos_val = [img[order[t]] for t in range(k)]
        ok += all(pos_val[s] > pos_val[t] for s, t in cons)
    assert ok == 1


def test_named_families_keep_their_plans():
    assert G.gpm_pattern_describe("diamond").startswith("family: diamond")
    assert G.gpm_pattern_describe("5-clique").startswith("family: k-clique (k = 5)")
    k, edges = EXTRA_PATTERNS["5-cycle"]
    assert G.gpm_pattern_describe(G.pattern_from_edges(k, edges)).startswith("family: generic")


def test_unsupported_patterns():
    for k, edges in ((4, [(0, 1), (2, 3)]),            # disconnected
                     (2, [(0, 1)]),                     # too small
                     (3, [(0, 1), (1, 1)])):            # self-loop
        with pytest.raises(G.GpmError) as ei:
            G.gpm_pattern_describe(G.pattern_from_edges(k, edges))
        assert ei.value.name == "GPM_E_UNSUPPORTED_PATTERN"
