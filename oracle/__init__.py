"""CPU oracle for pattern-aware subgraph enumeration — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path
(``paper_2112_09761_gb300``); see ``gpm_oracle.c`` for the three tiers
(O1 brute force = the definition of Section 2.1, O2 nested-loop plans after
Algorithm 1 / Sections 5-6, O3 closed-form decompositions after Section 5.4).

Pattern names and the vertex order of listed matches (the oracle's own
copies; a match tuple lists data vertices in the plan's matching order):

    triangle / k-clique   v1..vk, the DAG order of the clique
    diamond               (v1, v2) = the chord, v3 > v4 the two others
    4-cycle               v1 = max, cycle v1-v2-v3-v4-v1, v2 > v4
    tailed-triangle       v1 = degree-3 vertex, triangle v1 v2 v3 (v3 < v2), tail v4
    3-star                centre v1, leaves v2 > v3 > v4
    4-path                path v3-v1-v2-v4 (middle edge v1 > v2)
    wedge                 centre v1, ends v2 > v3

Parity status of every function is pinned (closed forms, brute force and
identities in ``tests/test_oracle.py``); no function here is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gpm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libgpm_oracle.so")
_lib = None

CLIQUE, DIAMOND, CYCLE4, TAILED_TRIANGLE, STAR3, PATH4, WEDGE = 1, 2, 3, 4, 5, 6, 7

# name -> (family code, k, pattern edges in the oracle's matching order)
PATTERNS = {
    "wedge": (WEDGE, 3, [(0, 1), (0, 2)]),
    "3-star": (STAR3, 4, [(0, 1), (0, 2), (0, 3)]),
    "4-path": (PATH4, 4, [(0, 1), (0, 2), (1, 3)]),
    "4-cycle": (CYCLE4, 4, [(0, 1), (1, 2), (2, 3), (3, 0)]),
    "tailed-triangle": (TAILED_TRIANGLE, 4, [(0, 1), (0, 2), (1, 2), (0, 3)]),
    "diamond": (DIAMOND, 4, [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3)]),
}
for _k in range(3, 9):
    PATTERNS[f"{_k}-clique"] = (CLIQUE, _k, [(i, j) for i in range(_k) for j in range(i + 1, _k)])
PATTERNS["triangle"] = PATTERNS["3-clique"]

MOTIF3 = ["wedge", "triangle"]
MOTIF4 = ["4-path", "3-star", "4-cycle", "tailed-triangle", "diamond", "4-clique"]


def build(force: bool = False) -> str:
    """Compile gpm_oracle.c into _build/libgpm_oracle.so (plain C, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
                               "-Wall", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i64p = ctypes.POINTER(ctypes.c_int64)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        lib.og_num_tasks.restype = ctypes.c_int64
        lib.og_num_tasks.argtypes = [i64p, u32p, ctypes.c_uint32, ctypes.c_int, ctypes.c_uint32]
        lib.og_count.restype = ctypes.c_int
        lib.og_count.argtypes = [i64p, u32p, ctypes.c_uint32, ctypes.c_int, ctypes.c_uint32,
                                 ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, u64p]
        lib.og_count_ranges.restype = ctypes.c_int
        lib.og_count_ranges.argtypes = [i64p, u32p, ctypes.c_uint32, ctypes.c_int, ctypes.c_uint32,
                                        ctypes.c_int, u64p, ctypes.c_uint64, ctypes.c_int, u64p,
                                        u64p, ctypes.POINTER(ctypes.c_double)]
        lib.og_list.restype = ctypes.c_int
        lib.og_list.argtypes = [i64p, u32p, ctypes.c_uint32, ctypes.c_int, ctypes.c_uint32,
                                ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, u32p,
                                ctypes.c_uint64, u64p]
        lib.og_brute.restype = ctypes.c_uint64
        lib.og_brute.argtypes = [i64p, u32p, ctypes.c_uint32, ctypes.c_uint32,
                                 ctypes.POINTER(ctypes.c_uint8), ctypes.c_uint32, ctypes.c_int]
        lib.og_automorphisms.restype = ctypes.c_uint64
        lib.og_automorphisms.argtypes = [ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint8),
                                         ctypes.c_uint32]
        lib.og_injhom.restype = ctypes.c_uint64
        lib.og_injhom.argtypes = [i64p, u32p, ctypes.c_uint32, ctypes.c_uint32,
                                  ctypes.POINTER(ctypes.c_uint8), ctypes.c_uint32, ctypes.c_int,
                                  ctypes.c_int]
        lib.og_connected_subsets.restype = ctypes.c_uint64
        lib.og_connected_subsets.argtypes = [i64p, u32p, ctypes.c_uint32, ctypes.c_uint32]
        lib.og_identities.restype = ctypes.c_int
        lib.og_identities.argtypes = [i64p, u32p, ctypes.c_uint32, ctypes.c_int, u64p]
        lib.og_motif4_inversion.argtypes = [u64p, u64p]
        _lib = lib
    return _lib


def _arrs(g):
    off = np.ascontiguousarray(g.offsets, dtype=np.int64)
    nbr = np.ascontiguousarray(g.nbrs, dtype=np.uint32)
    if len(nbr) == 0:
        nbr = np.zeros(1, dtype=np.uint32)
    return (off, nbr, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
            nbr.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))


def _check(rc: int):
    if rc == -2:
        raise ValueError("unsupported pattern family")
    if rc != 0:
        raise MemoryError("oracle allocation failed")


def num_tasks(g, pattern: str) -> int:
    fam, k, _ = PATTERNS[pattern]
    off, nbr, po, pn = _arrs(g)
    r = _L().og_num_tasks(po, pn, g.n, fam, k)
    _check(0 if r >= 0 else int(r))
    return int(r)


def count(g, pattern: str, induced: bool = False, task_lo: int = 0, task_hi: int | None = None,
          nthreads: int = 1) -> int:
    """O2: number of matches of `pattern` rooted at tasks [task_lo, task_hi)."""
    fam, k, _ = PATTERNS[pattern]
    off, nbr, po, pn = _arrs(g)
    out = ctypes.c_uint64(0)
    hi = (1 << 64) - 1 if task_hi is None else task_hi
    _check(_L().og_count(po, pn, g.n, fam, k, int(induced), task_lo, hi, nthreads,
                         ctypes.byref(out)))
    return out.value


def count_ranges(g, pattern: str, ranges, induced: bool = False, nthreads: int = 1,
                 per_range: bool = False):
    """O2 counts of task ranges [(lo, hi), ...] with one setup.  Returns
    (sum, seconds of the counting phase) or, with per_range, (list of counts,
    seconds)."""
    fam, k, _ = PATTERNS[pattern]
    off, nbr, po, pn = _arrs(g)
    rr = np.asarray(ranges, dtype=np.uint64).reshape(-1)
    if len(rr) == 0:
        return ([] if per_range else 0), 0.0
    nr = len(rr) // 2
    each = np.zeros(nr, dtype=np.uint64)
    out = ctypes.c_uint64(0)
    sec = ctypes.c_double(0.0)
    _check(_L().og_count_ranges(po, pn, g.n, fam, k, int(induced),
                                rr.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), nr, nthreads,
                                each.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                ctypes.byref(out), ctypes.byref(sec)))
    if per_range:
        return [int(x) for x in each], sec.value
    return out.value, sec.value


def list_matches(g, pattern: str, induced: bool = False, task_lo: int = 0,
                 task_hi: int | None = None, cap: int = 1 << 20) -> tuple[np.ndarray, int]:
    """O2 listing: (array [min(total, cap), k] of matches, total)."""
    fam, k, _ = PATTERNS[pattern]
    off, nbr, po, pn = _arrs(g)
    buf = np.zeros(max(1, cap) * k, dtype=np.uint32)
    total = ctypes.c_uint64(0)
    hi = (1 << 64) - 1 if task_hi is None else task_hi
    _check(_L().og_list(po, pn, g.n, fam, k, int(induced), task_lo, hi,
                        buf.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), cap,
                        ctypes.byref(total)))
    t = total.value
    return buf[: min(t, cap) * k].reshape(-1, k), t


def brute(g, k: int, edges, induced: bool) -> int:
    """O1: the definition of Section 2.1 by exhaustive search (tiny graphs)."""
    off, nbr, po, pn = _arrs(g)
    pe = np.asarray(edges, dtype=np.uint8).reshape(-1)
    if len(pe) == 0:
        pe = np.zeros(2, dtype=np.uint8)
    return int(_L().og_brute(po, pn, g.n, k, pe.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                             len(edges), int(induced)))


def brute_named(g, pattern: str, induced: bool) -> int:
    _, k, edges = PATTERNS[pattern]
    return brute(g, k, edges, induced)


def _pattern_bytes(edges):
    pe = np.asarray(edges, dtype=np.uint8).reshape(-1)
    if len(pe) == 0:
        pe = np.zeros(2, dtype=np.uint8)
    return pe


def automorphisms(k: int, edges) -> int:
    """|Aut(P)| by trying every permutation of the k pattern vertices."""
    pe = _pattern_bytes(edges)
    return int(_L().og_automorphisms(k, pe.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                     len(edges)))


def injhom(g, k: int, edges, induced: bool, nthreads: int = 1) -> int:
    """O1b: injective homomorphisms P -> G (embeddings before symmetry breaking)."""
    off, nbr, po, pn = _arrs(g)
    pe = _pattern_bytes(edges)
    return int(_L().og_injhom(po, pn, g.n, k, pe.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                              len(edges), int(induced), nthreads))


def count_any(g, k: int, edges, induced: bool, nthreads: int = 1) -> int:
    """Count of Section 2.1 for any pattern: injective homomorphisms / |Aut(P)|."""
    h = injhom(g, k, edges, induced, nthreads)
    a = automorphisms(k, edges)
    assert h % a == 0, "embeddings must split into whole automorphism classes"
    return h // a


def connected_subsets(g, k: int) -> int:
    off, nbr, po, pn = _arrs(g)
    return int(_L().og_connected_subsets(po, pn, g.n, k))


def identities(g, nthreads: int = 1) -> dict:
    """O3 closed forms (see og_identities in gpm_oracle.c)."""
    off, nbr, po, pn = _arrs(g)
    out = (ctypes.c_uint64 * 8)()
    _check(_L().og_identities(po, pn, g.n, nthreads, out))
    keys = ["triangle", "wedge_e", "3-star_e", "4-path_e", "tailed-triangle_e", "diamond_e",
            "4-cycle_e", "wedge_v"]
    return {k: int(v) for k, v in zip(keys, out)}


def motif4_induced_from_edge(edge_counts: list[int]) -> list[int]:
    """Vertex-induced 4-motif counts from edge-induced ones (MOTIF4 order)."""
    inp = (ctypes.c_uint64 * 6)(*[int(x) for x in edge_counts])
    out = (ctypes.c_uint64 * 6)()
    _L().og_motif4_inversion(inp, out)
    return [int(x) for x in out]


def motif_counts(g, k: int, nthreads: int = 1, method: str = "enumerate") -> list[int]:
    """Induced k-motif counts (k = 3: MOTIF3 order, k = 4: MOTIF4 order).

    method="enumerate" runs the O2 plans per pattern; method="identities"
    uses O3 closed forms plus the O2 4-clique count and the inversion.
    """
    names = MOTIF3 if k == 3 else MOTIF4
    if method == "enumerate":
        return [count(g, p, induced=True, nthreads=nthreads) for p in names]
    ids = identities(g, nthreads)
    if k == 3:
        return [ids["wedge_v"], ids["triangle"]]
    k4 = count(g, "4-clique", nthreads=nthreads)
    edge = [ids["4-path_e"], ids["3-star_e"], ids["4-cycle_e"], ids["tailed-triangle_e"],
            ids["diamond_e"], k4]
    return motif4_induced_from_edge(edge)


def canonical(match, edges) -> tuple:
    """A match as (sorted vertex tuple, sorted tuple of mapped edges)."""
    vs = tuple(sorted(int(x) for x in match))
    es = tuple(sorted(tuple(sorted((int(match[a]), int(match[b])))) for a, b in edges))
    return vs, es
