"""Seeded synthetic data graphs (inputs only; no pattern-matching arithmetic).

Both the CUDA path and the CPU oracle read the CSR arrays built here and share
nothing else.  The generators follow the workload shapes of the paper's
evaluation (Section 8, Table "tab:input": power-law degrees, maximum degree
10^3..10^6, |E| 10^7..10^9) with seeded stand-ins:

* ``er_graph``       Erdős–Rényi G(n, m), m distinct pairs without replacement.
* ``rmat_graph``     R-MAT (a, b, c, d) edge draws, symmetrised, deduplicated,
                     loops dropped, vertex IDs seed-permuted (Graph500 style).
* ``chung_lu_graph`` Chung–Lu power-law graph with hubs.
* small closed-form graphs (K_n, K_{a,b}, stars, paths, cycles) and G(n, p).

Every random draw is a pure function of (seed, stream, index), see
``graphgen.c``; the same seed yields byte-identical CSR arrays on x86-64 and
AArch64, which ``csr_checksum`` lets a test confirm.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libgraphgen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile graphgen.c into _build/libgraphgen.so (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u32p = ctypes.POINTER(ctypes.c_uint32)
        lib.gg_rand.restype = ctypes.c_uint64
        lib.gg_rand.argtypes = [ctypes.c_uint64] * 3
        lib.gg_build_csr.restype = ctypes.c_int
        lib.gg_build_csr.argtypes = [ctypes.c_uint32, u32p, u32p, ctypes.c_uint64,
                                     ctypes.POINTER(ctypes.c_int64),
                                     ctypes.POINTER(u32p), ctypes.POINTER(ctypes.c_uint64)]
        lib.gg_free.argtypes = [ctypes.c_void_p]
        lib.gg_permutation.argtypes = [ctypes.c_uint32, ctypes.c_uint64, u32p]
        lib.gg_apply_perm.argtypes = [u32p, u32p, ctypes.c_uint64]
        lib.gg_er.restype = ctypes.c_int
        lib.gg_er.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, u32p, u32p]
        lib.gg_rmat.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64, u32p, u32p]
        lib.gg_chung_lu.restype = ctypes.c_int
        lib.gg_chung_lu.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_uint64, u32p, u32p]
        lib.gg_gnp.restype = ctypes.c_uint64
        lib.gg_gnp.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64, u32p, u32p]
        lib.gg_fnv1a.restype = ctypes.c_uint64
        lib.gg_fnv1a.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64]
        _lib = lib
    return _lib


def _u32p(a: np.ndarray):
    assert a.dtype == np.uint32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


@dataclass
class CSR:
    """A simple undirected graph: ascending rows, both directions, no loops/dups."""
    n: int
    offsets: np.ndarray  # int64[n+1]
    nbrs: np.ndarray     # uint32[offsets[n]]
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.offsets[-1])

    @property
    def m(self) -> int:
        """Number of undirected edges."""
        return self.nnz // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.offsets)

    def max_degree(self) -> int:
        return int(self.degrees().max()) if self.n else 0


def from_pairs(n: int, us: np.ndarray, vs: np.ndarray, name: str = "") -> CSR:
    """Symmetrise, drop loops, sort rows and dedup a list of endpoint pairs."""
    L = _L()
    us = np.ascontiguousarray(us, dtype=np.uint32)
    vs = np.ascontiguousarray(vs, dtype=np.uint32)
    off = np.zeros(n + 1, dtype=np.int64)
    nbr_p = ctypes.POINTER(ctypes.c_uint32)()
    nnz = ctypes.c_uint64(0)
    rc = L.gg_build_csr(n, _u32p(us), _u32p(vs), len(us),
                        off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                        ctypes.byref(nbr_p), ctypes.byref(nnz))
    if rc != 0:
        raise MemoryError("gg_build_csr failed")
    count = nnz.value
    nbrs = np.empty(count, dtype=np.uint32)
    if count:
        ctypes.memmove(nbrs.ctypes.data, nbr_p, count * 4)
    L.gg_free(nbr_p)
    return CSR(n, off, nbrs, name)


def from_edges(n: int, edges, name: str = "") -> CSR:
    e = np.asarray(list(edges), dtype=np.int64).reshape(-1, 2)
    return from_pairs(n, e[:, 0].astype(np.uint32), e[:, 1].astype(np.uint32), name)


def permute(g: CSR, seed: int) -> CSR:
    """Relabel vertices by a seeded permutation (counts are invariant)."""
    L = _L()
    perm = np.empty(g.n, dtype=np.uint32)
    L.gg_permutation(g.n, seed, _u32p(perm))
    src = np.repeat(np.arange(g.n, dtype=np.uint32), np.diff(g.offsets))
    us, vs = perm[src], perm[g.nbrs]
    keep = us < vs
    return from_pairs(g.n, us[keep].copy(), vs[keep].copy(), g.name + f"~perm{seed}")


# ------------------------------------------------------------ generators

def er_graph(n: int, m: int, seed: int) -> CSR:
    """G(n, m): exactly m distinct undirected pairs, uniform without replacement."""
    L = _L()
    us = np.empty(m, dtype=np.uint32)
    vs = np.empty(m, dtype=np.uint32)
    if L.gg_er(n, m, seed, _u32p(us), _u32p(vs)) != 0:
        raise ValueError("invalid G(n,m) parameters")
    return from_pairs(n, us, vs, f"er-n{n}-m{m}-s{seed}")


def _fixed(p: float) -> int:
    return min(int(round(p * 2**32)), 2**32 - 1)


def rmat_graph(scale: int, edge_factor: int, seed: int, a=0.57, b=0.19, c=0.19,
               n: int | None = None, ndraws: int | None = None, permute_ids: bool = True) -> CSR:
    """R-MAT graph; `n` < 2^scale rejects and redraws out-of-range endpoints."""
    L = _L()
    nv = n if n is not None else (1 << scale)
    draws = ndraws if ndraws is not None else edge_factor * nv
    us = np.empty(draws, dtype=np.uint32)
    vs = np.empty(draws, dtype=np.uint32)
    L.gg_rmat(scale, draws, _fixed(a), _fixed(a + b), _fixed(a + b + c), nv, seed,
              _u32p(us), _u32p(vs))
    if permute_ids:
        perm = np.empty(nv, dtype=np.uint32)
        L.gg_permutation(nv, seed, _u32p(perm))
        L.gg_apply_perm(_u32p(perm), _u32p(us), draws)
        L.gg_apply_perm(_u32p(perm), _u32p(vs), draws)
    return from_pairs(nv, us, vs, f"rmat-s{scale}-ef{edge_factor}-seed{seed}")


def chung_lu_graph(n: int, npairs: int, seed: int, wmax: float = 80000.0, i0: float = 49.73,
                   gamma: float = 2.1, permute_ids: bool = True) -> CSR:
    """Chung–Lu power-law graph (degree exponent gamma), hubs seed-permuted."""
    L = _L()
    us = np.empty(npairs, dtype=np.uint32)
    vs = np.empty(npairs, dtype=np.uint32)
    if L.gg_chung_lu(n, npairs, wmax, i0, gamma, seed, _u32p(us), _u32p(vs)) != 0:
        raise MemoryError("gg_chung_lu failed")
    if permute_ids:
        perm = np.empty(n, dtype=np.uint32)
        L.gg_permutation(n, seed, _u32p(perm))
        L.gg_apply_perm(_u32p(perm), _u32p(us), npairs)
        L.gg_apply_perm(_u32p(perm), _u32p(vs), npairs)
    return from_pairs(n, us, vs, f"chunglu-n{n}-p{npairs}-seed{seed}")


def gnp_graph(n: int, p: float, seed: int) -> CSR:
    L = _L()
    cap = max(1, n * (n - 1) // 2)
    us = np.empty(cap, dtype=np.uint32)
    vs = np.empty(cap, dtype=np.uint32)
    k = L.gg_gnp(n, _fixed(p), seed, _u32p(us), _u32p(vs))
    return from_pairs(n, us[:k].copy(), vs[:k].copy(), f"gnp-n{n}-p{p}-s{seed}")


def complete(n: int) -> CSR:
    return from_edges(n, [(u, v) for u in range(n) for v in range(u + 1, n)], f"K{n}")


def complete_bipartite(a: int, b: int) -> CSR:
    return from_edges(a + b, [(u, a + v) for u in range(a) for v in range(b)], f"K{a},{b}")


def star(leaves: int) -> CSR:
    return from_edges(leaves + 1, [(0, i) for i in range(1, leaves + 1)], f"S{leaves}")


def path(n: int) -> CSR:
    return from_edges(n, [(i, i + 1) for i in range(n - 1)], f"P{n}")


def cycle(n: int) -> CSR:
    return from_edges(n, [(i, (i + 1) % n) for i in range(n)], f"C{n}")


def empty(n: int) -> CSR:
    return CSR(n, np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.uint32), f"E{n}")


def csr_checksum(g: CSR) -> str:
    """FNV-1a of the offsets and neighbour arrays (host-independent)."""
    L = _L()
    h = L.gg_fnv1a(g.offsets.ctypes.data, g.offsets.nbytes, 0)
    h = L.gg_fnv1a(g.nbrs.ctypes.data, g.nbrs.nbytes, h)
    return f"{h:016x}"


# ------------------------------------------------- named workload recipes

def workload(name: str) -> CSR:
    """The seeded synthetic workloads, by name.

    er-10k      G(n=10,000, m=80,000), seed 1 (average degree 16)
    rmat22      R-MAT scale 22, edge factor 16, (0.57, 0.19, 0.19, 0.05), seed 2
    chunglu-1m  Chung–Lu n=10^6, 32,000,000 endpoint pairs, gamma 2.1, seed 3
    rmat25      R-MAT scale 25, edge factor 16, same (a, b, c, d), seed 25
    batch-<i>   graph i of the 2,000-graph batch (seed 4000+i): n ~ U{1K..200K},
                average degree ~ U[4, 64]; even i G(n, floor(n d/2)), odd i
                R-MAT a=0.57 at scale ceil(log2 n) with floor(n d/2) draws
    rmat<s>     R-MAT scale s (smaller stand-ins for tests), seed s
    chunglu-<n> Chung–Lu with n vertices and 32 n endpoint pairs (scaled weights)
    """
    if name == "er-10k":
        return er_graph(10_000, 80_000, 1)
    if name == "rmat22":
        return rmat_graph(22, 16, 2)
    if name == "chunglu-1m":
        return chung_lu_graph(1_000_000, 32_000_000, 3)
    if name == "rmat25":
        return rmat_graph(25, 16, 25)
    if name.startswith("batch-"):
        return batch_graph(int(name.split("-")[1]))
    if name.startswith("rmat"):
        s = int(name[4:])
        return rmat_graph(s, 16, s)
    if name.startswith("chunglu-"):
        n = int(name.split("-")[1])
        # keep the same shape: weights scaled so that sum(w) ~ 64 n, hub ~ 0.08 n
        return chung_lu_graph(n, 32 * n, 3, wmax=0.08 * n, i0=49.73 * n / 1_000_000)
    raise KeyError(name)


def batch_params(i: int) -> tuple[int, float, str]:
    """(n, average degree, kind) of batch graph i, drawn from seed 4000+i."""
    L = _L()
    seed = 4000 + i
    r0 = L.gg_rand(seed, 7, 0)
    r1 = L.gg_rand(seed, 7, 1)
    n = 1000 + int((r0 * (200_000 - 1000 + 1)) >> 64)
    d = 4.0 + 60.0 * ((r1 >> 11) / float(1 << 53))
    return n, d, ("er" if i % 2 == 0 else "rmat")


def batch_graph(i: int) -> CSR:
    n, d, kind = batch_params(i)
    m = int(math.floor(n * d / 2))
    seed = 4000 + i
    if kind == "er":
        g = er_graph(n, m, seed)
    else:
        scale = max(1, math.ceil(math.log2(n)))
        g = rmat_graph(scale, 0, seed, n=n, ndraws=m)
    g.name = f"batch-{i}"
    return g
