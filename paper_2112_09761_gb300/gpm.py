"""Thin ctypes binding of the C ABI in include/gpm.h (argument marshalling only).

Every function here has the name of the C entry point it wraps and does no
computation of its own: all enumeration work runs in libgpm.so's CUDA kernels.
If the library has not been built, or the process has no GPU, calls fail
loudly (RuntimeError / GpmError with GPM_E_CUDA); there is no CPU fallback.

PyTorch is used only for device memory (listing buffers, device-resident CSR
arrays) and for the current CUDA stream.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

from . import _build

GPM_OK = 0
STATUS = {0: "GPM_OK", 1: "GPM_E_INVALID_ARG", 2: "GPM_E_UNSORTED", 3: "GPM_E_SELF_LOOP",
          4: "GPM_E_DUPLICATE", 5: "GPM_E_ASYMMETRIC", 6: "GPM_E_OOM",
          7: "GPM_E_UNSUPPORTED_PATTERN", 8: "GPM_E_CAPACITY", 9: "GPM_E_TIMEOUT",
          10: "GPM_E_CUDA", 11: "GPM_E_RANGE"}
GPM_E_CAPACITY = 8
GPM_DEVICE_PTRS, GPM_BORROW, GPM_SKIP_VALIDATE, GPM_RELABEL = 1, 2, 4, 8
GPM_COUNT, GPM_LIST = 0, 1


class GpmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status
        self.name = STATUS.get(status, str(status))


class gpm_pattern(ctypes.Structure):
    _fields_ = [("k", ctypes.c_uint32), ("n_edges", ctypes.c_uint32),
                ("edges", (ctypes.c_uint8 * 2) * 28)]

    def edge_list(self):
        return [(int(self.edges[i][0]), int(self.edges[i][1])) for i in range(self.n_edges)]


class gpm_plan_opts(ctypes.Structure):
    _fields_ = [("warps_per_block", ctypes.c_uint32), ("blocks_per_sm", ctypes.c_uint32),
                ("chunk", ctypes.c_uint32), ("bsearch_ratio", ctypes.c_uint32),
                ("no_count_only", ctypes.c_uint32), ("collect_stats", ctypes.c_uint32),
                ("no_lgs", ctypes.c_uint32), ("generic_plan", ctypes.c_uint32),
                ("vertex_parallel", ctypes.c_uint32)]


_lib = None


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libgpm.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libgpm.so is not built ({path}); run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        vp, u32, u64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
        u64p = ctypes.POINTER(ctypes.c_uint64)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        L.gpm_last_error.restype = ctypes.c_char_p
        L.gpm_version.restype = ctypes.c_char_p
        L.gpm_pattern_named.argtypes = [ctypes.c_char_p, ctypes.POINTER(gpm_pattern)]
        L.gpm_load_csr.argtypes = [vp, ctypes.c_int, vp, u32, u64, u32, vp, ctypes.POINTER(vp)]
        L.gpm_graph_info.argtypes = [vp, u32p, u64p, u32p, u32p]
        L.gpm_graph_export.argtypes = [vp, vp, vp, vp, vp]
        L.gpm_graph_free.argtypes = [vp]
        L.gpm_graph_free.restype = None
        L.gpm_plan.argtypes = [vp, ctypes.POINTER(gpm_pattern), ctypes.c_int, ctypes.c_int,
                               ctypes.POINTER(gpm_plan_opts), vp, ctypes.POINTER(vp)]
        L.gpm_plan_info.argtypes = [vp, u64p, u32p]
        L.gpm_plan_describe.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t]
        L.gpm_plan_launches.argtypes = [vp, u32p]
        L.gpm_pattern_describe.argtypes = [ctypes.POINTER(gpm_pattern), ctypes.c_int, u32, u64,
                                           ctypes.c_int, ctypes.c_char_p, ctypes.c_size_t]
        L.gpm_count.argtypes = [vp, u64p, vp]
        L.gpm_count_range.argtypes = [vp, u64, u64, u64p, vp]
        L.gpm_list.argtypes = [vp, vp, u64, u64p, u64p, vp]
        L.gpm_plan_stats.argtypes = [vp, u64p, u64p, u64p]
        L.gpm_motif_count.argtypes = [vp, u32, u64p, vp]
        L.gpm_batch_create.argtypes = [ctypes.POINTER(vp), u32, u32, ctypes.POINTER(gpm_plan_opts),
                                       vp, ctypes.POINTER(vp)]
        L.gpm_batch_count.argtypes = [vp, u64p, vp]
        L.gpm_batch_info.argtypes = [vp, u32p, u32p, u32p]
        L.gpm_batch_free.argtypes = [vp]
        L.gpm_batch_free.restype = None
        L.gpm_server_create.argtypes = [ctypes.c_size_t, u32, ctypes.POINTER(vp)]
        L.gpm_server_submit.argtypes = [vp, vp, ctypes.POINTER(gpm_pattern), ctypes.c_int, u64p]
        L.gpm_server_poll.argtypes = [vp, u64, ctypes.POINTER(ctypes.c_int), u64p,
                                      ctypes.POINTER(ctypes.c_double)]
        L.gpm_server_wait.argtypes = [vp, u64, ctypes.c_double, u64p, ctypes.POINTER(ctypes.c_double)]
        L.gpm_server_stats.argtypes = [vp, u64p, u64p, u64p, ctypes.POINTER(ctypes.c_size_t)]
        L.gpm_server_free.argtypes = [vp]
        L.gpm_server_free.restype = None
        L.gpm_count_triangles_noalloc.argtypes = [vp, vp, u32, vp, vp]
        L.gpm_plan_free.argtypes = [vp]
        L.gpm_plan_free.restype = None
        for name in ("gpm_pattern_named", "gpm_load_csr", "gpm_graph_info", "gpm_plan",
                     "gpm_plan_info", "gpm_count", "gpm_count_range", "gpm_list", "gpm_plan_stats",
                     "gpm_motif_count", "gpm_batch_create", "gpm_batch_count", "gpm_batch_info",
                     "gpm_server_create", "gpm_server_submit", "gpm_server_poll",
                     "gpm_server_wait", "gpm_server_stats", "gpm_count_triangles_noalloc"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def header_functions() -> list[str]:
    """Names of the functions declared in include/gpm.h."""
    path = os.path.join(_build.ROOT, "include", "gpm.h")
    with open(path) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gpm_[a-z_0-9]+)\s*\(", text)))


def _check(status: int):
    if status != GPM_OK:
        raise GpmError(status, gpm_last_error())


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return ctypes.c_void_p(0)


def gpm_last_error() -> str:
    return lib().gpm_last_error().decode()


def gpm_version() -> str:
    return lib().gpm_version().decode()


def gpm_pattern_named(name: str) -> gpm_pattern:
    p = gpm_pattern()
    _check(lib().gpm_pattern_named(name.encode(), ctypes.byref(p)))
    return p


def pattern_from_edges(k: int, edges) -> gpm_pattern:
    p = gpm_pattern()
    p.k = k
    edges = list(edges)
    p.n_edges = len(edges)
    for i, (a, b) in enumerate(edges):
        p.edges[i][0] = a
        p.edges[i][1] = b
    return p


def gpm_load_csr(offsets, nbrs, n: int | None = None, flags: int = 0, stream=None):
    """Load a CSR (numpy host arrays, or torch CUDA tensors with GPM_DEVICE_PTRS)."""
    keep = []
    if hasattr(offsets, "data_ptr"):  # torch tensor
        is64 = int(offsets.dtype.itemsize == 8)
        po, pn = offsets.data_ptr(), (nbrs.data_ptr() if nbrs.numel() else 0)
        nnz = int(nbrs.numel())
        nv = int(offsets.numel()) - 1 if n is None else n
        if offsets.is_cuda:
            flags |= GPM_DEVICE_PTRS
        keep = [offsets, nbrs]
    else:
        off = np.ascontiguousarray(offsets)
        if off.dtype not in (np.int64, np.int32):
            off = off.astype(np.int64)
        nb = np.ascontiguousarray(nbrs, dtype=np.uint32)
        is64 = int(off.dtype == np.int64)
        po, pn = off.ctypes.data, (nb.ctypes.data if len(nb) else 0)
        nnz = int(len(nb))
        nv = len(off) - 1 if n is None else n
        keep = [off, nb]
    h = ctypes.c_void_p()
    _check(lib().gpm_load_csr(ctypes.c_void_p(po), is64, ctypes.c_void_p(pn), nv, nnz, flags,
                              _stream(stream), ctypes.byref(h)))
    del keep
    return h


def gpm_graph_info(g) -> dict:
    n, m, d, do = ctypes.c_uint32(), ctypes.c_uint64(), ctypes.c_uint32(), ctypes.c_uint32()
    _check(lib().gpm_graph_info(g, ctypes.byref(n), ctypes.byref(m), ctypes.byref(d),
                                ctypes.byref(do)))
    return {"n": n.value, "n_edges": m.value, "max_degree": d.value, "max_out_degree": do.value}


def gpm_graph_export(g):
    """(offsets int64[n+1], nbrs uint32[nnz], perm uint32[n]) as the library holds the graph."""
    info = gpm_graph_info(g)
    n, nnz = info["n"], 2 * info["n_edges"]
    off = np.zeros(n + 1, dtype=np.int64)
    nbr = np.zeros(max(nnz, 1), dtype=np.uint32)
    perm = np.zeros(max(n, 1), dtype=np.uint32)
    _check(lib().gpm_graph_export(g, off.ctypes.data, nbr.ctypes.data, perm.ctypes.data, None))
    return off, nbr[:nnz], perm[:n]


def gpm_graph_free(g) -> None:
    lib().gpm_graph_free(g)


def gpm_plan(g, pattern, induced: bool = False, mode: int = GPM_COUNT, opts: dict | None = None,
             stream=None):
    if isinstance(pattern, str):
        pattern = gpm_pattern_named(pattern)
    o = None
    if opts:
        o = gpm_plan_opts()
        for key, val in opts.items():
            setattr(o, key, int(val))
    h = ctypes.c_void_p()
    _check(lib().gpm_plan(g, ctypes.byref(pattern), int(bool(induced)), mode,
                          ctypes.byref(o) if o is not None else None, _stream(stream),
                          ctypes.byref(h)))
    return h


def gpm_plan_info(p) -> dict:
    nt, k = ctypes.c_uint64(), ctypes.c_uint32()
    _check(lib().gpm_plan_info(p, ctypes.byref(nt), ctypes.byref(k)))
    return {"n_tasks": nt.value, "k": k.value}


def gpm_plan_launches(p) -> int:
    """Kernels one evaluation of the plan enqueues."""
    n = ctypes.c_uint32()
    _check(lib().gpm_plan_launches(p, ctypes.byref(n)))
    return n.value


def gpm_plan_describe(p) -> str:
    buf = ctypes.create_string_buffer(1024)
    _check(lib().gpm_plan_describe(p, buf, len(buf)))
    return buf.value.decode()


def gpm_pattern_describe(pattern, induced: bool = False, n: int = 0, nnz: int = 0,
                         generic: bool = False) -> str:
    """Host-side pattern analysis: the search plan text gpm_plan would use."""
    if isinstance(pattern, str):
        pattern = gpm_pattern_named(pattern)
    buf = ctypes.create_string_buffer(1024)
    _check(lib().gpm_pattern_describe(ctypes.byref(pattern), int(bool(induced)), n, nnz,
                                      int(bool(generic)), buf, len(buf)))
    return buf.value.decode()


def gpm_count(p, stream=None) -> int:
    out = ctypes.c_uint64()
    _check(lib().gpm_count(p, ctypes.byref(out), _stream(stream)))
    return out.value


def gpm_count_range(p, task_lo: int, task_hi: int, stream=None) -> int:
    out = ctypes.c_uint64()
    _check(lib().gpm_count_range(p, task_lo, task_hi, ctypes.byref(out), _stream(stream)))
    return out.value


def gpm_list(p, capacity: int, out=None, stream=None):
    """List matches into a device buffer; returns (tensor[n_written, k], n_total, truncated)."""
    import torch
    k = gpm_plan_info(p)["k"]
    if out is None:
        out = torch.empty((max(capacity, 1), k), dtype=torch.int32, device="cuda")
    nw, nt = ctypes.c_uint64(), ctypes.c_uint64()
    st = lib().gpm_list(p, ctypes.c_void_p(out.data_ptr()), capacity, ctypes.byref(nw),
                        ctypes.byref(nt), _stream(stream))
    if st not in (GPM_OK, GPM_E_CAPACITY):
        _check(st)
    return out[: nw.value], nt.value, st == GPM_E_CAPACITY


def gpm_plan_stats(p) -> dict:
    b, n, w = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().gpm_plan_stats(p, ctypes.byref(b), ctypes.byref(n), ctypes.byref(w)))
    return {"alg_bytes": b.value, "set_ops": n.value, "word_ops": w.value}


MOTIF3 = ["wedge", "triangle"]
MOTIF4 = ["4-path", "3-star", "4-cycle", "tailed-triangle", "diamond", "4-clique"]


def gpm_motif_count(g, k: int, stream=None) -> list[int]:
    """Vertex-induced k-motif counts (k = 3: MOTIF3 order, k = 4: MOTIF4 order)."""
    w = 2 if k == 3 else 6
    out = (ctypes.c_uint64 * w)()
    _check(lib().gpm_motif_count(g, k, out, _stream(stream)))
    return [int(x) for x in out]


def _opts(opts):
    if not opts:
        return None
    o = gpm_plan_opts()
    for key, val in opts.items():
        setattr(o, key, int(val))
    return o


def gpm_batch_create(graphs, k: int, opts: dict | None = None, stream=None):
    arr = (ctypes.c_void_p * len(graphs))(*[ctypes.c_void_p(getattr(h, "value", h)) for h in graphs])
    o = _opts(opts)
    h = ctypes.c_void_p()
    _check(lib().gpm_batch_create(arr, len(graphs), k, ctypes.byref(o) if o is not None else None,
                                  _stream(stream), ctypes.byref(h)))
    h._n = len(graphs)
    h._k = k
    return h


def gpm_batch_count(b, stream=None) -> np.ndarray:
    w = 2 if b._k == 3 else 6
    out = np.zeros((b._n, w), dtype=np.uint64)
    _check(lib().gpm_batch_count(b, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                 _stream(stream)))
    return out


def gpm_batch_info(b) -> dict:
    c, r, w = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    _check(lib().gpm_batch_info(b, ctypes.byref(c), ctypes.byref(r), ctypes.byref(w)))
    return {"chunk": c.value, "bsearch_ratio": r.value, "warps_per_block": w.value}


def gpm_batch_free(b) -> None:
    lib().gpm_batch_free(b)


def gpm_server_create(mem_budget: int, max_inflight: int = 8):
    h = ctypes.c_void_p()
    _check(lib().gpm_server_create(mem_budget, max_inflight, ctypes.byref(h)))
    return h


def gpm_server_submit(srv, g, pattern, induced: bool = False) -> int:
    if isinstance(pattern, str):
        pattern = gpm_pattern_named(pattern)
    t = ctypes.c_uint64()
    _check(lib().gpm_server_submit(srv, g, ctypes.byref(pattern), int(bool(induced)),
                                   ctypes.byref(t)))
    return t.value


def gpm_server_poll(srv, ticket: int):
    """(done, count, latency_s) — count/latency are None while running."""
    d, c, l = ctypes.c_int(), ctypes.c_uint64(), ctypes.c_double()
    _check(lib().gpm_server_poll(srv, ticket, ctypes.byref(d), ctypes.byref(c), ctypes.byref(l)))
    return (True, c.value, l.value) if d.value else (False, None, None)


def gpm_server_wait(srv, ticket: int, timeout_s: float = 600.0):
    """(count, latency_s)."""
    c, l = ctypes.c_uint64(), ctypes.c_double()
    _check(lib().gpm_server_wait(srv, ticket, timeout_s, ctypes.byref(c), ctypes.byref(l)))
    return c.value, l.value


def gpm_server_stats(srv) -> dict:
    c, p, pk, b = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_size_t()
    _check(lib().gpm_server_stats(srv, ctypes.byref(c), ctypes.byref(p), ctypes.byref(pk),
                                  ctypes.byref(b)))
    return {"completed": c.value, "pending": p.value, "peak_inflight": pk.value,
            "bytes_in_use": b.value}


def gpm_server_free(srv) -> None:
    lib().gpm_server_free(srv)


def gpm_count_triangles_noalloc(offsets_dev, nbrs_dev, n: int, count_dev, stream=None) -> None:
    """Triangle count into count_dev (device tensors in, device tensor out); the
    library allocates nothing for it.  Enqueued on the stream, not synchronised."""
    _check(lib().gpm_count_triangles_noalloc(
        ctypes.c_void_p(offsets_dev.data_ptr()),
        ctypes.c_void_p(nbrs_dev.data_ptr() if nbrs_dev.numel() else 0), n,
        ctypes.c_void_p(count_dev.data_ptr()), _stream(stream)))


def gpm_plan_free(p) -> None:
    lib().gpm_plan_free(p)


# ----------------------------------------------------------- conveniences

class Graph:
    """Owning wrapper: Graph(csr) loads once; .count()/.list() build cached plans."""

    def __init__(self, offsets, nbrs, n=None, flags=0, stream=None):
        self.handle = gpm_load_csr(offsets, nbrs, n, flags, stream)
        self._plans = {}

    @classmethod
    def from_csr(cls, csr, **kw):
        return cls(csr.offsets, csr.nbrs, csr.n, **kw)

    def info(self):
        return gpm_graph_info(self.handle)

    def plan(self, pattern, induced=False, mode=GPM_COUNT, opts=None, stream=None):
        key = (pattern if isinstance(pattern, str) else bytes(pattern), bool(induced), mode,
               tuple(sorted((opts or {}).items())))
        if key not in self._plans:
            self._plans[key] = gpm_plan(self.handle, pattern, induced, mode, opts, stream)
        return self._plans[key]

    def count(self, pattern, induced=False, opts=None, stream=None) -> int:
        return gpm_count(self.plan(pattern, induced, GPM_COUNT, opts, stream), stream)

    def list(self, pattern, induced=False, capacity=1 << 20, opts=None, stream=None):
        return gpm_list(self.plan(pattern, induced, GPM_LIST, opts, stream), capacity, stream=stream)

    def close(self):
        for p in self._plans.values():
            gpm_plan_free(p)
        self._plans.clear()
        if self.handle:
            gpm_graph_free(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
