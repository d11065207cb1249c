"""GB300-native pattern-aware subgraph enumeration (G2Miner, arXiv 2112.09761).

The product is the C-ABI library ``libgpm.so`` (declared in ``include/gpm.h``)
whose enumeration kernels are hand-written CUDA for sm_103a.  This package
holds its sources (``csrc/``), its in-tree build (``_build.py``) and a thin
ctypes binding with the same function names (``gpm.py``).
"""
from .gpm import (MOTIF3, MOTIF4, gpm_count_triangles_noalloc, gpm_server_create, gpm_server_free, gpm_server_poll,
                  gpm_server_stats, gpm_server_submit, gpm_server_wait, gpm_batch_count, gpm_batch_create, gpm_batch_free,
                  gpm_batch_info, gpm_motif_count, GPM_BORROW, GPM_COUNT, GPM_DEVICE_PTRS, GPM_LIST, GPM_RELABEL, GPM_SKIP_VALIDATE, Graph,
                  GpmError, gpm_count, gpm_count_range, gpm_graph_export, gpm_graph_free, gpm_graph_info,
                  gpm_last_error, gpm_list, gpm_load_csr, gpm_pattern_named, gpm_plan,
                  gpm_pattern_describe, gpm_plan_describe, gpm_plan_free, gpm_plan_launches, gpm_plan_info, gpm_plan_stats, gpm_version, header_functions, lib,
                  pattern_from_edges)
from ._build import build

__all__ = [n for n in dir() if not n.startswith("_")]
