"""C-ABI checks that need no GPU: the library builds for sm_103a, loads, exports
every function include/gpm.h declares, and refuses to run without a GPU."""
import ctypes
import subprocess

import pytest

import paper_2112_09761_gb300 as G


@pytest.fixture(scope="module")
def L():
    G.build()
    return G.lib()


def test_exports_every_declared_symbol(L):
    names = G.header_functions()
    assert "gpm_load_csr" in names and "gpm_plan" in names and "gpm_count" in names
    for n in names:
        assert hasattr(L, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", G.gpm.library_path()],
                         capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert set(names) <= exported


def test_build_targets_sm_103a_only(L):
    assert G._build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert "-lineinfo" in G._build.NVCC_FLAGS


NAMES = ["triangle", "3-clique", "4-clique", "5-clique", "6-clique", "7-clique", "8-clique",
         "diamond", "4-cycle", "tailed-triangle", "3-star", "4-path", "wedge"]


@pytest.mark.parametrize("name", NAMES)
def test_pattern_named(L, name):
    p = G.gpm_pattern_named(name)
    k = {"triangle": 3, "wedge": 3}.get(name, int(name[0]) if name[0].isdigit() else 4)
    if name in ("3-star", "4-path", "4-cycle"):
        k = 4
    assert p.k == k
    edges = p.edge_list()
    assert len(set(tuple(sorted(e)) for e in edges)) == len(edges) == p.n_edges
    if "clique" in name or name == "triangle":
        assert p.n_edges == k * (k - 1) // 2


def test_pattern_unknown_name(L):
    with pytest.raises(G.GpmError) as e:
        G.gpm_pattern_named("5-cycle")
    assert e.value.name == "GPM_E_UNSUPPORTED_PATTERN"
    assert "unknown pattern" in G.gpm_last_error()


def test_no_gpu_fails_loudly(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(G.GpmError) as e:
        G.gpm_load_csr([0, 1, 2], [1, 0])
    assert e.value.name == "GPM_E_CUDA"


def test_null_arguments_rejected(L):
    h = ctypes.c_void_p()
    assert L.gpm_load_csr(None, 1, None, 3, 4, 0, None, ctypes.byref(h)) == 1
    assert L.gpm_count(None, None, None) == 1
    assert L.gpm_plan(None, None, 0, 0, None, None, ctypes.byref(h)) == 1
    assert L.gpm_graph_info(None, None, None, None, None) == 1
    L.gpm_plan_free(None)
    L.gpm_graph_free(None)
