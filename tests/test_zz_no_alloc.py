"""The allocation-free triangle count (gpm_count_triangles_noalloc) against the
regular entry point (gpm_plan + gpm_count), through the C ABI.

Some callers cannot allocate device memory (real-time loops where an
allocation could synchronise the device, plug-ins whose host owns all device
memory, fully pre-reserved processes); this entry point takes device inputs
and a device output and works in a fixed array inside the library.  The file
is named to be collected last."""
import numpy as np
import pytest

import graphgen as gg
import paper_2112_09761_gb300 as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    G.build()
    return torch


GRAPHS = {
    "er-10k": lambda: gg.workload("er-10k"),
    "rmat13": lambda: gg.rmat_graph(13, 16, 41),
    "chunglu": lambda: gg.chung_lu_graph(20_000, 160_000, 42, wmax=2000.0, i0=2.0),
    "K50": lambda: gg.complete(50),
    "edgeless": lambda: gg.empty(5),
}


@pytest.mark.parametrize("name", list(GRAPHS))
def test_noalloc_equals_regular_count(torch_cuda, name):
    torch = torch_cuda
    g = GRAPHS[name]()
    with G.Graph.from_csr(g) as h:
        want = h.count("triangle")  # the existing entry point
    off_d = torch.from_numpy(g.offsets).cuda()
    nbr_d = torch.from_numpy(g.nbrs.view(np.int32)).cuda()
    out = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    for _ in range(2):  # two calls in a row share the library's array
        out.fill_(-1)
        G.gpm_count_triangles_noalloc(off_d, nbr_d, g.n, out)
        torch.cuda.synchronize()
        assert int(out.item()) == want


def test_noalloc_rejects_too_many_vertices(torch_cuda):
    torch = torch_cuda
    n = 131_070
    off_d = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    nbr_d = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(G.GpmError) as e:
        G.gpm_count_triangles_noalloc(off_d, nbr_d, n, out)
    assert e.value.name == "GPM_E_INVALID_ARG"
    assert "at most 131069" in str(e.value)
