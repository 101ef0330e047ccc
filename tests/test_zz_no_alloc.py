"""ipg_sssp_noalloc, the SSSP entry point for callers that may not allocate device
memory (their memory belongs to another allocator, or they run on a path where a
cudaMalloc could stall or fail), returns the same distances and superstep count as
ipg_sssp and as the CPU oracle.  Its scratch is one fixed array that keeps the previous
call's contents, so the check runs two calls in a row, then a smaller graph after a
larger one, and a graph of exactly the largest size the scratch holds.  After the first
call on the device, a call must not change the device's free memory.
Called through the C ABI; this file is collected last."""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ipg():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2010_01542_gb300 as ipg
    from paper_2010_01542_gb300 import _build

    _build.build()
    ipg.load_library()
    return ipg


def _device_csr(g, weighted=True):
    import torch

    offs = torch.from_numpy(g.offsets.view(np.int64)).cuda()
    cols = torch.from_numpy(g.cols.view(np.int32)).cuda()
    w = torch.from_numpy(g.weights.view(np.int32)).cuda() if weighted and g.weights is not None else None
    return offs, cols, w


def _compare(ipg, g, src, weighted=True):
    import torch

    h = ipg.ipg_graph_create(g.offsets, g.cols, g.weights if weighted else None, g.n, g.m, True)
    ref, count, _ = ipg.ipg_sssp(h, src)
    offs, cols, w = _device_csr(g, weighted)
    d = torch.empty(g.n, dtype=torch.int32, device="cuda")
    steps = ipg.ipg_sssp_noalloc(offs, cols, w, g.n, g.m, src, d)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(d.cpu().numpy().view(np.uint32), ref)
    assert steps == count
    w = g.weights if weighted else None
    o = oracle.sssp(g.n, g.offsets, g.cols, w, src)
    np.testing.assert_array_equal(d.cpu().numpy().view(np.uint32), o.values)
    assert steps == o.supersteps


def test_noalloc_matches_ipg_sssp_on_consecutive_calls(ipg):
    g = gen.rmat(14, 16, seed=21, weighted=True)
    hub = gen.max_out_degree_vertex(g)
    _compare(ipg, g, hub)  # first call
    _compare(ipg, g, hub)  # second call finds the first call's scratch contents
    _compare(ipg, g, 7)
    _compare(ipg, g, hub, weighted=False)
    small = gen.random_multigraph(300, 1500, seed=4, weighted=True)
    _compare(ipg, small, 0)  # a smaller graph after a larger one
    _compare(ipg, small, 299)


def test_noalloc_at_its_vertex_limit(ipg):
    """A graph of exactly IPG_NOALLOC_MAX_VERTICES vertices fills the scratch arrays."""
    g = gen.rmat(20, 16, seed=22, weighted=True)
    assert g.n == ipg.IPG_NOALLOC_MAX_VERTICES
    _compare(ipg, g, gen.max_out_degree_vertex(g))
    _compare(ipg, g, g.n - 1)  # the last vertex as the source
    _compare(ipg, g, gen.max_out_degree_vertex(g), weighted=False)


def test_noalloc_takes_no_device_memory_after_the_first_call(ipg):
    import torch

    g = gen.rmat(12, 16, seed=23, weighted=True)
    offs, cols, w = _device_csr(g)
    d = torch.empty(g.n, dtype=torch.int32, device="cuda")
    ipg.ipg_sssp_noalloc(offs, cols, w, g.n, g.m, 0, d)  # the first call on this device
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for src in (0, 1, g.n - 1):
        ipg.ipg_sssp_noalloc(offs, cols, w, g.n, g.m, src, d)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_graphs_above_its_limit(ipg):
    import torch

    n = ipg.IPG_NOALLOC_MAX_VERTICES + 1
    offs = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    d = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(ipg.IpgError) as e:
        ipg.ipg_sssp_noalloc(offs, None, None, n, 0, 0, d)
    assert e.value.status == 1 and "limit" in str(e.value)
