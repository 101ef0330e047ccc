"""Page-locked host buffers from ipg_host_alloc: a graph uploaded from them and results
read back into them equal the oracle's, buffers of at least one huge page are aligned
to it, and freeing is checked.  Called through the C ABI."""
import ctypes

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


def _copy(ipg, a):
    h = ipg.host_empty(a.shape, a.dtype)
    assert not h.any(), "ipg_host_alloc memory must come zero-filled"
    h[...] = a
    return h


def test_graph_from_host_buffers(ipg):
    g = gen.rmat(12, 16, seed=5, weighted=True)
    off, cols, w = _copy(ipg, g.offsets), _copy(ipg, g.cols), _copy(ipg, g.weights)
    h = ipg.ipg_graph_create(off, cols, w, g.n, g.m, True)
    src = int(gen.max_out_degree_vertex(g))
    dist = ipg.host_empty(g.n, np.uint32)
    ranks = ipg.host_empty(g.n, np.float32)
    _, cnt, _ = ipg.ipg_sssp(h, src, dist)
    ipg.ipg_pagerank(h, 10, ranks)
    ref = oracle.sssp(g.n, g.offsets, g.cols, g.weights, src)
    np.testing.assert_array_equal(dist, ref.values)
    assert cnt == ref.supersteps
    pr = oracle.pagerank(g.n, g.offsets, g.cols, 10)
    assert np.max(np.abs(ranks.astype(np.float64) - pr.values)) / np.max(pr.values) <= 1e-5
    # the same graph from ordinary pageable arrays gives the same bits
    h2 = ipg.ipg_graph_create(g.offsets, g.cols, g.weights, g.n, g.m, True)
    r2, _, _ = ipg.ipg_pagerank(h2, 10)
    assert np.array_equal(r2.view(np.uint32), ranks.view(np.uint32))


def test_alignment_and_free(ipg):
    lib = ipg.load_library()
    alloc, free = lib.ipg_host_alloc, lib.ipg_host_free
    alloc.argtypes, alloc.restype = [ctypes.c_size_t, ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int
    free.argtypes, free.restype = [ctypes.c_void_p], ctypes.c_int
    try:
        huge = int(open("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size").read())
    except (OSError, ValueError):
        huge = 2 << 20
    for nbytes in (1, 4097, (2 << 20) + 1, 48 << 20):
        p = ctypes.c_void_p()
        assert alloc(nbytes, ctypes.byref(p)) == 0, lib.ipg_last_error()
        assert p.value and p.value % 4096 == 0
        if nbytes >= huge:
            assert p.value % huge == 0
        ctypes.memset(p.value, 0xA5, nbytes)
        assert free(p) == 0
        assert free(p) == 1  # a second free is refused
