"""ipg_graph_check_symmetric against a brute-force multiset comparison of the stored
edges (u, v, w) with their reverses (v, u, w), on undirected graphs as the paper
stores them (Sec. VI-B: both directions of every edge, same weight) and on graphs
that break that in one place.  Called through the C ABI."""
import numpy as np
import pytest

import gen

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


def _brute(g):
    row = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.offsets.astype(np.int64)))
    col = g.cols.astype(np.int64)
    w = g.weights.astype(np.int64) if g.weights is not None else np.zeros_like(col)
    fwd = sorted(zip(row.tolist(), col.tolist(), w.tolist()))
    rev = sorted(zip(col.tolist(), row.tolist(), w.tolist()))
    return fwd == rev


def _check(ipg, g, directed=None):
    d = g.directed if directed is None else directed
    h = ipg.ipg_graph_create(g.offsets, g.cols, g.weights, g.n, g.m, d)
    got = ipg.ipg_graph_check_symmetric(h)
    assert got == _brute(g)
    return got


def _edges(n, triples, weighted=True):
    e = np.asarray(triples, dtype=np.int64).reshape(-1, 3)
    return gen.csr_from_edges(n, e[:, 0], e[:, 1], weights=e[:, 2] if weighted else None)


@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("scale", [6, 10, 16])
def test_undirected_rmat_is_symmetric(ipg, scale, weighted):
    g = gen.rmat(scale, 8, seed=scale, undirected=True, weighted=weighted)
    assert _check(ipg, g)
    assert _check(ipg, g, directed=True)  # the answer does not depend on how it was created


@pytest.mark.parametrize("weighted", [False, True])
def test_directed_rmat(ipg, weighted):
    assert not _check(ipg, gen.rmat(10, 8, seed=3, weighted=weighted))


def test_one_missing_direction(ipg):
    g = gen.rmat(10, 8, seed=4, undirected=True)
    row = np.repeat(np.arange(g.n), np.diff(g.offsets.astype(np.int64)))
    keep = np.ones(g.m, dtype=bool)
    keep[g.m // 2] = False
    h = gen.csr_from_edges(g.n, row[keep], g.cols[keep])
    assert not _check(ipg, h)


@pytest.mark.parametrize("wmax", [255, 1000])  # one-byte and four-byte weight storage
def test_one_changed_weight(ipg, wmax):
    g = gen.rmat(10, 8, seed=5, undirected=True, weighted=True)
    row = np.repeat(np.arange(g.n), np.diff(g.offsets.astype(np.int64)))
    key = np.minimum(row, g.cols) * g.n + np.maximum(row, g.cols)
    w = 1 + (key * 2654435761 % wmax)  # symmetric: a function of the unordered pair
    sym = gen.csr_from_edges(g.n, row, g.cols, weights=w)
    assert _check(ipg, sym)
    w2 = w.copy()
    i = int(np.flatnonzero(row != g.cols)[0])
    w2[i] = w2[i] % wmax + 1
    assert not _check(ipg, gen.csr_from_edges(g.n, row, g.cols, weights=w2))


def test_parallel_edges_compare_as_multisets(ipg):
    # u->v twice with weights 3 and 5; the reverse pair listed in the other order
    assert _check(ipg, _edges(4, [(0, 1, 3), (0, 1, 5), (1, 0, 5), (1, 0, 3), (2, 3, 7), (3, 2, 7)]))
    assert not _check(ipg, _edges(4, [(0, 1, 3), (0, 1, 5), (1, 0, 3), (1, 0, 3), (2, 3, 7), (3, 2, 7)]))
    assert not _check(ipg, _edges(4, [(0, 1, 3), (0, 1, 3), (1, 0, 3), (2, 3, 7), (3, 2, 7)]))


def test_self_loops_and_empty(ipg):
    assert _check(ipg, _edges(5, [(0, 0, 1), (3, 3, 9), (3, 3, 2)]))
    assert not _check(ipg, _edges(5, [(0, 0, 1), (3, 4, 2)]))
    empty = gen.csr_from_edges(5, [], [])
    h = ipg.ipg_graph_create(empty.offsets, empty.cols, None, 5, 0, False)
    assert ipg.ipg_graph_check_symmetric(h)
