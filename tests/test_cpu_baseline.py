"""The OpenMP CPU baseline (the paper's final design on the host cores) computes what the
oracle computes: Hashmin labels, SSSP distances, superstep counts and message totals
exactly, PageRank within float32 rounding.  CPU only."""
import numpy as np
import pytest

import cpu_baseline
import gen
import oracle


def _graphs():
    yield "rmat10-directed", gen.rmat(10, 8, seed=11, weighted=True)
    yield "rmat12-undirected", gen.rmat(12, 8, seed=12, undirected=True, weighted=True)
    yield "multigraph", gen.random_multigraph(400, 3000, seed=13, weighted=True)
    yield "path", gen.csr_from_edges(300, np.arange(299), np.arange(1, 300), weights=np.full(299, 255))
    yield "no-edges", gen.csr_from_edges(5, [], [])


GRAPHS = list(_graphs())


@pytest.mark.parametrize("name,g", GRAPHS, ids=[x[0] for x in GRAPHS])
def test_pagerank_matches_oracle(name, g):
    ref = oracle.pagerank(g.n, g.offsets, g.cols, 10)
    got = cpu_baseline.pagerank(g.n, g.offsets, g.cols, 10)
    assert got.messages == 10 * g.m
    assert np.max(np.abs(got.values.astype(np.float64) - ref.values)) / np.max(ref.values) <= 1e-5


@pytest.mark.parametrize("weighted", [True, False])
@pytest.mark.parametrize("name,g", GRAPHS, ids=[x[0] for x in GRAPHS])
def test_sssp_matches_oracle(name, g, weighted):
    w = g.weights if weighted else None
    for src in sorted({0, g.n - 1, int(gen.max_out_degree_vertex(g))}):
        ref = oracle.sssp(g.n, g.offsets, g.cols, w, src)
        got = cpu_baseline.sssp(g.n, g.offsets, g.cols, w, src)
        np.testing.assert_array_equal(got.values, ref.values)
        assert got.supersteps == ref.supersteps
        assert got.messages == sum(s.messages_sent for s in ref.stats)


@pytest.mark.parametrize("name,g", [x for x in GRAPHS if not x[1].directed or x[0] in ("no-edges",)],
                         ids=lambda x: x if isinstance(x, str) else "")
def test_hashmin_matches_oracle(name, g):
    ref = oracle.hashmin(g.n, g.offsets, g.cols)
    got = cpu_baseline.hashmin(g.n, g.offsets, g.cols)
    np.testing.assert_array_equal(got.values, ref.values)
    assert got.supersteps == ref.supersteps
    assert got.messages == sum(s.messages_sent for s in ref.stats)


def test_threads_reported():
    assert cpu_baseline.threads() >= 1
