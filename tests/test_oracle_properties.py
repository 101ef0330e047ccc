"""Property tests of the oracle on random tiny multigraphs (self-loops and parallel edges
included), each against a brute-force restatement written here from the definitions:
SSSP distances against scipy's Dijkstra and its superstep count against the hop-count
closed form (a vertex last improves at the fewest hops of its shortest paths, and only a
vertex with out-edges sends); Hashmin labels against union-find and its superstep count
against 2 + the largest eccentricity of a component's smallest vertex; PageRank against
the update rule summed edge by edge.  The OpenMP baseline is held to the oracle on the
same inputs.  CPU only."""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import cpu_baseline  # noqa: E402
import gen  # noqa: E402
import oracle  # noqa: E402

INF = 0xFFFFFFFF


@st.composite
def multigraphs(draw, max_n=9, max_m=24, undirected=False):
    n = draw(st.integers(1, max_n))
    k = draw(st.integers(0, max_m))
    edges = draw(st.lists(st.tuples(st.integers(0, n - 1), st.integers(0, n - 1), st.integers(1, 255)),
                          min_size=k, max_size=k))
    src = [e[0] for e in edges]
    dst = [e[1] for e in edges]
    w = [e[2] for e in edges]
    if undirected:
        src, dst, w = src + dst, dst + src, w + w
    return gen.csr_from_edges(n, src, dst, weights=w if edges else None) if edges else gen.csr_from_edges(n, [], [])


def _edges(g):
    row = np.repeat(np.arange(g.n), np.diff(g.offsets.astype(np.int64)))
    w = g.weights if g.weights is not None else np.ones(g.m, dtype=np.uint32)
    return list(zip(row.tolist(), g.cols.tolist(), w.tolist()))


def _hop_bounded(g, src, weighted):
    """best[k][v]: shortest distance using at most k edges (Bellman-Ford by hop count)."""
    E = [(u, v, w if weighted else 1) for u, v, w in _edges(g)]
    best = [[INF] * g.n]
    best[0][src] = 0
    for _ in range(g.n):
        prev = best[-1]
        cur = list(prev)
        for u, v, w in E:
            if prev[u] != INF and prev[u] + w < cur[v]:
                cur[v] = prev[u] + w
        best.append(cur)
    return best


@settings(max_examples=150, deadline=None)
@given(g=multigraphs(), weighted=st.booleans(), pick=st.integers(0, 1000))
def test_sssp_distances_and_superstep_count(g, weighted, pick):
    src = pick % g.n
    w = g.weights if weighted else None
    r = oracle.sssp(g.n, g.offsets, g.cols, w, src)
    best = _hop_bounded(g, src, weighted and g.weights is not None)
    dist = best[-1]
    np.testing.assert_array_equal(r.values, np.asarray(dist, dtype=np.uint32))
    if g.m:
        import scipy.sparse as sp
        from scipy.sparse.csgraph import dijkstra

        lengths = {}
        for u, v, ww in _edges(g):
            ln = ww if weighted and g.weights is not None else 1
            lengths[(u, v)] = min(lengths.get((u, v), ln), ln)
        rows, cols = zip(*lengths)
        mat = sp.csr_matrix((list(lengths.values()), (rows, cols)), shape=(g.n, g.n))
        d = dijkstra(mat, indices=src)
        d[src] = 0
        want = np.where(np.isinf(d), INF, d).astype(np.uint64)
        np.testing.assert_array_equal(r.values.astype(np.uint64), want)
    outdeg = np.diff(g.offsets.astype(np.int64))
    hops = [min(k for k in range(len(best)) if best[k][v] == dist[v]) for v in range(g.n) if dist[v] != INF]
    reached = [v for v in range(g.n) if dist[v] != INF]
    senders = [h for v, h in zip(reached, hops) if outdeg[v] > 0]
    want_steps = 2 + max(senders) if senders else 1
    assert r.supersteps == want_steps
    # superstep k's senders are the vertices whose k-hop distance dropped (the source at k = 0)
    msgs = int(outdeg[src]) + sum(int(outdeg[v]) for k in range(1, len(best)) for v in range(g.n)
                                  if best[k][v] < best[k - 1][v])
    assert sum(s.messages_sent for s in r.stats) == msgs
    # the OpenMP baseline computes the same run
    p = cpu_baseline.sssp(g.n, g.offsets, g.cols, w, src)
    np.testing.assert_array_equal(p.values, r.values)
    assert p.supersteps == r.supersteps and p.messages == sum(s.messages_sent for s in r.stats)


def _components(g):
    parent = list(range(g.n))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for u, v, _ in _edges(g):
        a, b = find(u), find(v)
        if a != b:
            parent[max(a, b)] = min(a, b)
    return [find(v) for v in range(g.n)]


@settings(max_examples=150, deadline=None)
@given(g=multigraphs(undirected=True))
def test_hashmin_labels_and_superstep_count(g):
    r = oracle.hashmin(g.n, g.offsets, g.cols)
    comp = _components(g)
    labels = [min(v for v in range(g.n) if comp[v] == comp[x]) for x in range(g.n)]
    np.testing.assert_array_equal(r.values, np.asarray(labels, dtype=np.uint32))
    if g.m == 0:
        assert r.supersteps == 1
    else:
        ecc = 0
        for root in set(labels):  # BFS from each component's smallest vertex
            level = {root: 0}
            frontier = [root]
            while frontier:
                nxt = []
                for u in frontier:
                    for e in range(int(g.offsets[u]), int(g.offsets[u + 1])):
                        v = int(g.cols[e])
                        if v not in level:
                            level[v] = level[u] + 1
                            nxt.append(v)
                frontier = nxt
            ecc = max(ecc, max(level.values()))
        assert r.supersteps == 2 + ecc
    p = cpu_baseline.hashmin(g.n, g.offsets, g.cols)
    np.testing.assert_array_equal(p.values, r.values)
    assert p.supersteps == r.supersteps and p.messages == sum(s.messages_sent for s in r.stats)


@settings(max_examples=100, deadline=None)
@given(g=multigraphs(), updates=st.integers(0, 6))
def test_pagerank_update_rule(g, updates):
    r = oracle.pagerank(g.n, g.offsets, g.cols, updates)
    outdeg = np.diff(g.offsets.astype(np.int64))
    rank = np.full(g.n, 1.0 / g.n)
    for _ in range(updates):
        nxt = np.full(g.n, 0.15 / g.n)
        for u, v, _ in _edges(g):
            nxt[v] += 0.85 * rank[u] / outdeg[u]
        rank = nxt
    np.testing.assert_allclose(r.values, rank, rtol=1e-12, atol=1e-15)
    assert r.supersteps == updates + 1
    p = cpu_baseline.pagerank(g.n, g.offsets, g.cols, updates)
    np.testing.assert_allclose(p.values, rank, rtol=1e-5, atol=1e-7)
