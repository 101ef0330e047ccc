"""Pins for the oracle's general-combiner functions (Sec. III, Fig. 1), each against
something other than the oracle itself.

* combine (the mailbox step alone): numpy's unbuffered ufunc.at reductions (xor, min,
  add modulo 2^64), a two-pass (minimum key, then sum of the counts at that key)
  formulation of the 128-bit kind, the has-message flag as a bincount, invariance
  under any permutation of the messages, and the empty-mailbox cases where the combined
  value equals the combine's neutral element (x xor x = 0, x + (2^64 - x) = 0) but the
  flag must still be raised.
* shortest-path tree: scipy Dijkstra distances, and the parent written out from its
  definition (the smallest in-neighbour u with dist[u] + w(u,v) = dist[v]); superstep
  counts from the same hop closed form as SSSP.
* shortest-path counting: scipy BFS levels; counts from the textbook recurrence over
  the BFS DAG (sigma[v] = sum over edges u -> v with level[u] + 1 = level[v]); closed
  forms on grids (binomials) and hypercubes (factorials); path enumeration by networkx;
  the wrap-around of 2^64 paths to a count of 0 on a chain of 64 diamonds, after which
  the search must still go on (the receiver got a message whose count is the neutral 0).
"""
import itertools
import math

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse import csgraph

import gen
import oracle

U64 = 1 << 64


# ---------------------------------------------------------------------------------------
# combine


def _random_messages(kind, n, k, seed, key_range=None):
    rng = np.random.default_rng(seed)
    # skewed destinations: a few vertices get most of the messages
    dst = np.minimum(rng.zipf(1.5, size=k) - 1, n - 1).astype(np.uint32)
    if kind == oracle.COMBINE_XOR_U32:
        msgs = rng.integers(0, 1 << 32, size=k, dtype=np.uint64).astype(np.uint32)
    elif kind == oracle.COMBINE_MINCOUNT_U128:
        keys = rng.integers(0, key_range or 4, size=k, dtype=np.uint64)
        counts = rng.integers(0, U64, size=k, dtype=np.uint64)
        msgs = np.stack([keys, counts], axis=1)
    else:
        msgs = rng.integers(0, U64, size=k, dtype=np.uint64)
    return dst, msgs


def _expected(kind, n, dst, msgs):
    has = np.bincount(dst, minlength=n)[:n] > 0
    if kind == oracle.COMBINE_XOR_U32:
        out = np.zeros(n, dtype=np.uint32)
        np.bitwise_xor.at(out, dst, msgs)
    elif kind == oracle.COMBINE_MIN_U64:
        out = np.full(n, np.iinfo(np.uint64).max, dtype=np.uint64)
        np.minimum.at(out, dst, msgs)
    elif kind == oracle.COMBINE_SUM_U64:
        out = np.zeros(n, dtype=np.uint64)
        np.add.at(out, dst, msgs)  # uint64 arithmetic wraps modulo 2^64
    else:
        key = np.full(n, np.iinfo(np.uint64).max, dtype=np.uint64)
        np.minimum.at(key, dst, msgs[:, 0])
        at_min = msgs[:, 0] == key[dst]
        cnt = np.zeros(n, dtype=np.uint64)
        np.add.at(cnt, dst[at_min], msgs[at_min, 1])
        out = np.stack([key, cnt], axis=1)
    return has, out


KINDS = [oracle.COMBINE_XOR_U32, oracle.COMBINE_MIN_U64, oracle.COMBINE_SUM_U64, oracle.COMBINE_MINCOUNT_U128]


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("n,k", [(1, 1), (7, 50), (300, 5000), (5000, 3000)])
def test_combine_matches_ufunc_reductions(kind, n, k):
    dst, msgs = _random_messages(kind, n, k, seed=n * 31 + k + kind)
    r = oracle.combine(kind, n, dst, msgs)
    has, out = _expected(kind, n, dst, msgs)
    np.testing.assert_array_equal(r.has, has)
    assert r.receivers == int(has.sum())
    np.testing.assert_array_equal(r.mail[has], out[has])


@pytest.mark.parametrize("kind", KINDS)
def test_combine_is_order_free(kind):
    dst, msgs = _random_messages(kind, 50, 2000, seed=9 + kind)
    base = oracle.combine(kind, 50, dst, msgs)
    for s in range(3):
        p = np.random.default_rng(s).permutation(dst.size)
        r = oracle.combine(kind, 50, dst[p], msgs[p])
        np.testing.assert_array_equal(r.has, base.has)
        np.testing.assert_array_equal(r.mail[r.has], base.mail[base.has])


def test_combine_neutral_results_still_count_as_messages():
    # xor of a message with itself and x + (2^64 - x) both give the neutral element 0;
    # the receivers got messages all the same (the empty-mailbox hazard, Sec. III)
    r = oracle.combine(oracle.COMBINE_XOR_U32, 4, [1, 1, 3], np.array([0xDEADBEEF, 0xDEADBEEF, 0], np.uint32))
    np.testing.assert_array_equal(r.has, [False, True, False, True])
    assert r.mail[1] == 0 and r.mail[3] == 0 and r.receivers == 2
    x = 0x123456789ABCDEF1
    r = oracle.combine(oracle.COMBINE_SUM_U64, 3, [2, 2], np.array([x, U64 - x], np.uint64))
    np.testing.assert_array_equal(r.has, [False, False, True])
    assert r.mail[2] == 0
    # (key, count) with counts that cancel modulo 2^64 at the smallest key
    m = np.array([[5, 7], [3, 1], [3, U64 - 1], [9, 4]], dtype=np.uint64)
    r = oracle.combine(oracle.COMBINE_MINCOUNT_U128, 2, [0, 0, 0, 0], m)
    assert r.has[0] and not r.has[1]
    np.testing.assert_array_equal(r.mail[0], [3, 0])


def test_combine_edge_cases():
    r = oracle.combine(oracle.COMBINE_MIN_U64, 5, np.zeros(0, np.uint32), np.zeros(0, np.uint64))
    assert not r.has.any() and r.receivers == 0
    r = oracle.combine(oracle.COMBINE_MIN_U64, 0, np.zeros(0, np.uint32), np.zeros(0, np.uint64))
    assert r.receivers == 0
    with pytest.raises(oracle.OracleError):
        oracle.combine(oracle.COMBINE_MIN_U64, 2, [2], np.array([1], np.uint64))
    with pytest.raises(ValueError):
        oracle.combine(oracle.COMBINE_MINCOUNT_U128, 2, [0], np.array([1], np.uint64))


# ---------------------------------------------------------------------------------------
# shortest-path tree


def _graphs(undirected=False):
    yield gen.csr_from_edges(1, [], [], undirected=undirected)
    yield gen.csr_from_edges(5, [], [], undirected=undirected)
    yield gen.csr_from_edges(3, [0, 1, 1], [0, 1, 1], undirected=undirected)
    yield gen.csr_from_edges(6, [0, 0, 2, 3, 3, 5], [1, 1, 3, 4, 4, 5], undirected=undirected)
    for seed in range(6):
        yield gen.random_multigraph(12 + seed, 20 + 3 * seed, seed=seed, undirected=undirected)
    for scale in (4, 5, 6, 7):
        yield gen.rmat(scale, 4, seed=scale, undirected=undirected)


def _min_weight_matrix(g, w):
    n = g.n
    rows = np.repeat(np.arange(n), g.out_degree())
    key = rows * n + g.cols.astype(np.int64)
    order = np.lexsort((w, key))
    key, ww = key[order], w[order].astype(np.float64)
    first = np.ones(key.size, dtype=bool)
    first[1:] = key[1:] != key[:-1]
    return sp.csr_matrix((ww[first], (key[first] // n, key[first] % n)), shape=(n, n))


def _dijkstra(g, w, src):
    d = csgraph.dijkstra(_min_weight_matrix(g, w), directed=True, indices=src)
    return np.where(np.isfinite(d), d, oracle.INF).astype(np.int64)


def _parent_by_definition(g, w, dist, src):
    rows = np.repeat(np.arange(g.n), g.out_degree())
    v = g.cols.astype(np.int64)
    ok = (dist[rows] != oracle.INF) & (dist[rows] + w.astype(np.int64) == dist[v])
    parent = np.full(g.n, oracle.INF, dtype=np.int64)
    np.minimum.at(parent, v[ok], rows[ok])
    parent[src] = src
    return parent


def _hop_closed_form_supersteps(g, w, src):
    big = g.n + 1
    d = csgraph.dijkstra(_min_weight_matrix(g, w.astype(np.int64) * big + 1), directed=True, indices=src)
    fin = np.isfinite(d)
    hops = np.full(g.n, -1, dtype=np.int64)
    hops[fin] = d[fin].astype(np.int64) % big
    outdeg = g.out_degree()
    if outdeg[src] == 0:
        return 1
    return 2 + int(hops[fin & (outdeg > 0)].max())


def test_sssp_tree_matches_dijkstra_and_parent_definition():
    for g in _graphs():
        rng = np.random.default_rng(g.n * 5 + g.m)
        for weighted in (True, False):
            # few distinct weights so that equal-length alternatives (parent ties) are common
            w = rng.integers(1, 4, size=g.m).astype(np.uint32) if weighted else np.ones(g.m, np.uint32)
            for src in sorted({0, g.n // 2, g.n - 1}):
                r = oracle.sssp_tree(g.n, g.offsets, g.cols, w if weighted else None, src)
                dist = _dijkstra(g, w, src)
                np.testing.assert_array_equal(r.dist.astype(np.int64), dist)
                np.testing.assert_array_equal(r.parent.astype(np.int64), _parent_by_definition(g, w, dist, src))
                assert r.supersteps == _hop_closed_form_supersteps(g, w, src)


def test_sssp_tree_tie_goes_to_the_smaller_parent():
    # 0 -> 3 -> 1 and 0 -> 2 -> 1 with equal lengths: parent of 1 is 2; vertex 4 unreached
    g = gen.csr_from_edges(5, [0, 0, 3, 2], [3, 2, 1, 1], [1, 1, 1, 1])
    r = oracle.sssp_tree(g.n, g.offsets, g.cols, g.weights, 0)
    np.testing.assert_array_equal(r.dist, [0, 2, 1, 1, oracle.INF])
    np.testing.assert_array_equal(r.parent, [0, 2, 0, 0, oracle.INF])
    # a longer path that arrives first does not fix the parent: 0 -> 1 (w 5), 0 -> 2 -> 1 (1 + 1)
    g = gen.csr_from_edges(3, [0, 0, 2], [1, 2, 1], [5, 1, 1])
    r = oracle.sssp_tree(g.n, g.offsets, g.cols, g.weights, 0)
    np.testing.assert_array_equal(r.dist, [0, 2, 1])
    np.testing.assert_array_equal(r.parent, [0, 2, 0])


def _walk_minima(g, w, src, kmax):
    """best[k][v] = smallest weight of a walk from src to v with at most k edges (brute force)."""
    adj = [[(int(g.cols[e]), int(w[e])) for e in range(int(g.offsets[u]), int(g.offsets[u + 1]))]
           for u in range(g.n)]
    best = []
    for k in range(kmax + 1):
        b = [np.inf] * g.n
        b[src] = 0
        frontier = {(src, 0)}
        seen = set(frontier)
        for _ in range(k):
            nxt = set()
            for u, d in frontier:
                for v, ww in adj[u]:
                    if (v, d + ww) not in seen:
                        seen.add((v, d + ww))
                        nxt.add((v, d + ww))
                        b[v] = min(b[v], d + ww)
            frontier = nxt
        best.append(b)
    return best


def test_sssp_tree_late_parent_change_sends_nothing():
    # vertex 1 first hears (3, parent 3) over 0 -> 3 -> 1 (weights 1, 2) in superstep 2,
    # then (3, parent 2) over 0 -> 4 -> 2 -> 1 (weights 1, 1, 1) in superstep 3: its parent
    # becomes 2, its distance stays 3, so it sends only once (in superstep 2)
    g = gen.csr_from_edges(5, [0, 3, 0, 4, 2, 1], [3, 1, 4, 2, 1, 0], [1, 2, 1, 1, 1, 1])
    r = oracle.sssp_tree(g.n, g.offsets, g.cols, g.weights, 0)
    np.testing.assert_array_equal(r.dist, [0, 3, 2, 1, 1])
    np.testing.assert_array_equal(r.parent, [0, 2, 4, 0, 0])
    assert [st.senders for st in r.stats] == [1, 2, 2, 0]
    assert r.supersteps == 4


@pytest.mark.parametrize("seed", range(30))
def test_sssp_tree_sends_only_when_the_distance_drops(seed):
    # a vertex whose parent changes but whose distance does not has nothing new to say:
    # the senders of superstep s are the vertices whose <= s-edge walk minimum dropped
    rng = np.random.default_rng(2000 + seed)
    n = int(rng.integers(3, 9))
    g = gen.random_multigraph(n, int(rng.integers(4, 18)), seed=seed)
    w = rng.integers(1, 4, size=g.m).astype(np.uint32)
    src = int(rng.integers(0, n))
    r = oracle.sssp_tree(g.n, g.offsets, g.cols, w, src)
    best = _walk_minima(g, w, src, r.supersteps)
    outdeg = g.out_degree()
    for s, st in enumerate(r.stats):
        prev = np.full(n, np.inf) if s == 0 else np.array(best[s - 1])
        send = np.array(best[s]) < prev
        assert st.senders == int(send.sum()), (s, st)
        assert st.messages_sent == int(outdeg[send].sum())


def test_sssp_tree_overflow_is_reported():
    g = gen.csr_from_edges(3, [0, 1], [1, 2], [0xFFFFFF00, 0xFFFFFF00])
    with pytest.raises(oracle.OracleError):
        oracle.sssp_tree(g.n, g.offsets, g.cols, g.weights, 0)


# ---------------------------------------------------------------------------------------
# shortest-path counting


def _bfs_levels(g, src):
    rows = np.repeat(np.arange(g.n), g.out_degree())
    A = sp.csr_matrix((np.ones(g.m), (rows, g.cols.astype(np.int64))), shape=(g.n, g.n))
    d = csgraph.shortest_path(A, directed=True, unweighted=True, indices=src)
    return np.where(np.isfinite(d), d, oracle.INF).astype(np.int64)


def _brandes_counts(g, level, src):
    """sigma[src] = 1; sigma[v] = sum over edges u -> v with level[u] + 1 = level[v] of sigma[u]."""
    sigma = [0] * g.n
    sigma[src] = 1
    order = sorted((int(level[v]), v) for v in range(g.n) if level[v] != oracle.INF)
    for lv, u in order:
        for e in range(int(g.offsets[u]), int(g.offsets[u + 1])):
            v = int(g.cols[e])
            if level[v] == lv + 1:
                sigma[v] = (sigma[v] + sigma[u]) % U64
    return np.array(sigma, dtype=np.uint64)


def test_bfs_paths_matches_bfs_and_recurrence():
    for g in _graphs():
        for src in sorted({0, g.n // 2, g.n - 1}):
            r = oracle.bfs_paths(g.n, g.offsets, g.cols, src)
            lev = _bfs_levels(g, src)
            np.testing.assert_array_equal(r.level.astype(np.int64), lev)
            np.testing.assert_array_equal(r.paths, _brandes_counts(g, lev, src))
            assert (r.paths[lev == oracle.INF] == 0).all()
            outdeg = g.out_degree()
            fin = lev != oracle.INF
            expect = 1 if outdeg[src] == 0 else 2 + int(lev[fin & (outdeg > 0)].max())
            assert r.supersteps == expect
            # per superstep: the vertices of level s send to all their out-neighbours
            rows = np.repeat(np.arange(g.n), outdeg)
            for s, st in enumerate(r.stats):
                at = lev == s
                assert st.senders == int(at.sum())
                assert st.messages_sent == int(outdeg[at].sum())
                assert st.receivers == np.unique(g.cols[at[rows]]).size


@pytest.mark.parametrize("a,b", [(1, 1), (2, 3), (6, 9), (12, 12)])
def test_bfs_paths_grid_binomials(a, b):
    # a x b grid, edges right and down: paths from the corner to (i, j) = C(i + j, i)
    idx = lambda i, j: i * b + j  # noqa: E731
    src, dst = [], []
    for i in range(a):
        for j in range(b):
            if j + 1 < b:
                src.append(idx(i, j)), dst.append(idx(i, j + 1))
            if i + 1 < a:
                src.append(idx(i, j)), dst.append(idx(i + 1, j))
    g = gen.csr_from_edges(a * b, src, dst)
    r = oracle.bfs_paths(g.n, g.offsets, g.cols, 0)
    for i in range(a):
        for j in range(b):
            assert r.level[idx(i, j)] == i + j
            assert int(r.paths[idx(i, j)]) == math.comb(i + j, i)


@pytest.mark.parametrize("d", [1, 3, 6])
def test_bfs_paths_hypercube_factorials(d):
    n = 1 << d
    src = [x for x in range(n) for k in range(d)]
    dst = [x ^ (1 << k) for x in range(n) for k in range(d)]
    g = gen.csr_from_edges(n, src, dst)
    r = oracle.bfs_paths(g.n, g.offsets, g.cols, 0)
    for x in range(n):
        h = bin(x).count("1")
        assert r.level[x] == h and int(r.paths[x]) == math.factorial(h)


@pytest.mark.parametrize("width,stages", [(2, 64), (2, 70), (3, 41), (3, 45)])
def test_bfs_paths_wraps_modulo_2_64(width, stages):
    # a chain of `stages` diamonds of `width` parallel two-edge routes, then a tail of two
    # vertices: width^stages paths reach the chain's end.  For 2^64 the count is 0 modulo
    # 2^64, yet the end vertex and the tail are still reached (a message with count 0 is a
    # message all the same).
    src, dst = [], []
    nxt = 1
    hub = 0
    for _ in range(stages):
        mids = list(range(nxt, nxt + width))
        end = nxt + width
        for m in mids:
            src += [hub, m]
            dst += [m, end]
        hub, nxt = end, end + 1
    src += [hub, hub + 1]
    dst += [hub + 1, hub + 2]
    n = hub + 3
    g = gen.csr_from_edges(n, src, dst)
    r = oracle.bfs_paths(g.n, g.offsets, g.cols, 0)
    assert r.level[hub] == 2 * stages and r.level[hub + 2] == 2 * stages + 2
    assert int(r.paths[hub]) == pow(width, stages, U64)
    assert int(r.paths[hub + 2]) == pow(width, stages, U64)
    assert r.supersteps == 2 * stages + 3


def test_bfs_paths_networkx_enumeration():
    nx = pytest.importorskip("networkx")
    for seed in range(10):
        g = gen.random_multigraph(9, 22, seed=seed)
        # networkx paths are vertex sequences: drop parallel edges so that they match
        rows = np.repeat(np.arange(g.n), g.out_degree())
        pairs = sorted(set(zip(rows.tolist(), g.cols.tolist())))
        g = gen.csr_from_edges(g.n, [p[0] for p in pairs], [p[1] for p in pairs])
        G = nx.DiGraph()
        G.add_nodes_from(range(g.n))
        G.add_edges_from(pairs)
        r = oracle.bfs_paths(g.n, g.offsets, g.cols, 0)
        for v in range(g.n):
            if v == 0:
                assert int(r.paths[0]) == 1
            elif nx.has_path(G, 0, v):
                assert int(r.paths[v]) == sum(1 for _ in nx.all_shortest_paths(G, 0, v))
            else:
                assert r.paths[v] == 0 and r.level[v] == oracle.INF


def test_bfs_paths_counts_parallel_edges():
    # two parallel edges 0 -> 1 and three 1 -> 2: 6 shortest paths as edge sequences
    g = gen.csr_from_edges(3, [0, 0, 1, 1, 1], [1, 1, 2, 2, 2])
    r = oracle.bfs_paths(g.n, g.offsets, g.cols, 0)
    np.testing.assert_array_equal(r.paths, [1, 2, 6])
    assert list(itertools.chain(r.level)) == [0, 1, 2]
