"""Pins for the CPU oracle: each test checks it against something other than itself.

* PageRank: closed forms on a directed cycle, an in-star and an out-star (the
  latter two catch a transposed graph), the fixed point of the update rule as a
  dense linear solve, the rank-mass identity, and brute-force per-superstep
  message counts.
* Hashmin CC: scipy connected components (min id per component), the superstep
  count closed form 2 + max eccentricity of each component's minimum vertex,
  and per-superstep sender / receiver counts from BFS hop distances.
* SSSP: scipy Dijkstra, BFS levels for the unweighted case (Sec. VI-C),
  the superstep count 2 + L where L is the largest hop count of a
  minimum-weight path to a vertex with out-edges, and per-superstep senders
  from brute-force enumeration of walks on tiny graphs.
"""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse import csgraph

import gen
import oracle

# ---------------------------------------------------------------------------------------
# helpers (library routines and brute force; none of the oracle's code)


def _unweighted_matrix(g):
    n = g.n
    rows = np.repeat(np.arange(n), g.out_degree())
    return sp.csr_matrix((np.ones(g.m), (rows, g.cols.astype(np.int64))), shape=(n, n))


def _min_weight_matrix(g, weights):
    """Sparse matrix holding the smallest weight among parallel edges (scipy would add them)."""
    n = g.n
    rows = np.repeat(np.arange(n), g.out_degree())
    cols = g.cols.astype(np.int64)
    key = rows * n + cols
    order = np.lexsort((weights, key))
    key, w = key[order], weights[order].astype(np.float64)
    first = np.ones(key.size, dtype=bool)
    first[1:] = key[1:] != key[:-1]
    key, w = key[first], w[first]
    return sp.csr_matrix((w, (key // n, key % n)), shape=(n, n))


def _small_graphs(undirected):
    yield gen.csr_from_edges(1, [], [], undirected=undirected)  # n = 1, m = 0
    yield gen.csr_from_edges(5, [], [], undirected=undirected)  # isolated vertices only
    yield gen.csr_from_edges(3, [0, 1, 1], [0, 1, 1], undirected=undirected)  # self-loops only
    yield gen.csr_from_edges(6, [0, 0, 2, 3, 3, 5], [1, 1, 3, 4, 4, 5], undirected=undirected)  # multi-edges
    for seed in range(6):
        yield gen.random_multigraph(12 + seed, 20 + 3 * seed, seed=seed, undirected=undirected)
    for scale in (4, 5, 6, 7):
        yield gen.rmat(scale, 4, seed=scale, undirected=undirected)


# ---------------------------------------------------------------------------------------
# PageRank


@pytest.mark.parametrize("N", [1, 2, 3, 7, 64])
@pytest.mark.parametrize("T", [1, 2, 10])
def test_pagerank_cycle_is_uniform(N, T):
    # directed N-cycle: every vertex has one in- and one out-edge, so 1/N is a fixed point
    g = gen.csr_from_edges(N, np.arange(N), (np.arange(N) + 1) % N)
    r = oracle.pagerank(g.n, g.offsets, g.cols, T)
    np.testing.assert_allclose(r.values, 1.0 / N, rtol=1e-14, atol=0)
    assert r.supersteps == T + 1


@pytest.mark.parametrize("N", [2, 5, 33])
@pytest.mark.parametrize("T", [1, 2, 3, 10])
def test_pagerank_in_star_closed_form(N, T):
    # leaves 1..N-1 -> centre 0; the centre is dangling, leaves receive nothing
    g = gen.csr_from_edges(N, np.arange(1, N), np.zeros(N - 1, dtype=int))
    r = oracle.pagerank(g.n, g.offsets, g.cols, T).values
    base = 0.15 / N
    np.testing.assert_allclose(r[1:], base, rtol=1e-14)
    centre = base + 0.85 * (N - 1) / N if T == 1 else base + 0.85 * (N - 1) * base
    np.testing.assert_allclose(r[0], centre, rtol=1e-14)


@pytest.mark.parametrize("N", [2, 5, 33])
@pytest.mark.parametrize("T", [1, 2, 3, 10])
def test_pagerank_out_star_closed_form(N, T):
    # centre 0 -> leaves; the centre receives nothing, the leaves are dangling
    g = gen.csr_from_edges(N, np.zeros(N - 1, dtype=int), np.arange(1, N))
    r = oracle.pagerank(g.n, g.offsets, g.cols, T).values
    base = 0.15 / N
    np.testing.assert_allclose(r[0], base, rtol=1e-14)
    prev_centre = 1.0 / N if T == 1 else base
    np.testing.assert_allclose(r[1:], base + 0.85 * prev_centre / (N - 1), rtol=1e-14)


def _transition(g):
    """M[v, u] = (number of u->v edges) / outdeg(u)."""
    A = _unweighted_matrix(g).toarray()  # A[u, v] = multiplicity (duplicates summed)
    out = A.sum(axis=1)
    M = np.zeros_like(A)
    nz = out > 0
    M[:, nz] = (A[nz, :] / out[nz, None]).T
    return M


@pytest.mark.parametrize("seed", range(5))
def test_pagerank_fixed_point_linear_solve(seed):
    # after many updates the iteration sits at the unique solution of x = 0.15/N + 0.85 M x
    g = gen.random_multigraph(24, 70, seed=100 + seed)
    N = g.n
    x = np.linalg.solve(np.eye(N) - 0.85 * _transition(g), np.full(N, 0.15 / N))
    r = oracle.pagerank(g.n, g.offsets, g.cols, 400).values
    np.testing.assert_allclose(r, x, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("seed", range(3))
def test_pagerank_one_update_dense(seed):
    # one update from the uniform start, written as a dense product (small n only)
    g = gen.random_multigraph(17, 40, seed=200 + seed)
    N = g.n
    expect = 0.15 / N + 0.85 * _transition(g) @ np.full(N, 1.0 / N)
    r = oracle.pagerank(g.n, g.offsets, g.cols, 1).values
    np.testing.assert_allclose(r, expect, rtol=1e-14)


@pytest.mark.parametrize("scale", [6, 9])
def test_pagerank_mass_identity_and_counts(scale):
    g = gen.rmat(scale, 8, seed=scale)
    outdeg = g.out_degree()
    indeg = np.bincount(g.cols, minlength=g.n)
    assert (outdeg == 0).any()  # dangling vertices present, so mass leaks
    for T in (1, 4, 10):
        prev = oracle.pagerank(g.n, g.offsets, g.cols, T - 1).values
        cur = oracle.pagerank(g.n, g.offsets, g.cols, T)
        # sum_v rank_T(v) = 0.15 + 0.85 * sum over non-dangling u of rank_{T-1}(u)
        np.testing.assert_allclose(cur.values.sum(), 0.15 + 0.85 * prev[outdeg > 0].sum(), rtol=1e-12)
        for s, st in enumerate(cur.stats):
            assert st.superstep == s and st.active == g.n
            if s < T:
                assert st.senders == g.n and st.messages_sent == g.m
                assert st.receivers == int((indeg > 0).sum())
            else:
                assert st.senders == 0 and st.messages_sent == 0 and st.receivers == 0


def test_pagerank_without_dangling_conserves_mass():
    g = gen.random_multigraph(50, 400, seed=7)
    g = gen.csr_from_edges(50, np.concatenate([np.repeat(np.arange(50), g.out_degree()), np.arange(50)]),
                           np.concatenate([g.cols, (np.arange(50) + 1) % 50]))
    r = oracle.pagerank(g.n, g.offsets, g.cols, 10).values
    assert abs(r.sum() - 1.0) < 1e-13


# ---------------------------------------------------------------------------------------
# Hashmin connected components


def _hop_distances(g):
    d = csgraph.shortest_path(_unweighted_matrix(g), directed=True, unweighted=True)
    return d  # inf where unreachable


def test_hashmin_matches_components_and_closed_forms():
    for g in _small_graphs(undirected=True):
        r = oracle.hashmin(g.n, g.offsets, g.cols)
        ncomp, comp = csgraph.connected_components(_unweighted_matrix(g), directed=False)
        minid = np.full(ncomp, g.n, dtype=np.int64)
        np.minimum.at(minid, comp, np.arange(g.n))
        np.testing.assert_array_equal(r.values, minid[comp])

        D = _hop_distances(g)
        if g.m == 0:
            assert r.supersteps == 1
        else:
            ecc = max(int(np.max(D[c][np.isfinite(D[c])])) for c in minid)
            assert r.supersteps == 2 + ecc

        # label after superstep s = smallest id within s hops; senders = vertices whose label dropped
        ids = np.arange(g.n, dtype=np.float64)
        outdeg = g.out_degree()
        rows = np.repeat(np.arange(g.n), outdeg)
        prev = None
        for s, st in enumerate(r.stats):
            lab = np.array([ids[D[:, v] <= s].min() for v in range(g.n)])
            send = np.ones(g.n, bool) if s == 0 else lab < prev
            assert st.senders == int(send.sum()), (s, st)
            assert st.messages_sent == int(outdeg[send].sum())
            assert st.receivers == np.unique(g.cols[send[rows]]).size
            assert st.active == (g.n if s == 0 else r.stats[s - 1].receivers)
            prev = lab


def test_hashmin_rmat_components():
    g = gen.rmat(10, 4, seed=3, undirected=True)
    r = oracle.hashmin(g.n, g.offsets, g.cols)
    ncomp, comp = csgraph.connected_components(_unweighted_matrix(g), directed=False)
    minid = np.full(ncomp, g.n, dtype=np.int64)
    np.minimum.at(minid, comp, np.arange(g.n))
    np.testing.assert_array_equal(r.values, minid[comp])


# ---------------------------------------------------------------------------------------
# SSSP


def _lexicographic_hops(g, weights, source):
    """Hop count of the fewest-hop minimum-weight path, via Dijkstra on w*BIG + 1."""
    big = g.n + 1
    W = _min_weight_matrix(g, weights.astype(np.int64) * big + 1)
    d = csgraph.dijkstra(W, directed=True, indices=source)
    fin = np.isfinite(d)
    hops = np.full(g.n, -1, dtype=np.int64)
    hops[fin] = (d[fin].astype(np.int64)) % big
    dist = np.full(g.n, oracle.INF, dtype=np.int64)
    dist[fin] = d[fin].astype(np.int64) // big
    return dist, hops


def _sssp_cases():
    for g in _small_graphs(undirected=False):
        rng = np.random.default_rng(g.n * 7 + g.m)
        w = rng.integers(1, 256, size=g.m).astype(np.uint32)
        for src in sorted({0, g.n - 1, g.n // 2}):
            yield g, w, src
            yield g, None, src


def test_sssp_matches_dijkstra_and_superstep_closed_form():
    for g, w, src in _sssp_cases():
        r = oracle.sssp(g.n, g.offsets, g.cols, w, src)
        ww = np.ones(g.m, dtype=np.int64) if w is None else w.astype(np.int64)
        dist, hops = _lexicographic_hops(g, ww, src)
        np.testing.assert_array_equal(r.values.astype(np.int64), dist)
        plain = csgraph.dijkstra(_min_weight_matrix(g, ww), directed=True, indices=src)
        np.testing.assert_array_equal(np.where(np.isfinite(plain), plain, oracle.INF).astype(np.int64), dist)
        outdeg = g.out_degree()
        senders = (hops >= 0) & (outdeg > 0)
        if outdeg[src] == 0:
            assert r.supersteps == 1
        else:
            assert r.supersteps == 2 + int(hops[senders].max())


def test_sssp_unweighted_is_bfs():
    for g in _small_graphs(undirected=False):
        for src in (0, g.n - 1):
            r = oracle.sssp(g.n, g.offsets, g.cols, None, src)
            d = csgraph.shortest_path(_unweighted_matrix(g), directed=True, unweighted=True, indices=src)
            np.testing.assert_array_equal(r.values.astype(np.int64),
                                          np.where(np.isfinite(d), d, oracle.INF).astype(np.int64))


def _walk_minima(g, w, src, kmax):
    """best[k][v] = smallest weight of a walk from src to v with at most k edges (brute force)."""
    n = g.n
    adj = [[(int(g.cols[e]), int(w[e])) for e in range(int(g.offsets[u]), int(g.offsets[u + 1]))] for u in range(n)]
    best = []
    for k in range(kmax + 1):
        b = [np.inf] * n
        b[src] = 0
        frontier = {(src, 0)}
        seen = set(frontier)
        for _ in range(k):
            nxt = set()
            for u, d in frontier:
                for v, ww in adj[u]:
                    item = (v, d + ww)
                    if item not in seen:
                        seen.add(item)
                        nxt.add(item)
                        b[v] = min(b[v], d + ww)
            frontier = nxt
        best.append(b)
    return best


@pytest.mark.parametrize("seed", range(8))
def test_sssp_per_superstep_senders_brute_force(seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(2, 8))
    g = gen.random_multigraph(n, int(rng.integers(1, 14)), seed=seed)
    w = rng.integers(1, 6, size=g.m).astype(np.uint32)
    src = int(rng.integers(0, n))
    r = oracle.sssp(g.n, g.offsets, g.cols, w, src)
    best = _walk_minima(g, w, src, r.supersteps)
    outdeg = g.out_degree()
    rows = np.repeat(np.arange(g.n), outdeg)
    for s, st in enumerate(r.stats):
        cur = np.array(best[s])
        prev = np.full(n, np.inf) if s == 0 else np.array(best[s - 1])
        send = cur < prev  # the vertex's best value improved in superstep s
        assert st.senders == int(send.sum()), (s, st)
        assert st.messages_sent == int(outdeg[send].sum())
        assert st.receivers == np.unique(g.cols[send[rows]]).size


def test_sssp_overflow_is_reported():
    g = gen.csr_from_edges(3, [0, 1], [1, 2], [0xFFFFFF00, 0xFFFFFF00])
    with pytest.raises(oracle.OracleError):
        oracle.sssp(g.n, g.offsets, g.cols, g.weights, 0)


def test_oracle_rejects_bad_csr():
    with pytest.raises(oracle.OracleError):
        oracle.hashmin(2, np.array([0, 1, 1], dtype=np.uint64), np.array([5], dtype=np.uint32))
    with pytest.raises(oracle.OracleError):
        oracle.sssp(2, np.array([0, 0, 0], dtype=np.uint64), np.zeros(0, np.uint32), None, 2)


def test_max_supersteps_stops_early():
    g = gen.csr_from_edges(6, np.arange(5), np.arange(1, 6))  # path 0->1->...->5
    full = oracle.sssp(g.n, g.offsets, g.cols, None, 0)
    assert full.supersteps == 2 + 4
    cut = oracle.sssp(g.n, g.offsets, g.cols, None, 0, max_supersteps=3)
    assert cut.supersteps == 3
    np.testing.assert_array_equal(cut.values[:3], [0, 1, 2])
    assert (cut.values[3:] == oracle.INF).all()
