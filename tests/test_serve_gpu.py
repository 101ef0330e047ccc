"""Serving loop (ipg_server_*): a mixed stream of SSSP, Hashmin and PageRank queries on a
resident set of graphs.  Every result is the same in the mix as alone (bit for bit: the
min combiners are exact and PageRank sums in a fixed order), SSSP queries that queue up
on one graph run batched, and a tight workspace budget forces least-recently-used
workspace releases without changing any result."""
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


def _graph_set():
    out = []
    for i, sc in enumerate((8, 10, 12, 13, 9, 14)):
        out.append(gen.rmat(sc, 16, seed=100 + i, undirected=True, weighted=True))
    return out


def _alone(ipg, h, kind, source):
    if kind == ipg.IPG_Q_SSSP:
        return ipg.ipg_sssp(h, source)
    if kind == ipg.IPG_Q_HASHMIN:
        return ipg.ipg_hashmin_cc(h)
    return ipg.ipg_pagerank(h, 10)


def _mixed_queries(graphs, count, seed):
    rng = np.random.default_rng(seed)
    qs = []
    for u in range(count):
        gi = int(rng.integers(0, len(graphs)))
        r = rng.random()
        kind = 0 if r < 0.6 else (1 if r < 0.9 else 2)
        qs.append((u, gi, kind, int(rng.integers(0, graphs[gi].n))))
    return qs


SERVER_MODES = {
    "default": {},
    "prepared-min4": dict(prepare=True, min_sssp_batch=4),  # workspaces made up front; batch from 4 queries
    "autotuned": dict(autotune=True),                      # every graph tuned first: same results
}


@pytest.mark.parametrize("mode", sorted(SERVER_MODES))
@pytest.mark.parametrize("budget", [0, 1 << 22])
def test_results_same_alone_and_in_the_mix(ipg, budget, mode):
    graphs = _graph_set()
    handles = [ipg.ipg_graph_create(g.offsets, g.cols, g.weights, g.n, g.m, False) for g in graphs]
    queries = _mixed_queries(graphs, 300, seed=budget % 7 + 1)
    # results alone, before the server exists
    ref = {}
    for u, gi, kind, src in queries:
        vals, cnt, _ = _alone(ipg, handles[gi], kind, src)
        ref[u] = (vals.copy(), cnt)
    srv = ipg.Server(handles, workers=4, max_batch=64, workspace_budget=budget, **SERVER_MODES[mode])
    done = []
    for u, gi, kind, src in queries:
        out = np.empty(graphs[gi].n, dtype=np.float32 if kind == 2 else np.uint32)
        srv.submit(gi, kind, out, source=src, updates=10, user=u)
        done += srv.poll(0)
    srv.drain()
    done += srv.poll(0)
    srv.close()
    assert len(done) == len(queries)
    batched = 0
    for c in done:
        assert c.status == 0
        vals, cnt = ref[c.user]
        np.testing.assert_array_equal(c.out.view(np.uint32), vals.view(np.uint32))
        assert c.supersteps == cnt
        assert c.t_submit <= c.t_start <= c.t_done
        batched += c.batch > 1
    assert batched > 0  # SSSP queries that queued on one graph ran together


def test_server_rejects_bad_queries(ipg):
    g = gen.rmat(8, 8, seed=1, weighted=True)
    hd = ipg.ipg_graph_create(g.offsets, g.cols, g.weights, g.n, g.m, True)
    srv = ipg.Server([hd], workers=1)
    out = np.empty(g.n, dtype=np.uint32)
    with pytest.raises(ipg.IpgError):
        srv.submit(1, ipg.IPG_Q_SSSP, out, source=0)
    with pytest.raises(ipg.IpgError):
        srv.submit(0, ipg.IPG_Q_SSSP, out, source=g.n)
    with pytest.raises(ipg.IpgError):
        srv.submit(0, ipg.IPG_Q_HASHMIN, out)  # directed graph
    srv.submit(0, ipg.IPG_Q_SSSP, out, source=0, user=5)
    srv.drain()
    (c,) = srv.poll(0)
    ref, cnt, _ = ipg.ipg_sssp(hd, 0)
    assert c.user == 5 and c.status == 0 and c.supersteps == cnt
    np.testing.assert_array_equal(c.out, ref)
    srv.close()


def test_cancel_queued_queries(ipg):
    """Queries cancelled while queued complete with IPG_ECANCELED and leave their output
    untouched; the others still equal ipg_sssp alone.  One worker is kept busy on another
    graph (a long PageRank) so that the SSSP queries queue up behind it."""
    big = gen.rmat(16, 16, seed=7, undirected=True, weighted=True)
    small = gen.rmat(10, 16, seed=8, undirected=True, weighted=True)
    hb = ipg.ipg_graph_create(big.offsets, big.cols, big.weights, big.n, big.m, False)
    hs = ipg.ipg_graph_create(small.offsets, small.cols, small.weights, small.n, small.m, False)
    ref = {u: ipg.ipg_sssp(hs, u)[:2] for u in range(20)}
    cancelled_total = 0
    for _ in range(3):  # a cancel can lose the race with a free worker; retry the scenario
        srv = ipg.Server([hb, hs], workers=1, min_sssp_batch=1000)  # SSSP one source at a time
        srv.submit(0, ipg.IPG_Q_PAGERANK, np.empty(big.n, dtype=np.float32), updates=300, user=1000)
        outs = {}
        for u in range(20):
            outs[u] = np.full(small.n, 0xA5A5A5A5, dtype=np.uint32)
            srv.submit(1, ipg.IPG_Q_SSSP, outs[u], source=u, user=u)
        k = sum(srv.cancel(u) for u in range(0, 20, 2))
        assert srv.cancel(12345) == 0  # no such query
        srv.drain()
        done = srv.poll(0)
        srv.close()
        by_user = {c.user: c for c in done}
        assert len(done) == 21 and len(by_user) == 21
        assert by_user[1000].status == 0
        n_cancel = 0
        for u in range(20):
            c = by_user[u]
            if c.status == ipg.IPG_ECANCELED:
                assert u % 2 == 0
                assert c.supersteps == 0 and c.batch == 0 and c.t_start == c.t_done
                assert np.all(outs[u] == 0xA5A5A5A5)  # never written
                n_cancel += 1
            else:
                assert c.status == 0
                vals, cnt = ref[u]
                np.testing.assert_array_equal(c.out, vals)
                assert c.supersteps == cnt
        assert n_cancel == k
        cancelled_total += k
        if k:
            break
    assert cancelled_total > 0


def test_queries_join_a_running_lane_session(ipg):
    """SSSP queries submitted while a lane session runs on the graph are seeded into free
    lanes at superstep boundaries (completion.joined == 1); every result equals the oracle's
    and the query run alone, whichever superstep it joined at.  The single worker is first
    kept busy by a long PageRank on another graph, so the first SSSP queries queue up and
    start a session; the rest arrive while it runs."""
    import time

    import oracle

    g = gen.rmat(15, 16, seed=31, undirected=True, weighted=True)
    big = gen.rmat(16, 16, seed=32, undirected=True, weighted=True)
    h = ipg.ipg_graph_create(g.offsets, g.cols, g.weights, g.n, g.m, False)
    hb = ipg.ipg_graph_create(big.offsets, big.cols, big.weights, big.n, big.m, False)
    rng = np.random.default_rng(31)
    sources = [int(x) for x in rng.integers(0, g.n, size=120)]
    srv = ipg.Server([h, hb], workers=1, min_sssp_batch=4, prepare=True)
    srv.submit(1, ipg.IPG_Q_PAGERANK, np.empty(big.n, dtype=np.float32), updates=200, user=10_000)
    outs = {}
    for u, src in enumerate(sources):
        outs[u] = np.empty(g.n, dtype=np.uint32)
        srv.submit(0, ipg.IPG_Q_SSSP, outs[u], source=src, user=u)
        if u >= 8 and u % 2 == 0:
            time.sleep(0.001)  # later queries arrive while the session runs
    srv.drain()
    done = [c for c in srv.poll(0) if c.user != 10_000]
    srv.close()
    assert len(done) == len(sources)
    joined = 0
    for c in done:
        assert c.status == 0
        ref, cnt, _ = ipg.ipg_sssp(h, sources[c.user])
        np.testing.assert_array_equal(c.out, ref)
        assert c.supersteps == cnt
        joined += c.joined
    assert joined > 0
    for u in range(0, len(sources), 15):  # a sample against the oracle
        o = oracle.sssp(g.n, g.offsets, g.cols, g.weights, sources[u])
        np.testing.assert_array_equal(outs[u], o.values)
