"""The five workload configurations at their stated sizes, held to the CPU oracle
through the C ABI.

* configuration 3: PageRank (10 updates) and SSSP from the max-out-degree vertex on the
  directed, weighted R-MAT scale 26, edge factor 28 graph (1.84e9 edges): every rank of
  all 67M vertices within max|d rank| / max(rank) <= 1e-5 of the float64 oracle;
  distances, the superstep count and every per-superstep counter bit-exact; plus the
  SSSP run's Bellman certificate as a second, oracle-free check;
* configuration 4(a): 256 seeded sources on the directed, weighted R-MAT 22/16 graph in
  one batched call: every row equal to a standalone ipg_sssp run, and 16 rows equal to
  the oracle;
* configuration 4(b): 64 undirected R-MAT graphs of scales 10..20 in one batch object:
  every instance's labels and superstep count equal to the oracle's;
* configuration 5: the 32-graph serving set (undirected, weighted, scales 12..22): a
  seeded mixed stream served concurrently; every result equal to the same query run
  alone, and a seeded sample equal to the oracle.
(Configurations 1 and 2 are compared with the full oracle in test_parity_gpu.py.)

The oracle calls run on host threads (the oracle is a C library called through ctypes,
which releases the interpreter lock), concurrently with the GPU work and with each other.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

PR_TOL = 1e-5
THREADS = max(2, min(16, os.cpu_count() or 2))


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


def _cmp_stats(gpu_stats, gpu_count, orc):
    assert gpu_count == orc.supersteps
    assert len(gpu_stats) == len(orc.stats)
    for a, b in zip(gpu_stats, orc.stats):
        assert (a.superstep, a.senders, a.messages_sent, a.receivers, a.active) == \
               (b.superstep, b.senders, b.messages_sent, b.receivers, b.active), (a, b)


def _rows_chunks(offsets, step):
    n = offsets.size - 1
    u = 0
    while u < n:
        e0 = int(offsets[u])
        v = int(np.searchsorted(offsets, e0 + step, side="right")) - 1
        v = min(max(v, u + 1), n)
        yield u, v, e0, int(offsets[v])
        u = v


def _bellman_certificate(g, src, dist, outdeg):
    """Oracle-free proof of SSSP distances: every edge out of a reached vertex is relaxed,
    every reached vertex other than the source is tight on some in-edge, unreached vertices
    have no reached in-neighbour.  Returns 2 + the largest fewest-hop count of a shortest
    path to a reached vertex with out-edges (the superstep count's closed form)."""
    n = g.n
    INF = np.uint64(0xFFFFFFFF)
    big = np.iinfo(np.uint64).max
    best = np.full(n, big, dtype=np.uint64)
    d64 = dist.astype(np.uint64)
    tight_src, tight_dst = [], []
    for u0, u1, e0, e1 in _rows_chunks(g.offsets, 200_000_000):
        rows = np.repeat(np.arange(u0, u1, dtype=np.int64), outdeg[u0:u1])
        du = d64[rows]
        ok = du != INF
        cand = du[ok] + g.weights[e0:e1][ok].astype(np.uint64)
        cols = g.cols[e0:e1][ok]
        assert (d64[cols] <= cand).all(), "an edge is not relaxed"
        np.minimum.at(best, cols, cand)
        t = d64[cols] == cand
        tight_src.append(rows[ok][t])
        tight_dst.append(cols[t])
    reached = d64 != INF
    reached[src] = False
    np.testing.assert_array_equal(best[reached], d64[reached])
    assert (best[d64 == INF] == big).all()
    ts, td = np.concatenate(tight_src), np.concatenate(tight_dst)
    far = np.iinfo(np.int64).max
    hops = np.full(n, far, dtype=np.int64)
    hops[src] = 0
    for _ in range(10_000):
        cand = np.full(n, far, dtype=np.int64)
        fin = hops[ts] != far
        np.minimum.at(cand, td[fin], hops[ts[fin]] + 1)
        new = np.minimum(hops, cand)
        if np.array_equal(new, hops):
            break
        hops = new
    senders = (d64 != INF) & (outdeg > 0)
    return 2 + int(hops[senders].max())


def test_config3_billion_edge_against_the_oracle(ipg):
    """R-MAT scale 26, edge factor 28, weights in [1,255], seed 1 (1.84e9 edges)."""
    import torch

    dg = gen.rmat_device(26, 28, seed=1, weighted=True)
    h = ipg.ipg_graph_create_dev(dg.offsets, dg.cols, dg.weights, dg.n, dg.m, True)
    g = dg.to_host()
    del dg
    torch.cuda.empty_cache()
    n, m = g.n, g.m
    assert m > 1_800_000_000
    src = gen.max_out_degree_vertex(g)
    outdeg = g.out_degree()
    with ThreadPoolExecutor(max_workers=2) as ex:
        f_pr = ex.submit(oracle.pagerank, n, g.offsets, g.cols, 10)
        f_sssp = ex.submit(oracle.sssp, n, g.offsets, g.cols, g.weights, src)
        ranks, c_pr, st_pr = ipg.ipg_pagerank(h, 10, stats_flags=ipg.IPG_STAT_RECEIVERS)
        dist, c_sssp, st_sssp = ipg.ipg_sssp(h, src, stats_flags=ipg.IPG_STAT_RECEIVERS)
        h.destroy()
        torch.cuda.empty_cache()
        # while the oracle runs: the oracle-free checks
        assert c_pr == 11 and all(s.messages_sent == m for s in st_pr[:10])
        assert dist[src] == 0
        assert c_sssp == _bellman_certificate(g, src, dist, outdeg)
        ref_pr = f_pr.result()
        ref_sssp = f_sssp.result()
    err = np.max(np.abs(ranks.astype(np.float64) - ref_pr.values)) / np.max(ref_pr.values)
    assert err <= PR_TOL, err
    _cmp_stats(st_pr, c_pr, ref_pr)
    np.testing.assert_array_equal(dist, ref_sssp.values)
    _cmp_stats(st_sssp, c_sssp, ref_sssp)


def test_config4a_256_sources_batched(ipg):
    """256 uniform random sources (seed 1) on the directed, weighted R-MAT 22/16 graph."""
    import torch

    dg = gen.rmat_device(22, 16, seed=1, weighted=True)
    n, m = dg.n, dg.m
    h = ipg.ipg_graph_create_dev(dg.offsets, dg.cols, dg.weights, n, m, True)
    g = dg.to_host()
    del dg
    sources = gen.batch_sources(n, 256, 1)
    checked = np.arange(0, 256, 16)  # 16 rows against the oracle
    with ThreadPoolExecutor(max_workers=THREADS) as ex:
        futs = {int(i): ex.submit(oracle.sssp, n, g.offsets, g.cols, g.weights, int(sources[i])) for i in checked}
        out = torch.empty(256 * n, dtype=torch.int32, device="cuda")
        steps = ipg.ipg_sssp_batch_dev(h, sources, out)
        torch.cuda.synchronize()
        single = torch.empty(n, dtype=torch.int32, device="cuda")
        for i, s in enumerate(sources):
            c, _ = ipg.ipg_sssp_dev(h, int(s), single)
            torch.cuda.synchronize()
            assert torch.equal(out[i * n:(i + 1) * n], single), f"row {i} (source {s})"
            assert int(steps[i]) == c, (i, int(steps[i]), c)
        rows = {i: out[i * n:(i + 1) * n].cpu().numpy().view(np.uint32) for i in futs}
        for i, f in futs.items():
            ref = f.result()
            np.testing.assert_array_equal(rows[i], ref.values, err_msg=f"row {i}")
            assert int(steps[i]) == ref.supersteps
    h.destroy()


def test_config4b_64_graphs_batched(ipg):
    """64 undirected R-MAT graphs, EF 16, scales 10..20 (seeded), graph seeds 1..64."""
    scales = gen.cc_batch_scales(64, 1)
    graphs = [gen.rmat_device(sc, 16, seed=i + 1, undirected=True).to_host() for i, sc in enumerate(scales)]
    with ThreadPoolExecutor(max_workers=THREADS) as ex:
        futs = [ex.submit(oracle.hashmin, gr.n, gr.offsets, gr.cols) for gr in graphs]
        hb = ipg.ipg_graph_create_batch(graphs, directed=False)
        count, bases = ipg.ipg_graph_instances(hb)
        assert count == 64
        labels, steps = ipg.ipg_hashmin_cc_batch(hb)
        for i, f in enumerate(futs):
            ref = f.result()
            np.testing.assert_array_equal(labels[bases[i]:bases[i + 1]], ref.values, err_msg=f"instance {i}")
            assert steps[i] == ref.supersteps, (i, steps[i], ref.supersteps)
    hb.destroy()


def _oracle_query(g, kind, source):
    if kind == 0:
        return oracle.sssp(g.n, g.offsets, g.cols, g.weights, source)
    if kind == 1:
        return oracle.hashmin(g.n, g.offsets, g.cols)
    return oracle.pagerank(g.n, g.offsets, g.cols, 10)


def test_config5_served_set_against_the_oracle(ipg):
    """The 32 served graphs (undirected, weighted, EF 16, scales 12..22, graph seeds 101..132)
    and a seeded stream of 300 mixed queries (60% SSSP from a uniform random source, 30%
    Hashmin, 10% PageRank with 10 updates), all submitted at once so that they queue,
    batch and overlap on the device."""
    scales = gen.serve_scales(32, 1)
    graphs = [gen.rmat_device(sc, 16, seed=101 + i, undirected=True, weighted=True).to_host()
              for i, sc in enumerate(scales)]
    handles = [ipg.ipg_graph_create(gr.offsets, gr.cols, gr.weights, gr.n, gr.m, False) for gr in graphs]
    rng = np.random.default_rng(5)
    queries = []
    for u in range(300):
        gi = int(rng.integers(0, 32))
        r = rng.random()
        kind = 0 if r < 0.6 else (1 if r < 0.9 else 2)
        queries.append((u, gi, kind, int(rng.integers(0, graphs[gi].n))))
    # a seeded sample for the oracle: 24 SSSP, 12 Hashmin, 6 PageRank queries
    sample = []
    for kind, k in ((0, 24), (1, 12), (2, 6)):
        of_kind = [q for q in queries if q[2] == kind]
        pick = rng.choice(len(of_kind), size=min(k, len(of_kind)), replace=False)
        sample += [of_kind[int(i)] for i in pick]
    with ThreadPoolExecutor(max_workers=THREADS) as ex:
        futs = {u: ex.submit(_oracle_query, graphs[gi], kind, src) for u, gi, kind, src in sample}
        srv = ipg.Server(handles, workers=8, max_batch=256, prepare=True)
        done = []
        for u, gi, kind, src in queries:
            out = np.empty(graphs[gi].n, dtype=np.float32 if kind == 2 else np.uint32)
            srv.submit(gi, kind, out, source=src, updates=10, user=u)
        srv.drain()
        done += srv.poll(0)
        srv.close()
        assert len(done) == len(queries)
        by_user = {c.user: c for c in done}
        batched = 0
        for u, gi, kind, src in queries:
            c = by_user[u]
            assert c.status == 0
            if kind == 0:
                vals, cnt, _ = ipg.ipg_sssp(handles[gi], src)
            elif kind == 1:
                vals, cnt, _ = ipg.ipg_hashmin_cc(handles[gi])
            else:
                vals, cnt, _ = ipg.ipg_pagerank(handles[gi], 10)
            np.testing.assert_array_equal(c.out.view(np.uint32), vals.view(np.uint32), err_msg=f"query {u}")
            assert c.supersteps == cnt
            batched += kind == 0 and c.batch > 1
        assert batched > 0
        for u, f in futs.items():
            ref = f.result()
            c = by_user[u]
            kind = queries[u][2]
            if kind == 2:
                err = np.max(np.abs(c.out.astype(np.float64) - ref.values)) / np.max(ref.values)
                assert err <= PR_TOL, (u, err)
            else:
                np.testing.assert_array_equal(c.out, ref.values, err_msg=f"query {u}")
            assert c.supersteps == ref.supersteps, (u, c.supersteps, ref.supersteps)
    for hnd in handles:
        hnd.destroy()
