"""Autotuner and launch-shape knobs, through the C ABI.

Tuning changes speed only: every candidate ipg_autotune times gives
bit-identical results (min combiners are order-free; both PageRank engines and
every carveout add in one fixed order).  The tests check that the tuned graph
reproduces the untuned results bit for bit, that the chosen values come from
the documented candidate sets, that the PageRank ranks are bit-identical under
every engine/carveout pair and still match the float64 oracle, and that the
tuning cache is used for a second call and for an identical graph.
"""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

DIVISORS = {0, 2, 4, 6, 10, 16, 32}
PR_SHAPES = {(0, -1), (0, 60), (1, -1), (1, 5)}


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


def _results(ipg, h, g, src, hashmin):
    ranks, cr, _ = ipg.ipg_pagerank(h, 10)
    dist, cs, _ = ipg.ipg_sssp(h, src)
    out = {"ranks": ranks.view(np.uint32).copy(), "pr_count": cr, "dist": dist.copy(), "sssp_count": cs}
    if hashmin:
        labels, cc, _ = ipg.ipg_hashmin_cc(h)
        out.update(labels=labels.copy(), cc_count=cc)
    return out


CASES = [
    ("rmat12-directed", dict(scale=12, ef=16, undirected=False)),
    ("rmat13-undirected", dict(scale=13, ef=8, undirected=True)),
    ("rmat10-directed-sparse", dict(scale=10, ef=2, undirected=False)),
]


@pytest.mark.parametrize("name,spec", CASES, ids=[c[0] for c in CASES])
def test_autotune_keeps_results(ipg, name, spec):
    g = gen.rmat(spec["scale"], spec["ef"], seed=7, weighted=True, undirected=spec["undirected"])
    h = ipg.ipg_graph_create(g.offsets, g.cols, g.weights, g.n, g.m, not spec["undirected"])
    src = gen.max_out_degree_vertex(g)
    hashmin = spec["undirected"]
    before = _results(ipg, h, g, src, hashmin)
    batch_src = np.random.default_rng(1).integers(0, g.n, size=40).astype(np.uint32)
    before["batch"], before["batch_steps"] = ipg.ipg_sssp_batch(h, batch_src)
    progs = ipg.IPG_TUNE_PAGERANK | ipg.IPG_TUNE_SSSP | ipg.IPG_TUNE_SSSP_BATCH | \
        (ipg.IPG_TUNE_HASHMIN if hashmin else 0)
    rep = ipg.ipg_autotune(h, progs | ipg.IPG_TUNE_FORCE, src)
    assert rep["programs"] == progs and rep["cached"] == 0 and rep["candidates_timed"] > 0
    assert rep["sssp_pull_divisor"] in DIVISORS and rep["sssp_batch_divisor"] in DIVISORS
    assert rep["sssp_batch_chunk"] in (64, 128, 256, 512, 1024)
    assert rep["sssp_batch_ms"] > 0
    assert (rep["pr_engine"], rep["pr_carveout"]) in PR_SHAPES
    if hashmin:
        assert rep["hashmin_pull_divisor"] in DIVISORS
    else:
        assert rep["hashmin_pull_divisor"] == -1
    assert rep["pagerank_ms"] > 0 and rep["sssp_ms"] > 0
    after = _results(ipg, h, g, src, hashmin)
    after["batch"], after["batch_steps"] = ipg.ipg_sssp_batch(h, batch_src)
    for k in before:
        assert np.array_equal(np.asarray(before[k]), np.asarray(after[k])), k
    # a second call and an identical graph come from the cache
    again = ipg.ipg_autotune(h, progs, src)
    assert again["cached"] == 1 and again["candidates_timed"] == 0
    h2 = ipg.ipg_graph_create(g.offsets, g.cols, g.weights, g.n, g.m, not spec["undirected"])
    rep2 = ipg.ipg_autotune(h2, progs, src)
    assert rep2["cached"] == 1 and rep2["candidates_timed"] == 0
    for k in ("sssp_pull_divisor", "sssp_batch_divisor", "sssp_batch_chunk", "pr_engine", "pr_carveout",
              "hashmin_pull_divisor"):
        assert rep2[k] == rep[k], k
    after2 = _results(ipg, h2, g, src, hashmin)
    after2["batch"], after2["batch_steps"] = ipg.ipg_sssp_batch(h2, batch_src)
    for k in before:
        assert np.array_equal(np.asarray(before[k]), np.asarray(after2[k])), k
    h.destroy()
    h2.destroy()


def test_autotune_rejects(ipg):
    g = gen.rmat(8, 4, seed=3)
    h = ipg.ipg_graph_create(g.offsets, g.cols, None, g.n, g.m, True)
    with pytest.raises(ipg.IpgError):
        ipg.ipg_autotune(h, ipg.IPG_TUNE_HASHMIN)  # directed graph
    with pytest.raises(ipg.IpgError):
        ipg.ipg_autotune(h, 0x80)  # unknown bit
    rep = ipg.ipg_autotune(h, 0)
    assert rep["programs"] == 0 and rep["candidates_timed"] == 0
    h.destroy()


def test_pagerank_shapes_bit_identical(ipg):
    """Every (engine, carveout) pair the tuner may choose adds in the same order."""
    g = gen.rmat(14, 16, seed=5)
    ref = oracle.pagerank(g.n, g.offsets, g.cols, 10)
    h = ipg.ipg_graph_create(g.offsets, g.cols, None, g.n, g.m, True)
    old = {k: ipg.ipg_get_tuning(k) for k in ("pr_engine", "pr_carveout")}
    outs = []
    try:
        for eng, carve in sorted(PR_SHAPES):
            ipg.ipg_set_tuning("pr_engine", eng)
            ipg.ipg_set_tuning("pr_carveout", carve)
            r, c, _ = ipg.ipg_pagerank(h, 10)
            assert c == ref.supersteps
            err = np.max(np.abs(r.astype(np.float64) - ref.values)) / ref.values.max()
            assert err <= 1e-5, (eng, carve, err)
            outs.append(r.view(np.uint32).copy())
    finally:
        for k, v in old.items():
            ipg.ipg_set_tuning(k, v)
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    h.destroy()


def test_pagerank_512_threads_within_tolerance(ipg):
    g = gen.rmat(13, 16, seed=9)
    ref = oracle.pagerank(g.n, g.offsets, g.cols, 10)
    h = ipg.ipg_graph_create(g.offsets, g.cols, None, g.n, g.m, True)
    old = ipg.ipg_get_tuning("pr_threads")
    try:
        for eng in (0, 1):
            ipg.ipg_set_tuning("pr_threads", 512)
            ipg.ipg_set_tuning("pr_engine", eng)
            r, c, _ = ipg.ipg_pagerank(h, 10)
            err = np.max(np.abs(r.astype(np.float64) - ref.values)) / ref.values.max()
            assert c == ref.supersteps and err <= 1e-5, (eng, err)
    finally:
        ipg.ipg_set_tuning("pr_threads", old)
        ipg.ipg_set_tuning("pr_engine", 0)
    h.destroy()


def test_pagerank_captured_loop_matches_timed_loop(ipg):
    """Without per-superstep timing PageRank replays a captured CUDA graph of its
    supersteps; with timing it launches them one by one.  Both are the same kernels
    in the same order: bit-identical ranks, including after the update count (and so
    the captured graph) changes."""
    g = gen.rmat(12, 16, seed=11)
    h = ipg.ipg_graph_create(g.offsets, g.cols, None, g.n, g.m, True)
    for updates in (10, 3, 10):
        r_graph, c1, _ = ipg.ipg_pagerank(h, updates)
        r_timed, c2, st = ipg.ipg_pagerank(h, updates, stats_flags=ipg.IPG_STAT_TIMING)
        assert c1 == c2 == updates + 1
        assert all(s.kernel_ms > 0 for s in st[:updates])
        assert np.array_equal(r_graph.view(np.uint32), r_timed.view(np.uint32))
    h.destroy()
