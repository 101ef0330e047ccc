"""Batched SSSP (ipg_sssp_batch): every row equals a standalone ipg_sssp run from the
same source — distances and superstep count, bit for bit — and the oracle on small
graphs.  Groups of 32 sources share supersteps, so the cases cover groups that end
early or late, more than 32 sources, repeated sources and sources without out-edges."""
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


@pytest.fixture(autouse=True, params=["auto", "pull", "push"])
def batch_direction(request, ipg):
    """Every batched SSSP test runs with the automatic push/pull switch, pull only
    (batch_divisor 0) and push whenever the senders hold fewer than all m edges (1)."""
    old = ipg.ipg_get_tuning("batch_divisor")
    ipg.ipg_set_tuning("batch_divisor", {"auto": old, "pull": 0, "push": 1}[request.param])
    yield request.param
    ipg.ipg_set_tuning("batch_divisor", old)


def _check_batch(ipg, g, sources, weights, use_oracle=False):
    h = ipg.ipg_graph_create(g.offsets, g.cols, weights, g.n, g.m, g.directed)
    dist, steps = ipg.ipg_sssp_batch(h, sources)
    assert dist.shape == (len(sources), g.n)
    for i, s in enumerate(sources):
        ref, cnt, _ = ipg.ipg_sssp(h, int(s))
        np.testing.assert_array_equal(dist[i], ref, err_msg=f"source {s}")
        assert steps[i] == cnt, (s, steps[i], cnt)
        if use_oracle:
            o = oracle.sssp(g.n, g.offsets, g.cols, weights, int(s))
            np.testing.assert_array_equal(dist[i], o.values)
            assert steps[i] == o.supersteps
    return dist, steps


@pytest.mark.parametrize("seed", range(6))
def test_batch_random_multigraphs(ipg, seed):
    rng = np.random.default_rng(50 + seed)
    n = int(rng.integers(2, 2500))
    g = gen.random_multigraph(n, int(rng.integers(1, 20000)), seed=seed, weighted=True)
    k = int(rng.integers(1, 70))
    sources = rng.integers(0, n, size=k)
    _check_batch(ipg, g, sources, g.weights, use_oracle=True)
    _check_batch(ipg, g, sources, None, use_oracle=True)


@pytest.mark.parametrize("scale", [8, 12, 16])
def test_batch_rmat(ipg, scale):
    g = gen.rmat(scale, 16, seed=scale, weighted=True)
    rng = np.random.default_rng(scale)
    sources = list(rng.integers(0, g.n, size=40)) + [gen.max_out_degree_vertex(g)] * 2
    zero_out = np.nonzero(g.out_degree() == 0)[0]
    if zero_out.size:
        sources.append(int(zero_out[0]))
    _check_batch(ipg, g, np.array(sources), g.weights, use_oracle=scale <= 12)


def test_batch_wide_weights_and_undirected(ipg):
    g = gen.rmat(11, 8, seed=3)
    rng = np.random.default_rng(3)
    w = rng.integers(1, 100000, size=g.m).astype(np.uint32)  # u32 weights (> 255)
    _check_batch(ipg, g, rng.integers(0, g.n, size=33), w, use_oracle=True)
    u = gen.rmat(11, 8, seed=4, undirected=True, weighted=True)
    _check_batch(ipg, u, rng.integers(0, u.n, size=17), u.weights, use_oracle=True)


def test_batch_device_entry_and_errors(ipg):
    import torch

    g = gen.rmat(10, 16, seed=5, weighted=True)
    h = ipg.ipg_graph_create(g.offsets, g.cols, g.weights, g.n, g.m, True)
    sources = np.arange(0, 40, dtype=np.uint32)
    ref, ref_steps = ipg.ipg_sssp_batch(h, sources)
    d = torch.empty(len(sources) * g.n, dtype=torch.int32, device="cuda")
    steps = ipg.ipg_sssp_batch_dev(h, sources, d)
    np.testing.assert_array_equal(d.cpu().numpy().view(np.uint32).reshape(len(sources), g.n), ref)
    np.testing.assert_array_equal(steps, ref_steps)
    with pytest.raises(ipg.IpgError) as e:
        ipg.ipg_sssp_batch(h, [0, g.n])
    assert e.value.status == 1
    big = gen.csr_from_edges(3, [0, 1], [1, 2], [0xFFFFFF00, 0xFFFFFF00])
    hb = ipg.ipg_graph_create(big.offsets, big.cols, big.weights, 3, 2, True)
    with pytest.raises(ipg.IpgError) as e:
        ipg.ipg_sssp_batch(hb, [0])
    assert e.value.status == 7
    dist, steps = ipg.ipg_sssp_batch(h, [])
    assert dist.shape == (0, g.n)


# ---------------------------------------------------------------------------------------
# many graphs in one object: Hashmin on every instance at once


@pytest.fixture(params=["graph-loop", "host-loop"])
def driver(request, ipg):
    """The union's superstep loop (and its per-instance superstep counts) on the device in a
    CUDA graph, or driven from the host."""
    old = ipg.ipg_get_tuning("push_loop")
    ipg.ipg_set_tuning("push_loop", 1 if request.param == "graph-loop" else 0)
    yield request.param
    ipg.ipg_set_tuning("push_loop", old)


@pytest.fixture(params=["auto", "push", "pull"])
def direction(request, ipg, driver):
    old = ipg.ipg_get_tuning("pull_divisor")
    ipg.ipg_set_tuning("pull_divisor", {"auto": old, "push": 0, "pull": 1 << 40}[request.param])
    yield request.param
    ipg.ipg_set_tuning("pull_divisor", old)


def _instances(seed):
    rng = np.random.default_rng(seed)
    out = [gen.csr_from_edges(0, [], [], undirected=True),  # an empty instance
           gen.csr_from_edges(1, [], [], undirected=True),
           gen.csr_from_edges(5, [0, 1, 3], [1, 2, 3], undirected=True)]
    for i in range(6):
        out.append(gen.random_multigraph(int(rng.integers(1, 400)), int(rng.integers(0, 900)), seed=seed * 10 + i,
                                         undirected=True))
    for sc in (6, 9, 12):
        out.append(gen.rmat(sc, 8, seed=sc + seed, undirected=True))
    return out


@pytest.mark.parametrize("seed", range(3))
def test_hashmin_batch_matches_each_instance(ipg, direction, seed):
    graphs = _instances(seed)
    hb = ipg.ipg_graph_create_batch(graphs, directed=False)
    count, bases = ipg.ipg_graph_instances(hb)
    assert count == len(graphs) and bases[-1] == sum(g.n for g in graphs)
    labels, steps = ipg.ipg_hashmin_cc_batch(hb)
    for i, g in enumerate(graphs):
        mine = labels[bases[i]:bases[i + 1]]
        ref = oracle.hashmin(g.n, g.offsets, g.cols)
        np.testing.assert_array_equal(mine, ref.values)
        assert steps[i] == ref.supersteps, (i, steps[i], ref.supersteps)
        if g.n:
            h = ipg.ipg_graph_create(g.offsets, g.cols, None, g.n, g.m, False)
            alone, cnt, _ = ipg.ipg_hashmin_cc(h)
            np.testing.assert_array_equal(mine, alone)
            assert cnt == steps[i]


def test_hashmin_batch_device_and_errors(ipg):
    import torch

    graphs = _instances(7)
    hb = ipg.ipg_graph_create_batch(graphs, directed=False)
    labels, steps = ipg.ipg_hashmin_cc_batch(hb)
    t = torch.empty(labels.size, dtype=torch.int32, device="cuda")
    steps2 = ipg.ipg_hashmin_cc_batch_dev(hb, t)
    np.testing.assert_array_equal(t.cpu().numpy().view(np.uint32), labels)
    np.testing.assert_array_equal(steps, steps2)
    bad = gen.csr_from_edges(3, [0], [1])
    bad.cols = np.array([7], dtype=np.uint32)  # column beyond its own instance
    with pytest.raises(ipg.IpgError) as e:
        ipg.ipg_graph_create_batch([graphs[3], bad], directed=False)
    assert e.value.status == 1
    # a plain graph is one instance
    g = gen.rmat(8, 8, seed=2, undirected=True)
    h = ipg.ipg_graph_create(g.offsets, g.cols, None, g.n, g.m, False)
    lab, st = ipg.ipg_hashmin_cc_batch(h)
    ref = oracle.hashmin(g.n, g.offsets, g.cols)
    np.testing.assert_array_equal(lab, ref.values)
    assert list(st) == [ref.supersteps]


def test_batch_long_paths_span_several_graph_launches(ipg):
    """A directed path of 300 vertices (plus a back edge and shortcuts) needs about
    300 supersteps from vertex 0: the device-side loop stops every 64 supersteps and
    the host relaunches it; counts and distances must still equal ipg_sssp's."""
    n = 300
    src = list(range(n - 1)) + [n - 1, 10, 100]
    dst = list(range(1, n)) + [0, 200, 250]
    w = np.array([1 + (i * 7) % 255 for i in range(len(src))], dtype=np.uint32)
    g = gen.csr_from_edges(n, np.array(src), np.array(dst), weights=w)
    sources = np.array([0, 1, 5, 150, 299, 0])
    dist, steps = _check_batch(ipg, g, sources, g.weights, use_oracle=True)
    assert steps.max() > 3 * 64


@pytest.mark.parametrize("chunk", [32, 128, 1024, 4096])
def test_batch_chunk_sizes_give_the_same_rows(ipg, chunk):
    """The pull forms' tile sizes (in-edges per warp task; batch_chunk with one line of
    lanes, batch_wide_chunk with more) change no row or count.  batch_tile_tasks = 0
    keeps the set sizes on this small graph; 3 (the default) halves them to the floor."""
    g = gen.rmat(12, 16, seed=12, weighted=True)
    rng = np.random.default_rng(12)
    names = ("batch_chunk", "batch_wide_chunk", "batch_tile_tasks")
    old = [ipg.ipg_get_tuning(x) for x in names]
    try:
        ipg.ipg_set_tuning("batch_chunk", chunk)
        ipg.ipg_set_tuning("batch_wide_chunk", chunk)
        for tasks in (0, 3):
            ipg.ipg_set_tuning("batch_tile_tasks", tasks)
            for k in (20, 45, 150):  # one, two and five lines
                _check_batch(ipg, g, rng.integers(0, g.n, size=k), g.weights)
    finally:
        for x, v in zip(names, old):
            ipg.ipg_set_tuning(x, v)


def _lines_for(g, sources):
    """Lines of 32 lanes a batched call uses: enough for the sources with out-edges, at most 8."""
    sending = int((g.out_degree()[np.asarray(sources)] > 0).sum())
    return min(8, max(1, (sending + 31) // 32))


@pytest.mark.parametrize("k", [33, 70, 140, 300])
def test_batch_wide_lines(ipg, k):
    """More than 32 queries run in up to 8 lines of 32 lanes; beyond 256 the lanes
    that finish take the rest.  Sources without out-edges are listed after the others,
    so every row must still land in its own output row.  u8, u32 and unit weights."""
    rng = np.random.default_rng(900 + k)
    g = gen.random_multigraph(3000, 24000, seed=k, weighted=True)
    zero = np.nonzero(g.out_degree() == 0)[0]
    sources = rng.integers(0, g.n, size=k)
    if zero.size:
        sources[::7] = zero[rng.integers(0, zero.size, size=sources[::7].size)]
    sources[1] = sources[0]  # a repeated source
    wide = rng.integers(1, 70000, size=g.m).astype(np.uint32)
    import torch

    for weights in (g.weights, wide, None):
        h = ipg.ipg_graph_create(g.offsets, g.cols, weights, g.n, g.m, True)
        # the device entry runs all k in one call (the host entry stages groups of 256)
        d = torch.empty(k * g.n, dtype=torch.int32, device="cuda")
        steps = ipg.ipg_sssp_batch_dev(h, sources, d)
        torch.cuda.synchronize()
        dist = d.cpu().numpy().view(np.uint32).reshape(k, g.n)
        info = ipg.ipg_sssp_batch_info(h)
        assert info["queries"] == k and info["lanes"] == 32 * _lines_for(g, sources), info
        for i in list(range(0, k, 5)) + [1, k - 1]:
            ref, cnt, _ = ipg.ipg_sssp(h, int(sources[i]))
            np.testing.assert_array_equal(dist[i], ref, err_msg=f"row {i} source {sources[i]}")
            assert steps[i] == cnt
        for i in (0, 2, k // 2):
            o = oracle.sssp(g.n, g.offsets, g.cols, weights, int(sources[i]))
            np.testing.assert_array_equal(dist[i], o.values)
            assert steps[i] == o.supersteps


def test_batch_wide_then_one_line_on_one_graph(ipg):
    """A graph whose workspace grew to 8 lines serves a one-line call next, and the
    reverse: the value arrays are re-laid out between calls without stale values."""
    g = gen.rmat(11, 16, seed=21, weighted=True)
    rng = np.random.default_rng(21)
    h = ipg.ipg_graph_create(g.offsets, g.cols, g.weights, g.n, g.m, True)
    few = rng.integers(0, g.n, size=9)
    many = rng.integers(0, g.n, size=250)
    for sources in (few, many, few, many[:40]):
        dist, steps = ipg.ipg_sssp_batch(h, sources)
        for i in range(0, len(sources), 3):
            ref, cnt, _ = ipg.ipg_sssp(h, int(sources[i]))
            np.testing.assert_array_equal(dist[i], ref)
            assert steps[i] == cnt


@pytest.mark.parametrize("first_weight", [0xFFFFFF00, 0xFFFFFFFF])
def test_batch_wide_overflow_is_reported(ipg, first_weight):
    """A path length that would reach UINT32_MAX fails the whole batched call with
    IPG_EOVERFLOW in the wide engine too (40 sending queries: two lines of lanes),
    whether the first message already overflows or the second one does."""
    n = 50
    src = [0, 1] + list(range(3, 43))
    dst = [1, 2] + [44] * 40
    w = [first_weight, 0xFFFFFF00] + [1] * 40
    g = gen.csr_from_edges(n, np.array(src), np.array(dst), weights=np.array(w, dtype=np.uint32))
    h = ipg.ipg_graph_create(g.offsets, g.cols, g.weights, n, g.m, True)
    sources = [0] + list(range(3, 43))
    with pytest.raises(ipg.IpgError) as e:
        ipg.ipg_sssp_batch(h, sources)
    assert e.value.status == 7
    # without the overflowing source the same graph runs
    dist, steps = ipg.ipg_sssp_batch(h, sources[1:])
    assert ipg.ipg_sssp_batch_info(h)["lanes"] == 64
    for i, s in enumerate(sources[1:]):
        ref, cnt, _ = ipg.ipg_sssp(h, s)
        np.testing.assert_array_equal(dist[i], ref)
        assert steps[i] == cnt


@pytest.mark.parametrize("k", [20, 150])
def test_batch_host_driven_loop_gives_the_same_rows(ipg, k):
    """batch_loop 0 launches every superstep's kernels from the host instead of the
    graph's WHILE node; one and eight lines give the same rows and counts."""
    g = gen.rmat(12, 16, seed=31, weighted=True)
    sources = np.random.default_rng(31 + k).integers(0, g.n, size=k)
    h = ipg.ipg_graph_create(g.offsets, g.cols, g.weights, g.n, g.m, True)
    ref, ref_steps = ipg.ipg_sssp_batch(h, sources)
    old = ipg.ipg_get_tuning("batch_loop")
    try:
        ipg.ipg_set_tuning("batch_loop", 0)
        dist, steps = ipg.ipg_sssp_batch(h, sources)
    finally:
        ipg.ipg_set_tuning("batch_loop", old)
    np.testing.assert_array_equal(dist, ref)
    np.testing.assert_array_equal(steps, ref_steps)
    for i in range(0, k, 7):
        o, cnt, _ = ipg.ipg_sssp(h, int(sources[i]))
        np.testing.assert_array_equal(dist[i], o)
        assert steps[i] == cnt


def test_batch_sources_without_out_edges_only(ipg):
    """Every source without out-edges: no lane runs, each row holds only its source at
    distance 0, and every count is 1 (superstep 0 alone); also on a graph with no edges."""
    g = gen.csr_from_edges(6, np.array([0, 1, 2]), np.array([1, 2, 0]), weights=np.array([3, 4, 5], dtype=np.uint32))
    empty = gen.csr_from_edges(4, np.array([], dtype=np.int64), np.array([], dtype=np.int64))
    for graph, weights, sources in ((g, g.weights, [3, 4, 5, 5, 3]), (empty, None, [0, 3, 1, 2, 0, 3])):
        h = ipg.ipg_graph_create(graph.offsets, graph.cols, weights, graph.n, graph.m, True)
        dist, steps = ipg.ipg_sssp_batch(h, sources)
        for i, s in enumerate(sources):
            want = np.full(graph.n, 0xFFFFFFFF, dtype=np.uint32)
            want[s] = 0
            np.testing.assert_array_equal(dist[i], want)
            o = oracle.sssp(graph.n, graph.offsets, graph.cols, weights, int(s))
            np.testing.assert_array_equal(dist[i], o.values)
            assert steps[i] == 1 == o.supersteps
        assert ipg.ipg_sssp_batch_info(h)["supersteps"] == 0


@pytest.mark.parametrize("k", [32, 33, 64, 256, 257])
def test_batch_line_boundaries(ipg, k):
    """Exactly full lines (32, 64, 256 sources with out-edges), one lane past a full
    line (33), and one query past the 256 lanes (257, refilled when a lane frees): every
    row and count equals the standalone run's, and the call uses the lanes it should."""
    rng = np.random.default_rng(1300 + k)
    n = 2000
    src = np.concatenate([np.arange(n), rng.integers(0, n, size=6 * n)])  # every vertex sends
    dst = rng.integers(0, n, size=src.size)
    w = rng.integers(1, 256, size=src.size).astype(np.uint32)
    g = gen.csr_from_edges(n, src, dst, weights=w)
    sources = rng.choice(n, size=k, replace=False)
    h = ipg.ipg_graph_create(g.offsets, g.cols, g.weights, g.n, g.m, True)
    import torch

    d = torch.empty(k * n, dtype=torch.int32, device="cuda")
    steps = ipg.ipg_sssp_batch_dev(h, sources, d)
    torch.cuda.synchronize()
    dist = d.cpu().numpy().view(np.uint32).reshape(k, n)
    assert ipg.ipg_sssp_batch_info(h)["lanes"] == 32 * min(8, (k + 31) // 32)
    for i in list(range(0, k, 9)) + [k - 1]:
        ref, cnt, _ = ipg.ipg_sssp(h, int(sources[i]))
        np.testing.assert_array_equal(dist[i], ref, err_msg=f"row {i}")
        assert steps[i] == cnt
    o = oracle.sssp(n, g.offsets, g.cols, g.weights, int(sources[-1]))
    np.testing.assert_array_equal(dist[-1], o.values)
    assert steps[-1] == o.supersteps
