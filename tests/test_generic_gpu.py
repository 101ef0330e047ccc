"""General combiners (Sec. III, Fig. 1) on the GPU vs the CPU oracle, through the C ABI.

Bars (all integer, all bit-exact): the shortest-path tree's distances and parents, the
shortest-path counts (modulo 2^64) and levels, superstep counts and every per-superstep
count (active, senders, messages sent, receivers); the combination step alone
(has-message flags, combined messages, receiver count) for every combine kind, with
and without warp pre-combination, under heavy contention on single mailboxes.
"""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

U64 = 1 << 64


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


@pytest.fixture(params=[0, 1], ids=["mailbox", "warp"])
def warp(request, ipg):
    """Runs a program test with and without warp pre-combination of same-destination messages."""
    old = ipg.ipg_get_tuning("combine_warp")
    ipg.ipg_set_tuning("combine_warp", request.param)
    yield request.param
    ipg.ipg_set_tuning("combine_warp", old)


def _cmp_stats(gpu_stats, gpu_count, orc):
    assert gpu_count == orc.supersteps
    assert len(gpu_stats) == len(orc.stats)
    for a, b in zip(gpu_stats, orc.stats):
        assert (a.superstep, a.senders, a.messages_sent, a.receivers, a.active) == \
               (b.superstep, b.senders, b.messages_sent, b.receivers, b.active), (a, b)


_GRAPH_WEIGHTS = object()


def check_tree(ipg, g, source, weights=_GRAPH_WEIGHTS, h=None):
    w = g.weights if weights is _GRAPH_WEIGHTS else weights
    if h is None:
        h = ipg.ipg_graph_create(g.offsets, g.cols, w, g.n, g.m, g.directed)
    dist, parent, cnt, st = ipg.ipg_sssp_tree(h, source)
    ref = oracle.sssp_tree(g.n, g.offsets, g.cols, w, source)
    np.testing.assert_array_equal(dist, ref.dist)
    np.testing.assert_array_equal(parent, ref.parent)
    _cmp_stats(st, cnt, ref)
    return h, dist, parent


def check_paths(ipg, g, source, h=None):
    if h is None:
        h = ipg.ipg_graph_create(g.offsets, g.cols, g.weights, g.n, g.m, g.directed)
    level, paths, cnt, st = ipg.ipg_bfs_paths(h, source)
    ref = oracle.bfs_paths(g.n, g.offsets, g.cols, source)
    np.testing.assert_array_equal(level, ref.level)
    np.testing.assert_array_equal(paths, ref.paths)
    _cmp_stats(st, cnt, ref)
    return h, level, paths


def _adversarial():
    yield gen.csr_from_edges(1, [], [])
    yield gen.csr_from_edges(7, [], [])
    yield gen.csr_from_edges(4, [0, 1, 1, 3], [0, 1, 1, 3])
    yield gen.csr_from_edges(6, [0, 0, 0, 2, 3, 3, 5], [1, 1, 1, 3, 4, 4, 5])
    p = 700
    yield gen.csr_from_edges(p, np.arange(p - 1), np.arange(1, p))
    leaves = 1 << 17  # one sender whose edges span many merge-path tiles
    yield gen.csr_from_edges(leaves + 1, np.zeros(leaves, dtype=np.int64), np.arange(1, leaves + 1))
    # many senders, one receiver: every message of superstep 1 goes to the same mailbox
    k = 300000
    src = np.concatenate([np.zeros(k, dtype=np.int64), np.arange(1, k + 1)])
    dst = np.concatenate([np.arange(1, k + 1), np.full(k, k + 1, dtype=np.int64)])
    yield gen.csr_from_edges(k + 2, src, dst)


def test_tree_adversarial(ipg, warp):
    for g in _adversarial():
        for s in sorted({0, g.n - 1, g.n // 2}):
            check_tree(ipg, g, s, weights=None)
            check_tree(ipg, g, s, weights=np.full(g.m, 255, dtype=np.uint32))
            check_tree(ipg, g, s, weights=np.full(g.m, 300, dtype=np.uint32))  # u32 weights


def test_paths_adversarial(ipg, warp):
    for g in _adversarial():
        for s in sorted({0, g.n - 1, g.n // 2}):
            check_paths(ipg, g, s)


@pytest.mark.parametrize("seed", range(10))
def test_random_multigraphs(ipg, seed, warp):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 3000))
    m = int(rng.integers(0, 25000))
    g = gen.random_multigraph(n, m, seed=seed, weighted=True)
    # few distinct weights: many equal-length alternatives, so parent ties are common
    w3 = rng.integers(1, 4, size=g.m).astype(np.uint32)
    for s in (0, int(rng.integers(0, n))):
        check_tree(ipg, g, s)
        check_tree(ipg, g, s, weights=w3)
        check_tree(ipg, g, s, weights=None)
        check_paths(ipg, g, s)


@pytest.mark.parametrize("scale", [6, 10, 14, 16])
def test_rmat_scales(ipg, scale, warp):
    g = gen.rmat(scale, 16, seed=scale, weighted=True)
    src = gen.max_out_degree_vertex(g)
    h, dist, _ = check_tree(ipg, g, src)
    # the tree's distances and counts are plain SSSP's
    d2, c2, st2 = ipg.ipg_sssp(h, src, stats_flags=ipg.IPG_STAT_RECEIVERS)
    np.testing.assert_array_equal(dist, d2)
    check_tree(ipg, g, src, weights=None)
    check_paths(ipg, g, src, h=h)
    u = gen.rmat(scale, 16, seed=scale, undirected=True)
    check_paths(ipg, u, gen.max_out_degree_vertex(u))


def test_paths_wrap_modulo_2_64(ipg, warp):
    # 64 diamonds in series: 2^64 paths, a count of 0 modulo 2^64 that still activates
    src, dst = [], []
    hub, nxt = 0, 1
    for _ in range(64):
        a, b, end = nxt, nxt + 1, nxt + 2
        src += [hub, hub, a, b]
        dst += [a, b, end, end]
        hub, nxt = end, end + 1
    src += [hub, hub + 1]
    dst += [hub + 1, hub + 2]
    g = gen.csr_from_edges(hub + 3, src, dst)
    _, level, paths = check_paths(ipg, g, 0)
    assert level[hub] == 128 and paths[hub] == 0 and level[hub + 2] == 130


def test_hypercube_counts_on_gpu(ipg, warp):
    d = 12
    n = 1 << d
    x = np.repeat(np.arange(n), d)
    bit = np.tile(np.arange(d), n)
    g = gen.csr_from_edges(n, x, x ^ (1 << bit))
    _, level, paths = check_paths(ipg, g, 0)
    pop = np.array([bin(v).count("1") for v in range(n)])
    import math

    np.testing.assert_array_equal(level, pop)
    np.testing.assert_array_equal(paths, [math.factorial(p) for p in pop])


def test_device_entry_points_match_host(ipg):
    import torch

    g = gen.rmat(12, 16, seed=3, weighted=True)
    h = ipg.ipg_graph_create(g.offsets, g.cols, g.weights, g.n, g.m, True)
    dist, parent, _, _ = ipg.ipg_sssp_tree(h, 5)
    d = torch.empty(g.n, dtype=torch.int32, device="cuda")
    p = torch.empty(g.n, dtype=torch.int32, device="cuda")
    ipg.ipg_sssp_tree_dev(h, 5, d, p)
    np.testing.assert_array_equal(d.cpu().numpy().view(np.uint32), dist)
    np.testing.assert_array_equal(p.cpu().numpy().view(np.uint32), parent)
    level, paths, _, _ = ipg.ipg_bfs_paths(h, 5)
    lv = torch.empty(g.n, dtype=torch.int32, device="cuda")
    pt = torch.empty(g.n, dtype=torch.int64, device="cuda")
    ipg.ipg_bfs_paths_dev(h, 5, lv, pt)
    np.testing.assert_array_equal(lv.cpu().numpy().view(np.uint32), level)
    np.testing.assert_array_equal(pt.cpu().numpy().view(np.uint64), paths)


def test_program_errors(ipg):
    g = gen.csr_from_edges(3, [0, 1], [1, 2], [0xFFFFFF00, 0xFFFFFF00])
    h = ipg.ipg_graph_create(g.offsets, g.cols, g.weights, g.n, g.m, True)
    with pytest.raises(ipg.IpgError) as e:
        ipg.ipg_sssp_tree(h, 0)
    assert e.value.status == ipg.IPG_EOVERFLOW
    for fn in (ipg.ipg_sssp_tree, ipg.ipg_bfs_paths):
        with pytest.raises(ipg.IpgError) as e:
            fn(h, 3)
        assert e.value.status == ipg.IPG_EINVAL
    # the graph is still usable after the errors
    level, paths, cnt, _ = ipg.ipg_bfs_paths(h, 0)
    np.testing.assert_array_equal(level, [0, 1, 2])
    np.testing.assert_array_equal(paths, [1, 1, 1])
    assert cnt == 3


# ---------------------------------------------------------------------------------------
# the combination step alone


KINDS = {oracle.COMBINE_XOR_U32: "xor32", oracle.COMBINE_MIN_U64: "min64", oracle.COMBINE_SUM_U64: "sum64",
         oracle.COMBINE_MINCOUNT_U128: "mincount128"}


def _messages(kind, n, k, seed, hot=0.0):
    rng = np.random.default_rng(seed)
    dst = rng.integers(0, n, size=k).astype(np.uint32)
    if hot:  # a fraction of all messages to vertex 0 and a few more hubs
        sel = rng.random(k) < hot
        dst[sel] = rng.integers(0, min(n, 4), size=int(sel.sum()))
    if kind == oracle.COMBINE_XOR_U32:
        msgs = rng.integers(0, 1 << 32, size=k, dtype=np.uint64).astype(np.uint32)
    elif kind == oracle.COMBINE_MINCOUNT_U128:
        msgs = np.stack([rng.integers(0, 3, size=k, dtype=np.uint64),
                         rng.integers(0, U64, size=k, dtype=np.uint64)], axis=1)
    else:
        msgs = rng.integers(0, U64, size=k, dtype=np.uint64)
    return dst, msgs


def _gpu_combine(ipg, kind, n, dst, msgs, options=0):
    import torch

    dt = torch.int32 if kind == oracle.COMBINE_XOR_U32 else torch.int64
    d = torch.from_numpy(dst.view(np.int32)).cuda()
    m = torch.from_numpy(msgs.view(np.int32 if dt == torch.int32 else np.int64)).cuda()
    shape = (max(n, 1), 2) if kind == oracle.COMBINE_MINCOUNT_U128 else (max(n, 1),)
    flags = torch.full((max(n, 1),), 7, dtype=torch.int32, device="cuda")  # the call must clear them
    mail = torch.zeros(shape, dtype=dt, device="cuda")
    r = ipg.ipg_combine_dev(kind, n, d, m, flags, mail, options)
    npdt = np.uint32 if dt == torch.int32 else np.uint64
    return r, flags.cpu().numpy()[:n], mail.cpu().numpy().view(npdt)[:n]


@pytest.mark.parametrize("kind", list(KINDS), ids=list(KINDS.values()))
@pytest.mark.parametrize("options", [0, 1], ids=["mailbox", "warp"])
@pytest.mark.parametrize("n,k,hot", [(1, 1, 0.0), (1, 100000, 0.0), (1000, 200000, 0.0), (100000, 1 << 20, 0.5),
                                     (1 << 20, 1 << 20, 0.0), (33, 77777, 0.9)])
def test_combine_matches_oracle(ipg, kind, options, n, k, hot):
    dst, msgs = _messages(kind, n, k, seed=n + k + kind, hot=hot)
    ref = oracle.combine(kind, n, dst, msgs)
    r, flags, mail = _gpu_combine(ipg, kind, n, dst, msgs, options)
    assert r == ref.receivers
    np.testing.assert_array_equal(flags.astype(bool), ref.has)
    assert set(np.unique(flags)) <= {0, 1}
    np.testing.assert_array_equal(mail[ref.has], ref.mail[ref.has])


@pytest.mark.parametrize("options", [2, 3], ids=["native", "native+warp"])
def test_native_min_matches(ipg, options):
    dst, msgs = _messages(oracle.COMBINE_MIN_U64, 5000, 1 << 20, seed=5, hot=0.3)
    ref = oracle.combine(oracle.COMBINE_MIN_U64, 5000, dst, msgs)
    r, flags, mail = _gpu_combine(ipg, oracle.COMBINE_MIN_U64, 5000, dst, msgs, options)
    assert r == ref.receivers
    np.testing.assert_array_equal(flags.astype(bool), ref.has)
    np.testing.assert_array_equal(mail[ref.has], ref.mail[ref.has])


def test_combine_neutral_results_are_messages(ipg):
    # x xor x = 0 and x + (2^64 - x) = 0: the flags still say "received"
    r, flags, mail = _gpu_combine(ipg, oracle.COMBINE_XOR_U32, 4, np.array([1, 1, 3], np.uint32),
                                  np.array([0xDEADBEEF, 0xDEADBEEF, 0], np.uint32))
    assert r == 2 and list(flags) == [0, 1, 0, 1] and mail[1] == 0 and mail[3] == 0
    x = 0x123456789ABCDEF1
    k = 4096  # many copies of +x and -x to one vertex, from many warps at once
    msgs = np.array([x, U64 - x] * (k // 2), dtype=np.uint64)
    for options in (0, 1):
        r, flags, mail = _gpu_combine(ipg, oracle.COMBINE_SUM_U64, 2, np.ones(k, np.uint32), msgs, options)
        assert r == 1 and list(flags) == [0, 1] and mail[1] == 0


def test_combine_errors(ipg):
    import torch

    n = 10
    flags = torch.zeros(n, dtype=torch.int32, device="cuda")
    mail = torch.zeros(n, dtype=torch.int64, device="cuda")
    d = torch.tensor([1, 10, 2], dtype=torch.int32, device="cuda")  # 10 >= n
    m = torch.tensor([5, 6, 7], dtype=torch.int64, device="cuda")
    with pytest.raises(ipg.IpgError) as e:
        ipg.ipg_combine_dev(oracle.COMBINE_MIN_U64, n, d, m, flags, mail)
    assert e.value.status == ipg.IPG_EINVAL
    with pytest.raises(ipg.IpgError):
        ipg.ipg_combine_dev(oracle.COMBINE_SUM_U64, n, d[:1], m[:1], flags, mail, ipg.IPG_COMBINE_NATIVE)
    with pytest.raises(ipg.IpgError):
        ipg.ipg_combine_dev(9, n, d[:1], m[:1], flags, mail)
    # k = 0: every flag cleared, no receiver
    flags.fill_(3)
    assert ipg.ipg_combine_dev(oracle.COMBINE_MIN_U64, n, d[:0], m[:0], flags, mail) == 0
    assert int(flags.sum()) == 0


@pytest.mark.parametrize("kind", list(KINDS), ids=list(KINDS.values()))
@pytest.mark.parametrize("options", [0, 1], ids=["mailbox", "warp"])
def test_combiner_bounded_wait_runs_out(ipg, kind, options):
    """Every mailbox starts CLAIMED by a first sender that never publishes (the state a
    stalled writer leaves): each send's bounded wait must run out, the device raises its
    timeout status and the call returns IPG_ETIMEOUT promptly, delivering nothing; the
    library stays usable afterwards."""
    import time

    import torch

    n, k = 1000, 1 << 16
    dst, msgs = _messages(kind, n, k, seed=11, hot=0.2)
    dt = torch.int32 if kind == oracle.COMBINE_XOR_U32 else torch.int64
    d = torch.from_numpy(dst.view(np.int32)).cuda()
    m = torch.from_numpy(msgs.view(np.int32 if dt == torch.int32 else np.int64)).cuda()
    shape = (n, 2) if kind == oracle.COMBINE_MINCOUNT_U128 else (n,)
    flags = torch.zeros(n, dtype=torch.int32, device="cuda")
    mail = torch.full(shape, 5, dtype=dt, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with pytest.raises(ipg.IpgError) as e:
        ipg.ipg_combine_dev(kind, n, d, m, flags, mail, options | ipg.IPG_COMBINE_STALLED)
    elapsed = time.perf_counter() - t0
    assert e.value.status == ipg.IPG_ETIMEOUT and "bounded wait" in str(e.value)
    assert elapsed < 5.0, elapsed
    assert (flags.cpu().numpy() == 2).all()  # still CLAIMED: nothing was published
    assert (mail.cpu().numpy() == 5).all()   # no slot was written
    # the same messages on ordinary empty mailboxes still combine exactly
    ref = oracle.combine(kind, n, dst, msgs)
    r, fl, ml = _gpu_combine(ipg, kind, n, dst, msgs, options)
    assert r == ref.receivers
    np.testing.assert_array_equal(ml[ref.has], ref.mail[ref.has])
    m64 = torch.zeros(k, dtype=torch.int64, device="cuda")
    mail64 = torch.zeros(n, dtype=torch.int64, device="cuda")
    with pytest.raises(ipg.IpgError) as e:  # the hardware atomic has no wait to run out
        ipg.ipg_combine_dev(oracle.COMBINE_MIN_U64, n, d, m64, flags, mail64,
                            ipg.IPG_COMBINE_NATIVE | ipg.IPG_COMBINE_STALLED)
    assert e.value.status == ipg.IPG_EINVAL
