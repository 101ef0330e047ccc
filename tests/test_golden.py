"""Hand-worked examples under tests/golden/: small graphs whose results and per-superstep
counters were derived by hand from the superstep model (Sec. I), the combining mailbox
(Sec. III, also with wider messages: shortest-path tree, path counting) and the three
benchmarks (Sec. VI-C), each derivation written out in its fixture.  The paper prints no worked example, so these are the stored values that pin
the oracle (CPU tests) and the CUDA path (GPU tests) to something outside both."""
import glob
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import gen
import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
FIXTURES = sorted(glob.glob(os.path.join(GOLDEN, "*.json")))
STAT_FIELDS = ("superstep", "active", "senders", "messages_sent", "receivers")


def _load(path):
    with open(path) as f:
        fx = json.load(f)
    g = fx["graph"]
    offsets = np.asarray(g["offsets"], dtype=np.uint64)
    cols = np.asarray(g["cols"], dtype=np.uint32)
    weights = np.asarray(g["weights"], dtype=np.uint32) if "weights" in g else None
    return fx, offsets, cols, weights


def _cases():
    for path in FIXTURES:
        fx = json.load(open(path))
        for i in range(len(fx["cases"])):
            yield pytest.param(path, i, id="%s-%d" % (os.path.basename(path)[:-5], i))


def test_every_program_has_a_fixture():
    programs = {json.load(open(p))["program"] for p in FIXTURES}
    assert programs == {"pagerank", "hashmin", "sssp", "sssp_tree", "bfs_paths"}


@pytest.mark.parametrize("path", FIXTURES, ids=[os.path.basename(p)[:-5] for p in FIXTURES])
def test_fixture_csr_matches_its_edge_list(path):
    """The CSR written in each fixture is the one its edge list defines."""
    fx, offsets, cols, weights = _load(path)
    g = fx["graph"]
    if "undirected_edges" in g:
        e = np.asarray(g["undirected_edges"])
        ref = gen.csr_from_edges(g["n"], e[:, 0], e[:, 1], undirected=True)
    else:
        e = np.asarray(g["edges"])
        ref = gen.csr_from_edges(g["n"], e[:, 0], e[:, 1], weights=e[:, 2] if e.shape[1] > 2 else None)
    np.testing.assert_array_equal(ref.offsets, offsets)
    # rows may list their neighbours in any order; compare (row, col, weight) multisets
    row = np.repeat(np.arange(g["n"]), np.diff(offsets.astype(np.int64)))
    mine = sorted(zip(row.tolist(), cols.tolist(), (weights if weights is not None else cols * 0).tolist()))
    theirs = sorted(zip(row.tolist(), ref.cols.tolist(),
                        (ref.weights if ref.weights is not None else ref.cols * 0).tolist()))
    assert mine == theirs


def _stats_rows(stats):
    return [[getattr(s, f) for f in STAT_FIELDS] for s in stats]


def _run_oracle(fx, offsets, cols, weights, case):
    n = fx["graph"]["n"]
    if fx["program"] == "pagerank":
        return oracle.pagerank(n, offsets, cols, case["updates"])
    if fx["program"] == "hashmin":
        return oracle.hashmin(n, offsets, cols)
    if fx["program"] == "sssp_tree":
        return oracle.sssp_tree(n, offsets, cols, weights, case["source"])
    if fx["program"] == "bfs_paths":
        return oracle.bfs_paths(n, offsets, cols, case["source"])
    return oracle.sssp(n, offsets, cols, weights if case["weighted"] else None, case["source"])


@pytest.mark.parametrize("path,i", list(_cases()))
def test_oracle_reproduces_hand_worked_example(path, i):
    fx, offsets, cols, weights = _load(path)
    case = fx["cases"][i]
    r = _run_oracle(fx, offsets, cols, weights, case)
    assert r.supersteps == case["supersteps"]
    assert _stats_rows(r.stats) == case["stats"]
    if fx["program"] == "pagerank":
        want = np.array([float(Fraction(x)) for x in case["ranks"]])
        np.testing.assert_allclose(r.values, want, rtol=1e-14, atol=0)
    elif fx["program"] == "sssp_tree":
        np.testing.assert_array_equal(r.dist, np.asarray(case["dist"], dtype=np.uint32))
        np.testing.assert_array_equal(r.parent, np.asarray(case["parent"], dtype=np.uint32))
    elif fx["program"] == "bfs_paths":
        np.testing.assert_array_equal(r.level, np.asarray(case["level"], dtype=np.uint32))
        np.testing.assert_array_equal(r.paths, np.asarray(case["paths"], dtype=np.uint64))
    else:
        want = case["labels"] if fx["program"] == "hashmin" else case["dist"]
        np.testing.assert_array_equal(r.values, np.asarray(want, dtype=np.uint32))


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


@pytest.mark.gpu
@pytest.mark.parametrize("path,i", list(_cases()))
def test_cuda_path_reproduces_hand_worked_example(ipg, path, i):
    fx, offsets, cols, weights = _load(path)
    case = fx["cases"][i]
    g = fx["graph"]
    n, m = g["n"], int(offsets[-1])
    flags = ipg.IPG_STAT_RECEIVERS
    if fx["program"] == "pagerank":
        h = ipg.ipg_graph_create(offsets, cols, None, n, m, True)
        vals, count, st = ipg.ipg_pagerank(h, case["updates"], stats_flags=flags)
        want = np.array([float(Fraction(x)) for x in case["ranks"]])
        assert np.max(np.abs(vals.astype(np.float64) - want)) / np.max(want) <= 1e-5
    elif fx["program"] == "hashmin":
        h = ipg.ipg_graph_create(offsets, cols, None, n, m, False)
        vals, count, st = ipg.ipg_hashmin_cc(h, stats_flags=flags)
        np.testing.assert_array_equal(vals, np.asarray(case["labels"], dtype=np.uint32))
    elif fx["program"] == "sssp_tree":
        h = ipg.ipg_graph_create(offsets, cols, weights, n, m, True)
        dist, parent, count, st = ipg.ipg_sssp_tree(h, case["source"], stats_flags=flags)
        np.testing.assert_array_equal(dist, np.asarray(case["dist"], dtype=np.uint32))
        np.testing.assert_array_equal(parent, np.asarray(case["parent"], dtype=np.uint32))
    elif fx["program"] == "bfs_paths":
        h = ipg.ipg_graph_create(offsets, cols, None, n, m, True)
        level, paths, count, st = ipg.ipg_bfs_paths(h, case["source"], stats_flags=flags)
        np.testing.assert_array_equal(level, np.asarray(case["level"], dtype=np.uint32))
        np.testing.assert_array_equal(paths, np.asarray(case["paths"], dtype=np.uint64))
    else:
        h = ipg.ipg_graph_create(offsets, cols, weights if case["weighted"] else None, n, m, True)
        vals, count, st = ipg.ipg_sssp(h, case["source"], stats_flags=flags)
        np.testing.assert_array_equal(vals, np.asarray(case["dist"], dtype=np.uint32))
    assert count == case["supersteps"]
    assert _stats_rows(st) == case["stats"]
