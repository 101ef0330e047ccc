"""The seeded input generator: deterministic, independent of the thread count, and
producing simple graphs (no self-loop, no duplicate, rows sorted, symmetric when
undirected) with the R-MAT skew; the GPU build of the generator matches the CPU
build bit for bit."""
import numpy as np
import pytest

import gen


def test_rmat_is_deterministic_and_thread_independent():
    a = gen.rmat(12, 8, seed=5, weighted=True, nthreads=1)
    b = gen.rmat(12, 8, seed=5, weighted=True, nthreads=7)
    np.testing.assert_array_equal(a.offsets, b.offsets)
    np.testing.assert_array_equal(a.cols, b.cols)
    np.testing.assert_array_equal(a.weights, b.weights)
    c = gen.rmat(12, 8, seed=6)
    assert not np.array_equal(a.cols[:1000], c.cols[:1000])


@pytest.mark.parametrize("undirected", [False, True])
def test_rmat_is_simple_and_sorted(undirected):
    g = gen.rmat(11, 16, seed=2, undirected=undirected, weighted=True)
    assert g.n == 2048 and g.offsets[0] == 0 and g.offsets[-1] == g.m
    rows = np.repeat(np.arange(g.n), g.out_degree())
    assert not (rows == g.cols).any()
    key = rows.astype(np.int64) * g.n + g.cols
    assert (np.diff(key) > 0).all()  # sorted within rows and no duplicates
    assert g.weights.min() >= 1 and g.weights.max() <= 255
    if undirected:
        rev = g.cols.astype(np.int64) * g.n + rows
        assert np.array_equal(np.sort(rev), key)
        order = np.argsort(rev)
        np.testing.assert_array_equal(g.weights[order], g.weights)  # both directions carry one weight


def test_rmat_skew():
    g = gen.rmat(14, 16, seed=1)
    deg = g.out_degree()
    # quadrant a = 0.57 concentrates edges on low ids: vertex 0 is the hub
    assert gen.max_out_degree_vertex(g) == 0
    assert deg[0] > 50 * deg.mean()
    assert 0.8 * 16 * g.n < g.m < 16 * g.n


def test_csr_from_edges_keeps_multi_edges_and_loops():
    g = gen.csr_from_edges(3, [2, 0, 0, 1], [2, 1, 1, 0], [5, 6, 7, 8])
    assert list(g.offsets) == [0, 2, 3, 4]
    assert list(g.cols) == [1, 1, 0, 2]
    assert list(g.weights) == [6, 7, 8, 5]
    u = gen.csr_from_edges(3, [0], [2], undirected=True)
    assert list(u.offsets) == [0, 1, 1, 2] and list(u.cols) == [2, 0]


@pytest.mark.gpu
@pytest.mark.parametrize("scale,ef,undirected", [(8, 4, False), (12, 16, True), (16, 16, False), (14, 8, True)])
def test_gpu_generator_matches_cpu(scale, ef, undirected):
    gen.build_cuda()
    cpu = gen.rmat(scale, ef, seed=3, undirected=undirected, weighted=True)
    dev = gen.rmat_device(scale, ef, seed=3, undirected=undirected, weighted=True).to_host()
    np.testing.assert_array_equal(cpu.offsets, dev.offsets)
    np.testing.assert_array_equal(cpu.cols, dev.cols)
    np.testing.assert_array_equal(cpu.weights, dev.weights)
