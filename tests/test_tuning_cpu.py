"""Tuning knobs and the autotuner's argument checks: host-side only, no GPU call."""
import ctypes

import pytest


@pytest.fixture(scope="module")
def ipg():
    import paper_2010_01542_gb300 as ipg
    from paper_2010_01542_gb300 import _build

    _build.build()
    ipg.load_library()
    return ipg


KNOBS = {
    "pull_divisor": ([0, 1, 6, 1 << 40], [-1]),
    "combine_warp": ([0, 1], [2, -1]),
    "pr_engine": ([0, 1], [2, -1]),
    "pr_threads": ([256, 512], [128, 1024, 0]),
    "pr_carveout": ([-1, 0, 50, 100], [-2, 101]),
    "batch_divisor": ([0, 1, 6, 1 << 40], [-1]),
    "push_loop": ([0, 1], [2, -1]),
    "pull_filter": ([0, 60, 100], [-1, 101]),
    "batch_chunk": ([32, 128, 256, 1024, 65536], [0, 16, 100, 65568]),
    "batch_loop": ([0, 1], [2, -1]),
    "batch_wide_chunk": ([32, 512, 1024, 65536], [0, 16, 100, 65568]),
    "batch_tile_tasks": ([0, 3, 64], [-1, 65]),
}


@pytest.mark.parametrize("name", sorted(KNOBS))
def test_knob_set_get_and_reject(ipg, name):
    good, bad = KNOBS[name]
    old = ipg.ipg_get_tuning(name)
    try:
        for v in good:
            ipg.ipg_set_tuning(name, v)
            assert ipg.ipg_get_tuning(name) == v
        for v in bad:
            with pytest.raises(ipg.IpgError):
                ipg.ipg_set_tuning(name, v)
            assert ipg.ipg_get_tuning(name) == good[-1]  # a rejected value changes nothing
    finally:
        ipg.ipg_set_tuning(name, old)


def test_unknown_knob(ipg):
    with pytest.raises(ipg.IpgError):
        ipg.ipg_set_tuning("no_such_knob", 1)
    with pytest.raises(ipg.IpgError):
        ipg.ipg_get_tuning("no_such_knob")


def test_autotune_null_graph(ipg):
    lib = ipg.load_library()
    lib.ipg_autotune.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p]
    lib.ipg_autotune.restype = ctypes.c_int
    assert lib.ipg_autotune(None, ipg.IPG_TUNE_PAGERANK, 0, None, None) == 1  # IPG_EINVAL
    assert "NULL" in ipg.ipg_last_error()
