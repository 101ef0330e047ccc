"""bench.py's contract on the host, without a GPU: the reference arm (the oracle on the
host cores, a bounded sample of the workload) prints one JSON line with the keys the
bench contract names; under several ranks only rank 0 prints; our arm fails loudly
instead of falling back to the CPU when no GPU is present."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(args, env_extra=None, timeout=300):
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", **(env_extra or {}))
    return subprocess.run([sys.executable, "bench.py"] + args, cwd=ROOT, env=env, capture_output=True, text=True,
                          timeout=timeout)


SMALL = ["--scale", "12", "--edge-factor", "8", "--steps", "2", "--warmup", "3"]


def test_reference_arm_prints_the_contract_line():
    r = _bench(["--impl", "reference"] + SMALL)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["config"]["n"] == 1 << 12 and "rmat12-ef8" in d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_without_work():
    r = _bench(["--impl", "reference"] + SMALL, env_extra={"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


def test_our_arm_fails_loudly_without_a_gpu():
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    r = _bench(["--steps", "1", "--warmup", "3", "--scale", "10", "--edge-factor", "4", "--e2e-steps", "0",
                "--no-cpu-baseline"])
    assert r.returncode != 0
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


def test_cpu_parallel_baseline_entry():
    """The bench's OpenMP baseline entry on a small graph: a positive rate, the threads used,
    and a description of the sample; errors would come back as an `unavailable` entry."""
    sys.path.insert(0, ROOT)
    import bench
    import gen

    g = gen.rmat(12, 8, seed=3, weighted=True)
    d = bench.cpu_parallel_baseline(g, int(gen.max_out_degree_vertex(g)), 0.2)
    assert "unavailable" not in d, d
    assert d["value"] > 0 and d["cores"] >= 1 and d["unit"] == "GTEPS" and "OpenMP" in d["kind"]
    assert "source rows" in d["sample"]


@pytest.mark.parametrize("pagerank", [True, False])
def test_cpu_parallel_whole_graph_entry(pagerank):
    sys.path.insert(0, ROOT)
    import bench
    import gen

    g = gen.rmat(12, 8, seed=4, undirected=not pagerank)
    d = bench.cpu_parallel_whole(g, pagerank)
    assert "unavailable" not in d, d
    assert d["value"] > 0 and d["cores"] >= 1 and "whole graph" in d["sample"]
