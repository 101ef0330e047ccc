"""The multi-GPU bench path is replicas (every rank runs the whole workload on its own GPU,
no data-path collective): the job's rate is all ranks' units over the slowest rank's time.
Checked with two gloo ranks on CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms_local = [40.0, 100.0][rank]  # rank 1 is the slow replica
    rate, ms = bench.replica_throughput(1e9, ms_local, world)
    bench.barrier(world)
    out[rank] = (rate, ms, bench.all_max(float(rank), world))
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_replica_throughput_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(90)
        assert p.exitcode == 0
    for r in range(2):
        rate, ms, mx = out[r]
        assert ms == 100.0  # the slowest rank's time
        assert rate == pytest.approx(2 * 1e9 / 0.1)  # both ranks' units over it
        assert mx == 1.0


def test_single_rank_needs_no_process_group():
    import bench

    rate, ms = bench.replica_throughput(5e8, 50.0, 1)
    assert ms == 50.0 and rate == pytest.approx(1e10)
