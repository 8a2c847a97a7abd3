"""Multi-GPU replicas (independent SFTs per rank, no data-path collective): the bench's host-side
aggregation over ranks, run as world_size-2 gloo process groups on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, elapsed, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, value = bench.aggregate_ranks(elapsed[rank], 40, world)
    out[rank] = (ms, value)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("elapsed", [(100.0, 250.0), (80.0, 20.0)])
def test_aggregate_takes_slowest_rank_and_sums_work(elapsed):
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, elapsed, out), nprocs=world, join=True,
                       start_method="spawn")
    slow = max(elapsed)
    for r in range(world):
        ms, value = out[r]
        assert ms == slow
        assert value == pytest.approx(40 * world / (slow / 1e3))


def test_single_rank_needs_no_process_group():
    import bench
    ms, value = bench.aggregate_ranks(50.0, 10, 1)
    assert ms == 50.0 and value == pytest.approx(200.0)
