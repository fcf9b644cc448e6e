"""The multi-rank path of bench.py on CPU (gloo, world_size 2): each rank
solves its own replica, the job time is the slowest rank's and the
iterations add up; a rank that raises is reported, not hung on."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out, fail_rank):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        if rank == fail_rank:
            raise RuntimeError("injected failure on rank %d" % rank)
        elapsed = [2.0, 3.0][rank]
        iters = [40, 40][rank]
        out[rank] = bench.aggregate_over_ranks(elapsed, iters, world)
    finally:
        dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, _free_port(), out, -1), nprocs=2, start_method="spawn")
    for r in range(2):
        elapsed_max, iters, value = out[r]
        assert elapsed_max == 3.0 and iters == 80.0
        assert abs(value - 80.0 / 3.0) < 1e-12


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.aggregate_over_ranks(2.0, 40, 1) == (2.0, 40.0, 20.0)


def test_failing_rank_is_reported():
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    with pytest.raises(Exception):
        mp.start_processes(_worker, args=(2, _free_port(), out, 1), nprocs=2, start_method="spawn",
                           join=True)
