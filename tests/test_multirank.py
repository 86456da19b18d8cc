"""The N-GPU bench path without GPUs: world_size-2 ranks over gloo on the CPU.

bench.py runs independent replicas (one mesh batch per rank, no collective on
the data path) and reduces only its result: the time is the maximum over the
ranks and the units are summed.  These tests run that reduction, and the
reference arm's rank rule (rank 0 alone works), in two processes.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, results):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import sys

        sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
        import bench

        ws, r, local = bench.dist_env()
        ms, units = bench.aggregate_over_ranks(10.0 + 5.0 * rank, 1000 * (rank + 1), torch.device("cpu"))
        results[rank] = (ws, r, local, ms, units, bench.reference_rank_works(r))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_ranks_reduce_time_by_max_and_units_by_sum():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        results = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, results), nprocs=world, join=True)
        res = dict(results)
    assert sorted(res) == [0, 1]
    for rank, (ws, r, local, ms, units, works) in res.items():
        assert (ws, r, local) == (2, rank, rank)
        assert ms == 15.0  # the slowest rank's time
        assert units == 3000.0  # every rank's units
        assert works == (rank == 0)  # the reference arm runs on rank 0 only
