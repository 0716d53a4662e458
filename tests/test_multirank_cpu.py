"""The multi-GPU form is replicas only (one independent graph per rank, no
data-path collective).  Its host logic -- distinct replica seeds, a barrier,
and the max over ranks of the step time -- runs here as two gloo ranks on
CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.barrier()
    ms = bench.max_over_ranks(1.0 + rank, dist)         # rank r "took" 1 + r ms
    seed = bench.replica_seed(rank)
    seeds = [None] * world
    dist.all_gather_object(seeds, seed)
    out[rank] = (ms, len(set(seeds)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_distinct_replicas():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()   # no fork of a multi-threaded test process
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        ms, distinct = out[r]
        assert ms == pytest.approx(2.0)     # every rank reports the slowest rank's time
        assert distinct == world             # every rank ran its own graph


def test_single_process_is_identity():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.max_over_ranks(3.5, None) == 3.5
