"""CPU test of the multi-rank reduction of bench.py: independent replicas (one per GPU in a
real run) report the slowest rank's time and the sum of all ranks' units. Two gloo ranks on
127.0.0.1 stand in for two GPUs."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    mx, sm = bench.combine_ranks([10.0 + rank, 1.0], [100.0 * (rank + 1), 0.5, 3.0], world, "cpu")
    out[rank] = (mx, sm)
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_take_max_time_and_sum_units():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    for r in range(world):
        mx, sm = out[r]
        assert mx == [11.0, 1.0]
        assert sm == [300.0, 1.0, 6.0]


def test_single_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks([2.0], [5.0], 1, "cpu") == ([2.0], [5.0])
