"""The multi-GPU path is replicas only: every rank runs independent
trajectories and the benchmark combines ranks by the maximum time and the
summed work. Checked here with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import workloads as W
    ms, work = bench.aggregate_over_ranks(10.0 * (rank + 1), 100.0 + rank, dist)
    g = W.rng(bench.replica_seed(W.SEEDS["L102x102x64"], rank, 0))
    first = float(g.normal())
    gathered = [None] * world
    dist.all_gather_object(gathered, first)
    out[rank] = (ms, work, gathered)
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_and_draw_independent_inputs():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        ms, work, firsts = out[r]
        assert ms == 20.0          # the slowest rank's time
        assert work == 201.0       # the summed work
        assert firsts[0] != firsts[1]  # replicas draw different inputs


def test_single_process_aggregation_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_over_ranks(3.5, 7.0, None) == (3.5, 7.0)
