"""The multi-rank path of bench.py on CPU: two gloo ranks (replicas, no data-path collective).

Each rank runs its own replica; the only collective is the maximum of the timings, and the
whole-job rate is world x units per rank / max time.  Runs here without a GPU.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as td  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    td.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [7.5, 3.25][rank]                      # each replica's own step time
    m = bench.max_over_ranks(ms)
    rate = bench.job_throughput(1000, world, m)
    out[rank] = (m, rate)
    td.barrier()
    td.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time():
    world, port = 2, _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    assert out[0] == out[1] == (7.5, 2 * 1000 / 7.5e-3)


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(4.0) == 4.0
    assert bench.job_throughput(10, 1, 2.0) == 5000.0
