"""Host logic of the multi-GPU replicas: max-over-ranks step time with gloo, 2 ranks."""
import os

import pytest
import torch.multiprocessing as mp


def _worker(rank, world, port, out):
    import torch.distributed as dist

    from paper_1908_05218_gb300 import replicas
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 100.0 + 25.0 * rank
    t = replicas.slowest(ms, dist, device="cpu")
    out[rank] = t
    dist.barrier()
    dist.destroy_process_group()


def test_slowest_replica_time_two_ranks():
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    assert out[0] == out[1] == 125.0


def test_throughput_counts_all_replicas():
    from paper_1908_05218_gb300 import replicas
    assert replicas.slowest(42.0) == 42.0
    assert replicas.throughput(2e9, 4, 1000.0) == pytest.approx(8.0)
