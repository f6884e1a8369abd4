"""The N > 1 bench path (independent replicas, max-over-ranks time, summed converged
eigenpairs) with world_size 2 on the gloo backend, CPU only."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, conv = bench.combine_ranks(dist, 100.0 + 50.0 * rank, 206 + rank, "cpu")
    out[rank] = (ms, conv)
    dist.destroy_process_group()


def test_two_ranks_gloo():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    assert out[0] == (150.0, 413) and out[1] == (150.0, 413)
