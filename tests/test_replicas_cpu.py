"""Multi-rank replica bookkeeping on CPU (gloo, world size 2): disjoint seeds,
max-over-ranks time and summed work; no GPU involved."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2208_06559_gb300 import inputs, replicas
    seed = replicas.replica_seed(1237, rank)
    r = inputs.random_walk([50], seed)
    ms = 10.0 + 5.0 * rank          # rank 1 is the slow one
    units, ms_max = replicas.aggregate(ms, 64 * 10, world)
    out[rank] = (seed, float(r[-1, 0]), units, ms_max)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn")
    s0, x0, u0, m0 = out[0]
    s1, x1, u1, m1 = out[1]
    assert s0 != s1 and x0 != x1                 # different chains per rank
    assert u0 == u1 == 2 * 640                   # work summed over ranks
    assert m0 == m1 == 15.0                      # slowest rank's time
