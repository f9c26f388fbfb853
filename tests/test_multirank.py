"""The multi-GPU bench's host logic on CPU ranks (gloo, world size 2): each
rank simulates its own unitary, the slowest rank's time is the job's time,
and the rate counts the work of every rank."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as td
    import bench
    import pcv_inputs as pin
    td.init_process_group("gloo", rank=rank, world_size=world)
    t = 1.0 + rank                                       # rank 1 is the slower one
    slowest = bench.max_over_ranks(t, world, torch.device("cpu"))
    U = pin.haar_unitary(6, bench.rank_unitary_seed(rank))
    gathered = [None] * world
    td.all_gather_object(gathered, U.tobytes())
    td.destroy_process_group()
    out[rank] = (slowest, gathered)


def test_two_cpu_ranks():
    import torch.multiprocessing as mp
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for r in (0, 1):
        slowest, gathered = out[r]
        assert slowest == 2.0
        assert gathered[0] != gathered[1]                # independent problems per rank
    import bench
    assert bench.whole_job_rate(100, 10, 2, 2.0) == 1000.0
