"""Multi-GPU is replicas only: every rank solves its own source set and the
job's value is all ranks' solves over the slowest rank's time.  The
rank-side logic runs here as two gloo processes on the CPU."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    nv = 1025 * 1025
    src = bench.rank_sources(rank, nv, np.array([123], np.int32))
    local_ms = 100.0 + 50.0 * rank          # the second replica is slower
    slow = bench.max_over_ranks(local_ms, dist)
    value = bench.whole_job_value(world, 2, 5, slow)
    out[rank] = (int(src[0]), slow, value)
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_two_ranks():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    (s0, t0, v0), (s1, t1, v1) = out[0], out[1]
    assert s0 == 123 and s1 != 123                      # each rank its own query
    assert t0 == t1 == 150.0                            # max over ranks
    assert v0 == v1 == pytest.approx(2 * 2 * 5 / 0.150)  # whole-job solves/s
