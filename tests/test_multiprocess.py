"""The N > 1 host logic of bench.py on CPU ranks (gloo, world size 2): every
rank searches its own stack (weak scaling), the job's time is the slowest
rank's, and its throughput is all ranks' work over that time.  No GPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench._dist()
    ms_local = [120.0, 150.0][rank]  # rank 1 is the slow one
    ms = bench.reduce_max(ms_local, dist)
    units = 1000.0
    out[rank] = (ws, r, local, ms, bench.job_throughput(units, ws, ms * 1e-3))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_weak_scaling_max_time():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        ws, r, local, ms, value = res[rank]
        assert ws == 2 and r == rank and local == rank
        assert ms == 150.0
        assert value == pytest.approx(2 * 1000.0 / 0.150)


def test_single_process_is_identity():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.reduce_max(3.5) == 3.5
    assert bench.job_throughput(10.0, 1, 2.0) == 5.0
