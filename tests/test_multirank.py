"""The N > 1 path of bench.py on CPU: two gloo ranks, as torchrun would
start them (RANK / WORLD_SIZE / MASTER_* in the environment).  Each rank is
an independent replica; the job's value is all ranks' units over the
slowest rank's time, and rank 0 alone reports."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    import torch.distributed as dist
    r, w, local = bench.dist_setup(world)
    assert (r, w) == (rank, world) and dist.get_backend() == "gloo"
    bench.barrier(w)
    # rank k did (k + 1) * 10 units in (k + 1) * 100 ms
    units, ms = (rank + 1) * 10, (rank + 1) * 100.0
    out[rank] = (bench.max_over_ranks(ms, w), bench.sum_over_ranks(units, w),
                 bench.replica_value(units, ms, w))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        mx, sm, val = res[rank]
        assert mx == 200.0 and sm == 30.0
        assert val == pytest.approx(30 / 0.2)


def test_single_rank_is_local():
    import bench
    assert bench.dist_setup(1) == (0, 1, 0)
    assert bench.max_over_ranks(5.0, 1) == 5.0 and bench.sum_over_ranks(3.0, 1) == 3.0
    assert bench.replica_value(10, 500.0, 1) == pytest.approx(20.0)
