"""Host-side multi-rank logic of bench.py on CPU (gloo, world size 2): each
rank times its own independent batch; the job's throughput divides all
ranks' units by the slowest rank's time."""
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
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    r, w, local = bench.dist_setup("gloo")
    assert (r, w, local) == (rank, world, rank)
    bench.barrier(w)
    my_ms = 100.0 * (rank + 1)             # rank 1 is the slowest
    mx = bench.max_over_ranks(my_ms, w)
    out[rank] = (mx, bench.weak_scaling_value(8192, 5, w, mx))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_rank_max_time_and_weak_scaling():
    import torch.multiprocessing as mp
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for rank in (0, 1):
        mx, value = out[rank]
        assert mx == 200.0
        assert value == pytest.approx(8192 * 5 * 2 / 0.2)
