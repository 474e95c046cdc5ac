"""The multi-rank timing path of bench.py (one process per GPU, weak scaling),
run as two gloo ranks on the CPU: the job time is the slowest rank's and the
value counts every rank's windows; no collective touches the data."""
import os
import socket

import torch
import torch.distributed as dist
import torch.multiprocessing as tmp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    total_ms, value = bench.aggregate_over_ranks(10.0 * (rank + 1), windows=961, steps=4, world=world,
                                                 device=torch.device("cpu"))
    out[rank] = (total_ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    port = _free_port()
    mgr = tmp.Manager()
    out = mgr.dict()
    tmp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 20.0
    assert abs(out[0][1] - 2 * 961 * 4 / 0.020) < 1e-6


def test_single_rank_is_a_no_op():
    import bench
    assert bench.aggregate_over_ranks(5.0, 961, 2, 1) == (5.0, 961 * 2 / 0.005)
