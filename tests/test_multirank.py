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


# --------------------------------------------------------------------------- #
# window partition: row bands, concatenated results, summed dL/dw
# --------------------------------------------------------------------------- #
def test_row_bands_cover_the_grid_once():
    from paper_1612_04787_gb300 import shard
    for n_rows in (0, 1, 5, 31):
        for world in (1, 2, 3, 4, 8):
            b = shard.row_bands(n_rows, world)
            assert len(b) == world and b[0][0] == 0 and b[-1][1] == n_rows
            assert all(b[i][1] == b[i + 1][0] for i in range(world - 1))
            sizes = [s - a for a, s in b]
            assert max(sizes) - min(sizes) <= 1


def _grid_case():
    """A 5 x 4 grid of 32 x 32 windows on a 256 x 256 EM-like pair, moving
    windows resampled under one affine warp, with the oracle as each rank's
    compute (result records and dL/dw)."""
    import numpy as np

    import synth
    from oracle import swim
    a, b = synth.em_section_pair(256, seed_content=3, seed_warp=4, seed_noise=(5, 6))
    rows, cols, n = 5, 4, 32
    org = np.array([(32 * i + 8, 32 * j + 8) for i in range(rows) for j in range(cols)], np.int32)
    lv = swim.Level(n, 0.5, swim.APOD_HANN, 1.0, 2.0)
    theta = np.array([1.0, 0.0, 0.3, 0.0, 1.0, -0.2])
    return a, b, rows, cols, n, org, lv, theta


def _compute(a, b, org, n, lv, theta):
    """Per-window results as [b, 8] int32 records and the summed dL/dw."""
    import numpy as np

    from oracle import swim
    recs = np.zeros((len(org), 8), np.int32)
    f = recs.view(np.float32)
    gw = 0.0
    for i, o in enumerate(org):
        ref_w = swim.gather(a, o, n).astype(np.float64)
        r = swim.match_pair(swim.resample(b.astype(np.float64), o, n, theta), ref_w, lv)
        recs[i, 0], recs[i, 1], recs[i, 6] = r["dy"], r["dx"], r["status"]
        f[i, 2], f[i, 3], f[i, 4], f[i, 5] = r["sy"], r["sx"], r["snr"], r["peak"]
        gw += swim.match_backward(b.astype(np.float64), o, theta, ref_w, lv, 1.0, 0.5)[2]
    return recs, gw


def _shard_rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1612_04787_gb300 import shard
    a, b, rows, cols, n, org, lv, theta = _grid_case()
    mine = shard.shard_rows(org, rows, cols, rank, world)
    recs, gw = _compute(a, b, mine, n, lv, theta)
    full = shard.gather_results(torch.from_numpy(recs))
    g = shard.allreduce_grad_w(torch.tensor([gw], dtype=torch.float64))
    out[rank] = (full.numpy().tobytes(), float(g[0]), len(mine))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_partition_equals_one_rank():
    """World size 2 on gloo: rank 0 takes grid rows 0-2, rank 1 rows 3-4; the
    concatenated records equal a single rank's, byte for byte, and the summed
    dL/dw equals the single rank's sum."""
    import numpy as np
    world = 2
    port = _free_port()
    mgr = tmp.Manager()
    out = mgr.dict()
    tmp.spawn(_shard_rank, args=(world, port, out), nprocs=world, join=True)
    a, b, rows, cols, n, org, lv, theta = _grid_case()
    recs, gw = _compute(a, b, org, n, lv, theta)
    assert out[0][2] == 12 and out[1][2] == 8
    for r in range(world):
        assert out[r][0] == recs.tobytes()
        assert abs(out[r][1] - gw) <= 1e-12 * max(1.0, abs(gw))
    assert (np.frombuffer(out[0][0], np.int32).reshape(-1, 8)[:, 6] == 0).all()
