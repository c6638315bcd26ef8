"""Replicas on several GPUs, host logic on CPU: two gloo ranks (127.0.0.1) each take their own
receiver batch, and the whole-job timing is the slowest rank's time over the units of all ranks."""
import os
import socket

import numpy as np

from paper_2402_13034_gb300.replicas import combine_over_ranks, rank_receivers


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        grid = np.stack([np.linspace(0.0, 1.0, 7), np.zeros(7), np.full(7, 1.2)], 1).astype(np.float32)
        mine = rank_receivers(grid, rank)
        t, u = combine_over_ranks(10.0 + 3.0 * rank, 100.0 * (rank + 1))
        x = torch.from_numpy(mine[:, 0].astype(np.float64))
        xs = [torch.zeros_like(x) for _ in range(world)]
        dist.all_gather(xs, x)
        out[rank] = (t, u, [v.numpy().tolist() for v in xs])
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_combine_timing_and_own_batches():
    import torch.multiprocessing as mp
    world = 2
    with mp.get_context("spawn").Manager() as m:      # no fork of a threaded process
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for r in range(world):
        t, u, xs = res[r]
        assert t == 13.0                         # the slowest rank's time
        assert u == 300.0                        # the units of both ranks
        a, b = np.array(xs[0]), np.array(xs[1])
        assert a.shape == b.shape == (7,)        # same batch size per rank (weak scaling)
        assert np.allclose(b - a, 1e-3, atol=1e-7) and not np.any(np.isin(a, b))


def test_single_process_returns_its_own_timing():
    assert combine_over_ranks(5.0, 42.0) == (5.0, 42.0)
    rx = np.ones((3, 3), np.float32)
    assert np.array_equal(rank_receivers(rx, 0), rx)
    assert rank_receivers(rx, 0) is not rx
