"""Host-side logic of the multi-GPU benchmark path, on CPU with two gloo
ranks: every rank gets the slowest rank's time, and the whole-job value is
the sum of all ranks' point-steps over that time (weak scaling: each rank
advances its own independent pulses; there is no data-path collective)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [120.0, 150.0][rank]
    t = bench.reduce_max(local_ms, dist, "cpu")
    v = bench.weak_scaling_value(world, 1000, 10, t)
    out[rank] = (t, v)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_weak_scaling_value():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert out[0][0] == 150.0 and out[1][0] == 150.0
    assert out[0][1] == pytest.approx(2 * 1000 * 10 / 0.150)


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_max(3.5, None, "cpu") == 3.5
    assert bench.weak_scaling_value(1, 100, 4, 1000.0) == pytest.approx(400.0)
