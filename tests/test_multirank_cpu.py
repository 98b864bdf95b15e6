"""The multi-rank logic of bench.py on CPU with the gloo backend (world size
2): the step time is the maximum over ranks, and each rank's units add up to
the whole-job value (independent problems per rank, weak scaling)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        local_ms = 10.0 + 5.0 * rank        # rank 1 is the slower one
        ms = bench.max_over_ranks(local_ms)
        units_per_rank = 3.0
        value = world * units_per_rank / (ms * 1e-3)
        out[rank] = (ms, value)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    world, port = 2, _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert out[0][0] == pytest.approx(15.0) and out[1][0] == pytest.approx(15.0)
    assert out[0][1] == pytest.approx(2 * 3.0 / 0.015)


def test_max_over_ranks_single_process():
    import bench
    assert bench.max_over_ranks(7.5) == 7.5
