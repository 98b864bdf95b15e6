"""The partitioned sketch (one problem split over ranks, the paper's Case 1
with no data exchange) on CPU with the gloo backend, world size 2: the block
ownership covers the output exactly once with aligned boundaries, and the
blocks each rank computes from its own part of A, assembled, are the
unsplit sketch bit for bit.  Each rank's local compute is the CPU oracle
(every column of a left sketch and every row of a right sketch is computed
independently, in index order, so splitting changes no bit)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2603_20966_gb300.partition import (block_range, column_align, left_column_ranges,
                                              right_row_ranges)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("total,parts,align", [(0, 3, 1), (1, 4, 1), (10, 3, 1), (512, 8, 64),
                                              (100, 8, 4), (7, 2, 4), (1 << 20, 5, 1),
                                              (130, 2, 64)])
def test_blocks_cover_once_with_aligned_boundaries(total, parts, align):
    rs = [block_range(total, parts, i, align) for i in range(parts)]
    assert rs[0][0] == 0 and rs[-1][1] == total
    for (a0, a1), (b0, b1) in zip(rs, rs[1:]):
        assert a1 == b0
    for a, b in rs:
        assert a <= b and a % align == 0 and (b == total or b % align == 0)
    sizes = [b - a for a, b in rs]
    assert sum(sizes) == total
    assert max(sizes) - min(sizes) <= align  # near-equal


def test_column_alignment_rule():
    assert column_align(512, 8) == 64 and column_align(512, 16) == 4
    for n, w in [(512, 2), (96, 2), (33, 3)]:
        for c0, _ in left_column_ranges(n, w):
            assert c0 % 4 == 0  # 16-byte aligned column views of a row-major matrix


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2603_20966_gb300.partition import gather_blocks
        from paper_2603_20966_gb300.workloads import gaussian_matrix
        seed, k = 7, 24
        res = {}
        for dist_id in (0, 1):
            # left: this rank's columns of A
            m, n = 300, 150
            A = gaussian_matrix(m, n, 5, device="cpu").numpy()
            c0, c1 = left_column_ranges(n, world)[rank]
            Yb = oracle.apply_left(seed, dist_id, 0, k, np.ascontiguousarray(A[:, c0:c1]),
                                   nthreads=1)
            Y = gather_blocks(torch.from_numpy(Yb), left_column_ranges(n, world), 1)
            res[("left", dist_id)] = Y.numpy()
            # right: this rank's rows of A
            m, n = 77, 40
            A = gaussian_matrix(m, n, 6, device="cpu").numpy()
            r0, r1 = right_row_ranges(m, world)[rank]
            Yb = oracle.apply_right(seed, dist_id, 0, k, np.ascontiguousarray(A[r0:r1]),
                                    nthreads=1)
            Y = gather_blocks(torch.from_numpy(Yb), right_row_ranges(m, world), 0)
            res[("right", dist_id)] = Y.numpy()
        out[rank] = res
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_partitioned_sketch_assembles_to_the_unsplit_sketch_gloo_world2(orc):
    from paper_2603_20966_gb300.workloads import gaussian_matrix
    world, port = 2, _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for dist_id in (0, 1):
        A = gaussian_matrix(300, 150, 5, device="cpu").numpy()
        ref = orc.apply_left(7, dist_id, 0, 24, A, nthreads=1)
        for r in range(world):
            assert np.array_equal(out[r][("left", dist_id)], ref)
        A = gaussian_matrix(77, 40, 6, device="cpu").numpy()
        ref = orc.apply_right(7, dist_id, 0, 24, A, nthreads=1)
        for r in range(world):
            assert np.array_equal(out[r][("right", dist_id)], ref)
