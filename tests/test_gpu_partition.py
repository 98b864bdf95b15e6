"""The partitioned sketch's per-rank work on one GPU: the ranks of a split
problem run one after the other (each on its own block of A, as on its own
GPU; nothing waits on another rank), and the blocks of Y they write, views
of one row-major Y, make up the unsplit sketch within the tolerance of each
form against the oracle."""
import numpy as np
import pytest
import torch

from gpu_util import rel_frob, require_gpu

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def P():
    require_gpu()
    import paper_2603_20966_gb300 as P
    return P


@pytest.mark.parametrize("form", [0, 1])  # FP32, BF16 split-A
@pytest.mark.parametrize("world", [2, 3, 8])
def test_left_split_by_columns(P, orc, form, world):
    from paper_2603_20966_gb300.partition import PartitionedSketch
    from paper_2603_20966_gb300.workloads import gaussian_matrix
    m, n, k, seed = 20000, 520, 256, 9
    A_cpu = gaussian_matrix(m, n, 41, device="cpu")
    A = A_cpu.cuda()
    Y = torch.full((k, n), float("nan"), dtype=torch.float32, device="cuda")
    for r in range(world):
        with PartitionedSketch(seed, 0, k, world, r, precision=form) as ps:
            c0, c1 = ps.left_columns(n)
            ps.left(A[:, c0:c1], Y[:, c0:c1])
            assert P.sk_stream_status(ps.handle) == 0
    ref = orc.apply_left(seed, 0, form, k, A_cpu.numpy())
    got = Y.cpu().numpy()
    assert np.all(np.isfinite(got))
    assert rel_frob(got, ref) <= TOL


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("world", [2, 5])
def test_right_split_by_rows(P, orc, form, world):
    from paper_2603_20966_gb300.partition import PartitionedSketch
    from paper_2603_20966_gb300.workloads import gaussian_matrix
    m, n, k, seed = 3001, 700, 96, 4
    A_cpu = gaussian_matrix(m, n, 42, device="cpu")
    A = A_cpu.cuda()
    Y = torch.full((m, k), float("nan"), dtype=torch.float32, device="cuda")
    for r in range(world):
        with PartitionedSketch(seed, 1, k, world, r, precision=form) as ps:
            r0, r1 = ps.right_rows(m)
            ps.right(A[r0:r1], Y[r0:r1])
            assert P.sk_stream_status(ps.handle) == 0
    ref = orc.apply_right(seed, 1, form, k, A_cpu.numpy())
    got = Y.cpu().numpy()
    assert np.all(np.isfinite(got))
    assert rel_frob(got, ref) <= TOL
