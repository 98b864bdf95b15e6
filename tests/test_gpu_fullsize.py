"""Full-size accuracy of the tensor-core sketches on every output entry, where
the CPU oracle would take hours: the reference is an FP64 product on the GPU
(cuBLAS DGEMM through torch) of A with S materialized by the library in
chunks.  sk_materialize is itself pinned bit-exact against the oracle
(test_gpu_generator.py), and these references are cross-checked against the
CPU oracle on sampled rows / columns in test_gpu_tc.py."""
import numpy as np
import pytest
import torch

from gpu_util import require_gpu

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def P():
    require_gpu()
    import paper_2603_20966_gb300 as P
    return P


def _materialize(P, h, r0, c0, rows, cols, fmt):
    out = torch.empty((rows, cols), dtype=torch.bfloat16 if fmt == 1 else torch.float32,
                      device="cuda")
    P.sk_materialize(h, r0, c0, rows, cols, fmt, 0, out, cols)
    return out.double()


def _rel(got, ref):
    return (torch.linalg.norm(got.double() - ref) / torch.linalg.norm(ref)).item()


@pytest.mark.parametrize("dist", [1, 0])
def test_c2_left_full_size(P, dist):
    from paper_2603_20966_gb300.workloads import gaussian_matrix
    m, n, k = 1 << 20, 512, 2048
    A = gaussian_matrix(m, n, 1, device="cuda")
    h = P.sk_create(7, dist, k)
    P.sk_set_precision(h, 1)
    Y = torch.empty((k, n), device="cuda")
    try:
        P.sk_apply_left(h, A, m, n, n, Y, n)
        assert P.sk_stream_status(h) == 0
        ref = torch.zeros((k, n), dtype=torch.float64, device="cuda")
        s = P.sk_get_info(h)["scale"]
        step = 1 << 16
        for r0 in range(0, m, step):  # S[:, r0:r0+step] @ A[r0:r0+step]
            S = _materialize(P, h, 0, r0, k, step, 1)
            ref += S @ A[r0:r0 + step].double()
        ref *= s
        err = _rel(Y, ref)
        print(f"C2 full size, dist {dist}: relative Frobenius error {err:.3e}")
        assert err <= TOL
    finally:
        P.sk_destroy(h)


def test_c3_right_full_size(P):
    from paper_2603_20966_gb300.workloads import lowrank_plus_noise
    m, n, k = 65536, 16384, 256
    A = lowrank_plus_noise(m, n, device="cuda")
    h = P.sk_create(7, 0, k)
    P.sk_set_precision(h, 1)
    Y = torch.empty((m, k), device="cuda")
    try:
        P.sk_apply_right(h, A, m, n, n, Y, k)
        assert P.sk_stream_status(h) == 0
        s = P.sk_get_info(h)["scale"]
        S = _materialize(P, h, 0, 0, k, n, 1)  # 256 x 16384 values, exact in FP64
        ref = torch.empty((m, k), dtype=torch.float64, device="cuda")
        step = 8192
        for r0 in range(0, m, step):
            ref[r0:r0 + step] = A[r0:r0 + step].double() @ S.T
        ref *= s
        err = _rel(Y, ref)
        print(f"C3 full size: relative Frobenius error {err:.3e}")
        assert err <= TOL
    finally:
        P.sk_destroy(h)
