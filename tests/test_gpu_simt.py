"""GPU parity of the FP32 CUDA-core fused sketch (sk_set_precision(SK_FP32))
against the FP64 CPU oracle: relative Frobenius error <= 1e-5 on Y, at small
ragged shapes spanning several tiles and split-K ranges, and at the full
4096 x 256, k = 64 Gaussian workload; special inputs (identity) are exact."""
import numpy as np
import pytest
import torch

from gpu_util import rel_frob, require_gpu

pytestmark = pytest.mark.gpu

G, R, U = 0, 1, 2
TOL = 1e-5  # relative Frobenius error bound for FP32 forms vs the FP64 oracle


@pytest.fixture(scope="module")
def P():
    require_gpu()
    import paper_2603_20966_gb300 as P
    return P


def _A(m, n, seed):
    from paper_2603_20966_gb300.workloads import gaussian_matrix
    return gaussian_matrix(m, n, seed, device="cpu")


def run(P, side, seed, dist, k, A_cpu, prec=0, lda=None, ldy=None):
    m, n = A_cpu.shape
    lda = lda or n
    A = torch.zeros((m, lda), dtype=torch.float32, device="cuda")
    A[:, :n] = A_cpu.cuda()
    yr, yc = (k, n) if side == "left" else (m, k)
    ldy = ldy or yc
    Y = torch.full((yr, ldy), float("nan"), dtype=torch.float32, device="cuda")
    h = P.sk_create(seed, dist, k)
    try:
        P.sk_set_precision(h, prec)
        fn = P.sk_apply_left if side == "left" else P.sk_apply_right
        fn(h, A, m, n, lda, Y, ldy)
        assert P.sk_stream_status(h) == 0
    finally:
        P.sk_destroy(h)
    return Y[:, :yc].cpu().numpy()


SHAPES = [(1, 1, 1), (3, 5, 7), (64, 4096, 256), (130, 1000, 129), (257, 333, 31),
          (64, 100000, 40), (5, 70000, 3)]


@pytest.mark.parametrize("dist", [G, R])
@pytest.mark.parametrize("k,m,n", SHAPES)
def test_left_fp32_matches_oracle(P, orc, dist, k, m, n):
    A = _A(m, n, k + m + n)
    got = run(P, "left", 7, dist, k, A)
    ref = orc.apply_left(7, dist, 0, k, A.numpy())
    assert np.all(np.isfinite(got))
    assert rel_frob(got, ref) <= TOL


@pytest.mark.parametrize("dist", [G, R, U])
@pytest.mark.parametrize("k,m,n", [(1, 1, 1), (7, 3, 5), (256, 300, 1000), (129, 1025, 257),
                                   (31, 17, 70000)])
def test_right_fp32_matches_oracle(P, orc, dist, k, m, n):
    A = _A(m, n, 3 * k + m + n)
    got = run(P, "right", 11, dist, k, A)
    ref = orc.apply_right(11, dist, 0, k, A.numpy())
    assert rel_frob(got, ref) <= TOL


def test_config1_full_size(P, orc):
    # left sketch, A 4096 x 256 ~ N(0,1) (seed 1), S 64 x 4096 Gaussian (seed 7)
    A = _A(4096, 256, 1)
    got = run(P, "left", 7, G, 64, A)
    ref = orc.apply_left(7, G, 0, 64, A.numpy())
    err = rel_frob(got, ref)
    assert err <= TOL, err


def test_leading_dimensions(P, orc):
    A = _A(300, 50, 5)
    got = run(P, "left", 3, G, 20, A, lda=64, ldy=77)
    assert rel_frob(got, orc.apply_left(3, G, 0, 20, A.numpy())) <= TOL
    got = run(P, "right", 3, G, 20, A, lda=51, ldy=21)
    assert rel_frob(got, orc.apply_right(3, G, 0, 20, A.numpy())) <= TOL


def test_identity_gives_scaled_matrix_exactly(P, orc):
    m, k = 512, 96
    got = run(P, "left", 13, G, k, torch.eye(m))
    ref = orc.generate(13, G, 0, 0, 0, k, m) * orc.scale(k)
    np.testing.assert_array_equal(got, ref.astype(np.float32))


def test_deterministic_and_host_entry_point(P):
    A = _A(5000, 70, 2)
    a = run(P, "left", 5, G, 33, A)
    b = run(P, "left", 5, G, 33, A)
    np.testing.assert_array_equal(a, b)
    h = P.sk_create(5, G, 33)
    try:
        Yh = np.full((33, 70), np.nan, np.float32)
        An = np.ascontiguousarray(A.numpy())
        P.sk_apply_left_host(h, An.ctypes.data, 5000, 70, 70, Yh.ctypes.data, 70)
    finally:
        P.sk_destroy(h)
    np.testing.assert_array_equal(Yh, a)


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("side", ["left", "right"])
def test_host_entry_points_unpadded_rows(P, side, form):
    """Host buffers whose rows need no padding (n and the output width
    multiples of 4) take the linear-copy path; the result is the device
    path's bit for bit, and nothing outside Y is written."""
    m, n, k = 3000, 64, 48
    A = _A(m, n, 11)
    h = P.sk_create(21, G, k)
    try:
        P.sk_set_precision(h, form)
        yshape = (k, n) if side == "left" else (m, k)
        Yd = torch.empty(yshape, dtype=torch.float32, device="cuda")
        f = P.sk_apply_left if side == "left" else P.sk_apply_right
        f(h, A.cuda(), m, n, n, Yd, yshape[1])
        torch.cuda.synchronize()
        Yh = np.full((yshape[0] * yshape[1] + 8,), np.nan, np.float32)
        An = np.ascontiguousarray(A.numpy())
        g = P.sk_apply_left_host if side == "left" else P.sk_apply_right_host
        g(h, An.ctypes.data, m, n, n, Yh.ctypes.data, yshape[1])
    finally:
        P.sk_destroy(h)
    np.testing.assert_array_equal(Yh[:-8].reshape(yshape), Yd.cpu().numpy())
    assert np.isnan(Yh[-8:]).all()


def test_transposition_identity(P):
    A = _A(300, 200, 9)
    right = run(P, "right", 4, R, 24, A)
    left = run(P, "left", 4, R, 24, A.t().contiguous())
    assert rel_frob(right, left.T) <= 1e-6


def test_workspace_lent_by_caller(P, orc):
    A = _A(20000, 64, 4)
    h = P.sk_create(8, G, 64)
    try:
        nbytes = P.sk_workspace_size(h, 0, 20000, 64)
        ws = torch.empty(max(nbytes, 16) // 4 + 4, dtype=torch.float32, device="cuda")
        P.sk_set_workspace(h, ws, ws.numel() * 4)
        Ad = A.cuda()
        Y = torch.empty((64, 64), device="cuda")
        P.sk_apply_left(h, Ad, 20000, 64, 64, Y, 64)
        assert P.sk_stream_status(h) == 0
        if nbytes:
            P.sk_set_workspace(h, ws, 16)  # too small: rejected, not overrun
            with pytest.raises(P.SketchError):
                P.sk_apply_left(h, Ad, 20000, 64, 64, Y, 64)
    finally:
        P.sk_destroy(h)
    assert rel_frob(Y.cpu().numpy(), orc.apply_left(8, G, 0, 64, A.numpy())) <= TOL


def test_invalid_arguments(P):
    h = P.sk_create(1, G, 8)
    A = torch.zeros((4, 4), device="cuda")
    Y = torch.zeros((8, 4), device="cuda")
    try:
        for args in [(A, 0, 4, 4, Y, 4), (A, 4, 4, 3, Y, 4), (A, 4, 4, 4, Y, 3),
                     (None, 4, 4, 4, Y, 4), (A, 4, 4, 4, None, 4)]:
            with pytest.raises(P.SketchError) as e:
                P.sk_apply_left(h, *args)
            assert e.value.status == 1
    finally:
        P.sk_destroy(h)


def test_right_fp32_beyond_65535_row_tiles(P, orc):
    """A right sketch whose m needs more than 65535 tiles of 256 rows (the
    long side runs along the launch grid's x extent): sampled rows of Y,
    including the last tile's, against the oracle."""
    m, n, k, seed = 65536 * 256 + 300, 6, 24, 13
    A = torch.randn((m, n), generator=torch.Generator().manual_seed(seed))
    Y = torch.full((m, k), float("nan"), dtype=torch.float32, device="cuda")
    h = P.sk_create(seed, G, k)
    try:
        P.sk_apply_right(h, A.cuda(), m, n, n, Y, k)
        assert P.sk_stream_status(h) == 0
    finally:
        P.sk_destroy(h)
    rows = np.unique(np.r_[np.arange(0, 8), np.linspace(0, m - 1, 200).astype(np.int64),
                           np.arange(m - 300, m)])
    got = Y[torch.from_numpy(rows).cuda()].cpu().numpy()
    ref = orc.apply_right(seed, G, 0, k, A.numpy(), rows=rows)
    assert np.all(np.isfinite(got))
    assert rel_frob(got, ref) <= TOL
