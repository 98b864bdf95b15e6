"""GPU parity of the BF16 split-A tensor-core form (sk_set_precision(SK_BF16X2),
tcgen05 + TMEM + TMA) against the FP64 CPU oracle of the product with
S = bf16(g): relative Frobenius error <= 1e-5 at ragged shapes spanning
several tiles, splits and a ragged tail, and on sampled entries at the full
2^20 x 512, k = 2048 workload in the launch configuration bench.py times."""
import numpy as np
import pytest
import torch

from gpu_util import rel_frob, require_gpu

pytestmark = pytest.mark.gpu

G, R, U = 0, 1, 2
BF16 = 1
TOL = 1e-5


@pytest.fixture(scope="module")
def P():
    require_gpu()
    import paper_2603_20966_gb300 as P
    return P


def _A(m, n, seed, device="cpu"):
    from paper_2603_20966_gb300.workloads import gaussian_matrix
    return gaussian_matrix(m, n, seed, device=device)


def run_left(P, seed, dist, k, A, prec=BF16, lda=None, ldy=None):
    m, n = A.shape
    lda = lda or (n + 3) // 4 * 4
    ldy = ldy or (n + 3) // 4 * 4
    Ad = torch.zeros((m, lda), dtype=torch.float32, device="cuda")
    Ad[:, :n] = A.cuda()
    Y = torch.full((k, ldy), float("nan"), dtype=torch.float32, device="cuda")
    h = P.sk_create(seed, dist, k)
    try:
        P.sk_set_precision(h, prec)
        P.sk_apply_left(h, Ad, m, n, lda, Y, ldy)
        assert P.sk_stream_status(h) == 0
    finally:
        P.sk_destroy(h)
    # the padding columns of Y's rows are never written
    assert torch.isnan(Y[:, n:]).all()
    return Y[:, :n].cpu().numpy()


SHAPES = [(128, 4096, 512), (64, 4096, 256), (100, 1000, 48), (130, 777, 300), (1, 16, 16),
          (3, 5, 7), (256, 70000, 1000), (2048, 65536, 512), (200, 300000, 20),
          # CTA pairs split A in place (one 3D box per stage when n is a
          # multiple of 32, else a 2D box per 32 columns): ragged m, a partly
          # filled second column tile, 96 columns, a chain longer than the
          # item (m below one chain), n = 40 (one chunk per CTA: the second
          # set of converting warps idle)
          (384, 10007, 544), (256, 3000, 96), (512, 1500, 256), (256, 20000, 40),
          # 4 and 5 pair tiles of k: the last Gaussian sketch that splits A in
          # the kernel, the first that runs the split pass
          (1024, 9000, 256), (1280, 9000, 256)]


@pytest.mark.parametrize("dist", [R, G])
@pytest.mark.parametrize("k,m,n", SHAPES)
def test_left_bf16x2_matches_oracle(P, orc, dist, k, m, n):
    A = _A(m, n, 31 * k + m + n)
    got = run_left(P, 7, dist, k, A)
    assert np.all(np.isfinite(got))
    ref = orc.apply_left(7, dist, BF16, k, A.numpy())
    err = rel_frob(got, ref)
    assert err <= TOL, err


@pytest.mark.parametrize("k,m,n", [(96, 3000, 64), (300, 5000, 200)])  # one CTA; pairs
def test_left_bf16x2_uniform(P, orc, k, m, n):
    A = _A(m, n, 5)
    got = run_left(P, 11, U, k, A)
    assert rel_frob(got, orc.apply_left(11, U, BF16, k, A.numpy())) <= TOL


@pytest.mark.parametrize("dist", [R, G])
def test_identity_gives_scaled_bf16_matrix_exactly(P, orc, dist):
    m, k = 512, 200
    got = run_left(P, 13, dist, k, torch.eye(m))
    ref = orc.generate(13, dist, BF16, 0, 0, k, m) * orc.scale(k)  # fl32(s * bf16(g))
    np.testing.assert_array_equal(got, ref.astype(np.float32))


@pytest.mark.parametrize("dist", [R, G])
def test_in_place_split_with_padded_rows(P, orc, dist):
    # lda > n: the FP32 tile the kernel splits in place (Rademacher: the
    # workers; Gaussian: the epilogue warps) is read with the row pitch
    A = _A(5003, 160, 9)
    got = run_left(P, 21, dist, 300, A, lda=176, ldy=164)
    assert rel_frob(got, orc.apply_left(21, dist, BF16, 300, A.numpy())) <= TOL


def test_rademacher_bf16x2_agrees_with_fp32_form(P):
    # S is exactly +-1 in both forms, so both approximate the same exact product;
    # each is within TOL of it, hence within 2*TOL of each other
    A = _A(100000, 512, 3)
    a = run_left(P, 5, R, 512, A, prec=BF16)
    b = run_left(P, 5, R, 512, A, prec=0)
    assert rel_frob(a, b) <= 2 * TOL


def test_deterministic(P):
    A = _A(50000, 300, 4)
    a = run_left(P, 2, G, 256, A)
    b = run_left(P, 2, G, 256, A)
    np.testing.assert_array_equal(a, b)


def test_leading_dimensions_and_alignment(P, orc):
    A = _A(2000, 100, 6)
    got = run_left(P, 3, G, 64, A, lda=128, ldy=104)
    assert rel_frob(got, orc.apply_left(3, G, BF16, 64, A.numpy())) <= TOL
    h = P.sk_create(3, G, 64)
    Ad = torch.zeros((2000, 101), device="cuda")
    Y = torch.zeros((64, 104), device="cuda")
    try:
        P.sk_set_precision(h, BF16)
        with pytest.raises(P.SketchError):  # lda not a multiple of 4 (TMA row pitch)
            P.sk_apply_left(h, Ad, 2000, 100, 101, Y, 104)
        with pytest.raises(P.SketchError):  # misaligned base pointer
            P.sk_apply_left(h, Ad.data_ptr() + 4, 2000, 100, 104, Y, 104)
    finally:
        P.sk_destroy(h)


def _full_size_left(P, dist, m, n, k, seed, lda):
    A = torch.zeros((m, lda), device="cuda")
    A[:, :n] = _A(m, n, seed, device="cuda")
    Y = torch.empty((k, lda), device="cuda")
    h = P.sk_create(7, dist, k)
    try:
        P.sk_set_precision(h, BF16)
        P.sk_apply_left(h, A, m, n, lda, Y, lda)
        assert P.sk_stream_status(h) == 0
    finally:
        P.sk_destroy(h)
    return A, Y


def _check_row_blocks(orc, dist, k, A, Y, cols, blocks):
    idx = torch.from_numpy(cols).cuda()
    a_cols = A[:, idx].cpu().numpy()
    for rows in blocks:
        ref = orc.apply_left(7, dist, BF16, k, a_cols, rows=rows)
        got = Y[rows[0]:rows[0] + rows[1]][:, idx].cpu().numpy()
        err = rel_frob(got, ref)
        assert err <= TOL, (rows, err)


@pytest.mark.parametrize("dist", [R, G])
def test_full_size_tall_skinny_sampled(P, orc, dist):
    # the 2^20 x 512, k = 2048 workload exactly as bench.py launches it; rows
    # in the first, an inner and the last 256-row tile of k (each tile shifts
    # its accumulation-chain boundaries differently), columns in both
    # 256-column halves
    m, n, k = 1 << 20, 512, 2048
    A, Y = _full_size_left(P, dist, m, n, k, 1, n)
    cols = np.array([0, 1, 255, 256, 511])
    _check_row_blocks(orc, dist, k, A, Y, cols, [(0, 32), (1000, 96), (k - 48, 48)])
    assert torch.isfinite(Y[:, :n]).all()


@pytest.mark.parametrize("dist", [R, G])
def test_full_size_ragged_sampled(P, orc, dist):
    # near-full size with a ragged tail everywhere: m not a multiple of a
    # stage or a split of m, n = 500 (second column tile partly filled, A
    # split in place by 32-column boxes), k = 2000 (last 256-row tile of k
    # partly filled)
    m, n, k = (1 << 20) - 37, 500, 2000
    A, Y = _full_size_left(P, dist, m, n, k, 2, 500)
    cols = np.array([0, 255, 256, 480, 499])
    _check_row_blocks(orc, dist, k, A, Y, cols, [(0, 16), (1790, 16), (k - 32, 32)])
    assert torch.isfinite(Y[:, :n]).all()


def run_right(P, seed, dist, k, A, prec=BF16, lda=None, ldy=None):
    m, n = A.shape
    lda = lda or (n + 3) // 4 * 4
    ldy = ldy or (k + 3) // 4 * 4
    Ad = torch.zeros((m, lda), dtype=torch.float32, device="cuda")
    Ad[:, :n] = A.cuda()
    Y = torch.full((m, ldy), float("nan"), dtype=torch.float32, device="cuda")
    h = P.sk_create(seed, dist, k)
    try:
        P.sk_set_precision(h, prec)
        P.sk_apply_right(h, Ad, m, n, lda, Y, ldy)
        assert P.sk_stream_status(h) == 0
    finally:
        P.sk_destroy(h)
    # the padding columns of Y's rows are never written
    assert torch.isnan(Y[:, k:]).all()
    return Y[:, :k].cpu().numpy()


# k tiles of 32 to 256 rows (each CTA pair's S tile split between the two
# pairs of a cluster in whole 8-row groups), including 96 and 224
RIGHT_SHAPES = [(512, 4096, 256), (1000, 3000, 100), (300, 17, 31), (5, 5, 3), (2048, 1000, 512),
                (700, 70000, 48), (4096, 2048, 256), (3000, 2000, 200), (2500, 1500, 90),
                # more 1024-row blocks than clusters, two tiles of k, ragged m
                (40000, 600, 300)]


@pytest.mark.parametrize("dist", [R, G])
@pytest.mark.parametrize("m,n,k", RIGHT_SHAPES)
def test_right_bf16x2_matches_oracle(P, orc, dist, m, n, k):
    A = _A(m, n, 17 * k + m + n)
    got = run_right(P, 11, dist, k, A)
    assert np.all(np.isfinite(got))
    ref = orc.apply_right(11, dist, BF16, k, A.numpy())
    err = rel_frob(got, ref)
    assert err <= TOL, err


def test_right_identity_gives_transposed_scaled_matrix(P, orc):
    n, k = 384, 200
    got = run_right(P, 5, G, k, torch.eye(n))
    ref = (orc.generate(5, G, BF16, 0, 0, k, n) * orc.scale(k)).T  # Y = S^T scaled
    np.testing.assert_array_equal(got, ref.astype(np.float32))


@pytest.mark.parametrize("dist", [G, R])
def test_right_full_size_lowrank_sampled(P, orc, dist):
    # A = U V^T + 1e-3 E, 65536 x 16384, k = 256: the right-sketch workload
    from paper_2603_20966_gb300.workloads import lowrank_plus_noise
    m, n, k = 65536, 16384, 256
    A = lowrank_plus_noise(m, n, device="cuda")
    Y = torch.empty((m, k), device="cuda")
    h = P.sk_create(7, dist, k)
    try:
        P.sk_set_precision(h, BF16)
        P.sk_apply_right(h, A, m, n, n, Y, k)
        assert P.sk_stream_status(h) == 0
    finally:
        P.sk_destroy(h)
    rows = np.array([0, 1, 511, 512, 30000, 65535])
    a_rows = A[torch.from_numpy(rows).cuda()].cpu().numpy()
    ref = orc.apply_right(7, dist, BF16, k, a_rows)
    got = Y[torch.from_numpy(rows).cuda()].cpu().numpy()
    assert rel_frob(got, ref) <= TOL
    assert torch.isfinite(Y).all()
