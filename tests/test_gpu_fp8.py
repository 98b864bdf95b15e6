"""GPU parity of the FP8 (E4M3) right sketch: the row quantizer bit-exact
against the oracle (codes and row exponents), the sketch within 1e-5 of the
oracle's FP64 product of the same E4M3 values (FP32 tensor-core
accumulation), in-call quantization identical to quantize + sketch, the
error against the exact FP64 product reported (a few percent)."""
import numpy as np
import pytest
import torch

from gpu_util import rel_frob, require_gpu

pytestmark = pytest.mark.gpu

FP8 = 2
TOL = 1e-5


@pytest.fixture(scope="module")
def P():
    require_gpu()
    import paper_2603_20966_gb300 as P
    return P


def _quantize(P, A):
    m, n = A.shape
    ldq = (n + 15) // 16 * 16
    Aq = torch.full((m, ldq), 0x7F, dtype=torch.uint8, device="cuda")
    ex = torch.full((m,), 12345, dtype=torch.int32, device="cuda")
    P.sk_quantize_e4m3(A, m, n, A.stride(0), Aq, ldq, ex)
    torch.cuda.synchronize()
    return Aq, ex, ldq


@pytest.mark.parametrize("m,n,scale", [(100, 1000, 1.0), (37, 4099, 1e-20), (256, 160, 1e6),
                                       (5, 17, 1.0)])
def test_quantize_bit_exact(P, orc, m, n, scale):
    g = torch.Generator(device="cpu").manual_seed(m * 7 + n)
    A = (torch.randn((m, n), generator=g) * scale).to("cuda")
    A[min(3, m - 1)] = 0.0                      # a zero row
    A[0, 0] = 448.0 * 2.0 ** 4                  # an exact boundary
    Aq, ex, ldq = _quantize(P, A)
    codes, exps = orc.quantize_rows_e4m3(A.cpu().numpy())
    got = Aq.cpu().numpy()
    assert np.array_equal(ex.cpu().numpy(), exps)
    assert np.array_equal(got[:, :n], codes)
    assert np.all(got[:, n:] == 0)


def test_quantize_unaligned_rows(P, orc):
    base = torch.randn((64 * 131 + 1,), device="cuda")
    A = base[1:].view(64, 131)[:, :130]        # rows 4-byte aligned only, lda 131
    Aq, ex, ldq = _quantize(P, A)
    codes, exps = orc.quantize_rows_e4m3(A.cpu().numpy())
    assert np.array_equal(ex.cpu().numpy(), exps)
    assert np.array_equal(Aq.cpu().numpy()[:, :130], codes)


SHAPES = [(300, 1000, 64, 0), (700, 4099, 200, 1), (1024, 2048, 256, 0), (513, 777, 48, 2),
          (2000, 16384, 256, 0)]


@pytest.mark.parametrize("m,n,k,dist", SHAPES)
def test_right_fp8_matches_oracle(P, orc, m, n, k, dist):
    A = torch.randn((m, n), device="cuda")
    Aq, ex, ldq = _quantize(P, A)
    h = P.sk_create(23, dist, k)
    P.sk_set_precision(h, FP8)
    ldy = (k + 3) // 4 * 4
    Y = torch.full((m, ldy), float("nan"), device="cuda")
    try:
        P.sk_apply_right_e4m3(h, Aq, ex, m, n, ldq, Y, ldy)
        assert P.sk_stream_status(h) == 0
        rows = np.unique(np.linspace(0, m - 1, min(m, 96)).astype(np.int64))
        Ah = A.cpu().numpy()[rows]
        codes, exps = orc.quantize_rows_e4m3(Ah)
        ref = orc.apply_right_q8(23, dist, k, codes, exps)
        got = Y[:, :k].cpu().numpy()[rows]
        assert rel_frob(got, ref) <= TOL, (m, n, k, dist, rel_frob(got, ref))
        # in-call quantization: the same numbers
        Y2 = torch.empty_like(Y)
        P.sk_apply_right(h, A, m, n, n, Y2, ldy)
        assert P.sk_stream_status(h) == 0
        assert torch.equal(Y2[:, :k], Y[:, :k])
        # the FP8 sketch against the exact product: a few percent, reported
        exact = orc.apply_right(23, dist, 0, k, Ah)
        err = rel_frob(got, exact)
        print(f"fp8 right m={m} n={n} k={k} dist={dist}: vs E4M3 oracle {rel_frob(got, ref):.2e}, "
              f"vs exact {err:.2e}")
        assert err < 0.1
    finally:
        P.sk_destroy(h)


def test_right_fp8_lowrank_workload_sampled(P, orc):
    from paper_2603_20966_gb300.workloads import lowrank_plus_noise
    m, n, k = 65536, 16384, 256
    A = lowrank_plus_noise(m, n, device="cuda")
    h = P.sk_create(7, 0, k)
    P.sk_set_precision(h, FP8)
    Y = torch.empty((m, k), device="cuda")
    try:
        P.sk_apply_right(h, A, m, n, n, Y, k)
        assert P.sk_stream_status(h) == 0
        rows = np.linspace(0, m - 1, 64).astype(np.int64)
        Ah = A[torch.from_numpy(rows).cuda()].cpu().numpy()
        codes, exps = orc.quantize_rows_e4m3(Ah)
        ref = orc.apply_right_q8(7, 0, k, codes, exps)
        got = Y.cpu().numpy()[rows]
        assert rel_frob(got, ref) <= TOL
    finally:
        P.sk_destroy(h)


def test_left_fp8_unsupported(P):
    h = P.sk_create(1, 0, 64)
    P.sk_set_precision(h, FP8)
    A = torch.zeros((128, 64), device="cuda")
    Y = torch.zeros((64, 64), device="cuda")
    try:
        with pytest.raises(P.SketchError) as ei:
            P.sk_apply_left(h, A, 128, 64, 64, Y, 64)
        assert ei.value.status == 6  # SK_EUNSUPPORTED
    finally:
        P.sk_destroy(h)
