"""The stored-S left sketch (sk_apply_left_stored), the communicated-Omega
side of the generate-versus-communicate trade (Sec. 6.2): with the handle's
own S materialized by the library it must give the fused sketch's Y bit for
bit (same operand values, same MMA order); with any other BF16 S it must be
the product s S A (checked against an FP64 product of the same values)."""
import pytest
import torch

from gpu_util import require_gpu

pytestmark = pytest.mark.gpu

G, R, U = 0, 1, 2
BF16 = 1
TOL = 1e-5


@pytest.fixture(scope="module")
def P():
    require_gpu()
    import paper_2603_20966_gb300 as P
    return P


def _A(m, n, seed, lda):
    from paper_2603_20966_gb300.workloads import gaussian_matrix
    A = torch.zeros((m, lda), dtype=torch.float32, device="cuda")
    A[:, :n] = gaussian_matrix(m, n, seed, device="cuda")
    return A


def _lds(m):
    return (m + 15) // 16 * 16


SHAPES = [(128, 4096, 512), (64, 4096, 256), (104, 1000, 48), (8, 40, 16), (256, 70000, 1000),
          (2048, 65536, 512), (136, 777, 300)]


@pytest.mark.parametrize("dist", [R, G, U])
@pytest.mark.parametrize("k,m,n", SHAPES)
def test_stored_equals_fused(P, dist, k, m, n):
    ld = (n + 3) // 4 * 4
    A = _A(m, n, 3 * k + m + n, ld)
    lds = _lds(m)
    S = torch.zeros((k, lds), dtype=torch.bfloat16, device="cuda")
    Yf = torch.full((k, ld), float("nan"), device="cuda")
    Ys = torch.full((k, ld), float("nan"), device="cuda")
    h = P.sk_create(9, dist, k)
    try:
        P.sk_set_precision(h, BF16)
        P.sk_apply_left(h, A, m, n, ld, Yf, ld)
        P.sk_materialize(h, 0, 0, k, m, BF16, 0, S, lds)
        P.sk_apply_left_stored(h, S, lds, A, m, n, ld, Ys, ld)
        assert P.sk_stream_status(h) == 0
    finally:
        P.sk_destroy(h)
    assert torch.isfinite(Ys[:, :n]).all()
    assert torch.equal(Ys[:, :n], Yf[:, :n])


@pytest.mark.parametrize("k,m,n", [(256, 30000, 512), (40, 999, 64)])
def test_stored_arbitrary_s(P, k, m, n):
    # an S the generator would never produce: the kernel must read it
    g = torch.Generator(device="cuda").manual_seed(k + m)
    lds = _lds(m) + 16
    S = torch.randn((k, lds), generator=g, device="cuda").to(torch.bfloat16)
    S[:, m:] = 0
    A = _A(m, n, 77, n)
    Y = torch.empty((k, n), device="cuda")
    h = P.sk_create(1, G, k)
    try:
        P.sk_set_precision(h, BF16)
        P.sk_apply_left_stored(h, S, lds, A, m, n, n, Y, n)
        assert P.sk_stream_status(h) == 0
        s = P.sk_get_info(h)["scale"]
    finally:
        P.sk_destroy(h)
    ref = s * (S[:, :m].double() @ A.double())
    err = (torch.linalg.norm(Y.double() - ref) / torch.linalg.norm(ref)).item()
    assert err <= TOL, err


def test_stored_argument_checks(P):
    k, m, n = 64, 1000, 64
    A = _A(m, n, 1, n)
    Y = torch.empty((k, n), device="cuda")
    S = torch.zeros((k, 1024 + 8), dtype=torch.bfloat16, device="cuda")
    h = P.sk_create(1, R, k)
    try:
        with pytest.raises(P.SketchError):  # the FP32 form has no stored-S path
            P.sk_apply_left_stored(h, S, 1024, A, m, n, n, Y, n)
        P.sk_set_precision(h, BF16)
        with pytest.raises(P.SketchError):  # lds below m rounded up to 16
            P.sk_apply_left_stored(h, S, 1000, A, m, n, n, Y, n)
        with pytest.raises(P.SketchError):  # lds not a multiple of 8
            P.sk_apply_left_stored(h, S, 1028, A, m, n, n, Y, n)
        with pytest.raises(P.SketchError):  # S not 16-byte aligned
            P.sk_apply_left_stored(h, S.data_ptr() + 2, 1024, A, m, n, n, Y, n)
        P.sk_apply_left_stored(h, S, 1024, A, m, n, n, Y, n)  # S = 0: Y = 0
        assert P.sk_stream_status(h) == 0
        assert torch.count_nonzero(Y).item() == 0
    finally:
        P.sk_destroy(h)
    h = P.sk_create(1, R, 12)  # k not a multiple of 8
    try:
        P.sk_set_precision(h, BF16)
        with pytest.raises(P.SketchError):
            P.sk_apply_left_stored(h, S, 1024, A, m, n, n, Y[:12], n)
    finally:
        P.sk_destroy(h)
