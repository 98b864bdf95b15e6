"""GPU parity of the Nystrom pair (sk_nystrom: B = A Omega, C = Omega^T B):
both outputs within 1e-5 of the FP64 oracle in the FP32 and BF16 split-A
forms, C symmetric, and the Nystrom formula recovering a low-rank PSD
matrix."""
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


@pytest.mark.parametrize("n,k,dist,prec", [(500, 64, 0, 0), (1000, 200, 1, 1), (2048, 256, 0, 1),
                                           (780, 96, 2, 1), (300, 40, 1, 0)])
def test_nystrom_matches_oracle(P, orc, n, k, dist, prec):
    g = torch.Generator(device="cpu").manual_seed(n + k)
    G = torch.randn((n, n), generator=g)
    A = ((G + G.T) / 2).contiguous().cuda()
    from paper_2603_20966_gb300 import Sketch
    with Sketch(17, dist, k, precision=prec) as sk:
        B, C = sk.nystrom(A)
        assert sk.status() == 0
        Bref, Cref = orc.nystrom(17, dist, prec, k, A.cpu().numpy())
        assert rel_frob(B.cpu().numpy(), Bref) <= TOL
        assert rel_frob(C.cpu().numpy(), Cref) <= TOL
        Cn = C.double().cpu().numpy()
        assert np.linalg.norm(Cn - Cn.T) / np.linalg.norm(Cn) <= 2 * TOL


def test_nystrom_low_rank_recovery(P):
    n, k, rank = 4096, 128, 32
    U = torch.randn((n, rank), dtype=torch.float64, device="cuda")
    A = (U @ U.T).float().contiguous()
    from paper_2603_20966_gb300 import Sketch
    with Sketch(5, 0, k, precision=1) as sk:
        B, C = sk.nystrom(A)
        rec = B.double() @ torch.linalg.pinv(C.double(), rtol=1e-7) @ B.double().T
        assert (torch.linalg.norm(rec - A.double()) / torch.linalg.norm(A.double())).item() < 1e-4


def test_nystrom_fp8_unsupported(P):
    h = P.sk_create(1, 0, 16)
    P.sk_set_precision(h, 2)
    A = torch.zeros((64, 64), device="cuda")
    B = torch.zeros((64, 16), device="cuda")
    C = torch.zeros((16, 16), device="cuda")
    try:
        with pytest.raises(P.SketchError):
            P.sk_nystrom(h, A, 64, 64, B, 16, C, 16)
    finally:
        P.sk_destroy(h)
