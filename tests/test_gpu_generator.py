"""GPU parity of the generated matrix: sk_materialize is bit-exact against the
CPU oracle for every distribution and storage format, at ragged offsets and
at the top of the 32-bit index range; the oracle's Philox also matches
cuRAND's device API at counters with all four words non-zero."""
import ctypes

import numpy as np
import pytest
import torch

from gpu_util import build_test_so, require_gpu

pytestmark = pytest.mark.gpu

G, R, U = 0, 1, 2
FP32, BF16, E4M3 = 0, 1, 2


@pytest.fixture(scope="module")
def P():
    require_gpu()
    import paper_2603_20966_gb300 as P
    return P


def _materialize(P, seed, dist, k, row0, col0, rows, cols, fmt, scaled=0, ld=None):
    ld = ld or cols
    dt = {FP32: torch.float32, BF16: torch.bfloat16, E4M3: torch.uint8}[fmt]
    out = torch.full((rows, ld), 7, dtype=dt, device="cuda") if ld > cols else torch.empty(
        (rows, cols), dtype=dt, device="cuda")
    h = P.sk_create(seed, dist, k)
    try:
        P.sk_materialize(h, row0, col0, rows, cols, fmt, scaled, out, ld)
        torch.cuda.synchronize()
    finally:
        P.sk_destroy(h)
    return out


CASES = [
    (7, 0, 0, 64, 4096), (7, 5, 3, 17, 1001), (123456789012345, 100, 131, 33, 517),
    (1, 2**32 - 20, 2**32 - 777, 20, 777), (2**64 - 1, 0, 2**31, 8, 4099),
]


@pytest.mark.parametrize("dist", [G, R, U])
@pytest.mark.parametrize("case", CASES)
def test_materialize_fp32_bit_exact(P, orc, dist, case):
    seed, r0, c0, rows, cols = case
    got = _materialize(P, seed, dist, 64, r0, c0, rows, cols, FP32).cpu().numpy()
    ref = orc.generate(seed, dist, FP32, r0, c0, rows, cols)
    np.testing.assert_array_equal(got.view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("dist", [G, R])
@pytest.mark.parametrize("case", CASES[:4])
def test_materialize_bf16_bit_exact(P, orc, dist, case):
    seed, r0, c0, rows, cols = case
    got = _materialize(P, seed, dist, 64, r0, c0, rows, cols, BF16)
    got = got.view(torch.int16).cpu().numpy().view(np.uint16)
    ref = orc.bf16_rne(orc.generate(seed, dist, FP32, r0, c0, rows, cols))
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("dist", [G, R])
@pytest.mark.parametrize("case", CASES[:4])
def test_materialize_e4m3_bit_exact(P, orc, dist, case):
    seed, r0, c0, rows, cols = case
    got = _materialize(P, seed, dist, 64, r0, c0, rows, cols, E4M3).cpu().numpy()
    ref = orc.e4m3_rne(orc.generate(seed, dist, FP32, r0, c0, rows, cols))
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("k", [64, 2048, 100])
def test_materialize_scaled(P, orc, k):
    got = _materialize(P, 9, G, k, 0, 0, 16, 300, FP32, scaled=1).cpu().numpy()
    ref = orc.generate(9, G, FP32, 0, 0, 16, 300) * orc.scale(k)  # FP32 multiply, RN
    np.testing.assert_array_equal(got.view(np.uint32), ref.astype(np.float32).view(np.uint32))


def test_materialize_respects_leading_dimension(P, orc):
    got = _materialize(P, 3, G, 8, 0, 0, 5, 13, FP32, ld=20).cpu().numpy()
    np.testing.assert_array_equal(got[:, :13], orc.generate(3, G, FP32, 0, 0, 5, 13))
    assert np.all(got[:, 13:] == 7)


def test_materialize_rejects_bad_arguments(P):
    h = P.sk_create(1, G, 8)
    buf = torch.empty(16, device="cuda")
    try:
        for args in [(0, 0, 0, 4, FP32, 0, buf, 4), (0, 0, 2, 4, FP32, 0, buf, 3),
                     (2**32 - 1, 0, 2, 4, FP32, 0, buf, 4), (0, 0, 2, 4, BF16, 1, buf, 4),
                     (0, 0, 2, 4, 7, 0, buf, 4)]:
            with pytest.raises(P.SketchError):
                P.sk_materialize(h, *args)
    finally:
        P.sk_destroy(h)


def test_oracle_philox_matches_curand_device_api(orc):
    require_gpu()
    lib = ctypes.CDLL(build_test_so("curand_philox_ref"))
    lib.curand_ref_words.argtypes = [ctypes.c_ulonglong] * 3 + [ctypes.c_void_p, ctypes.c_int]
    n = 4096
    for seed, subseq0, off_blocks in [(7, 0, 0), (0x0123456789ABCDEF, 2**32 + 5, 3 * 2**32 + 7),
                                      (2**64 - 1, 2**64 - n, 2**32 - 1)]:
        out = torch.zeros((n, 4), dtype=torch.int32, device="cuda")
        assert lib.curand_ref_words(seed, subseq0, 4 * off_blocks, out.data_ptr(), n) == 0
        got = out.cpu().numpy().view(np.uint32)
        sub = np.array([(subseq0 + i) % 2**64 for i in range(n)], dtype=np.uint64)
        ctr = np.stack([np.full(n, off_blocks & 0xFFFFFFFF, np.uint64),
                        np.full(n, off_blocks >> 32, np.uint64),
                        sub & np.uint64(0xFFFFFFFF), sub >> np.uint64(32)], 1).astype(np.uint32)
        ref = orc.philox4x32_10(ctr, [seed & 0xFFFFFFFF, seed >> 32])
        np.testing.assert_array_equal(got, ref)
