"""Pins for the oracle's round-to-nearest-even conversions to BF16 and to
E4M3 (the storage precisions of the generated matrix in the tensor-core
forms).  Reference: torch's dtype casts (library routines) on a structured
sample that includes every tie pattern, and on every E4M3 code."""
import numpy as np
import pytest
import torch


def _structured_floats():
    hi = np.arange(1 << 16, dtype=np.uint32) << 16
    lows = np.array([0, 1, 0x7FFF, 0x8000, 0x8001, 0xFFFF, 0x4000, 0xC000, 0x10, 0x7FF0],
                    dtype=np.uint32)
    rng = np.random.default_rng(11)
    lows = np.concatenate([lows, rng.integers(0, 1 << 16, size=22, dtype=np.uint32)])
    bits = (hi[:, None] | lows[None, :]).reshape(-1)
    f = bits.view(np.float32)
    return f[np.isfinite(f)]


def test_bf16_rne_matches_torch(orc):
    x = _structured_floats()
    got = orc.bf16_rne(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    np.testing.assert_array_equal(got, ref)


def test_bf16_rne_random_full_range(orc):
    rng = np.random.default_rng(5)
    bits = rng.integers(0, 1 << 32, size=1 << 22, dtype=np.uint64).astype(np.uint32)
    x = bits.view(np.float32)
    x = x[np.isfinite(x)]
    got = orc.bf16_rne(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    np.testing.assert_array_equal(got, ref)


def _e4m3_torch_codes(x):
    return torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()


def test_e4m3_rne_matches_torch_in_range(orc):
    x = _structured_floats()
    x = x[np.abs(x) <= 448.0]
    got = orc.e4m3_rne(x)
    np.testing.assert_array_equal(got, _e4m3_torch_codes(x))


def test_e4m3_rne_dense_generator_range(orc):
    # every FP32 value in [-8, 8] with the low 12 bits fixed to a tie-rich set
    base = np.arange(0, 0x41000000 >> 12, dtype=np.uint32) << 12
    lows = np.array([0, 0x7FF, 0x800, 0x801, 0xFFF], dtype=np.uint32)
    bits = (base[:, None] | lows[None, :]).reshape(-1)
    x = np.concatenate([bits.view(np.float32), -bits.view(np.float32)])
    got = orc.e4m3_rne(x)
    np.testing.assert_array_equal(got, _e4m3_torch_codes(x))


def test_e4m3_saturates(orc):
    x = np.array([448.0, 463.9, 464.0, 1000.0, -5000.0, 3.0e38], dtype=np.float32)
    got = orc.e4m3_rne(x)
    np.testing.assert_array_equal(got, [0x7E, 0x7E, 0x7E, 0x7E, 0xFE, 0x7E])


def test_e4m3_decode_all_codes(orc):
    codes = np.arange(256, dtype=np.uint8)
    got = orc.e4m3_value(codes)
    ref = torch.from_numpy(codes).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    finite = np.isfinite(ref)
    np.testing.assert_array_equal(got[finite], ref[finite])
    assert np.all(np.isnan(got[~finite]))


@pytest.mark.parametrize("v", [0.0, 1.0, -1.0, 0.5, 5.765, -5.765, 2.0**-9, 2.0**-10])
def test_e4m3_round_trip_values(orc, v):
    code = orc.e4m3_rne(np.array([v], np.float32))
    ref = _e4m3_torch_codes(np.array([v], np.float32))
    assert code[0] == ref[0]
