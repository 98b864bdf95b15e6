"""Pins of the oracle's FP8 (E4M3) form of A against things other than itself:
torch's float8_e4m3fn conversion (round to nearest even), the definition of
the row exponent (smallest power of two that keeps every entry within 448),
closed forms, and brute-force products on tiny inputs."""
import math

import numpy as np
import pytest
import torch

import oracle


def _torch_e4m3(x: np.ndarray):
    """(codes, values) of float32 x by torch's E4M3 cast (no value exceeds 448)."""
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(torch.float8_e4m3fn)
    return t.view(torch.uint8).numpy(), t.to(torch.float64).numpy()


def _rows():
    rng = np.random.default_rng(5)
    rows = [
        rng.standard_normal(64) * 10.0 ** rng.integers(-6, 7),
        np.zeros(64),
        np.full(64, 448.0),                        # already at the top: exponent 0
        np.full(64, -448.0 * 2.0 ** 5),            # exact boundary, negative
        np.concatenate([[1e6], rng.standard_normal(63) * 1e-3]),  # one large, many tiny
        2.0 ** rng.integers(-20, 20, 64).astype(np.float64),       # powers of two
        np.concatenate([[449.0], np.ones(63)]),    # just above the top: exponent 1
        rng.standard_normal(64) * 1e-30,           # very small row
    ]
    return np.stack([np.asarray(r, dtype=np.float32) for r in rows])


def test_row_exponent_is_the_smallest_that_fits():
    A = _rows()
    codes, exps = oracle.quantize_rows_e4m3(A)
    for i in range(A.shape[0]):
        amax = float(np.max(np.abs(A[i].astype(np.float64))))
        e = int(exps[i])
        if amax == 0.0:
            assert e == 0 and np.all(codes[i] == 0)
            continue
        assert math.ldexp(amax, -e) <= 448.0 < math.ldexp(amax, -(e - 1)), (i, e, amax)
    assert exps[2] == 0 and exps[3] == 5 and exps[6] == 1


def test_codes_match_torch_rounding():
    A = _rows()
    codes, exps = oracle.quantize_rows_e4m3(A)
    for i in range(A.shape[0]):
        scaled = np.ldexp(A[i].astype(np.float64), -int(exps[i])).astype(np.float32)
        tcodes, tvals = _torch_e4m3(scaled)
        # +0 and -0 both decode to zero; compare values, and codes away from zero
        vals = oracle.e4m3_value(codes[i])
        assert np.array_equal(vals, tvals), i
        nz = tvals != 0
        assert np.array_equal(codes[i][nz], tcodes[nz]), i
        assert np.all(np.abs(vals) <= 448.0)


def test_nearest_by_enumeration():
    # every finite E4M3 value by torch's decode of all 256 codes; each code the
    # oracle picks is a nearest one (ties to the even significand)
    allv = torch.arange(256, dtype=torch.uint8).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    finite = np.isfinite(allv)
    grid = np.unique(allv[finite])
    rng = np.random.default_rng(9)
    A = (rng.standard_normal((16, 128)) * 50).astype(np.float32)
    codes, exps = oracle.quantize_rows_e4m3(A)
    vals = oracle.e4m3_value(codes)
    for i in range(16):
        x = np.ldexp(A[i].astype(np.float64), -int(exps[i]))
        d = np.abs(grid[None, :] - x[:, None])
        best = d.min(axis=1)
        assert np.all(np.abs(vals[i] - x) == best)


def test_right_q8_brute_force():
    rng = np.random.default_rng(3)
    for dist in (0, 1):
        m, n, k = 5, 37, 6
        A = (rng.standard_normal((m, n)) * 3).astype(np.float32)
        codes, exps = oracle.quantize_rows_e4m3(A)
        Y = oracle.apply_right_q8(11, dist, k, codes, exps)
        S = oracle.generate(11, dist, oracle.E4M3, 0, 0, k, n).astype(np.float64)
        s = float(oracle.scale(k))
        Aval = oracle.e4m3_value(codes) * np.ldexp(1.0, exps.astype(np.int64))[:, None]
        want = (Aval @ S.T) * s
        assert np.allclose(Y, want, rtol=1e-14, atol=1e-14)
        rows = np.array([4, 0, 2])
        assert np.array_equal(oracle.apply_right_q8(11, dist, k, codes, exps, rows=rows), Y[rows])


def test_right_q8_identity_gives_the_e4m3_matrix():
    # A = I: every row max is 1, exponent -8, the code is 256 exactly, so
    # Y = S^T with S in E4M3, bit for bit
    n, k = 24, 8
    codes, exps = oracle.quantize_rows_e4m3(np.eye(n, dtype=np.float32))
    assert np.all(exps == -8)
    Y = oracle.apply_right_q8(2, 0, k, codes, exps)
    S = oracle.materialize_scaled(2, 0, oracle.E4M3, k, 0, 0, k, n)
    assert np.array_equal(Y, S.T.astype(np.float64))


def test_right_q8_error_against_exact_product_is_fp8_sized():
    rng = np.random.default_rng(4)
    m, n, k = 64, 512, 32
    A = rng.standard_normal((m, n)).astype(np.float32)
    codes, exps = oracle.quantize_rows_e4m3(A)
    Yq = oracle.apply_right_q8(7, 0, k, codes, exps)
    Y = oracle.apply_right(7, 0, oracle.FP32, k, A)
    rel = np.linalg.norm(Yq - Y) / np.linalg.norm(Y)
    # 3 significand bits on both operands: a few percent, never exact
    assert 1e-3 < rel < 0.1, rel
