"""Pins for the oracle's own FP32 ln and sincospi (the Box-Muller steps of
the generator).  Reference: FP64 libm through numpy, exhaustively over every
input the generator can produce (u1 = j 2^-24, j = 1..2^24 for ln;
t = 2 j 2^-24, j = 0..2^24-1 for sincospi)."""
import numpy as np


def ulp32(ref64):
    """Size of one FP32 ulp at each reference value (FP32 spacing at |ref|)."""
    r = np.abs(ref64).astype(np.float32)
    r = np.where(r == 0, np.float32(np.finfo(np.float32).tiny), r)
    return (np.nextafter(r, np.float32(np.inf)) - r).astype(np.float64)


def test_ln_exhaustive_within_2ulp(orc):
    j = np.arange(1, (1 << 24) + 1, dtype=np.float64)
    u = (j * 2.0**-24).astype(np.float32)
    assert np.all(u.astype(np.float64) == j * 2.0**-24)  # the inputs are exact
    got = orc.ln(u).astype(np.float64)
    ref = np.log(u.astype(np.float64))
    err = np.abs(got - ref) / ulp32(ref)
    err[ref == 0] = np.abs(got[ref == 0]) / 2.0**-149
    assert err.max() <= 2.0, err.max()
    assert got[-1] == 0.0  # ln 1 = 0 exactly


def test_ln_special_values(orc):
    x = np.array([1.0, 0.5, 0.25, 2.0**-24, 2.0**-1 * 1.5], dtype=np.float32)
    got = orc.ln(x).astype(np.float64)
    np.testing.assert_allclose(got, np.log(x.astype(np.float64)), rtol=2.0**-22)


def test_sincospi_exhaustive_within_2ulp(orc):
    j = np.arange(0, 1 << 24, dtype=np.float64)
    t = (2.0 * j * 2.0**-24).astype(np.float32)
    s, c = orc.sincospi(t)
    t64 = t.astype(np.float64)
    rs, rc = np.sin(np.pi * t64), np.cos(np.pi * t64)
    # exact zeros of sin/cos on the grid (t in {0, 1/2, 1, 3/2}) must come out as +-0
    for ref, got in ((rs, s), (rc, c)):
        g = got.astype(np.float64)
        zero = np.isin(t64 * 2, [0.0, 1.0, 2.0, 3.0]) & (np.abs(ref) < 1e-12)
        assert np.all(g[zero] == 0.0)
        nz = ~zero
        err = np.abs(g[nz] - ref[nz]) / ulp32(ref[nz])
        assert err.max() <= 2.0, err.max()


def test_sincospi_quadrants(orc):
    t = np.array([0.0, 0.5, 1.0, 1.5, 0.25, 0.75, 1.25, 1.75], dtype=np.float32)
    s, c = orc.sincospi(t)
    h = np.sqrt(0.5)
    np.testing.assert_allclose(s, [0, 1, 0, -1, h, h, -h, -h], atol=1e-7)
    np.testing.assert_allclose(c, [1, 0, -1, 0, h, -h, -h, h], atol=1e-7)
