"""Pins for the oracle's own FP32 ln, sinpi / cospi and circle map (the
Box-Muller steps of the generator).  References: FP64 libm through numpy,
exhaustively over every input the generator can produce (u1 = j 2^-24,
j = 1..2^24 for ln; r = w 2^-23 - 1/4, w = 0..2^22-1 for the polynomials;
every one of the 2^24 angle words for the circle map)."""
import numpy as np


def ulp32(ref64):
    """Size of one FP32 ulp at each reference value (FP32 spacing at |ref|)."""
    r = np.abs(ref64).astype(np.float32)
    r = np.where(r == 0, np.float32(np.finfo(np.float32).tiny), r)
    return (np.nextafter(r, np.float32(np.inf)) - r).astype(np.float64)


def test_ln_exhaustive_within_1ulp(orc):
    j = np.arange(1, (1 << 24) + 1, dtype=np.float64)
    u = (j * 2.0**-24).astype(np.float32)
    assert np.all(u.astype(np.float64) == j * 2.0**-24)  # the inputs are exact
    got = orc.ln(u).astype(np.float64)
    ref = np.log(u.astype(np.float64))
    err = np.abs(got - ref) / ulp32(ref)
    err[ref == 0] = np.abs(got[ref == 0]) / 2.0**-149
    assert err.max() <= 1.0, err.max()
    assert got[-1] == 0.0  # ln 1 = 0 exactly


def test_ln_special_values(orc):
    x = np.array([1.0, 0.5, 0.25, 2.0**-24, 2.0**-1 * 1.5], dtype=np.float32)
    got = orc.ln(x).astype(np.float64)
    np.testing.assert_allclose(got, np.log(x.astype(np.float64)), rtol=2.0**-22)


def test_ln_across_the_fold(orc):
    # mantissas on both sides of sqrt 2, where the reduction switches from f
    # to f / 2, in several binades
    base = np.frombuffer(np.array([0x3F3504F0 + i for i in range(8)], np.uint32).tobytes(),
                         np.float32)
    x = np.concatenate([base * np.float32(2.0**-e) for e in range(1, 24, 5)]).astype(np.float32)
    got = orc.ln(x).astype(np.float64)
    ref = np.log(x.astype(np.float64))
    assert (np.abs(got - ref) / ulp32(ref)).max() <= 1.0


def test_sincospi_quarter_exhaustive_within_2ulp(orc):
    w = np.arange(0, 1 << 22, dtype=np.float64)
    r = (w * 2.0**-23 - 0.25).astype(np.float32)
    assert np.all(r.astype(np.float64) == w * 2.0**-23 - 0.25)  # exact grid
    s, c = orc.sincospi_quarter(r)
    r64 = r.astype(np.float64)
    rs, rc = np.sin(np.pi * r64), np.cos(np.pi * r64)
    zero = r64 == 0
    assert np.all(s[zero] == 0.0) and np.all(c[zero] == 1.0)
    for ref, got in ((rs[~zero], s[~zero]), (rc, c)):
        g = got.astype(np.float64)
        nz = slice(None)
        err = np.abs(g[nz] - ref[nz]) / ulp32(ref[nz])
        assert err.max() <= 2.0, err.max()


def test_circle_words_give_every_grid_angle_once(orc):
    # the 2^24 values of a word's top 24 bits map to points on the unit
    # circle whose angles are exactly the multiples of 2 pi / 2^24, each
    # once: the four turned quarters tile the circle with no overlap and no
    # gap
    n = 1 << 24
    words = (np.arange(n, dtype=np.uint64) << 8).astype(np.uint32) | np.uint32(0x5A)
    x, y = orc.circle(words)
    x64, y64 = x.astype(np.float64), y.astype(np.float64)
    assert np.abs(x64 * x64 + y64 * y64 - 1.0).max() < 4e-7
    step = 2 * np.pi / n
    k = np.arctan2(y64, x64) / step
    ki = np.rint(k)
    assert np.abs(k - ki).max() < 0.25  # every point sits on a grid angle
    idx = np.mod(ki.astype(np.int64), n)
    assert np.unique(idx).size == n  # ... and every grid angle is hit once
    # the low 8 bits of the word do not move the point
    x2, y2 = orc.circle(words ^ np.uint32(0xFF))
    assert np.array_equal(x, x2) and np.array_equal(y, y2)


def test_circle_quarters(orc):
    # position bits 29..8 = 2^21 (r = 0, the centre of each quarter): the
    # four quarter circles centred on angles 0, pi, pi/2 and 3 pi/2
    centre = np.uint32(1 << 29)
    words = np.array([centre, centre | 0x80000000, centre | 0x40000000, centre | 0xC0000000],
                     np.uint32)
    x, y = orc.circle(words)
    np.testing.assert_array_equal(x, np.array([1, -1, 0, 0], np.float32))
    np.testing.assert_array_equal(y, np.array([0, 0, 1, -1], np.float32))
    # r = -1/4 (position 0): the lower end of each quarter, angle -pi/4 + q pi/2
    # for q = 0, 2, 1, 3
    h = np.float32(np.sqrt(0.5))
    x, y = orc.circle(words & np.uint32(0xC0000000))
    np.testing.assert_allclose(x, [h, -h, h, -h], atol=1e-7)
    np.testing.assert_allclose(y, [-h, h, h, -h], atol=1e-7)
