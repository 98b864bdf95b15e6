"""Pins for the oracle's generated entries g(r, c): Box-Muller identities
against FP64 libm on the (cuRAND-pinned) Philox words, distribution tests
(moments, Kolmogorov-Smirnov), and the Rademacher/uniform bit mappings
checked through invariants rather than by restating them."""
import numpy as np
import pytest
from scipy import stats

G, R, U = 0, 1, 2


def _words(orc, seed, row, c_block, dom=0):
    n = c_block.size
    ctr = np.stack([c_block.astype(np.uint32), np.full(n, row, np.uint32),
                    np.full(n, dom, np.uint32), np.zeros(n, np.uint32)], 1)
    return orc.philox4x32_10(ctr, [seed & 0xFFFFFFFF, seed >> 32])


@pytest.mark.parametrize("seed,row", [(7, 0), (7, 5), (0xDEADBEEFCAFE, 1234567), (1, 2**32 - 1)])
def test_box_muller_radius_and_angle(orc, seed, row):
    ncols = 4096
    g = orc.generate(seed, G, 0, row, 0, 1, ncols)[0].astype(np.float64)
    x = _words(orc, seed, row, np.arange(ncols // 4))
    for pair in (0, 1):
        xa = x[:, 2 * pair].astype(np.float64)
        u1 = (np.floor(xa / 256) + 1) / 2.0**24
        z0 = g[2 * pair::4]
        z1 = g[2 * pair + 1::4]
        r2 = z0 * z0 + z1 * z1
        np.testing.assert_allclose(r2, -2.0 * np.log(u1), rtol=2e-6, atol=1e-6)
        # the angle is the circle point's (pinned on its own) of the pair's
        # second word
        cx, cy = orc.circle(x[:, 2 * pair + 1])
        big = r2 > 1e-6
        d = np.abs(np.angle((z0[big] + 1j * z1[big]) / (cx[big] + 1j * cy[big].astype(np.float64))))
        assert d.max() < 1e-5


def test_gaussian_moments_and_ks(orc):
    rows, cols = 64, 1 << 17  # 2^23 samples from many counters and rows
    g = orc.generate(99, G, 0, 0, 0, rows, cols).astype(np.float64).ravel()
    n = g.size
    assert abs(g.mean()) < 5 / np.sqrt(n)
    assert abs(g.var() - 1.0) < 5 * np.sqrt(2.0 / n)
    assert abs((g**4).mean() - 3.0) < 5 * np.sqrt(96.0 / n)
    assert abs((g**3).mean()) < 5 * np.sqrt(15.0 / n)
    assert stats.kstest(g[:1 << 21], "norm").pvalue > 1e-3
    assert np.abs(g).max() <= np.sqrt(-2 * np.log(2.0**-24)) * (1 + 1e-6)


def test_gaussian_columns_are_independent(orc):
    # neighbouring entries share a Philox call; their correlation must vanish
    g = orc.generate(5, G, 0, 0, 0, 16, 1 << 16).astype(np.float64)
    n = g.size // 2
    for lag in (1, 2, 3, 4):
        rho = np.mean(g[:, :-lag] * g[:, lag:])
        assert abs(rho) < 5 / np.sqrt(n)


def test_rademacher_signs_carry_the_philox_popcount(orc):
    seed, row = 0x1234567890, 77
    ncols = 128 * 256
    g = orc.generate(seed, R, 0, row, 0, 1, ncols)[0]
    assert set(np.unique(g)) <= {-1.0, 1.0}
    x = _words(orc, seed, row, np.arange(ncols // 128))
    neg_per_block = (g.reshape(-1, 128) < 0).sum(axis=1)
    popcnt = np.unpackbits(x.view(np.uint8), axis=1).sum(axis=1)
    np.testing.assert_array_equal(neg_per_block, popcnt)
    # each 32-entry group tracks one word: its count of -1 is that word's popcount
    neg_per_word = (g.reshape(-1, 4, 32) < 0).sum(axis=2)
    pc_word = np.unpackbits(x.view(np.uint8).reshape(-1, 4, 4), axis=2).sum(axis=2)
    np.testing.assert_array_equal(neg_per_word, pc_word)


def test_rademacher_balanced(orc):
    g = orc.generate(3, R, 0, 0, 0, 32, 1 << 16)
    n = g.size
    assert abs(g.mean()) < 5 / np.sqrt(n)


def test_uniform_range_and_ks(orc):
    u = orc.generate(11, U, 0, 0, 0, 16, 1 << 16).astype(np.float64).ravel()
    assert u.min() >= 0.0 and u.max() < 1.0
    assert np.all(u * 2**24 == np.floor(u * 2**24))
    assert stats.kstest(u[:1 << 20], "uniform").pvalue > 1e-3
    x = _words(orc, 11, 3, np.arange(1024))
    u3 = orc.generate(11, U, 0, 3, 0, 1, 4096)[0].astype(np.float64)
    # every uniform draw is the top 24 bits of one of the four Philox words of its counter
    top = np.floor(x.astype(np.float64) / 256) / 2.0**24
    assert np.all(np.isin(u3.reshape(-1, 4), top).reshape(-1))


def test_precisions_quantize_the_same_draw(orc):
    g32 = orc.generate(8, G, 0, 0, 0, 8, 512)
    gbf = orc.generate(8, G, 1, 0, 0, 8, 512)
    g8 = orc.generate(8, G, 2, 0, 0, 8, 512)
    np.testing.assert_allclose(gbf, g32, rtol=2.0**-8)
    np.testing.assert_allclose(g8, g32, rtol=2.0**-4, atol=2.0**-10)
    import torch
    ref_bf = torch.from_numpy(g32).to(torch.bfloat16).float().numpy()
    np.testing.assert_array_equal(gbf, ref_bf)
    r32 = orc.generate(8, R, 0, 0, 0, 8, 512)
    for p in (1, 2):
        np.testing.assert_array_equal(orc.generate(8, R, p, 0, 0, 8, 512), r32)


def test_offsets_and_domains(orc):
    full = orc.generate(21, G, 0, 10, 0, 4, 300)
    part = orc.generate(21, G, 0, 12, 37, 2, 101)
    np.testing.assert_array_equal(full[2:4, 37:138], part)
    other_dom = orc.generate(21, G, 0, 10, 0, 4, 300, dom=1)
    assert not np.any(other_dom == full)
    edge = orc.generate(21, R, 0, 2**32 - 2, 2**32 - 300, 2, 300)
    assert edge.shape == (2, 300)
    with pytest.raises(ValueError):
        orc.generate(21, G, 0, 2**32 - 1, 0, 2, 4)


def test_scale(orc):
    for k in (1, 2, 3, 64, 100, 256, 2048, 1 << 20):
        s = float(orc.scale(k))
        assert abs(s - 1 / np.sqrt(k)) <= 0.5 * np.spacing(np.float32(1 / np.sqrt(k)))
    assert orc.scale(64) == 0.125


def test_box_muller_every_input_against_fp64(orc):
    """orc_box_muller over every u1 (with the angle word running through
    every value of its top 24 bits in the same order): the radius matches
    sqrt(-2 ln u1) in FP64 and the angle is the multiple of 2 pi / 2^24 that
    the circle map assigns to the word."""
    n = 1 << 24
    i = np.arange(n, dtype=np.uint64)
    words = np.stack([((i << 8) | 0x11).astype(np.uint32),
                      (((n - 1 - i) << 8) | 0xEE).astype(np.uint32)], 1)
    z = orc.box_muller(words).astype(np.float64)
    u1 = (i.astype(np.float64) + 1) / 2.0**24
    r = np.sqrt(z[:, 0] ** 2 + z[:, 1] ** 2)
    rho = np.sqrt(-2.0 * np.log(u1))
    assert np.all(np.abs(r - rho) <= 4e-7 * np.maximum(rho, 1.0))
    assert r[-1] == 0.0  # u1 = 1: ln 1 = 0 exactly
    big = rho > 1e-2
    cx, cy = orc.circle(words[:, 1])
    d = np.abs(np.angle((z[big, 0] + 1j * z[big, 1]) / (cx[big] + 1j * cy[big].astype(np.float64))))
    assert d.max() < 2e-6
    # the generator's Gaussian entries are these pairs of its Philox words
    x = _words(orc, 7, 3, np.arange(64))
    g = orc.generate(7, G, 0, 3, 0, 1, 256)[0]
    np.testing.assert_array_equal(orc.box_muller(x.reshape(-1, 2)).reshape(-1), g)
