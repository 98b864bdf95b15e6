"""Pins for the oracle's Philox4x32-10 (Salmon et al. 2011, the generator the
paper names in Sec. 6.2).  The reference is cuRAND's host-side
PHILOX4_32_10 generator, a library implementation run on the CPU: for outputs
0 .. N-1 with N <= 2^16 its block j (4 words) is Philox(counter=(0,0,j,0),
key=(seed lo, seed hi)), which exercises every round, both multipliers, both
Weyl constants and both key words."""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _curand():
    cands = [os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib64", "libcurand.so"),
             ctypes.util.find_library("curand")]
    for c in cands:
        if c and (os.path.exists(c) or not c.startswith("/")):
            try:
                return ctypes.CDLL(c)
            except OSError:
                continue
    pytest.skip("libcurand not available")


def _curand_host_words(L, seed, n):
    g = ctypes.c_void_p()
    if L.curandCreateGeneratorHost(ctypes.byref(g), CURAND_RNG_PSEUDO_PHILOX4_32_10) != 0:
        pytest.skip("cuRAND host generator unavailable")
    try:
        assert L.curandSetPseudoRandomGeneratorSeed(g, ctypes.c_ulonglong(seed)) == 0
        out = np.zeros(n, np.uint32)
        assert L.curandGenerate(g, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
    finally:
        L.curandDestroyGenerator(g)
    return out.reshape(-1, 4)


@pytest.mark.parametrize("seed", [0, 7, 1000, 0xFFFFFFFF, 0x100000007, 0x0123456789ABCDEF,
                                  0xFFFFFFFFFFFFFFFF])
def test_philox_matches_curand_host(orc, seed):
    L = _curand()
    n_words = 1 << 16
    ref = _curand_host_words(L, seed, n_words)
    j = np.arange(ref.shape[0], dtype=np.uint32)
    z = np.zeros_like(j)
    ctr = np.stack([z, z, j, z], axis=1)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    got = orc.philox4x32_10(ctr, key)
    np.testing.assert_array_equal(got, ref)


def test_philox_is_a_bijection_of_the_counter(orc):
    # For a fixed key Philox is a permutation of the 128-bit counter space:
    # distinct counters that differ in any single word never collide.
    rng = np.random.default_rng(3)
    base = rng.integers(0, 2**32, size=(1, 4), dtype=np.uint64).astype(np.uint32)
    ctrs = np.repeat(base, 4 * 4096, axis=0)
    for w in range(4):
        ctrs[w * 4096:(w + 1) * 4096, w] = np.arange(4096, dtype=np.uint32)
    out = orc.philox4x32_10(ctrs, [123, 456])
    as_bytes = {bytes(r) for r in out}
    distinct_ctrs = {bytes(r) for r in ctrs}
    assert len(as_bytes) == len(distinct_ctrs)


def test_philox_word_balance(orc):
    # Each output bit is 1 with probability 1/2 (5-sigma band over 2^20 words).
    j = np.arange(1 << 18, dtype=np.uint32)
    z = np.zeros_like(j)
    out = orc.philox4x32_10(np.stack([j, z, z, z], 1), [7, 0]).reshape(-1)
    bits = np.unpackbits(out.view(np.uint8)).reshape(-1, 32).mean(axis=0)
    sigma = 0.5 / np.sqrt(out.size)
    assert np.all(np.abs(bits - 0.5) < 5 * sigma)
