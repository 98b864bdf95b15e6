"""Derivation of the coefficients of the generator's logarithm (run by hand;
nothing imports it).

ln x for x in (0, 1] reduces to ln f, f = x 2^-e in [sqrt(1/2), sqrt 2)
(the folded mantissa), and ln f = t + t^2 Q(t) with t = f - 1 in
[sqrt(1/2) - 1, sqrt 2 - 1].  Q is the degree-8 polynomial that minimises, in
the least-squares sense on 4000 Chebyshev nodes of that interval, the error of
t + t^2 Q(t) relative to ln(1 + t): a near-minimax fit, computed in double
precision and rounded once to FP32.  The printed hexadecimal values are the
ones the oracle uses; tests/test_oracle_transcendentals.py checks the
resulting FP32 logarithm against FP64 libm on every input the generator can
produce.

Run:  python oracle/fit_ln.py
"""
import numpy as np

DEGREE = 8
NODES = 4000


def q_true(t: np.ndarray) -> np.ndarray:
    """(ln(1 + t) - t) / t^2 in double precision: the series near 0, where
    the difference cancels, log1p elsewhere."""
    out = np.empty_like(t)
    small = np.abs(t) < 1e-3
    ts = t[small]
    # -1/2 + t/3 - t^2/4 + t^3/5 - t^4/6 (the next term is below 1e-16)
    out[small] = -0.5 + ts * (1 / 3 + ts * (-0.25 + ts * (0.2 + ts * (-1 / 6))))
    tl = t[~small]
    out[~small] = (np.log1p(tl) - tl) / (tl * tl)
    return out


def fit():
    bits_lo, bits_hi = np.uint32(0x3F3504F4), np.uint32(0x3F3504F4 + 0x7FFFFF)
    a = float(bits_lo.view(np.float32)) - 1.0
    b = float(bits_hi.view(np.float32)) - 1.0
    k = np.arange(NODES)
    t = 0.5 * (a + b) + 0.5 * (b - a) * np.cos(np.pi * (k + 0.5) / NODES)
    w = t * t / np.abs(np.log1p(t))  # error of t + t^2 Q relative to ln(1 + t)
    V = np.vander(t, DEGREE + 1, increasing=True)
    c, *_ = np.linalg.lstsq(V * w[:, None], q_true(t) * w, rcond=None)
    return c.astype(np.float32), (a, b)


if __name__ == "__main__":
    c32, (a, b) = fit()
    print(f"t in [{a:.9f}, {b:.9f}], Q(t) = sum c_i t^i:")
    for i, v in enumerate(c32):
        print(f"  c{i} = {float(v).hex()}")
