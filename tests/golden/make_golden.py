"""Writes tests/golden/generator_samples.txt from the oracle alone.

The file freezes a few generated entries g(r, c) (FP32 bit patterns) and the
Philox words behind them, so that any later change to the generator
specification (key/counter layout, Box-Muller mapping, Rademacher bit order,
the own ln and circle map) is visible as a diff.  Values come only from oracle/;
the Philox words are the ones pinned to cuRAND's host generator by
tests/test_oracle_philox.py.

Run:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
import oracle  # noqa: E402

CASES = [
    # seed, dist, prec, row, col
    (7, 0, 0, 0, 0), (7, 0, 0, 0, 1), (7, 0, 0, 0, 2), (7, 0, 0, 0, 3),
    (7, 0, 0, 63, 4095), (7, 0, 1, 5, 17), (7, 0, 2, 5, 17),
    (0x0123456789ABCDEF, 0, 0, 2047, 1048575), (1, 0, 0, 4294967295, 4294967295),
    (7, 1, 0, 0, 0), (7, 1, 0, 0, 127), (7, 1, 0, 3, 1000), (7, 1, 2, 2047, 1048575),
    (11, 2, 0, 0, 0), (11, 2, 0, 9, 4097),
]


def main():
    lines = ["# seed dist prec row col value_f32_hex  (dist 0=Gaussian 1=Rademacher 2=uniform;"
             " prec 0=FP32 1=BF16 2=E4M3; value unscaled)"]
    for seed, dist, prec, r, c in CASES:
        v = oracle.generate(seed, dist, prec, r, c, 1, 1)[0, 0]
        lines.append(f"{seed} {dist} {prec} {r} {c} {np.float32(v).view(np.uint32):08x}")
    lines.append("# philox: key0 key1 c0 c1 c2 c3 -> x0 x1 x2 x3")
    for key, ctr in [((7, 0), (0, 0, 0, 0)), ((7, 0), (1023, 63, 0, 0)),
                     ((0x89ABCDEF, 0x01234567), (262143, 2047, 0, 0)),
                     ((0xFFFFFFFF, 0xFFFFFFFF), (0xFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF))]:
        x = oracle.philox4x32_10(np.array([ctr], np.uint32), key)[0]
        lines.append(" ".join(f"{v:08x}" for v in (*key, *ctr)) + " -> " +
                     " ".join(f"{v:08x}" for v in x))
    with open(os.path.join(HERE, "generator_samples.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
