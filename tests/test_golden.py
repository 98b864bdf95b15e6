"""The oracle still produces the frozen generator samples in
tests/golden/generator_samples.txt (written by tests/golden/make_golden.py
from the oracle; see that script)."""
import os

import numpy as np

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows():
    vals, phil = [], []
    with open(os.path.join(HERE, "generator_samples.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            if "->" in line:
                a, b = line.split("->")
                phil.append(([int(t, 16) for t in a.split()], [int(t, 16) for t in b.split()]))
            else:
                seed, dist, prec, r, c, hx = line.split()
                vals.append((int(seed), int(dist), int(prec), int(r), int(c), int(hx, 16)))
    return vals, phil


def test_generator_samples_unchanged(orc):
    vals, phil = _rows()
    assert len(vals) >= 10 and len(phil) >= 3
    for seed, dist, prec, r, c, hx in vals:
        v = orc.generate(seed, dist, prec, r, c, 1, 1)[0, 0]
        assert int(np.float32(v).view(np.uint32)) == hx, (seed, dist, prec, r, c)
    for inp, out in phil:
        got = orc.philox4x32_10(np.array([inp[2:]], np.uint32), inp[:2])[0]
        assert list(got) == out
