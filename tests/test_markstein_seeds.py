"""The device generator's square root (Markstein's correction of the
hardware reciprocal-square-root approximation) gives the IEEE result on every
radicand Box-Muller can produce, from every seed within 6 ulp:
tests/host/markstein_seeds.c, linked with the oracle's ln for the radicands.  Host-only; the GPU side is pinned exhaustively by
test_gpu_box_muller_all.py."""
import os
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_markstein_sequences_round_correctly_from_any_nearby_seed(orc, tmp_path):
    exe = str(tmp_path / "markstein_seeds")
    src = os.path.join(HERE, "host", "markstein_seeds.c")
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                    "-frounding-math", src, orc.build(), "-o", exe, "-lm"], check=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "root mismatches 0" in r.stdout
