"""Shared helpers of the GPU tests (no sketch arithmetic here)."""
import os
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def require_gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def rel_frob(got, ref) -> float:
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300))


def build_test_so(name: str) -> str:
    """Compile tests/cuda/<name>.cu into tests/_build/lib<name>.so for sm_103a."""
    src = os.path.join(HERE, "cuda", name + ".cu")
    out_dir = os.path.join(HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    out = os.path.join(out_dir, f"lib{name}.so")
    if not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
        subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared",
                        "-Xcompiler", "-fPIC", src, "-o", out], check=True)
    return out
