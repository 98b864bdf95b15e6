"""The device Box-Muller transform against the oracle on every input it can
see: a Gaussian entry depends on its Philox word pair only through
xa >> 8 (u1) and xb >> 8 (u2), 2^24 values each, and the words below run
both through all of them (in both pairs of a call, in different orders) with
arbitrary low bytes.  Together with the Philox parity tests this covers the
Gaussian generator exhaustively."""
import ctypes

import numpy as np
import pytest
import torch

from gpu_util import build_test_so, require_gpu

pytestmark = pytest.mark.gpu

N = 1 << 24


def _words():
    i = np.arange(N, dtype=np.uint64)
    w = np.empty((N, 4), dtype=np.uint32)
    w[:, 0] = ((i << 8) | (i & 0xFF)).astype(np.uint32)                   # u1 = (i + 1) 2^-24
    w[:, 1] = ((i << 8) | 0x5A).astype(np.uint32)                         # every angle word
    w[:, 2] = ((((i * 0x9E3779B1) & 0xFFFFFF) << 8) | 0xC3).astype(np.uint32)  # a permutation
    w[:, 3] = ((((~i) & 0xFFFFFF) << 8) | ((i >> 16) & 0xFF)).astype(np.uint32)
    return w


def test_device_box_muller_bit_exact_on_every_input(orc):
    require_gpu()
    lib = ctypes.CDLL(build_test_so("box_muller_all"))
    lib.box_muller_all.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    w = _words()
    assert len(np.unique(w[:, 2] >> 8)) == N and len(np.unique(w[:, 3] >> 8)) == N
    wd = torch.from_numpy(w.view(np.int32)).cuda()
    out = torch.empty((N, 4), dtype=torch.float32, device="cuda")
    assert lib.box_muller_all(wd.data_ptr(), out.data_ptr(), N) == 0
    got = out.cpu().numpy().view(np.uint32)
    ref = orc.box_muller(w.reshape(-1, 2)).reshape(N, 4).view(np.uint32)
    bad = np.nonzero((got != ref).any(axis=1))[0]
    assert bad.size == 0, f"{bad.size} mismatching calls, first words {w[bad[0]]}"
