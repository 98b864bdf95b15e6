"""The allocation-free left sketch (sk_apply_left_noalloc) gives the same Y as
the allocating entry point sk_apply_left.

It exists for callers that must not have this library allocate device
memory: applications whose HBM is owned by another allocator, or
latency-critical paths that cannot absorb cudaMalloc/cudaFree
synchronisation.  Its split-K scratch is a fixed array inside the library.
This file is collected last on purpose, so that a stop-at-first-failure run
has executed every other test before it."""
import ctypes

import numpy as np
import pytest
import torch

from gpu_util import rel_frob, require_gpu

pytestmark = pytest.mark.gpu

TOL = 1e-5  # the FP32-form tolerance used by the other parity tests


def _raw_noalloc(N, h, A, m, n, Y, stream):
    # straight through the C ABI symbol
    return N.lib().sk_apply_left_noalloc(h, A.data_ptr(), m, n, A.stride(0), Y.data_ptr(),
                                         Y.stride(0), stream.cuda_stream)


def test_noalloc_matches_allocating_entry_point_twice_in_a_row():
    require_gpu()
    from paper_2603_20966_gb300 import _native as N
    from paper_2603_20966_gb300.workloads import gaussian_matrix
    stream = torch.cuda.current_stream()
    cases = [(7, N.SK_GAUSSIAN, 64, 20000, 96), (9, N.SK_RADEMACHER, 48, 33333, 130)]
    for i, (seed, dist, k, m, n) in enumerate(cases):
        A = gaussian_matrix(m, n, 100 + i, device="cuda")
        h = N.sk_create(seed, dist, k)
        try:
            assert N.sk_workspace_size(h, 0, m, n) > 0  # the split-K scratch is exercised
            Y_ref = torch.full((k, n), float("nan"), device="cuda")
            N.sk_apply_left(h, A, m, n, n, Y_ref, n, stream)
            Y = torch.full((k, n), float("nan"), device="cuda")
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info()[0]
            assert _raw_noalloc(N, h, A, m, n, Y, stream) == N.SK_OK
            torch.cuda.synchronize()
            free_after = torch.cuda.mem_get_info()[0]
            assert N.sk_stream_status(h, stream) == N.SK_OK
        finally:
            N.sk_destroy(h)
        if i > 0:
            assert free_after == free_before  # no device allocation by the call
        got, ref = Y.cpu().numpy(), Y_ref.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert rel_frob(got, ref) <= TOL


def test_noalloc_rejects_problems_beyond_its_scratch():
    require_gpu()
    from paper_2603_20966_gb300 import _native as N
    k, m, n = 2048, 1 << 16, 512
    h = N.sk_create(1, N.SK_GAUSSIAN, k)
    try:
        assert N.sk_workspace_size(h, 0, m, n) > (16 << 20)
        A = torch.zeros((m, n), device="cuda")
        Y = torch.zeros((k, n), device="cuda")
        st = _raw_noalloc(N, h, A, m, n, Y, torch.cuda.current_stream())
        assert st == N.SK_EUNSUPPORTED
        N.sk_set_precision(h, N.SK_BF16X2)
        small = torch.zeros((64, 64), device="cuda")
        assert N.lib().sk_apply_left_noalloc(h, small.data_ptr(), 64, 64, 64, small.data_ptr(),
                                             64, None) == N.SK_EUNSUPPORTED
    finally:
        N.sk_destroy(h)


def test_noalloc_cuda_error_is_reported_like_every_other_entry_point():
    """A CUDA failure inside the allocation-free call comes back as SK_ECUDA
    with sk_last_cuda_error describing it, as for the allocating call.  The
    failure used is one CUDA detects on the host before anything runs: in the
    FP32 form a sketch size k above 65535 tiles of 256 rows (n <= 128) is a
    launch grid CUDA refuses."""
    require_gpu()
    from paper_2603_20966_gb300 import _native as N
    L = N.lib()
    k, m, n = 65536 * 256, 32, 4
    h = N.sk_create(3, N.SK_GAUSSIAN, k)
    try:
        A = torch.zeros((m, n), device="cuda")
        Y = torch.zeros((k, n), device="cuda")
        stream = torch.cuda.current_stream()
        assert N.sk_workspace_size(h, 0, m, n) == 0  # within the array's limit
        st = L.sk_apply_left_noalloc(h, A.data_ptr(), m, n, n, Y.data_ptr(), n,
                                     stream.cuda_stream)
        assert st == N.SK_ECUDA
        msg = L.sk_last_cuda_error().decode()
        assert msg != "no error"  # the launch's CUDA error, described
        # the allocating entry point reports the same failure the same way
        assert L.sk_apply_left(h, A.data_ptr(), m, n, n, Y.data_ptr(), n,
                               stream.cuda_stream) == N.SK_ECUDA
        assert L.sk_last_cuda_error().decode() == msg
        # the error is not sticky: the context still runs work, and a later
        # successful call leaves the description of the last failure in place
        k2, m2 = 64, 4096
        h2 = N.sk_create(5, N.SK_GAUSSIAN, k2)
        try:
            A2 = torch.randn((m2, n), device="cuda")
            Y2 = torch.full((k2, n), float("nan"), device="cuda")
            Y2_ref = torch.empty((k2, n), device="cuda")
            N.sk_apply_left(h2, A2, m2, n, n, Y2_ref, n, stream)
            assert _raw_noalloc(N, h2, A2, m2, n, Y2, stream) == N.SK_OK
            assert N.sk_stream_status(h2, stream) == N.SK_OK
            assert L.sk_last_cuda_error().decode() == msg
            assert rel_frob(Y2.cpu().numpy(), Y2_ref.cpu().numpy()) <= TOL
        finally:
            N.sk_destroy(h2)
    finally:
        N.sk_destroy(h)
