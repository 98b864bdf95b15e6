"""Failure detection on the GPU without a fault: a bounded device wait that
runs out.

The test-only hook sk_debug_set_wait shortens the wait limit of a handle and
makes the TMA producer of the BF16 left sketch issue no copy for one pipeline
stage, so the waits that depend on that stage can never complete.  The
kernel must give up after the limit, record SK_ETIMEOUT and the waiting site,
wait (bounded) for its own copies and MMAs in flight, free its tensor memory
and exit; the context stays usable, and the next normal call on the same
handle and stream is correct against the oracle."""
import time

import numpy as np
import pytest
import torch

from gpu_util import rel_frob, require_gpu

pytestmark = pytest.mark.gpu

G = 0
TOL = 1e-5
LIMIT_NS = 20_000_000  # 20 ms: a healthy stage of these sizes takes microseconds

# Wait sites (role * 16 + barrier) that depend on the stage whose copy is never
# issued: the MMA issuer waiting for that stage's operands (0x22), a worker
# waiting for its A tile (0x40; one CTA), an epilogue warp waiting for the A
# tile it splits in place (0x30; Gaussian sketches on CTA pairs) or for the
# accumulation chain that needs it (0x34), the TMA producer or a worker
# waiting for a ring slot that stage holds (0x13, 0x43).
DEPENDENT_SITES = {0x22, 0x40, 0x30, 0x34, 0x13, 0x43}


@pytest.fixture(scope="module")
def P():
    require_gpu()
    import paper_2603_20966_gb300 as P
    return P


def _sketch(P, h, A, m, n, k, stream):
    Y = torch.full((k, n), float("nan"), dtype=torch.float32, device="cuda")
    P.sk_apply_left(h, A, m, n, n, Y, n, stream)
    return Y


@pytest.mark.parametrize("k", [64, 256])  # one CTA (cta_group::1); CTA pairs (cta_group::2)
def test_bounded_wait_gives_up_and_the_handle_recovers(P, orc, k):
    from paper_2603_20966_gb300.workloads import gaussian_matrix
    m, n, seed, stall = 4096, 96, 7, 1
    A_cpu = gaussian_matrix(m, n, 31, device="cpu")
    A = A_cpu.cuda()
    ref = orc.apply_left(seed, G, 1, k, A_cpu.numpy())
    stream = torch.cuda.current_stream()
    h = P.sk_create(seed, G, k)
    try:
        P.sk_set_precision(h, P.SK_BF16X2)
        Y = _sketch(P, h, A, m, n, k, stream)
        assert P.sk_stream_status(h, stream) == 0
        assert rel_frob(Y.cpu().numpy(), ref) <= TOL

        P.sk_debug_set_wait(h, LIMIT_NS, stall)
        t0 = time.perf_counter()
        _sketch(P, h, A, m, n, k, stream)  # enqueued; the kernel gives up on the device
        words = P.sk_debug_status(h, stream)  # synchronises the stream
        elapsed = time.perf_counter() - t0
        assert words[0] == 4, words  # SK_ETIMEOUT
        assert words[1] in DEPENDENT_SITES, hex(words[1])
        if words[1] in (0x22, 0x40, 0x30):
            assert words[2] == stall, words
        assert words[3] >= 0
        assert elapsed < 5.0, elapsed  # the limit plus bounded drains, not a hang
        assert P.sk_stream_status(h, stream) == 4  # reported once, then cleared
        assert P.sk_debug_status(h, stream)[0] == 0

        # the injection off again: same handle, same stream, correct result
        P.sk_debug_set_wait(h, 0, -1)
        for _ in range(2):
            Y = _sketch(P, h, A, m, n, k, stream)
            assert P.sk_stream_status(h, stream) == 0
            got = Y.cpu().numpy()
            assert np.all(np.isfinite(got))
            assert rel_frob(got, ref) <= TOL
    finally:
        P.sk_destroy(h)


def test_wait_limit_arguments(P):
    h = P.sk_create(1, G, 64)
    try:
        with pytest.raises(P.SketchError):
            P.sk_debug_set_wait(h, 1000, -1)  # below 1 ms
        P.sk_debug_set_wait(h, 0, -1)
    finally:
        P.sk_destroy(h)
