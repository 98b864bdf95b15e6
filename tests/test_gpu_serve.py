"""GPU tests of the request server (sk_server_*): results within 1e-5 of the
FP64 oracle for both forms, bit-identical alone and in a concurrent mix,
admission bounded by the HBM budget and the slot count, oversize requests
rejected, early release, host-resident inputs."""
import threading
import time

import numpy as np
import pytest
import torch

from gpu_util import rel_frob, require_gpu

pytestmark = pytest.mark.gpu

FP32, BF16 = 0, 1
TOL = 1e-5
MB = 1 << 20


@pytest.fixture(scope="module")
def P():
    require_gpu()
    import paper_2603_20966_gb300 as P
    return P


# (m, n, k, dist, seed, form): uneven shapes, both distributions, both forms
REQS = [(1024, 32, 64, 0, 1000, BF16), (5000, 100, 200, 1, 1001, BF16),
        (20000, 256, 512, 0, 1002, BF16), (3000, 37, 74, 1, 1003, FP32),
        (65536, 48, 96, 0, 1004, BF16), (1500, 257, 514, 0, 1005, FP32),
        (12345, 64, 128, 1, 1006, BF16), (4096, 131, 262, 1, 1007, BF16),
        (777, 5, 10, 0, 1008, FP32), (30000, 96, 192, 1, 1009, BF16)]


def _inputs(reqs, base_seed=40):
    from paper_2603_20966_gb300.workloads import gaussian_matrix
    # no synchronisation: each submission records an event on torch's stream
    return [gaussian_matrix(m, n, base_seed + i, device="cuda")
            for i, (m, n, *_rest) in enumerate(reqs)]


def _handles(P, reqs):
    hs = []
    for (m, n, k, dist, seed, form) in reqs:
        h = P.sk_create(seed, dist, k)
        if form != FP32:
            P.sk_set_precision(h, form)
        hs.append(h)
    return hs


def _fetch(P, srv, t, k, n):
    st, _ = P.sk_server_wait(srv, t, 60.0)
    assert st == 0, P.status_string(st)
    # the NaN fill is still queued on torch's stream: the copy is ordered after it
    Y = torch.full((k, n), float("nan"), device="cuda")
    P.sk_server_fetch(srv, t, Y, n, torch.cuda.current_stream())
    return Y


def test_server_matches_oracle(P, orc):
    As = _inputs(REQS)
    hs = _handles(P, REQS)
    srv = P.sk_server_create(2 << 30, 64)
    try:
        ts = [P.sk_server_submit(srv, h, A, A.shape[0], A.shape[1], A.stride(0))
              for h, A in zip(hs, As)]
        for t, A, (m, n, k, dist, seed, form) in zip(ts, As, REQS):
            Y = _fetch(P, srv, t, k, n)
            ref = orc.apply_left(seed, dist, form, k, A.cpu().numpy())
            assert rel_frob(Y.cpu().numpy(), ref) <= TOL, (m, n, k, dist, form)
        s = P.sk_server_stats_get(srv)
        assert s["completed"] == len(REQS) and s["failed"] == 0
        assert s["resident"] == 0 and s["pending"] == 0
        assert 0 < s["p50_ms"] <= s["p99_ms"] <= s["max_ms"]
        want = sum(2.0 * k * m * n for (m, n, k, *_r) in REQS)
        assert abs(s["flops"] - want) <= 1e-9 * want
    finally:
        P.sk_server_destroy(srv)
        for h in hs:
            P.sk_destroy(h)


def test_alone_equals_in_the_mix(P):
    As = _inputs(REQS)
    hs = _handles(P, REQS)
    srv = P.sk_server_create(2 << 30, 64)
    try:
        alone = []
        for h, A, (m, n, k, *_r) in zip(hs, As, REQS):
            t = P.sk_server_submit(srv, h, A, m, n, A.stride(0))
            alone.append(_fetch(P, srv, t, k, n))
        assert P.sk_server_stats_get(srv)["max_step_requests"] == 1
        # the mix: everything at once, in another order, with repeats, and a
        # second wave submitted from another thread while the first runs
        order = [4, 0, 9, 2, 7, 1, 3, 5, 8, 6, 2, 4]
        wave1 = [(i, P.sk_server_submit(srv, hs[i], As[i], *As[i].shape, As[i].stride(0)))
                 for i in order]
        wave2 = []

        def second_wave():
            for i in reversed(order):
                wave2.append((i, P.sk_server_submit(srv, hs[i], As[i], *As[i].shape,
                                                    As[i].stride(0))))
                time.sleep(0.0002)

        th = threading.Thread(target=second_wave)
        th.start()
        th.join()
        for i, t in wave1 + wave2:
            m, n, k, *_r = REQS[i]
            Y = _fetch(P, srv, t, k, n)
            assert torch.equal(Y, alone[i]), (i, REQS[i])
        s = P.sk_server_stats_get(srv)
        assert s["max_step_requests"] > 1  # the burst was batched
        assert s["completed"] == len(REQS) + 2 * len(order)
    finally:
        P.sk_server_destroy(srv)
        for h in hs:
            P.sk_destroy(h)


def _footprint(m, n, k):
    ldp = (n + 3) // 4 * 4
    return 4 * ldp * (m + k)


def test_budget_and_slots_bound_admission(P, orc):
    reqs = [(40000, 128, 256, i % 2, 2000 + i, BF16) for i in range(6)]
    As = _inputs(reqs, 80)
    hs = _handles(P, reqs)
    one = _footprint(40000, 128, 256)
    # room for about two requests (A, Y and partials) at a time
    budget = int(2.6 * one)
    srv = P.sk_server_create(budget, 64)
    try:
        ts = [P.sk_server_submit(srv, h, A, *A.shape, A.stride(0)) for h, A in zip(hs, As)]
        Ys = [_fetch(P, srv, t, 256, 128) for t in ts]
        s = P.sk_server_stats_get(srv)
        assert s["peak_bytes"] <= s["pool_bytes"]
        assert s["peak_bytes"] >= one
        assert s["steps"] >= 3          # at most two resident at a time
        assert s["max_step_requests"] <= 2
        for Y, A, (m, n, k, dist, seed, form) in zip(Ys, As, reqs):
            ref = orc.apply_left(seed, dist, form, k, A.cpu().numpy())
            assert rel_frob(Y.cpu().numpy(), ref) <= TOL
    finally:
        P.sk_server_destroy(srv)
    srv = P.sk_server_create(1 << 30, 1)  # one slot: every step holds one request
    try:
        ts = [P.sk_server_submit(srv, h, A, *A.shape, A.stride(0)) for h, A in zip(hs, As)]
        for t, Y in zip(ts, Ys):
            assert torch.equal(_fetch(P, srv, t, 256, 128), Y)
        s = P.sk_server_stats_get(srv)
        assert s["steps"] == len(reqs) and s["max_step_requests"] == 1
    finally:
        P.sk_server_destroy(srv)
        for h in hs:
            P.sk_destroy(h)


def test_oversize_rejected_and_release(P):
    h = P.sk_create(5, 0, 128)
    P.sk_set_precision(h, BF16)
    A = torch.randn((70000, 64), device="cuda")
    srv = P.sk_server_create(8 * MB, 8)
    try:
        with pytest.raises(P.SketchError) as ei:   # 70000 x 64 floats > 8 MB
            P.sk_server_submit(srv, h, A, 70000, 64, 64)
        assert ei.value.status == 5  # SK_EBUDGET
        small = A[:2000]
        t = P.sk_server_submit(srv, h, small, 2000, 64, 64)
        P.sk_server_release(srv, t)        # dropped when it finishes
        t2 = P.sk_server_submit(srv, h, small, 2000, 64, 64)
        Y = _fetch(P, srv, t2, 128, 64)
        assert torch.isfinite(Y).all()
        deadline = time.time() + 30
        while P.sk_server_stats_get(srv)["resident"] and time.time() < deadline:
            time.sleep(0.01)
        s = P.sk_server_stats_get(srv)
        assert s["resident"] == 0 and s["completed"] == 2
        st, _ = P.sk_server_poll(srv, t)
        assert st == 1  # released: unknown ticket
        with pytest.raises(P.SketchError):
            P.sk_server_submit(srv, h, small, 2000, 64, 63)  # lda < n
    finally:
        P.sk_server_destroy(srv)
        P.sk_destroy(h)


def test_host_input(P, orc):
    m, n, k = 3000, 40, 80
    h = P.sk_create(9, 1, k)
    P.sk_set_precision(h, BF16)
    A = torch.randn((m, n)).pin_memory()
    srv = P.sk_server_create(256 * MB, 4)
    try:
        A_pageable = A.clone()          # not registered: copied by the copy engine
        A_dev = A.cuda()
        ts = [P.sk_server_submit(srv, h, X, m, n, n, torch.cuda.current_stream())
              for X in (A, A_pageable, A_dev)]
        Ys = []
        for t in ts:
            Yh = torch.empty((k, n)).pin_memory()
            assert P.sk_server_wait(srv, t, 60.0)[0] == 0
            P.sk_server_fetch(srv, t, Yh, n, torch.cuda.current_stream())
            Ys.append(Yh)
        ref = orc.apply_left(9, 1, BF16, k, A.numpy())
        assert rel_frob(Ys[0].numpy(), ref) <= TOL
        assert torch.equal(Ys[0], Ys[1]) and torch.equal(Ys[0], Ys[2])
    finally:
        P.sk_server_destroy(srv)
        P.sk_destroy(h)


def test_server_class(P, orc):
    from paper_2603_20966_gb300 import Server, Sketch
    A = torch.randn((9000, 72), device="cuda")
    with Sketch(11, 0, 144, precision=BF16) as sk, Server(512 * MB, 8) as srv:
        ts = [srv.submit(sk, A) for _ in range(3)]
        Ys = [srv.result(t) for t in ts]
        assert torch.equal(Ys[0], Ys[1]) and torch.equal(Ys[0], Ys[2])
        ref = orc.apply_left(11, 0, BF16, 144, A.cpu().numpy())
        assert rel_frob(Ys[0].cpu().numpy(), ref) <= TOL
        assert srv.stats()["completed"] == 3
