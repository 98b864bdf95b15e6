"""GPU parity of batched left sketches (sk_batch_*): one persistent launch
over problems of uneven m, n, k and distribution, each member within 1e-5 of
the FP64 oracle, bit-identical alone and in the mix, repeatable, and still
correct after the autotuner chose its decomposition."""
import numpy as np
import pytest
import torch

from gpu_util import rel_frob, require_gpu

pytestmark = pytest.mark.gpu

BF16 = 1
TOL = 1e-5


@pytest.fixture(scope="module")
def P():
    require_gpu()
    import paper_2603_20966_gb300 as P
    return P


# (m, n, k, dist, seed): a small cross-section of the batched workload
PROBS = [(1024, 32, 64, 0, 1000), (5000, 100, 200, 1, 1001), (20000, 512, 1024, 0, 1002),
         (3000, 300, 600, 1, 1003), (65536, 48, 96, 0, 1004), (1500, 257, 514, 0, 1005),
         (12345, 64, 128, 1, 1006), (4096, 511, 1022, 1, 1007)]


def _make(P, probs, seeds_a=7):
    from paper_2603_20966_gb300.workloads import gaussian_matrix
    data = []
    for i, (m, n, k, dist, seed) in enumerate(probs):
        lda = (n + 3) // 4 * 4
        A = torch.zeros((m, lda), device="cuda")
        A[:, :n] = gaussian_matrix(m, n, seeds_a + i, device="cuda")
        Y = torch.full((k, lda), float("nan"), device="cuda")
        h = P.sk_create(seed, dist, k)
        P.sk_set_precision(h, BF16)
        data.append(dict(m=m, n=n, k=k, dist=dist, seed=seed, A=A, Y=Y, h=h, lda=lda))
    return data


_STREAM = None


def _stream():
    # a created stream, so that runs go through the captured graph
    global _STREAM
    if _STREAM is None:
        _STREAM = torch.cuda.Stream()
    return _STREAM


def _batch(P, data, tune=False):
    b = P.sk_batch_create()
    for d in data:
        P.sk_batch_add(b, d["h"], d["A"], d["m"], d["n"], d["lda"], d["Y"], d["lda"])
    torch.cuda.synchronize()
    chosen = P.sk_batch_tune(b, _stream()) if tune else None
    P.sk_batch_run(b, _stream())
    assert P.sk_batch_status(b, _stream()) == 0
    return b, chosen


def _free(P, data, b):
    P.sk_batch_destroy(b)
    for d in data:
        P.sk_destroy(d["h"])


def test_batch_matches_oracle(P, orc):
    data = _make(P, PROBS)
    b, _ = _batch(P, data)
    try:
        assert P.sk_batch_size(b) == len(PROBS)
        for d in data:
            got = d["Y"][:, :d["n"]].cpu().numpy()
            assert np.all(np.isfinite(got))
            A = d["A"][:, :d["n"]].cpu().numpy()
            ref = orc.apply_left(d["seed"], d["dist"], BF16, d["k"], A)
            assert rel_frob(got, ref) <= TOL, (d["m"], d["n"], d["k"], d["dist"])
    finally:
        _free(P, data, b)


def test_alone_equals_in_the_mix_and_repeatable(P):
    data = _make(P, PROBS)
    b, _ = _batch(P, data)
    mix = [d["Y"][:, :d["n"]].clone() for d in data]
    P.sk_batch_run(b, _stream())  # graph replay
    assert P.sk_batch_status(b, _stream()) == 0
    for d, y in zip(data, mix):
        assert torch.equal(d["Y"][:, :d["n"]], y)
    _free(P, data, b)
    for i in (0, 2, 4):
        alone = _make(P, [PROBS[i]], seeds_a=7 + i)
        b1, _ = _batch(P, alone)
        assert torch.equal(alone[0]["Y"][:, :alone[0]["n"]], mix[i]), i
        _free(P, alone, b1)


def test_batch_agrees_with_single_calls(P):
    data = _make(P, PROBS[:4])
    b, _ = _batch(P, data)
    try:
        for d in data:
            Y1 = torch.empty_like(d["Y"])
            P.sk_apply_left(d["h"], d["A"], d["m"], d["n"], d["lda"], Y1, d["lda"])
            assert P.sk_stream_status(d["h"]) == 0
            assert rel_frob(Y1[:, :d["n"]].cpu().numpy(),
                            d["Y"][:, :d["n"]].cpu().numpy()) <= 2 * TOL
    finally:
        _free(P, data, b)


# (item stages, tile columns, ring stages): the kernel configurations the
# autotuner chooses from
CONFIGS = [(512, 512, 4), (256, 256, 4), (1024, 256, 8)]


def _batch_cfg(P, data, cfg):
    b = P.sk_batch_create()
    for d in data:
        P.sk_batch_add(b, d["h"], d["A"], d["m"], d["n"], d["lda"], d["Y"], d["lda"])
    P.sk_batch_set_config(b, *cfg)
    assert P.sk_batch_config(b) == dict(zip(("item_stages", "tile_cols", "ring_stages"), cfg))
    P.sk_batch_run(b, _stream())
    assert P.sk_batch_status(b, _stream()) == 0
    return b


@pytest.mark.parametrize("cfg", CONFIGS)
def test_every_configuration_matches_oracle(P, orc, cfg):
    data = _make(P, PROBS)
    b = _batch_cfg(P, data, cfg)
    try:
        for d in data:
            A = d["A"][:, :d["n"]].cpu().numpy()
            ref = orc.apply_left(d["seed"], d["dist"], BF16, d["k"], A)
            assert rel_frob(d["Y"][:, :d["n"]].cpu().numpy(), ref) <= TOL, (cfg, d["n"])
        mix = [d["Y"][:, :d["n"]].clone() for d in data]
    finally:
        _free(P, data, b)
    # the same configuration alone gives the same bits
    for i in (1, 2):
        alone = _make(P, [PROBS[i]], seeds_a=7 + i)
        b1 = _batch_cfg(P, alone, cfg)
        assert torch.equal(alone[0]["Y"][:, :alone[0]["n"]], mix[i]), (cfg, i)
        _free(P, alone, b1)


def test_set_config_rejects_bad_values(P):
    b = P.sk_batch_create()
    try:
        for bad in [(0, 512, 4), (512, 384, 4), (512, 512, 5), (512, 512, 8)]:
            with pytest.raises(P.SketchError):
                P.sk_batch_set_config(b, *bad)
        assert P.sk_batch_config(b) == {"item_stages": 512, "tile_cols": 512, "ring_stages": 4}
    finally:
        P.sk_batch_destroy(b)


def test_autotune_then_correct(P, orc, tmp_path, monkeypatch):
    monkeypatch.setenv("SK_TUNE_CACHE", str(tmp_path / "tune.json"))
    data = _make(P, PROBS[:5])
    b, chosen = _batch(P, data, tune=True)
    try:
        assert chosen in (128, 256, 512, 1024, 2048, 4096)
        cfg = P.sk_batch_config(b)
        assert cfg["item_stages"] == chosen
        assert cfg["tile_cols"] in (256, 512) and cfg["ring_stages"] in (4, 8)
        assert cfg["ring_stages"] == 4 or cfg["tile_cols"] == 256
        assert (tmp_path / "tune.json").exists()
        for d in data:
            A = d["A"][:, :d["n"]].cpu().numpy()
            ref = orc.apply_left(d["seed"], d["dist"], BF16, d["k"], A)
            assert rel_frob(d["Y"][:, :d["n"]].cpu().numpy(), ref) <= TOL
    finally:
        _free(P, data, b)


def test_batch_rejects_bad_members(P):
    b = P.sk_batch_create()
    h = P.sk_create(1, 0, 64)
    A = torch.zeros((100, 64), device="cuda")
    Y = torch.zeros((64, 64), device="cuda")
    try:
        with pytest.raises(P.SketchError):   # FP32 form is not batched
            P.sk_batch_add(b, h, A, 100, 64, 64, Y, 64)
        P.sk_set_precision(h, BF16)
        with pytest.raises(P.SketchError):   # lda not a multiple of 4
            P.sk_batch_add(b, h, A, 100, 63, 63, Y, 64)
        with pytest.raises(P.SketchError):   # empty batch
            P.sk_batch_run(b)
        P.sk_batch_add(b, h, A, 100, 64, 64, Y, 64)
        P.sk_batch_run(b)                    # legacy default stream: direct launches
        assert P.sk_batch_status(b) == 0
    finally:
        P.sk_destroy(h)
        P.sk_batch_destroy(b)
