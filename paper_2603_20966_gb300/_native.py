"""ctypes binding of ``libsketch.so`` (the C ABI in include/sketch.h).

Argument marshalling only: every step of the sketch runs in the library's
CUDA kernels.  The functions keep the C names; tensors may be passed where
the C ABI takes pointers (their ``data_ptr()`` is used) and a torch stream
where it takes a ``cudaStream_t``.  The library is loaded on first use; if
it is missing or stale every call raises ImportError -- there is no
fallback path.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsketch.so")

SK_OK, SK_EINVAL, SK_ENOMEM, SK_ECUDA, SK_ETIMEOUT, SK_EBUDGET, SK_EUNSUPPORTED, SK_EBUSY, \
    SK_ECANCELLED = range(9)
SK_GAUSSIAN, SK_RADEMACHER, SK_UNIFORM = 0, 1, 2
SK_FP32, SK_BF16X2, SK_FP8E4M3 = 0, 1, 2

# C prototypes: name -> (restype, argtypes)
_i64, _u64, _int, _vp, _sz = ctypes.c_int64, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p, \
    ctypes.c_size_t
_P = ctypes.POINTER
PROTOTYPES = {
    "sk_create": (_int, [_u64, _int, _i64, _P(_vp)]),
    "sk_set_precision": (_int, [_vp, _int]),
    "sk_get_info": (_int, [_vp, _P(_u64), _P(_int), _P(_i64), _P(_int), _P(ctypes.c_float)]),
    "sk_apply_left": (_int, [_vp, _vp, _i64, _i64, _i64, _vp, _i64, _vp]),
    "sk_apply_right": (_int, [_vp, _vp, _i64, _i64, _i64, _vp, _i64, _vp]),
    "sk_apply_left_noalloc": (_int, [_vp, _vp, _i64, _i64, _i64, _vp, _i64, _vp]),
    "sk_apply_left_host": (_int, [_vp, _vp, _i64, _i64, _i64, _vp, _i64, _vp]),
    "sk_apply_right_host": (_int, [_vp, _vp, _i64, _i64, _i64, _vp, _i64, _vp]),
    "sk_materialize": (_int, [_vp, _i64, _i64, _i64, _i64, _int, _int, _vp, _i64, _vp]),
    "sk_workspace_size": (_int, [_vp, _int, _i64, _i64, _P(_sz)]),
    "sk_set_workspace": (_int, [_vp, _vp, _sz]),
    "sk_stream_status": (_int, [_vp, _vp]),
    "sk_debug_status": (_int, [_vp, _vp, _P(ctypes.c_int32)]),
    "sk_debug_set_wait": (_int, [_vp, _u64, _i64]),
    "sk_batch_create": (_int, [_P(_vp)]),
    "sk_batch_add": (_int, [_vp, _vp, _vp, _i64, _i64, _i64, _vp, _i64]),
    "sk_batch_run": (_int, [_vp, _vp]),
    "sk_batch_tune": (_int, [_vp, _vp, _P(_i64)]),
    "sk_batch_set_config": (_int, [_vp, _i64, ctypes.c_int32, ctypes.c_int32]),
    "sk_batch_config": (_int, [_vp, _P(_i64), _P(ctypes.c_int32), _P(ctypes.c_int32)]),
    "sk_batch_status": (_int, [_vp, _vp]),
    "sk_batch_size": (_int, [_vp, _P(_i64)]),
    "sk_batch_destroy": (_int, [_vp]),
    "sk_apply_left_stored": (_int, [_vp, _vp, _i64, _vp, _i64, _i64, _i64, _vp, _i64, _vp]),
    "sk_nystrom": (_int, [_vp, _vp, _i64, _i64, _vp, _i64, _vp, _i64, _vp]),
    "sk_quantize_e4m3": (_int, [_vp, _i64, _i64, _i64, _vp, _i64, _vp, _vp]),
    "sk_apply_right_e4m3": (_int, [_vp, _vp, _vp, _i64, _i64, _i64, _vp, _i64, _vp]),
    "sk_server_create": (_int, [_u64, ctypes.c_int32, _P(_vp)]),
    "sk_server_submit": (_int, [_vp, _vp, _vp, _i64, _i64, _i64, _vp, _P(_i64)]),
    "sk_server_poll": (_int, [_vp, _i64, _P(ctypes.c_double)]),
    "sk_server_wait": (_int, [_vp, _i64, ctypes.c_double, _P(ctypes.c_double)]),
    "sk_server_fetch": (_int, [_vp, _i64, _vp, _i64, _vp]),
    "sk_server_release": (_int, [_vp, _i64]),
    "sk_server_stats_get": (_int, [_vp, _vp]),
    "sk_server_reset_stats": (_int, [_vp]),
    "sk_server_destroy": (_int, [_vp]),
    "sk_destroy": (_int, [_vp]),
    "sk_profile_events": (_int, [_vp, _vp, _vp]),
    "sk_launch_count": (ctypes.c_uint64, []),
    "sk_status_string": (ctypes.c_char_p, [_int]),
    "sk_last_cuda_error": (ctypes.c_char_p, []),
    "sk_version": (_int, []),
}


class SketchError(RuntimeError):
    def __init__(self, fn: str, status: int):
        self.status = status
        detail = ""
        if status in (SK_ECUDA, SK_ENOMEM):
            detail = f" ({_lib.sk_last_cuda_error().decode()})"
        super().__init__(f"{fn}: {status_string(status)}{detail}")


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -m paper_2603_20966_gb300.build` (no CPU fallback exists)")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in PROTOTYPES.items():
        try:
            f = getattr(lib, name)
        except AttributeError as e:
            raise ImportError(f"{LIB_PATH} lacks {name}: rebuild it") from e
        f.restype = res
        f.argtypes = args
    return lib


class _Lazy:
    """Loads libsketch.so on first attribute access."""
    _lib = None

    def __getattr__(self, name):
        if _Lazy._lib is None:
            _Lazy._lib = _load()
        return getattr(_Lazy._lib, name)


_lib = _Lazy()


def lib():
    if _Lazy._lib is None:
        _Lazy._lib = _load()
    return _Lazy._lib


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream  # torch.cuda.Stream


def _check(fn, st):
    if st != SK_OK:
        raise SketchError(fn, st)


def status_string(status: int) -> str:
    return _lib.sk_status_string(int(status)).decode()


def sk_version() -> int:
    return _lib.sk_version()


def sk_create(seed: int, dist: int, k: int) -> int:
    h = ctypes.c_void_p()
    _check("sk_create", _lib.sk_create(int(seed) & (2**64 - 1), int(dist), int(k),
                                       ctypes.byref(h)))
    return h.value


def sk_set_precision(h: int, precision: int) -> None:
    _check("sk_set_precision", _lib.sk_set_precision(h, int(precision)))


def sk_get_info(h: int) -> dict:
    seed, dist, k, prec, scale = (ctypes.c_uint64(), ctypes.c_int(), ctypes.c_int64(),
                                  ctypes.c_int(), ctypes.c_float())
    _check("sk_get_info", _lib.sk_get_info(h, ctypes.byref(seed), ctypes.byref(dist),
                                           ctypes.byref(k), ctypes.byref(prec),
                                           ctypes.byref(scale)))
    return {"seed": seed.value, "dist": dist.value, "k": k.value, "precision": prec.value,
            "scale": scale.value}


def _apply(fn, h, A, m, n, lda, Y, ldy, stream):
    _check(fn, getattr(_lib, fn)(h, _ptr(A), int(m), int(n), int(lda), _ptr(Y), int(ldy),
                                 _stream(stream)))


def sk_apply_left(h, A, m, n, lda, Y, ldy, stream=None):
    _apply("sk_apply_left", h, A, m, n, lda, Y, ldy, stream)


def sk_apply_right(h, A, m, n, lda, Y, ldy, stream=None):
    _apply("sk_apply_right", h, A, m, n, lda, Y, ldy, stream)


def sk_apply_left_noalloc(h, A, m, n, lda, Y, ldy, stream=None):
    """FP32 left sketch whose scratch is a fixed array inside the library:
    for callers that must not have this library allocate device memory."""
    _apply("sk_apply_left_noalloc", h, A, m, n, lda, Y, ldy, stream)


def sk_apply_left_stored(h, S, lds, A, m, n, lda, Y, ldy, stream=None):
    """BF16 left sketch reading a caller-stored BF16 S instead of generating
    it (the communicated-S side of the generate-vs-communicate trade)."""
    _check("sk_apply_left_stored",
           _lib.sk_apply_left_stored(h, _ptr(S), int(lds), _ptr(A), int(m), int(n), int(lda),
                                     _ptr(Y), int(ldy), _stream(stream)))


def sk_apply_left_host(h, A, m, n, lda, Y, ldy, stream=None):
    _apply("sk_apply_left_host", h, A, m, n, lda, Y, ldy, stream)


def sk_apply_right_host(h, A, m, n, lda, Y, ldy, stream=None):
    _apply("sk_apply_right_host", h, A, m, n, lda, Y, ldy, stream)


def sk_materialize(h, row0, col0, rows, cols, fmt, scaled, out, ld, stream=None):
    _check("sk_materialize", _lib.sk_materialize(h, int(row0), int(col0), int(rows), int(cols),
                                                 int(fmt), int(scaled), _ptr(out), int(ld),
                                                 _stream(stream)))


def sk_workspace_size(h, side, m, n) -> int:
    b = ctypes.c_size_t()
    _check("sk_workspace_size", _lib.sk_workspace_size(h, int(side), int(m), int(n),
                                                       ctypes.byref(b)))
    return b.value


def sk_set_workspace(h, ptr, nbytes):
    _check("sk_set_workspace", _lib.sk_set_workspace(h, _ptr(ptr), int(nbytes)))


def sk_stream_status(h, stream=None) -> int:
    return _lib.sk_stream_status(h, _stream(stream))


def sk_profile_events(h, start_event, stop_event) -> None:
    """start_event/stop_event: torch.cuda.Event (or raw cudaEvent_t ints), or None."""
    def ev(e):
        if e is None or isinstance(e, int):
            return e
        return e.cuda_event
    _check("sk_profile_events", _lib.sk_profile_events(h, ev(start_event), ev(stop_event)))


def sk_launch_count() -> int:
    return int(_lib.sk_launch_count())


def sk_debug_status(h, stream=None) -> list[int]:
    """The four device status words (status, wait site, stage, CTA); see sketch.h."""
    out = (ctypes.c_int32 * 4)()
    _check("sk_debug_status", _lib.sk_debug_status(h, _stream(stream), out))
    return list(out)


def sk_debug_set_wait(h, limit_ns: int = 0, stall_stage: int = -1) -> None:
    """Failure-injection hook of the tests: bounded-wait limit (0 = default)
    and a pipeline stage whose copy is never issued (-1 = none); see sketch.h."""
    _check("sk_debug_set_wait", _lib.sk_debug_set_wait(h, int(limit_ns), int(stall_stage)))


def sk_batch_create() -> int:
    b = ctypes.c_void_p()
    _check("sk_batch_create", _lib.sk_batch_create(ctypes.byref(b)))
    return b.value


def sk_batch_add(b, h, A, m, n, lda, Y, ldy) -> None:
    _check("sk_batch_add", _lib.sk_batch_add(b, h, _ptr(A), int(m), int(n), int(lda), _ptr(Y),
                                             int(ldy)))


def sk_batch_run(b, stream=None) -> None:
    _check("sk_batch_run", _lib.sk_batch_run(b, _stream(stream)))


def sk_batch_tune(b, stream=None) -> int:
    c = ctypes.c_int64()
    _check("sk_batch_tune", _lib.sk_batch_tune(b, _stream(stream), ctypes.byref(c)))
    return c.value


def sk_batch_set_config(b, item_stages, tile_cols, ring_stages) -> None:
    _check("sk_batch_set_config",
           _lib.sk_batch_set_config(b, int(item_stages), int(tile_cols), int(ring_stages)))


def sk_batch_config(b) -> dict:
    t, c, r = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
    _check("sk_batch_config",
           _lib.sk_batch_config(b, ctypes.byref(t), ctypes.byref(c), ctypes.byref(r)))
    return {"item_stages": t.value, "tile_cols": c.value, "ring_stages": r.value}


def sk_batch_status(b, stream=None) -> int:
    return _lib.sk_batch_status(b, _stream(stream))


def sk_batch_size(b) -> int:
    c = ctypes.c_int64()
    _check("sk_batch_size", _lib.sk_batch_size(b, ctypes.byref(c)))
    return c.value


def sk_batch_destroy(b) -> None:
    _check("sk_batch_destroy", _lib.sk_batch_destroy(b))


def sk_destroy(h) -> None:
    _check("sk_destroy", _lib.sk_destroy(h))


class ServerStats(ctypes.Structure):
    """Mirror of ``sk_server_stats``."""
    _fields_ = [
        ("submitted", _i64), ("completed", _i64), ("failed", _i64), ("pending", _i64),
        ("resident", _i64), ("steps", _i64), ("max_step_requests", _i64),
        ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
        ("max_ms", ctypes.c_double), ("mean_wait_ms", ctypes.c_double),
        ("flops", ctypes.c_double), ("busy_s", ctypes.c_double),
        ("pool_bytes", _u64), ("peak_bytes", _u64),
    ]


def sk_server_create(hbm_budget_bytes: int, max_slots: int) -> int:
    s = ctypes.c_void_p()
    _check("sk_server_create", _lib.sk_server_create(int(hbm_budget_bytes), int(max_slots),
                                                     ctypes.byref(s)))
    return s.value


def sk_server_submit(s, h, A, m, n, lda, stream=None) -> int:
    """`stream`: the stream producing A (the copy of A waits for it)."""
    t = ctypes.c_int64()
    _check("sk_server_submit", _lib.sk_server_submit(s, h, _ptr(A), int(m), int(n), int(lda),
                                                     _stream(stream), ctypes.byref(t)))
    return t.value


def sk_server_poll(s, ticket) -> tuple[int, float]:
    """(status, latency_ms): SK_OK when done, SK_EBUSY while pending or running."""
    lat = ctypes.c_double(0.0)
    st = _lib.sk_server_poll(s, int(ticket), ctypes.byref(lat))
    return st, lat.value


def sk_server_wait(s, ticket, timeout_s: float) -> tuple[int, float]:
    lat = ctypes.c_double(0.0)
    st = _lib.sk_server_wait(s, int(ticket), float(timeout_s), ctypes.byref(lat))
    return st, lat.value


def sk_server_fetch(s, ticket, Y, ldy, stream=None) -> None:
    """Copy Y out on `stream` (after the work queued there) and release it."""
    _check("sk_server_fetch", _lib.sk_server_fetch(s, int(ticket), _ptr(Y), int(ldy),
                                                   _stream(stream)))


def sk_server_release(s, ticket) -> None:
    _check("sk_server_release", _lib.sk_server_release(s, int(ticket)))


def sk_server_stats_get(s) -> dict:
    out = ServerStats()
    _check("sk_server_stats_get", _lib.sk_server_stats_get(s, ctypes.byref(out)))
    return {name: getattr(out, name) for name, _ in ServerStats._fields_}


def sk_server_reset_stats(s) -> None:
    _check("sk_server_reset_stats", _lib.sk_server_reset_stats(s))


def sk_server_destroy(s) -> None:
    _check("sk_server_destroy", _lib.sk_server_destroy(s))


def sk_quantize_e4m3(A, m, n, lda, Aq, ldq, row_exp, stream=None) -> None:
    _check("sk_quantize_e4m3", _lib.sk_quantize_e4m3(_ptr(A), int(m), int(n), int(lda), _ptr(Aq),
                                                     int(ldq), _ptr(row_exp), _stream(stream)))


def sk_apply_right_e4m3(h, Aq, row_exp, m, n, ldq, Y, ldy, stream=None) -> None:
    _check("sk_apply_right_e4m3", _lib.sk_apply_right_e4m3(h, _ptr(Aq), _ptr(row_exp), int(m),
                                                           int(n), int(ldq), _ptr(Y), int(ldy),
                                                           _stream(stream)))


def sk_nystrom(h, A, n, lda, B, ldb, C, ldc, stream=None) -> None:
    """B = A Omega, C = Omega^T B (see sketch.h)."""
    _check("sk_nystrom", _lib.sk_nystrom(h, _ptr(A), int(n), int(lda), _ptr(B), int(ldb), _ptr(C),
                                         int(ldc), _stream(stream)))
