"""CPU oracle for the random-sketch hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
product library (``paper_2603_20966_gb300``) never imports, loads or calls
it, and the two share no code.

The arithmetic lives in ``sk_oracle.c`` (plain C, FP32 generator steps exactly
as specified, FP64 accumulation); this module compiles it with gcc and wraps
it with numpy marshalling.  See the header of ``sk_oracle.c`` for what each
function computes and which passage of arXiv 2603.20966 it follows.

Every function here is pinned by ``tests/test_oracle_*.py`` against things
other than itself: cuRAND's host Philox4x32-10 generator, FP64 libm, torch
dtype casts, Box-Muller identities, moment invariants and brute-force
products on tiny inputs.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sk_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libskoracle.so")

GAUSSIAN, RADEMACHER, UNIFORM = 0, 1, 2
FP32, BF16, E4M3 = 0, 1, 2

# Flags fix IEEE single-precision semantics: no contraction of a*b+c into an
# fma unless written as fmaf, no fast-math reassociation, no x87.
CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
          "-fno-unsafe-math-optimizations", "-frounding-math", "-Wall", "-Wno-unused-function"]

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile sk_oracle.c into a shared library (idempotent)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm", "-lpthread"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            i64, u64, i32, u32 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32
            vp = ctypes.c_void_p
            L.orc_philox4x32_10.argtypes = [vp, vp, vp, i64]
            L.orc_philox4x32_10.restype = None
            L.orc_ln.argtypes = [vp, vp, i64]
            L.orc_ln.restype = None
            L.orc_sincospi_quarter.argtypes = [vp, vp, vp, i64]
            L.orc_sincospi_quarter.restype = None
            L.orc_circle.argtypes = [vp, vp, vp, i64]
            L.orc_circle.restype = None
            L.orc_box_muller.argtypes = [vp, vp, i64]
            L.orc_box_muller.restype = None
            L.orc_bf16_rne.argtypes = [vp, vp, i64]
            L.orc_bf16_rne.restype = None
            L.orc_e4m3_rne.argtypes = [vp, vp, i64]
            L.orc_e4m3_rne.restype = None
            L.orc_e4m3_value.argtypes = [vp, vp, i64]
            L.orc_e4m3_value.restype = None
            L.orc_quantize_rows_e4m3.argtypes = [vp, i64, i64, i64, vp, i64, vp]
            L.orc_quantize_rows_e4m3.restype = ctypes.c_int
            L.orc_apply_right_q8.argtypes = [u64, i32, i64, vp, vp, i64, i64, i64, vp, i64, vp,
                                             i64, i32]
            L.orc_apply_right_q8.restype = ctypes.c_int
            L.orc_scale.argtypes = [i64]
            L.orc_scale.restype = ctypes.c_float
            L.orc_generate.argtypes = [u64, i32, i32, u32, i64, i64, i64, i64, vp, i64]
            L.orc_generate.restype = i32
            L.orc_apply_left_rows.argtypes = [u64, i32, i32, i64, i64, i64, vp, i64, i64, i64, vp,
                                              i64, vp, i64, i32]
            L.orc_apply_left_rows.restype = i32
            for f in (L.orc_apply_left, L.orc_apply_right):
                f.argtypes = [u64, i32, i32, i64, vp, i64, i64, i64, vp, i64, vp, i64, i32]
                f.restype = i32
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def philox4x32_10(ctr: np.ndarray, key) -> np.ndarray:
    """Philox4x32-10 of each row of ``ctr`` (shape [N, 4], uint32) under ``key`` (2 x uint32)."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(2))
    out = np.empty_like(ctr)
    lib().orc_philox4x32_10(_p(ctr), _p(key), _p(out), ctr.shape[0])
    return out


def ln(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.empty_like(x)
    lib().orc_ln(_p(x), _p(y), x.size)
    return y


def sincospi_quarter(r: np.ndarray):
    """(sin(pi r), cos(pi r)) for r in [-1/4, 1/4], the generator's FP32 polynomials."""
    r = np.ascontiguousarray(r, dtype=np.float32)
    s = np.empty_like(r)
    c = np.empty_like(r)
    lib().orc_sincospi_quarter(_p(r), _p(s), _p(c), r.size)
    return s, c


def circle(words: np.ndarray):
    """The circle point (X, Y) of each angle word (uint32): the position of
    bits 29..8 turned by the quarter turns of bits 31..30."""
    w = np.ascontiguousarray(words, dtype=np.uint32)
    x = np.empty(w.shape, dtype=np.float32)
    y = np.empty(w.shape, dtype=np.float32)
    lib().orc_circle(_p(w), _p(x), _p(y), w.size)
    return x, y


def box_muller(words: np.ndarray) -> np.ndarray:
    """Box-Muller of each word pair (row of ``words``, shape [N, 2], uint32):
    the generator's Gaussian pair (rho X, rho Y) with (X, Y) the circle
    point of the second word, shape [N, 2]."""
    w = np.ascontiguousarray(words, dtype=np.uint32).reshape(-1, 2)
    z = np.empty(w.shape, dtype=np.float32)
    lib().orc_box_muller(_p(w), _p(z), w.shape[0])
    return z


def bf16_rne(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.empty(x.shape, dtype=np.uint16)
    lib().orc_bf16_rne(_p(x), _p(y), x.size)
    return y


def e4m3_rne(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.empty(x.shape, dtype=np.uint8)
    lib().orc_e4m3_rne(_p(x), _p(y), x.size)
    return y


def e4m3_value(code: np.ndarray) -> np.ndarray:
    code = np.ascontiguousarray(code, dtype=np.uint8)
    y = np.empty(code.shape, dtype=np.float64)
    lib().orc_e4m3_value(_p(code), _p(y), code.size)
    return y


def scale(k: int) -> np.float32:
    return np.float32(lib().orc_scale(int(k)))


def generate(seed: int, dist: int, prec: int, row0: int, col0: int, rows: int, cols: int,
             dom: int = 0) -> np.ndarray:
    """Unscaled generated values q(g(r, c)) for r in [row0, row0+rows), c in [col0, col0+cols)."""
    out = np.empty((rows, cols), dtype=np.float32)
    rc = lib().orc_generate(int(seed), int(dist), int(prec), int(dom), int(row0), int(col0),
                            int(rows), int(cols), _p(out), max(int(cols), 1))
    if rc != 0:
        raise ValueError("orc_generate: bad arguments")
    return out


def materialize_scaled(seed: int, dist: int, prec: int, k: int, row0: int, col0: int,
                       rows: int, cols: int) -> np.ndarray:
    """S(r, c) = s * q(g(r, c)) as exact FP64 values."""
    return generate(seed, dist, prec, row0, col0, rows, cols).astype(np.float64) * float(scale(k))


def apply_left(seed: int, dist: int, prec: int, k: int, A: np.ndarray, cols=None,
               nthreads: int | None = None, rows: tuple[int, int] | None = None) -> np.ndarray:
    """Y = S[k x m] A[m x n] in FP64 (optionally only the columns ``cols`` and
    the rows ``rows = (row0, count)``)."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    m, n = A.shape
    if cols is None:
        idx, nidx = None, n
    else:
        idx = np.ascontiguousarray(cols, dtype=np.int64)
        nidx = idx.size
    row0, nrows = (0, k) if rows is None else (int(rows[0]), int(rows[1]))
    Y = np.empty((nrows, nidx), dtype=np.float64)
    rc = lib().orc_apply_left_rows(int(seed), int(dist), int(prec), int(k), row0, nrows, _p(A),
                                   m, n, n, None if idx is None else _p(idx), nidx, _p(Y),
                                   max(nidx, 1), int(nthreads or os.cpu_count() or 1))
    if rc != 0:
        raise ValueError("orc_apply_left failed")
    return Y


def apply_right(seed: int, dist: int, prec: int, k: int, A: np.ndarray, rows=None,
                nthreads: int | None = None) -> np.ndarray:
    """Y = A[m x n] S^T, S[k x n], in FP64 (optionally only the rows ``rows``)."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    m, n = A.shape
    if rows is None:
        idx, nidx = None, m
    else:
        idx = np.ascontiguousarray(rows, dtype=np.int64)
        nidx = idx.size
    Y = np.empty((nidx, k), dtype=np.float64)
    rc = lib().orc_apply_right(int(seed), int(dist), int(prec), int(k), _p(A), m, n, n,
                               None if idx is None else _p(idx), nidx, _p(Y), k,
                               int(nthreads or os.cpu_count() or 1))
    if rc != 0:
        raise ValueError("orc_apply_right failed")
    return Y


def quantize_rows_e4m3(A: np.ndarray):
    """(codes, exps): E4M3 codes of A[m x n] with one power-of-two scale 2^exps[i]
    per row, the smallest with max_j |a_ij| <= 448 * 2^exps[i] (0 for a zero
    row); codes[i, j] = RNE_e4m3(a_ij * 2^-exps[i])."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    m, n = A.shape
    codes = np.empty((m, n), dtype=np.uint8)
    exps = np.empty(m, dtype=np.int32)
    if lib().orc_quantize_rows_e4m3(_p(A), m, n, n, _p(codes), n, _p(exps)) != 0:
        raise ValueError("orc_quantize_rows_e4m3 failed")
    return codes, exps


def apply_right_q8(seed: int, dist: int, k: int, codes: np.ndarray, exps: np.ndarray, rows=None,
                   nthreads: int | None = None) -> np.ndarray:
    """FP8 right sketch in FP64: Y[i, j] = 2^exps[i] s sum_c value(codes[i, c])
    value(RNE_e4m3(g(j, c))) (optionally only the rows ``rows``)."""
    codes = np.ascontiguousarray(codes, dtype=np.uint8)
    exps = np.ascontiguousarray(exps, dtype=np.int32)
    m, n = codes.shape
    if rows is None:
        idx, nidx = None, m
    else:
        idx = np.ascontiguousarray(rows, dtype=np.int64)
        nidx = idx.size
    Y = np.empty((nidx, k), dtype=np.float64)
    rc = lib().orc_apply_right_q8(int(seed), int(dist), int(k), _p(codes), _p(exps), m, n, n,
                                  None if idx is None else _p(idx), nidx, _p(Y), k,
                                  int(nthreads or os.cpu_count() or 1))
    if rc != 0:
        raise ValueError("orc_apply_right_q8 failed")
    return Y


def nystrom(seed: int, dist: int, prec: int, k: int, A: np.ndarray, nthreads: int | None = None):
    """The two products of the paper's Nystrom computation (Sec. 5, Alg. 2),
    B = A Omega and C = Omega^T B with Omega = S^T (S[k x n] the sketching
    matrix, k = r), in FP64: B[n x k] by the right sketch, then C[k x k] as
    S B with S's exact values (a library matmul as the step)."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    n = A.shape[0]
    if A.shape != (n, n):
        raise ValueError("A must be square")
    Bm = apply_right(seed, dist, prec, k, A, nthreads=nthreads)
    S = materialize_scaled(seed, dist, prec, k, 0, 0, k, n)
    return Bm, S @ Bm
