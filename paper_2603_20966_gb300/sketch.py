"""Convenience wrapper over the C ABI for torch tensors.

``Sketch(seed, dist, k)`` owns one library handle.  ``left(A)`` /
``right(A)`` allocate Y with torch on A's device and call the library on
torch's current stream; nothing is computed in Python.  ``Server`` wraps the
library's request server (admission by an HBM budget, continuous batching).
"""
from __future__ import annotations

import torch

from . import _native as N


class Sketch:
    def __init__(self, seed: int, dist: int, k: int, precision: int = N.SK_FP32):
        self.handle = N.sk_create(seed, dist, k)
        self.k = int(k)
        if precision != N.SK_FP32:
            N.sk_set_precision(self.handle, precision)

    def close(self):
        if self.handle:
            N.sk_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def precision(self) -> int:
        return N.sk_get_info(self.handle)["precision"]

    @precision.setter
    def precision(self, p: int):
        N.sk_set_precision(self.handle, p)

    @property
    def scale(self) -> float:
        return N.sk_get_info(self.handle)["scale"]

    @staticmethod
    def _check(A: torch.Tensor):
        if A.dtype != torch.float32 or not A.is_cuda or A.dim() != 2 or A.stride(1) != 1:
            raise ValueError("A must be a CUDA float32 matrix with unit column stride")

    def left(self, A: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        self._check(A)
        m, n = A.shape
        Y = out if out is not None else torch.empty((self.k, n), dtype=torch.float32,
                                                      device=A.device)
        N.sk_apply_left(self.handle, A, m, n, A.stride(0), Y, Y.stride(0),
                        torch.cuda.current_stream(A.device))
        return Y

    def right(self, A: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        self._check(A)
        m, n = A.shape
        Y = out if out is not None else torch.empty((m, self.k), dtype=torch.float32,
                                                      device=A.device)
        N.sk_apply_right(self.handle, A, m, n, A.stride(0), Y, Y.stride(0),
                         torch.cuda.current_stream(A.device))
        return Y

    def nystrom(self, A: torch.Tensor) -> tuple[torch.Tensor, torch.Tensor]:
        """(B, C) = (A Omega, Omega^T A Omega) for a symmetric n x n A."""
        self._check(A)
        n = A.shape[0]
        ld = (self.k + 3) // 4 * 4
        B = torch.empty((n, ld), dtype=torch.float32, device=A.device)
        C = torch.empty((self.k, ld), dtype=torch.float32, device=A.device)
        N.sk_nystrom(self.handle, A, n, A.stride(0), B, ld, C, ld,
                     torch.cuda.current_stream(A.device))
        return B[:, :self.k], C[:, :self.k]

    def materialize(self, row0: int, col0: int, rows: int, cols: int, fmt: int = N.SK_FP32,
                    scaled: bool = False, device="cuda") -> torch.Tensor:
        dt = {N.SK_FP32: torch.float32, N.SK_BF16X2: torch.bfloat16,
              N.SK_FP8E4M3: torch.uint8}[fmt]
        out = torch.empty((rows, cols), dtype=dt, device=device)
        N.sk_materialize(self.handle, row0, col0, rows, cols, fmt, int(scaled), out, cols,
                         torch.cuda.current_stream(out.device))
        return out

    def status(self) -> int:
        return N.sk_stream_status(self.handle, torch.cuda.current_stream())


class Server:
    """Request server of left sketches (``sk_server_*``).

    ``submit(sketch, A)`` enqueues Y = S A for a CUDA (or host) float32
    matrix A and returns a ticket; ``result(ticket)`` waits and returns Y as
    a new tensor; ``release(ticket)`` discards a result (or drops it when it
    finishes).  A must stay valid until its request has finished.
    """

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 1024):
        self.handle = N.sk_server_create(hbm_budget_bytes, max_slots)
        self._shapes: dict[int, tuple[int, int]] = {}

    def close(self):
        if self.handle:
            N.sk_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def submit(self, sketch: Sketch, A: torch.Tensor) -> int:
        if A.dtype != torch.float32 or A.dim() != 2 or A.stride(1) != 1:
            raise ValueError("A must be a float32 matrix with unit column stride")
        m, n = A.shape
        stream = torch.cuda.current_stream(A.device) if A.is_cuda else None
        t = N.sk_server_submit(self.handle, sketch.handle, A, m, n, A.stride(0), stream)
        self._shapes[t] = (sketch.k, n)
        return t

    def poll(self, ticket: int) -> tuple[int, float]:
        return N.sk_server_poll(self.handle, ticket)

    def wait(self, ticket: int, timeout_s: float = 60.0) -> float:
        st, lat = N.sk_server_wait(self.handle, ticket, timeout_s)
        if st != N.SK_OK:
            raise N.SketchError("sk_server_wait", st)
        return lat

    def result(self, ticket: int, device="cuda", timeout_s: float = 60.0) -> torch.Tensor:
        self.wait(ticket, timeout_s)
        k, n = self._shapes.pop(ticket)
        Y = torch.empty((k, n), dtype=torch.float32, device=device)
        stream = torch.cuda.current_stream(Y.device) if Y.is_cuda else None
        N.sk_server_fetch(self.handle, ticket, Y, n, stream)
        return Y

    def release(self, ticket: int) -> None:
        self._shapes.pop(ticket, None)
        N.sk_server_release(self.handle, ticket)

    def stats(self) -> dict:
        return N.sk_server_stats_get(self.handle)

    def reset_stats(self) -> None:
        N.sk_server_reset_stats(self.handle)
