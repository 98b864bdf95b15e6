"""One sketch split over several GPUs with no data exchange.

This is the paper's Case 1 of the processor-grid selection (Sec. 3.3, P no
larger than the long dimension): Alg. 1 with a one-dimensional grid, whose
All-Gather of A and Reduce-Scatter of the result are both empty, because
every processor regenerates the block of the random matrix it needs
(GenRandom with the shared seed, Sec. 6.2) instead of receiving it.

* Right sketch Y[m x k] = A[m x n] S^T: A is split by rows.  Rank r owns rows
  [r0, r1) of A and computes rows [r0, r1) of Y with the whole S, which it
  regenerates from the seed.
* Left sketch Y[k x n] = S[k x m] A[m x n]: A is split by columns.  Rank r
  owns columns [c0, c1) of A and computes columns [c0, c1) of Y with the
  whole S.

Each rank's block of Y is final: no partial sums, nothing to reduce.  A rank
computes its block with the library's ordinary single-GPU entry points on its
own device; the only collective here is the optional assembly of the full Y
(an all-gather of the blocks), which the sketch itself does not need.  The
block boundaries are multiples of `align` (4 keeps every block's first
column 16-byte aligned, as the tensor-core forms require of a column block
that is a view of a row-major matrix).
"""
from __future__ import annotations

import torch

from . import _native as N


def block_range(total: int, parts: int, index: int, align: int = 1) -> tuple[int, int]:
    """Block `index` of `parts` contiguous blocks of range(total): near-equal
    sizes in units of `align` (the last block takes the remainder), so every
    boundary but the end is a multiple of `align`.  Blocks may be empty when
    total < parts * align."""
    if parts < 1 or not 0 <= index < parts or align < 1 or total < 0:
        raise ValueError("block_range: bad arguments")
    units = (total + align - 1) // align
    u0 = units * index // parts
    u1 = units * (index + 1) // parts
    return min(total, u0 * align), min(total, u1 * align)


def column_align(n: int, parts: int) -> int:
    """Column-block granularity of a left sketch: whole 64-column chunks of
    the split A when every rank gets at least one, else 4 columns."""
    return 64 if n >= 64 * parts else 4


def left_column_ranges(n: int, world: int) -> list[tuple[int, int]]:
    """Columns [c0, c1) of A (and of Y) each rank owns in a left sketch."""
    al = column_align(n, world)
    return [block_range(n, world, r, al) for r in range(world)]


def right_row_ranges(m: int, world: int) -> list[tuple[int, int]]:
    """Rows [r0, r1) of A (and of Y) each rank owns in a right sketch."""
    return [block_range(m, world, r, 1) for r in range(world)]


class PartitionedSketch:
    """The share of rank `rank` (of `world`) of one sketch.

    Every rank creates the operator with the same (seed, dist, k,
    precision), so all of them regenerate the same S.  `left` / `right`
    compute this rank's block of Y from this rank's block of A on the current
    device and stream; `assemble_*` gather the blocks into the full Y on
    every rank (torch.distributed all_gather over `group`), for callers that
    want it."""

    def __init__(self, seed: int, dist: int, k: int, world: int, rank: int,
                 precision: int = N.SK_FP32):
        if world < 1 or not 0 <= rank < world:
            raise ValueError("PartitionedSketch: bad world/rank")
        self.world, self.rank, self.k = int(world), int(rank), int(k)
        self.handle = N.sk_create(seed, dist, k)
        if precision != N.SK_FP32:
            N.sk_set_precision(self.handle, precision)

    def close(self):
        if self.handle:
            N.sk_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- ownership ----
    def left_columns(self, n: int) -> tuple[int, int]:
        """Columns [c0, c1) of A (and of Y) this rank owns in a left sketch."""
        return left_column_ranges(n, self.world)[self.rank]

    def right_rows(self, m: int) -> tuple[int, int]:
        """Rows [r0, r1) of A (and of Y) this rank owns in a right sketch."""
        return right_row_ranges(m, self.world)[self.rank]

    # ---- this rank's block ----
    def left(self, A_block: torch.Tensor, Y_block: torch.Tensor, stream=None) -> torch.Tensor:
        """Y_block[k x n_r] = S A_block[m x n_r]; both may be column views of
        full row-major matrices (leading dimensions are their row strides)."""
        m, nb = A_block.shape
        if nb == 0:
            return Y_block
        N.sk_apply_left(self.handle, A_block, m, nb, A_block.stride(0), Y_block,
                        Y_block.stride(0), stream if stream is not None else
                        torch.cuda.current_stream(A_block.device))
        return Y_block

    def right(self, A_block: torch.Tensor, Y_block: torch.Tensor, stream=None) -> torch.Tensor:
        """Y_block[m_r x k] = A_block[m_r x n] S^T."""
        mb, n = A_block.shape
        if mb == 0:
            return Y_block
        N.sk_apply_right(self.handle, A_block, mb, n, A_block.stride(0), Y_block,
                         Y_block.stride(0), stream if stream is not None else
                         torch.cuda.current_stream(A_block.device))
        return Y_block

    # ---- optional assembly (the sketch itself needs none) ----
    def assemble_left(self, Y_block: torch.Tensor, n: int, group=None) -> torch.Tensor:
        """The full Y[k x n] on every rank from the column blocks."""
        return gather_blocks(Y_block, left_column_ranges(n, self.world), 1, group)

    def assemble_right(self, Y_block: torch.Tensor, m: int, group=None) -> torch.Tensor:
        """The full Y[m x k] on every rank from the row blocks."""
        return gather_blocks(Y_block, right_row_ranges(m, self.world), 0, group)


def gather_blocks(block: torch.Tensor, ranges, dim: int, group=None) -> torch.Tensor:
    """all_gather of blocks of unequal size along `dim`: each rank's block is
    padded to the largest, gathered, and the padding dropped."""
    import torch.distributed as dist
    sizes = [b - a for a, b in ranges]
    width = max(sizes)
    shape = list(block.shape)
    shape[dim] = width
    pad = torch.zeros(shape, dtype=block.dtype, device=block.device)
    pad.narrow(dim, 0, block.shape[dim]).copy_(block)
    parts = [torch.empty_like(pad) for _ in ranges]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([p.narrow(dim, 0, s) for p, s in zip(parts, sizes)], dim=dim)
