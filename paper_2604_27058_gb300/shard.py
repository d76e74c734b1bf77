"""Shot-range sharding for runs on several GPUs (one process per GPU).

Shots are independent and every random draw is keyed by the global shot
index (Sec. 3.2 sampling, counter-based Philox), so a rank that samples
global shots [offset, offset + n) produces exactly the records a single run
would produce for those shots. There is no data exchange; only timings and
counts are reduced across ranks.
"""

from __future__ import annotations

ALIGN = 128  # shot_offset must be a multiple of 128 (one block draw covers 128 shots)


def weak(shots_per_rank: int, rank: int) -> tuple[int, int]:
    """Every rank samples `shots_per_rank` shots (weak scaling): returns the
    rank's (shot_offset, shots)."""
    stride = -(-shots_per_rank // ALIGN) * ALIGN
    return rank * stride, shots_per_rank


def strong(total: int, rank: int, world: int) -> tuple[int, int]:
    """`total` shots split into `world` contiguous 128-aligned ranges (strong
    scaling): returns the rank's (shot_offset, shots)."""
    blocks = -(-total // ALIGN)
    per, extra = divmod(blocks, world)
    first = rank * per + min(rank, extra)
    n_blocks = per + (1 if rank < extra else 0)
    off = first * ALIGN
    return off, max(0, min(total, off + n_blocks * ALIGN) - off)
