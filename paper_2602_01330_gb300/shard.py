"""Split a symmetric Gram matrix into per-GPU row blocks (§II-D: blocks of the kernel
matrix go to different GPU workers and are gathered on the host).

Row block r of an m x m symmetric Gram holds rows [lo, hi) and the unique pairs
(i, j) with lo <= i < hi, i <= j < m, i.e. sum_{i in [lo,hi)} (m - i) pairs. The split
below balances that count over `world` workers; each worker then needs one dk_gram_tile
call over rows [lo, hi) x columns [lo, m) (its mirror half is the transpose) and no data
exchange until the gather.
"""
from __future__ import annotations


def upper_pairs(m: int, lo: int, hi: int) -> int:
    """Pairs (i, j), lo <= i < hi, i <= j < m."""
    return sum(m - i for i in range(lo, hi))


def balanced_row_blocks(m: int, world: int):
    """[(lo, hi)] for each rank, contiguous, covering [0, m), with near-equal pair counts."""
    if world < 1:
        raise ValueError("world must be >= 1")
    total = m * (m + 1) // 2
    bounds = [0]
    acc = 0
    i = 0
    for r in range(1, world):
        target = total * r / world
        while i < m and acc + (m - i) <= target:
            acc += m - i
            i += 1
        bounds.append(i)
    bounds.append(m)
    return [(bounds[r], bounds[r + 1]) for r in range(world)]
