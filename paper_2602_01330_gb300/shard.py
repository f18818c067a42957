"""The symmetric Gram matrix split over GPU workers by row blocks (§II-D: blocks of the
kernel matrix are evaluated by different GPU workers and gathered on the host).

Row block r of an m x m symmetric Gram holds rows [lo, hi) and the unique pairs (i, j)
with lo <= i < hi, i <= j < m, i.e. sum_{i in [lo, hi)} (m - i) pairs. The split balances
that count over `world` workers. Worker r computes its pairs with two library calls and no
data exchange: the symmetric diagonal square [lo, hi) x [lo, hi) and the rectangle
[lo, hi) x [hi, m). Each pair is contracted with the same operand roles (row sample i <= j)
as in a one-process symmetric Gram, so the gathered matrix equals it bit for bit.

The gather is one collective per output (all_gather of equal-sized, zero-padded row
blocks); the assembly places every block by its known bounds and fills the lower triangle
as the transpose of the upper one, so no value (an exact zero included) is ever inferred.
"""
from __future__ import annotations

import torch

OUTPUTS = ("k", "kq", "kc", "logkq")


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


def gram_row_block(ctx, mps, rank: int, world: int, w: float = 0.5, gamma: float | None = None,
                   want=OUTPUTS, out: dict | None = None, stream=None):
    """This worker's share of the symmetric Gram of `mps`: a dict of (hi - lo) x (m - lo)
    float32 device tensors holding rows [lo, hi) and columns [lo, m) (entries left of the
    diagonal inside the square part are the mirrored values). Returns (block dict, (lo, hi))."""
    from . import dualk
    m = mps.m
    lo, hi = balanced_row_blocks(m, world)[rank]
    rows, cols = hi - lo, m - lo
    if out is None:
        out = {k: (torch.empty((rows, cols), dtype=torch.float32, device=mps.data.device) if k in want else None)
               for k in OUTPUTS}
    if rows == 0:
        return out, (lo, hi)
    ld = cols
    dualk.gram_tile(ctx, mps, mps, row0=lo, nrows=rows, col0=lo, ncols=rows, gamma=gamma, w=w, symmetric=True,
                    out=out, ld=ld, stream=stream)
    if hi < m:
        rect = {k: (v[:, rows:] if v is not None else None) for k, v in out.items()}
        dualk.gram_tile(ctx, mps, mps, row0=lo, nrows=rows, col0=hi, ncols=m - hi, gamma=gamma, w=w,
                        symmetric=False, out=rect, ld=ld, stream=stream)
    return out, (lo, hi)


def assemble(blocks, bounds, m: int) -> torch.Tensor:
    """The m x m symmetric matrix from the row blocks of every rank: block r's rows are
    [lo, hi) x [lo, m); the upper triangle is placed, the lower one is its transpose."""
    full = torch.zeros((m, m), dtype=blocks[0].dtype)
    for blk, (lo, hi) in zip(blocks, bounds):
        full[lo:hi, lo:] = blk[: hi - lo, : m - lo]
    upper = torch.triu(full)
    return upper + torch.triu(full, 1).T


def gather_gram(block: dict, m: int, world: int, group=None, device=None) -> dict:
    """All-gather every rank's row block (gram_row_block output) and assemble the full
    matrices on every rank, on the host. Collectives run on `device` tensors (CPU for gloo,
    the GPU for NCCL); each block is padded to the largest block's shape."""
    import torch.distributed as dist
    bounds = balanced_row_blocks(m, world)
    max_rows = max(hi - lo for lo, hi in bounds)
    res = {}
    for key in OUTPUTS:
        v = block.get(key)
        if v is None:
            continue
        dev = v.device if device is None else torch.device(device)
        pad = torch.zeros((max_rows, m), dtype=v.dtype, device=dev)
        pad[: v.shape[0], : v.shape[1]] = v.to(dev)
        parts = [torch.empty_like(pad) for _ in range(world)]
        dist.all_gather(parts, pad, group=group)
        res[key] = assemble([p.cpu() for p in parts], bounds, m)
    return res
