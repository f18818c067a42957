"""Run the FP64 oracle over many pairs on all host cores (test infrastructure only).

The oracle itself is unchanged: each worker process builds the oracle MPS of the samples
it needs (``oracle.mps.build_mps``) and contracts its share of the pairs with
``oracle.gram.pair_values``. Workers are started with the ``spawn`` method, which is safe
after the parent process has initialised CUDA (a forked child of a CUDA process can hang).
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np


def _procs(n_tasks: int) -> int:
    return max(1, min(n_tasks, os.cpu_count() or 1, 32))


def _aligned_worker(args):
    from oracle import gram, mps
    xa, xb, reps = args
    sa, _ = mps.build_mps(xa, reps)
    sb, _ = mps.build_mps(xb, reps)
    p = np.arange(xa.shape[0])
    return gram.pair_values(sa, sb, p, p)


def _block_worker(args):
    from oracle import gram, mps
    xa, xb, reps, ii, jj = args
    sa, _ = mps.build_mps(xa, reps)
    sb, _ = mps.build_mps(xb, reps)
    return gram.pair_values(sa, sb, ii, jj)


def _pool(n):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    return mp.get_context("spawn").Pool(n)


def aligned_pairs(x_rows, x_cols, reps: int):
    """(K_q, log K_q) of the pairs (x_rows[p], x_cols[p]), p = 0 .. len - 1."""
    xa = np.asarray(x_rows, dtype=np.float64)
    xb = np.asarray(x_cols, dtype=np.float64)
    n = _procs(max(1, xa.shape[0] // 8))
    cuts = [c for c in np.array_split(np.arange(xa.shape[0]), n) if c.size]
    with _pool(len(cuts)) as pool:
        parts = pool.map(_aligned_worker, [(xa[c], xb[c], reps) for c in cuts])
    return np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts])


def block(x_rows, x_cols, reps: int, symmetric: bool = False):
    """(K_q, log K_q) matrices of all pairs of x_rows x x_cols. symmetric: x_cols is x_rows
    and only the pairs i <= j are contracted; the lower triangle is their mirror."""
    xa = np.asarray(x_rows, dtype=np.float64)
    xb = xa if symmetric else np.asarray(x_cols, dtype=np.float64)
    mr, mc = xa.shape[0], xb.shape[0]
    n = _procs(max(1, mr // 4))
    # symmetric: row chunks of equal pair counts (row i holds mc - i pairs)
    if symmetric:
        w = np.cumsum(mc - np.arange(mr))
        edges = np.searchsorted(w, np.linspace(0, w[-1], n + 1)[1:-1])
        cuts = [c for c in np.split(np.arange(mr), edges) if c.size]
    else:
        cuts = [c for c in np.array_split(np.arange(mr), n) if c.size]
    tasks = []
    for c in cuts:
        cols = np.arange(c[0], mc) if symmetric else np.arange(mc)
        ii, jj = np.meshgrid(np.arange(c.size), np.arange(cols.size), indexing="ij")
        keep = (c[ii] <= cols[jj]) if symmetric else np.ones(ii.shape, dtype=bool)
        tasks.append((xa[c], xb[cols], reps, ii[keep], jj[keep], c, cols))
    kq = np.full((mr, mc), np.nan)
    lkq = np.full((mr, mc), np.nan)
    with _pool(len(tasks)) as pool:
        parts = pool.map(_block_worker, [t[:5] for t in tasks])
    for (_, _, _, ii, jj, c, cols), (k, lk) in zip(tasks, parts):
        kq[c[ii], cols[jj]] = k
        lkq[c[ii], cols[jj]] = lk
        if symmetric:
            kq[cols[jj], c[ii]] = k
            lkq[cols[jj], c[ii]] = lk
    assert not np.isnan(kq).any()
    return kq, lkq
