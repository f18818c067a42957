"""The multi-GPU split on the CPU: two gloo ranks each compute their balanced row block of
a symmetric Gram with the oracle and all-gather; the assembly equals the one-process Gram.
(No GPU: this checks the partition and gather logic of the sharded path.)"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2602_01330_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, x, result_q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import gram, mps
    m = x.shape[0]
    lo, hi = shard.balanced_row_blocks(m, world)[rank]
    sites, _ = mps.build_mps(x, 2)
    block = np.zeros((m, m))
    ii, jj = [], []
    for i in range(lo, hi):
        for j in range(i, m):
            ii.append(i)
            jj.append(j)
    kq, _ = gram.pair_values(sites, sites, ii, jj)
    block[ii, jj] = kq
    block[jj, ii] = kq
    t = torch.from_numpy(block)
    gathered = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(gathered, t)
    if rank == 0:
        full = torch.zeros_like(t)
        for g in gathered:
            full = torch.where(g != 0, g, full)
        result_q.put(full.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_balanced_row_blocks_cover_and_balance():
    for m in (1, 7, 100, 2001):
        for world in (1, 2, 3, 8):
            blocks = shard.balanced_row_blocks(m, world)
            assert blocks[0][0] == 0 and blocks[-1][1] == m
            assert all(a[1] == b[0] for a, b in zip(blocks, blocks[1:]))
            counts = [shard.upper_pairs(m, lo, hi) for lo, hi in blocks]
            assert sum(counts) == m * (m + 1) // 2
            if m >= 100 * world:
                assert max(counts) - min(counts) <= m


@pytest.mark.timeout(300)
def test_two_rank_gather_matches_single_process():
    from oracle import gram, mps
    from paper_2602_01330_gb300 import synthetic
    x = synthetic.fmnist_like(30, 0, 12)["x_train"].astype(np.float64)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, x, q)) for r in range(2)]
    for p in procs:
        p.start()
    full = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sites, _ = mps.build_mps(x, 2)
    ref, _ = gram.gram_from_mps(sites, sites)
    assert np.max(np.abs(full - ref)) < 1e-12
