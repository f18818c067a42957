"""The sharded Gram (§II-D: blocks to workers, gathered on the host) on two gloo ranks.

CPU tests: the row-block split covers the pairs in balance; the product gather
(shard.gather_gram, one all_gather per output, placement by the known bounds) rebuilds a
symmetric matrix exactly, exact zeros and negative values included; and row blocks filled
with the oracle's pair values assemble into the oracle's one-process Gram.
GPU test (marked gpu): two processes on one device, each with its own library context,
compute their row blocks with shard.gram_row_block (dk_gram_tile) and gather them over
gloo; the result equals the single-process Gram bit for bit and the oracle within 1e-6.
The two processes' kernels never wait on one another, so sharing one GPU is safe.
"""
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


def _init(rank, world, port):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)


def _matrix_worker(rank, world, port, g, result_q):
    _init(rank, world, port)
    m = g.shape[0]
    lo, hi = shard.balanced_row_blocks(m, world)[rank]
    block = {"kq": torch.from_numpy(np.ascontiguousarray(g[lo:hi, lo:])), "logkq": None}
    full = shard.gather_gram(block, m, world, device="cpu")
    if rank == 0:
        result_q.put(full["kq"].numpy())
    dist.barrier()
    dist.destroy_process_group()


def _oracle_worker(rank, world, port, x, result_q):
    _init(rank, world, port)
    from oracle import gram, mps
    m = x.shape[0]
    lo, hi = shard.balanced_row_blocks(m, world)[rank]
    sites, _ = mps.build_mps(x, 2)
    ii, jj = np.triu_indices(m)
    mine = (ii >= lo) & (ii < hi)
    kq, _ = gram.pair_values(sites, sites, ii[mine], jj[mine])
    block = np.zeros((hi - lo, m - lo))
    block[ii[mine] - lo, jj[mine] - lo] = kq
    full = shard.gather_gram({"kq": torch.from_numpy(block)}, m, world, device="cpu")
    if rank == 0:
        result_q.put(full["kq"].numpy())
    dist.barrier()
    dist.destroy_process_group()


def _run(target, world, *args):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, world, port, *args, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


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


def test_assemble_places_blocks_by_bounds():
    rng = np.random.Generator(np.random.PCG64(3))
    m, world = 23, 3
    g = rng.normal(size=(m, m)).astype(np.float32)
    g = np.triu(g) + np.triu(g, 1).T
    g[g > 0.8] = 0.0  # exact zeros must survive
    bounds = shard.balanced_row_blocks(m, world)
    blocks = [torch.from_numpy(np.ascontiguousarray(g[lo:hi, lo:])) for lo, hi in bounds]
    assert np.array_equal(shard.assemble(blocks, bounds, m).numpy(), g)


@pytest.mark.timeout(300)
def test_two_rank_gather_keeps_zeros_and_signs():
    rng = np.random.Generator(np.random.PCG64(4))
    m = 41
    g = rng.normal(size=(m, m)).astype(np.float32)
    g = np.triu(g) + np.triu(g, 1).T
    g[np.abs(g) < 0.5] = 0.0
    full = _run(_matrix_worker, 2, g)
    assert np.array_equal(full, g)


@pytest.mark.timeout(300)
def test_two_rank_oracle_blocks_match_single_process():
    from oracle import gram, mps
    from paper_2602_01330_gb300 import synthetic
    x = synthetic.fmnist_like(30, 0, 12)["x_train"].astype(np.float64)
    full = _run(_oracle_worker, 2, x)
    sites, _ = mps.build_mps(x, 2)
    ref, _ = gram.gram_from_mps(sites, sites)
    assert np.max(np.abs(full - ref)) < 1e-12


def _gpu_worker(rank, world, port, x, result_q):
    _init(rank, world, port)
    from paper_2602_01330_gb300 import dualk
    torch.cuda.set_device(0)
    ctx = dualk.Context(0)
    m = x.shape[0]
    mp_ = dualk.mps_build(ctx, torch.from_numpy(x).cuda(), dualk.FeatureMap(reps=2, chi_max=4))
    block, _ = shard.gram_row_block(ctx, mp_, rank, world, w=0.5)
    torch.cuda.synchronize()
    ctx.sync_status()
    full = shard.gather_gram(block, m, world, device="cpu")
    if rank == 0:
        result_q.put({k: v.numpy() for k, v in full.items()})
    dist.barrier()
    dist.destroy_process_group()
    ctx.close()


@pytest.mark.gpu
@pytest.mark.timeout(600)
def test_two_ranks_on_one_device_match_single_process_and_oracle():
    """d = 64, 300 samples of which 200..299 are near copies of 0..99 (K_q of order one),
    reps 2, w = 0.5: the gathered K, K_q, K_c, log K_q equal the one-process symmetric Gram
    bit for bit; K_q and K within 1e-6 of the oracle."""
    import oracle_pool
    from oracle import gram as og
    from paper_2602_01330_gb300 import build, dualk, synthetic
    build.build()
    x = synthetic.fmnist_like(300, 0, 64)["x_train"].copy()
    x[200:300] = synthetic.near_copies(x[0:100], 1e-3, 1e-1, seed=66)
    full = _run(_gpu_worker, 2, x)
    ctx = dualk.Context(0)
    mp_ = dualk.mps_build(ctx, torch.from_numpy(x).cuda(), dualk.FeatureMap(reps=2, chi_max=4))
    one = dualk.gram(ctx, mp_, w=0.5)
    torch.cuda.synchronize()
    ctx.sync_status()
    for k in ("k", "kq", "kc", "logkq"):
        assert np.array_equal(full[k], one[k].cpu().numpy()), k
    kq_ref, _ = oracle_pool.block(x, None, 2, symmetric=True)
    kc_ref = og.rbf(x, x, 1 / 64)
    assert np.max(np.abs(full["kq"] - kq_ref)) <= 1e-6
    assert np.max(np.abs(full["k"] - og.dual_kernel(kq_ref, kc_ref, 0.5))) <= 1e-6
    assert (kq_ref[np.arange(100), np.arange(200, 300)] > 1e-3).sum() >= 50
    ctx.close()
