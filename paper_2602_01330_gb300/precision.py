"""Precision form: the same Gram in FP32 on CUDA cores and in split-BF16 (bf16x3) on
tensor cores, timed and compared with each other (§II-C Eqs. 7-10).

Data: the Fashion-MNIST-shaped generator at d = 256. reps = 3 gives the exact bond 8
(FP32 only: the tensor-core path needs bond 32); reps = 5 reaches bond 32, where the
transfer step is a dense 16 x 16 x 16 complex contraction per block.

``compare`` returns, per path, the Gram throughput on an m-sample block, and the largest
difference between the two bond-32 paths over the whole block and over sampled pairs
(uniform pairs, nearest-neighbour pairs whose K is far from 0, diagonal). The errors
against the FP64 oracle on the same sampled pairs are measured by the GPU test suite
(tests/test_precision_gpu.py), which owns the oracle.
"""
from __future__ import annotations

import json

import numpy as np
import torch

from . import dualk, synthetic, workload


def _time(fn, reps=2):
    fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        b.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def sample_pairs(x: np.ndarray, n_uniform: int, n_near: int, n_diag: int, seed: int = 0):
    """Uniform pairs i < j, nearest-neighbour pairs (K far from 0) and diagonal pairs."""
    rng = np.random.Generator(np.random.PCG64(seed))
    m = x.shape[0]
    pairs = []
    while len(pairs) < n_uniform:
        i, j = sorted(rng.integers(0, m, size=2))
        if i < j:
            pairs.append((int(i), int(j)))
    d2 = ((x[:, None, :].astype(np.float64) - x[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(d2, np.inf)
    for i in rng.choice(m, size=n_near, replace=False):
        j = int(np.argmin(d2[i]))
        pairs.append((min(int(i), j), max(int(i), j)))
    for i in rng.choice(m, size=n_diag, replace=False):
        pairs.append((int(i), int(i)))
    return pairs


def compare(m: int = 512, d: int = 256, pool: int = 128, n_uniform: int = 40, n_near: int = 20, n_diag: int = 10,
            ctx: dualk.Context | None = None, return_blocks: bool = False):
    own = ctx is None
    ctx = ctx or dualk.Context(0)
    x = synthetic.fmnist_like(m, 0, d)["x_train"]
    xt = torch.from_numpy(x).cuda()
    pairs = sample_pairs(x[:pool], n_uniform, n_near, n_diag)
    res = {"workload": f"fmnist d={d} m={m} (Gram timing), {len(pairs)} sampled pairs from the first {pool}"}
    kq_block = {}
    for reps, chi, precs in ((3, 8, (("fp32", dualk.DK_PREC_F32),)),
                             (5, 32, (("fp32", dualk.DK_PREC_F32), ("bf16x3", dualk.DK_PREC_BF16X3)))):
        fm = dualk.FeatureMap(reps=reps, chi_max=chi)
        mps = dualk.mps_build(ctx, xt, fm)
        out = {"kq": torch.empty((m, m), device="cuda")}
        for name, prec in precs:
            ms = _time(lambda: dualk.gram_tile(ctx, mps, mps, symmetric=True, out=out, ld=m, w=1.0, prec=prec))
            kq = out["kq"].cpu().numpy().astype(np.float64)
            kq_block[(chi, name)] = kq
            units = workload.gram_entries(m) * d
            res[f"chi{chi}_{name}"] = {
                "gram_ms": ms, "entry_qubits_per_s": units / (ms / 1e3),
                "tflops_block_count": workload.gram_entries(m) * workload.flops_per_pair(d, reps) / ms / 1e9,
            }
    diff = np.abs(kq_block[(32, "fp32")] - kq_block[(32, "bf16x3")])
    res["chi32_max_abs_dK_bf16x3_vs_fp32_block"] = float(diff.max())
    res["chi32_max_abs_dK_bf16x3_vs_fp32_sampled"] = float(max(diff[i, j] for i, j in pairs))
    ctx.sync_status()
    if own:
        ctx.close()
    if return_blocks:
        return res, pairs, kq_block, x
    return res


def main():
    import argparse

    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--m", type=int, default=1024)
    ap.add_argument("--pool", type=int, default=256)
    ap.add_argument("--uniform", type=int, default=100)
    ap.add_argument("--near", type=int, default=60)
    ap.add_argument("--diag", type=int, default=20)
    args = ap.parse_args()
    print(json.dumps(compare(args.m, 256, args.pool, args.uniform, args.near, args.diag)))


if __name__ == "__main__":
    main()
