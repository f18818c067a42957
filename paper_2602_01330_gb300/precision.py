"""Precision form: the same Gram in FP32 on CUDA cores and in split-BF16 (bf16x3) on
tensor cores, timed and compared with each other (§II-C Eqs. 7-10); and the bond-4 MPS
build with its QR sweep in FP32 against FP64 (``compare_build_qr``).

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
            split_ms = None
            if prec == dualk.DK_PREC_BF16X3:  # the split operands, made once per MPS (not in the Gram time)
                mps.log_norm_for(ctx, prec)
                torch.cuda.synchronize()
                split_ms = _event_ms(lambda: mps.split_for(ctx))
            ms = _time(lambda: dualk.gram_tile(ctx, mps, mps, symmetric=True, out=out, ld=m, w=1.0, prec=prec))
            kq = out["kq"].cpu().numpy().astype(np.float64)
            kq_block[(chi, name)] = kq
            units = workload.gram_entries(m) * d
            res[f"chi{chi}_{name}"] = {
                "gram_ms": ms, "entry_qubits_per_s": units / (ms / 1e3),
                "tflops_block_count": workload.gram_entries(m) * workload.flops_per_pair(d, reps) / ms / 1e9,
            }
            if split_ms is not None:
                res[f"chi{chi}_{name}"]["split_operands_ms"] = split_ms
    diff = np.abs(kq_block[(32, "fp32")] - kq_block[(32, "bf16x3")])
    res["chi32_max_abs_dK_bf16x3_vs_fp32_block"] = float(diff.max())
    res["chi32_max_abs_dK_bf16x3_vs_fp32_sampled"] = float(max(diff[i, j] for i, j in pairs))
    off = ~np.eye(m, dtype=bool)
    res["chi32_offdiag_entries_with_K>1e-3"] = int((kq_block[(32, "fp32")][off] > 1e-3).sum())
    ctx.sync_status()
    if own:
        ctx.close()
    if return_blocks:
        return res, pairs, kq_block, x
    return res


def _event_ms(fn):
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    fn()
    b.record()
    b.synchronize()
    return a.elapsed_time(b)


def sampled_pairs_full_size(pairs, near_base, m: int = 4000, d: int = 256, near_sigma=(1e-4, 2.5e-2),
                            near_seed: int = 65, ctx: dualk.Context | None = None):
    """The precision form at full size: the whole m x m Gram of the d-feature Fashion-MNIST-shaped
    set at reps = 3 (bond 8, FP32) and reps = 5 (bond 32, FP32 and split-BF16 tensor cores),
    each timed once, and the rows of the near copies of the samples `near_base` against the
    set. Returns, per path, the timings and the K_q and log K_q of the listed pairs:
    pairs = [(group, i, j)], group "near_copy" meaning (set sample i, copy j), else the Gram
    entry (i, j)."""
    own = ctx is None
    ctx = ctx or dualk.Context(0)
    x = synthetic.fmnist_like(m, 0, d)["x_train"]
    xn = synthetic.near_copies(x[np.asarray(near_base)], near_sigma[0], near_sigma[1], seed=near_seed)
    xt = torch.from_numpy(x).cuda()
    xnt = torch.from_numpy(xn).cuda()
    gi = torch.tensor([i for g, i, j in pairs if g != "near_copy"], device="cuda", dtype=torch.long)
    gj = torch.tensor([j for g, i, j in pairs if g != "near_copy"], device="cuda", dtype=torch.long)
    ri = torch.tensor([j for g, i, j in pairs if g == "near_copy"], device="cuda", dtype=torch.long)
    rj = torch.tensor([i for g, i, j in pairs if g == "near_copy"], device="cuda", dtype=torch.long)
    is_row = np.array([g == "near_copy" for g, _, _ in pairs])
    res = {"workload": f"fmnist d={d} m={m}: full symmetric Gram + rows of {len(near_base)} near copies"}
    out = {"kq": torch.empty((m, m), device="cuda"), "logkq": torch.empty((m, m), device="cuda")}
    rows = {"kq": torch.empty((len(near_base), m), device="cuda"),
            "logkq": torch.empty((len(near_base), m), device="cuda")}
    for reps, chi, precs in ((3, 8, (("fp32", dualk.DK_PREC_F32),)),
                             (5, 32, (("fp32", dualk.DK_PREC_F32), ("bf16x3", dualk.DK_PREC_BF16X3)))):
        fm = dualk.FeatureMap(reps=reps, chi_max=chi)
        mp = dualk.mps_build(ctx, xt, fm)
        mpn = dualk.mps_build(ctx, xnt, fm)
        for name, prec in precs:
            mp.log_norm_for(ctx, prec)
            mpn.log_norm_for(ctx, prec)
            torch.cuda.synchronize()
            split_ms = None
            if prec == dualk.DK_PREC_BF16X3:  # the split operands, made once per MPS
                split_ms = _event_ms(lambda: (mp.split_for(ctx), mpn.split_for(ctx)))
            g_ms = _event_ms(lambda: dualk.gram_tile(ctx, mp, mp, symmetric=True, out=out, ld=m, w=1.0, prec=prec,
                                                     want=("kq", "logkq")))
            r_ms = _event_ms(lambda: dualk.dual_kernel_rows(ctx, mpn, mp, w=1.0, out=rows, prec=prec,
                                                            want=("kq", "logkq")))
            kq = np.empty(len(pairs))
            lkq = np.empty(len(pairs))
            kq[~is_row] = out["kq"][gi, gj].double().cpu().numpy()
            lkq[~is_row] = out["logkq"][gi, gj].double().cpu().numpy()
            kq[is_row] = rows["kq"][ri, rj].double().cpu().numpy()
            lkq[is_row] = rows["logkq"][ri, rj].double().cpu().numpy()
            units = workload.gram_entries(m) * d
            res[f"chi{chi}_{name}"] = {
                "gram_ms": g_ms, "rows_ms": r_ms, "gram_entry_qubits_per_s": units / (g_ms / 1e3),
                "gram_tflops_block_count": workload.gram_entries(m) * workload.flops_per_pair(d, reps) / g_ms / 1e9,
                "kq": kq, "logkq": lkq}
            if split_ms is not None:
                res[f"chi{chi}_{name}"]["split_operands_ms"] = split_ms
        del mp, mpn
    ctx.sync_status()
    if own:
        ctx.close()
    return res


def compare_build_qr(m: int = 2000, d: int = 784, block: int = 256, ctx: dualk.Context | None = None):
    """The bond-4 MPS build with its QR sweep in FP32 (default) and in FP64, both stored as
    complex64: build time for m samples at d features, and the largest |dK| and |d log K|
    between the two Gram blocks of the first `block` samples; plus the same on 96
    uniform-angle samples at d = 8, where many K_q are O(1) (largest relative dK there)."""
    own = ctx is None
    ctx = ctx or dualk.Context(0)
    res = {"workload": f"fmnist d={d} m={m} (build timing), Gram of the first {block}; uniform d=8 m=96"}
    cases = {"fmnist": torch.from_numpy(synthetic.fmnist_like(m, 0, d)["x_train"]).cuda(),
             "uniform8": torch.from_numpy(synthetic.uniform_angles(96, 8, seed=5).astype(np.float32)).cuda()}
    out = {}
    for name, prec in (("fp32_qr", dualk.DK_PREC_F32), ("fp64_qr", dualk.DK_PREC_F64)):
        fm = dualk.FeatureMap(reps=2, chi_max=4, qr_prec=prec)
        x = cases["fmnist"]
        buf = torch.empty(dualk.mps_bytes(m, d, 4), dtype=torch.uint8, device="cuda")
        res[f"build_ms_{name}"] = _time(lambda: dualk.mps_build(ctx, x, fm, out=buf), reps=3)
        mp = dualk.mps_build(ctx, x[:block].contiguous(), fm)
        g = dualk.gram(ctx, mp, w=1.0, want=("kq", "logkq"))
        mu = dualk.mps_build(ctx, cases["uniform8"], fm)
        gu = dualk.gram(ctx, mu, w=1.0, want=("kq",))
        out[name] = ({k: v.cpu().numpy().astype(np.float64) for k, v in g.items() if v is not None},
                     gu["kq"].cpu().numpy().astype(np.float64))
    a, b = out["fp32_qr"], out["fp64_qr"]
    res["max_abs_dK_fmnist"] = float(np.abs(a[0]["kq"] - b[0]["kq"]).max())
    res["max_abs_dlogK_fmnist"] = float(np.abs(a[0]["logkq"] - b[0]["logkq"]).max())
    big = b[1] > 1e-3
    res["max_abs_dK_uniform8"] = float(np.abs(a[1] - b[1]).max())
    res["max_rel_dK_uniform8_K>1e-3"] = float((np.abs(a[1] - b[1])[big] / b[1][big]).max())
    ctx.sync_status()
    if own:
        ctx.close()
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
