"""Kernel matrices of block-structured feature maps (§II-C: entanglers only inside blocks of b
consecutive qubits) by per-block statevector overlaps: ``dk_block_states`` builds every
block's 2^b amplitudes, ``dk_gram_blocks`` contracts the Gram and the decision rows, exact at
any n (no bond, no truncation). This module drives those two calls for a training set and a
test batch and times them; all arithmetic runs in libdualk's kernels.

    python -m paper_2602_01330_gb300.blockmap --m 2000 --m-test 500 --n 784 --block 10
"""
from __future__ import annotations

import argparse
import json
import os
import statistics

import torch

from . import dualk, synthetic, workload


def gram_flops(m_rows: int, m_cols: int, n: int, block: int, symmetric: bool) -> float:
    """Algorithmic FP32 flops: 8 per amplitude (one complex multiply-accumulate) per block and
    pair, over the unique pairs (m (m + 1) / 2 for a symmetric Gram)."""
    nb = -(-n // block)
    pairs = m_rows * (m_rows + 1) / 2 if symmetric else m_rows * m_cols
    return pairs * nb * 8 * max(2 ** block, 16)


def bf16_peak_tflops() -> tuple[float, str]:
    """Dense BF16 tensor peak: the measured burst figure of this machine's GPUs when the
    measurement file is present at the repository root, else 1900 (an earlier GB300 run)."""
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback"


def run_benchmark(ctx: dualk.Context, m: int = 2000, m_test: int = 500, n: int = 784, block: int = 10,
                  reps: int = 2, entangler: int = dualk.DK_ENT_FULL, w: float = 0.5, iters: int = 3,
                  prec: int = dualk.DK_PREC_F32, form: int = dualk.DK_BLOCK_TCGEN05) -> dict:
    """Block states of both sets, the symmetric training Gram and the test rows, timed with
    CUDA events; for prec = DK_PREC_BF16X3 `form` selects the tcgen05 or mma.sync kernels."""
    ctx.set_block_gram_form(form)
    try:
        return _run_benchmark(ctx, m, m_test, n, block, reps, entangler, w, iters, prec, form)
    finally:
        ctx.set_block_gram_form(dualk.DK_BLOCK_TCGEN05)


def _run_benchmark(ctx, m, m_test, n, block, reps, entangler, w, iters, prec, form) -> dict:
    d = synthetic.fmnist_like(m, m_test, n)
    xtr = torch.from_numpy(d["x_train"]).cuda()
    xte = torch.from_numpy(d["x_test"]).cuda()
    fm = dualk.FeatureMap(reps=reps, block=block)
    st = torch.cuda.current_stream()
    times = {"states_ms": [], "gram_ms": [], "rows_ms": []}
    for it in range(iters + 1):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(st)
        tr = dualk.block_states(ctx, xtr, fm, entangler, prec=prec)
        te = dualk.block_states(ctx, xte, fm, entangler, prec=prec) if m_test > 0 else None
        ev[1].record(st)
        g = dualk.gram_blocks(ctx, tr, w=w, want=("k", "kq", "kc", "logkq"))
        ev[2].record(st)
        r = dualk.gram_blocks(ctx, te, tr, w=w, want=("k", "kq", "kc", "logkq")) if m_test > 0 else None
        ev[3].record(st)
        torch.cuda.synchronize()
        if it == 0:
            continue  # warm-up
        times["states_ms"].append(ev[0].elapsed_time(ev[1]))
        times["gram_ms"].append(ev[1].elapsed_time(ev[2]))
        times["rows_ms"].append(ev[2].elapsed_time(ev[3]))
    ctx.sync_status()
    t = {k: statistics.mean(v) for k, v in times.items()}
    props = torch.cuda.get_device_properties(0)
    achieved = gram_flops(m, m, n, block, True) / (t["gram_ms"] * 1e-3) / 1e12
    if prec == dualk.DK_PREC_BF16X3:
        bf16, src = bf16_peak_tflops()
        kern = ("gram_blocks_umma_kernel<128, wide> (symmetric Gram, tcgen05 bf16x3, N = 256 MMAs)" if form == dualk.DK_BLOCK_TCGEN05
                else "gram_blocks_tc_kernel (symmetric Gram, mma.sync bf16x3)")
        roof = {"bound": "tensor", "kernel": kern,
                "achieved": achieved, "peak": bf16 / 3, "unit": "TFLOP/s (FP32-equivalent)",
                "frac": achieved / (bf16 / 3),
                "peak_source": f"dense BF16 {bf16:.1f} TFLOP/s ({src}) / 3 products per FP32-equivalent product"}
    else:
        peak = workload.fp32_peak_tflops(props.multi_processor_count, 2070.0)
        roof = {"bound": "alu", "kernel": "gram_blocks_kernel (symmetric Gram)", "achieved": achieved,
                "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "peak_source": f"FP32 FMA peak {props.multi_processor_count} SMs x 128 lanes x 2 x 2070 MHz"}
    entries = m * (m + 1) / 2 + m * m_test
    diag = torch.diagonal(g["kq"])
    return {
        "workload": f"fmnist-shaped n={n}, blocks of {block} "
                    f"({'all-to-all' if entangler == dualk.DK_ENT_FULL else 'chain'} ZZ), reps {reps}, "
                    f"{m} train (symmetric Gram) + {m_test} test rows",
        **t,
        "entry_qubits_per_s": entries * n / ((t["gram_ms"] + t["rows_ms"]) * 1e-3),
        "precision": "bf16x3" if prec == dualk.DK_PREC_BF16X3 else "f32",
        "form": ("tcgen05" if form == dualk.DK_BLOCK_TCGEN05 else "mma_sync") if prec == dualk.DK_PREC_BF16X3 else None,
        "roofline": roof,
        "diag_kq_exactly_1": bool(torch.all(diag == 1.0).item()),
        "mean_offdiag_log_kq": float((g["logkq"].sum() - g["logkq"].diagonal().sum()).item() / (m * m - m)),
        "max_row_k": float(r["k"].max().item()) if r is not None else None,
    }


def concentration(ctx: dualk.Context, dims=(8, 16, 32, 64, 128, 256, 784), m: int = 1000, reps: int = 2,
                  blocks=(8,), entangler: int = dualk.DK_ENT_FULL) -> dict:
    """Kernel concentration against the qubit count (§I; the diagnostics of §IV): per n, the
    mean and variance of the off-diagonal K_q and log K_q of a symmetric Gram of m samples,
    for the chain (MPS path) and for block-structured maps with the given block sizes
    (block-statevector path). dk_gram_stats forms the FP64 sums."""
    res = {}
    for d in dims:
        x = torch.from_numpy(synthetic.fmnist_like(m, 0, d)["x_train"]).cuda()
        row = {}
        g = dualk.gram(ctx, dualk.mps_build(ctx, x, dualk.FeatureMap(reps=reps, chi_max=4)), w=1.0,
                       want=("kq", "logkq"))
        row["chain"] = dualk.gram_stats(ctx, g["kq"], g["logkq"], symmetric=True)
        for b in blocks:
            st = dualk.block_states(ctx, x, dualk.FeatureMap(reps=reps, block=b), entangler)
            gb = dualk.gram_blocks(ctx, st, w=1.0, want=("kq", "logkq"))
            row[f"blocks_of_{b}"] = dualk.gram_stats(ctx, gb["kq"], gb["logkq"], symmetric=True)
        res[d] = {k: {q: v[q] for q in ("kq_mean", "kq_var", "logkq_mean", "logkq_var")} for k, v in row.items()}
    ctx.sync_status()
    return res


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--m", type=int, default=2000)
    ap.add_argument("--m-test", type=int, default=500)
    ap.add_argument("--n", type=int, default=784)
    ap.add_argument("--block", type=int, default=10)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--entangler", choices=("full", "chain"), default="full")
    ap.add_argument("--iters", type=int, default=3)
    ap.add_argument("--prec", choices=("f32", "bf16x3"), default="f32")
    ap.add_argument("--form", choices=("tcgen05", "mma_sync"), default="tcgen05",
                    help="tensor-core kernels of the bf16x3 block Gram")
    ap.add_argument("--concentration", action="store_true",
                    help="report kernel concentration against n for the chain and block maps instead")
    args = ap.parse_args()
    ctx = dualk.Context(0)
    if args.concentration:
        ent = dualk.DK_ENT_FULL if args.entangler == "full" else dualk.DK_ENT_CHAIN
        print(json.dumps(concentration(ctx, m=1000, reps=args.reps, blocks=(4, 8, args.block), entangler=ent)))
        ctx.close()
        return
    ent = dualk.DK_ENT_FULL if args.entangler == "full" else dualk.DK_ENT_CHAIN
    prec = dualk.DK_PREC_BF16X3 if args.prec == "bf16x3" else dualk.DK_PREC_F32
    form = dualk.DK_BLOCK_TCGEN05 if args.form == "tcgen05" else dualk.DK_BLOCK_MMA_SYNC
    print(json.dumps(run_benchmark(ctx, args.m, args.m_test, args.n, args.block, args.reps, ent, iters=args.iters,
                                   prec=prec, form=form)))
    ctx.close()


if __name__ == "__main__":
    main()
