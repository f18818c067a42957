#!/usr/bin/env python3
"""Benchmark of the quantum-kernel Gram hot path: Gram entries x qubits per second.

Workload (one step, all of the hot path): Fashion-MNIST-shaped synthetic data at d = 784
features (raw pixels, one qubit per feature), 2000 training + 500 test samples, ZZ-chain
map with reps = 2 (bond chi = 4), complex64 / FP32:
  MPS build of the 2000 training and the 500 test samples (closed-form sites, FP32 QR sweep),
  the symmetric 2000 x 2000 Gram with the fused RBF kernel and mix (w = 0.5; K, K_q,
  K_c and log K_q written), and the 500 x 2000 dual-kernel rows.
Unit of work: one entry x qubit (one pair through one site). Entries per step =
2000*2001/2 + 500*2000 = 3,001,000; x 784 qubits = 2.353e9 entry-qubits.

Default arm: our CUDA library (libdualk.so) through its Python binding. `--impl reference`
times the FP64 CPU oracle on a bounded sample of the same workload.
Multi-GPU (torchrun, one rank per GPU): each rank runs its own independent problem of the
same size (weak scaling, no collective on the data path). `--split` instead splits one
8000-sample Gram at n = 784 into balanced row blocks over the ranks (strong scaling; the
blocks are gathered to the hosts in the end-to-end leg only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

os.environ.setdefault("OMP_NUM_THREADS", "1")
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")

import numpy as np  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

WL = dict(workload="fmnist784_gram2000_rows500", d=784, n_train=2000, n_test=500, reps=2, chi=4, w=0.5)
METRIC = "Gram entries*qubits/s (n=784,chi=4)"
UNIT = "entry-qubits/s"


def entries_per_step(n_train, n_test):
    return n_train * (n_train + 1) // 2 + n_test * n_train


# DRAM bytes (read + write) of one Gram launch of the benchmarked workload, from one ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum, 1 pass) of this bench's own launch;
# the command and figures are in profiles/gram_kernel_dram_traffic_fmnist784_gram2000.md.
# Reported only while the kernel sources hash to the value they had when it was taken.
GRAM_TRAFFIC = {"n_train": 2000, "sources_sha256": "d7100897afe176cb8d2918401f2fa29e7df0cb977e028484a2892cc168a8062d",
                "bytes_by_tile_shape": {17: 2002821376 + 59936768}}
GRAM_SOURCES = ["gram.cu", "gram_common.cuh", "transfer.cuh", "common.cuh"]


def gram_sources_sha256() -> str:
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2602_01330_gb300", "csrc")
    for f in GRAM_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def gram_traffic(n_train: int, tile_shape_id: int):
    """Measured DRAM bytes per Gram launch, or None if the kernel, its tile shape or the
    workload differs."""
    if n_train != GRAM_TRAFFIC["n_train"] or tile_shape_id not in GRAM_TRAFFIC["bytes_by_tile_shape"]:
        return None
    if gram_sources_sha256() != GRAM_TRAFFIC["sources_sha256"]:
        return None
    return GRAM_TRAFFIC["bytes_by_tile_shape"][tile_shape_id]


def measured_peaks():
    try:
        with open(os.path.join(HERE, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.device_index = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device_index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names[1:], parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def oracle_rate(n_train, n_test, d, reps, seed_train=1, seed_test=2):
    """The FP64 oracle on a sample of the workload: MPS of n_train + n_test samples, the
    unique pairs of the train Gram and the test x train rows. Returns (entry-qubits/s, seconds)."""
    from oracle import gram, mps
    from paper_2602_01330_gb300 import synthetic
    data = synthetic.fmnist_like(n_train, n_test, d, seed_train=seed_train, seed_test=seed_test)
    xtr = data["x_train"].astype(np.float64)
    xte = data["x_test"].astype(np.float64)
    t0 = time.perf_counter()
    otr, _ = mps.build_mps(xtr, reps)
    ote, _ = mps.build_mps(xte, reps)
    iu, ju = np.triu_indices(n_train)
    kq, _ = gram.pair_values(otr, otr, iu, ju)
    kc = gram.rbf_pairs(xtr, xtr, iu, ju, 1.0 / d)
    gram.dual_kernel(kq, kc, WL["w"])
    ii, jj = np.meshgrid(np.arange(n_test), np.arange(n_train), indexing="ij")
    kq2, _ = gram.pair_values(ote, otr, ii.ravel(), jj.ravel())
    kc2 = gram.rbf_pairs(xte, xtr, ii.ravel(), jj.ravel(), 1.0 / d)
    gram.dual_kernel(kq2, kc2, WL["w"])
    dt = time.perf_counter() - t0
    units = (n_train * (n_train + 1) // 2 + n_test * n_train) * d
    return units / dt, dt


def _oracle_build(args):
    """Worker: the oracle MPS of one chunk of samples."""
    from oracle import mps
    x, reps = args
    return mps.build_mps(x, reps)[0]


def _oracle_pairs(args):
    """Worker: the oracle log K_q of all pairs between two chunks (i_idx x j_idx lists)."""
    from oracle import gram
    rows, cols, ii, jj = args
    return gram.pair_values(rows, cols, ii, jj)[1]


def oracle_rate_all_cores(n_train, n_test, d, reps, procs):
    """The same oracle sample as oracle_rate, its work split over `procs` spawned processes:
    the MPS builds by sample chunk, then the Gram and row entries by (row chunk, column
    chunk) block, each block contracted by the oracle's own pair_values. Returns
    (entry-qubits/s, seconds)."""
    import multiprocessing as mp
    from paper_2602_01330_gb300 import synthetic
    data = synthetic.fmnist_like(n_train, n_test, d)
    xtr = data["x_train"].astype(np.float64)
    xte = data["x_test"].astype(np.float64)
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        pool.map(_oracle_build, [(xtr[:1, :8], 1)] * procs)  # start-up and imports, untimed
        t0 = time.perf_counter()
        cut_tr = np.array_split(np.arange(n_train), procs)
        cut_te = np.array_split(np.arange(n_test), max(1, procs // 4))
        chunks = [xtr[c] for c in cut_tr if c.size] + [xte[c] for c in cut_te if c.size]
        built = pool.map(_oracle_build, [(c, reps) for c in chunks])
        n_tr_chunks = sum(1 for c in cut_tr if c.size)
        tasks = []
        for a in range(len(built)):
            for b in range(n_tr_chunks):
                if a < n_tr_chunks and b < a:
                    continue  # the symmetric Gram needs each unordered pair once
                ma, mb = built[a][0].shape[0], built[b][0].shape[0]
                ii, jj = np.meshgrid(np.arange(ma), np.arange(mb), indexing="ij")
                sel = (ii <= jj) if a == b else np.ones_like(ii, dtype=bool)
                tasks.append((built[a], built[b], ii[sel], jj[sel]))
        pool.map(_oracle_pairs, tasks)
        dt = time.perf_counter() - t0
    units = (n_train * (n_train + 1) // 2 + n_test * n_train) * d
    return units / dt, dt


GOLDEN_CFG3 = os.path.join(HERE, "tests", "golden", "cfg3_sampled_pairs.txt")


def load_cfg3_golden(path=GOLDEN_CFG3):
    """Stored FP64 oracle values of the precision form's sampled pairs (written by
    tests/golden/make_cfg3_golden.py from the oracle): rows of (group, i, j, K_q and log K_q
    at reps 3 and 5), the input checksum and the near-copy parameters."""
    rows, meta = [], {}
    with open(path) as f:
        for line in f:
            if line.startswith("# input_sha256"):
                meta["sha256"] = line.split()[2]
            if line.startswith("#"):
                continue
            g, i, j, a, b, c, d = line.split()
            rows.append((g, int(i), int(j), float(a), float(b), float(c), float(d)))
    return rows, meta


def precision_vs_oracle(ctx):
    """The precision form at its stated size (d = 256, 4000 samples, reps 3 / 5): full Grams on
    the GPU (FP32 at bond 8; FP32 and split-BF16 at bond 32) and the error of each path
    against the stored FP64 oracle values on 2000 sampled pairs (1000 uniform, 500 nearest
    neighbours, 500 diagonal) plus 200 near-duplicate pairs, per group."""
    import hashlib
    from paper_2602_01330_gb300 import precision, synthetic
    rows, meta = load_cfg3_golden()
    pairs = [(g, i, j) for g, i, j, *_ in rows]
    base = [i for g, i, j, *_ in rows if g == "near_copy"]
    x = synthetic.fmnist_like(4000, 0, 256)["x_train"]
    xn = synthetic.near_copies(x[np.asarray(base)], 1e-4, 2.5e-2, seed=65)
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(x, dtype=np.float32).tobytes())
    h.update(np.ascontiguousarray(xn, dtype=np.float32).tobytes())
    got = precision.sampled_pairs_full_size(pairs, base, ctx=ctx)
    groups = np.array([g for g, *_ in rows])
    ref = {3: (np.array([r[3] for r in rows]), np.array([r[4] for r in rows])),
           5: (np.array([r[5] for r in rows]), np.array([r[6] for r in rows]))}
    out = {"workload": got["workload"] + "; errors against the stored FP64 oracle values",
           "inputs_match_stored": h.hexdigest() == meta.get("sha256")}
    for key, reps in (("chi8_fp32", 3), ("chi32_fp32", 5), ("chi32_bf16x3", 5)):
        kq_ref, lkq_ref = ref[reps]
        kq, lkq = got[key]["kq"], got[key]["logkq"]
        entry = {k: v for k, v in got[key].items() if k not in ("kq", "logkq")}
        for g in ("uniform", "nearest", "diagonal", "near_copy"):
            sel = groups == g
            dk = np.abs(kq[sel] - kq_ref[sel])
            fin = sel & (lkq_ref > -700)
            big = sel & (kq_ref > 1e-3)
            entry[g] = {"pairs": int(sel.sum()), "max_abs_dK": float(dk.max()),
                        "max_rel_dlogK": float(np.max(np.abs(lkq[fin] - lkq_ref[fin]) /
                                                      np.maximum(1.0, np.abs(lkq_ref[fin])))) if fin.any() else None,
                        "pairs_K_gt_1e-3": int(big.sum()),
                        "max_rel_dK_K_gt_1e-3": float(np.max(np.abs(kq[big] - kq_ref[big]) / kq_ref[big]))
                        if big.any() else None}
        entry["max_abs_dK"] = max(entry[g]["max_abs_dK"] for g in ("uniform", "nearest", "diagonal", "near_copy"))
        entry["tolerance"] = 1e-4 if "bf16x3" in key else 1e-6
        entry["within_tolerance"] = entry["max_abs_dK"] <= entry["tolerance"]
        out[key] = entry
    return out


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    sample = dict(n_train=24, n_test=8)
    for _ in range(args.warmup):
        oracle_rate(sample["n_train"], sample["n_test"], WL["d"], WL["reps"])
    rates, secs = [], []
    for _ in range(args.steps):
        r, s = oracle_rate(sample["n_train"], sample["n_test"], WL["d"], WL["reps"])
        rates.append(r)
        secs.append(s)
    total_units = sum(r * s for r, s in zip(rates, secs))
    value = total_units / sum(secs)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(secs) / len(secs),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (Fashion-MNIST-shaped, seeded)",
        "config": {"workload": WL["workload"], "d": WL["d"], "reps": WL["reps"], "chi": WL["chi"],
                   "sample_per_step": f"{sample['n_train']} train + {sample['n_test']} test samples"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"per step: MPS of {sample['n_train']}+{sample['n_test']} samples at n=784, "
                                   f"{sample['n_train'] * (sample['n_train'] + 1) // 2} Gram + "
                                   f"{sample['n_train'] * sample['n_test']} row entries"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def end_to_end(torch, tdist, args, world, stream, flush, x_tr, x_te, g_out, r_out, data, step, units_step,
               barrier, dev):
    """The same metric through the public API: pinned host inputs copied in and the K blocks
    copied out inside the timed region, every step."""
    n_tr, n_te = x_tr.shape[0], x_te.shape[0]
    h_xtr = torch.from_numpy(data["x_train"]).pin_memory()
    h_xte = torch.from_numpy(data["x_test"]).pin_memory()
    h_k = torch.empty((n_tr, n_tr), dtype=torch.float32).pin_memory()
    h_r = torch.empty((n_te, n_tr), dtype=torch.float32).pin_memory()
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        flush.zero_()
        x_tr.copy_(h_xtr, non_blocking=True)
        x_te.copy_(h_xte, non_blocking=True)
        step()
        h_k.copy_(g_out["k"], non_blocking=True)
        h_r.copy_(r_out["k"], non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    e2e_ms = e0.elapsed_time(e1)
    if world > 1:
        tt = torch.tensor([e2e_ms], device=dev)
        tdist.all_reduce(tt, op=tdist.ReduceOp.MAX)
        e2e_ms = float(tt.item())
    e2e_value = world * units_step * args.steps / (e2e_ms / 1e3)
    h2d = h_xtr.numel() * 4 + h_xte.numel() * 4
    d2h = h_k.numel() * 4 + h_r.numel() * 4
    return {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}



def run_ours(args):
    import torch
    import torch.distributed as tdist

    from paper_2602_01330_gb300 import build as libbuild
    from paper_2602_01330_gb300 import dualk, synthetic, workload

    world, rank, local = dist_setup()
    if world > 1:
        tdist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if not os.path.exists(dualk.LIB_PATH):
        libbuild.build()

    n_tr, n_te, d, reps, chi, w = WL["n_train"], WL["n_test"], WL["d"], WL["reps"], WL["chi"], WL["w"]
    data = synthetic.fmnist_like(n_tr, n_te, d, seed_train=1 + 100 * rank, seed_test=2 + 100 * rank)
    ctx = dualk.Context(local)
    fm = dualk.FeatureMap(reps=reps, chi_max=chi)
    stream = torch.cuda.current_stream()

    x_tr = torch.from_numpy(data["x_train"]).to(dev)
    x_te = torch.from_numpy(data["x_test"]).to(dev)
    mps_tr = torch.empty(dualk.mps_bytes(n_tr, d, chi), dtype=torch.uint8, device=dev)
    mps_te = torch.empty(dualk.mps_bytes(n_te, d, chi), dtype=torch.uint8, device=dev)
    g_out = {k: torch.empty((n_tr, n_tr), dtype=torch.float32, device=dev) for k in ("k", "kq", "kc", "logkq")}
    r_out = {k: torch.empty((n_te, n_tr), dtype=torch.float32, device=dev) for k in ("k", "kq", "kc", "logkq")}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2
    bond_tr = torch.empty(d + 1, dtype=torch.int32, device=dev)
    bond_te = torch.empty(d + 1, dtype=torch.int32, device=dev)
    ln_tr = torch.empty(n_tr, dtype=torch.float32, device=dev)
    ln_te = torch.empty(n_te, dtype=torch.float32, device=dev)
    side = torch.cuda.Stream(device=dev)  # the test-set build runs beside the training-set build
    ref_ws = dualk.refine_workspace(n_tr, n_tr, dev)  # the refinement passes' workspace (once-per-sample norms)

    # Tile shapes for the two Gram launches, picked by the library's autotuner (sweep.py) on a
    # 48-site probe of the same sample sets, before anything is timed.
    # --tile-shapes G,R fixes them instead (profiling runs, where the tuner's launches would
    # shift the launch indices).
    if args.tile_shapes:
        cfg_gram, cfg_rows = (int(v) for v in args.tile_shapes.split(","))
    else:
        from paper_2602_01330_gb300.sweep import Autotuner
        tuner = Autotuner(ctx)
        mtr0 = dualk.mps_build(ctx, x_tr, fm, out=mps_tr, bond=bond_tr, log_norm=ln_tr)
        mte0 = dualk.mps_build(ctx, x_te, fm, out=mps_te, bond=bond_te, log_norm=ln_te)
        cfg_gram = tuner.best(mtr0, symmetric=True)
        cfg_rows = tuner.best(mte0, symmetric=False, cols=mtr0)

    phase_events = []  # per timed step: events around build, Gram, its refinement, rows, theirs

    def step(record=False):
        # The test-set build runs on a side stream beside the training-set build (each is a
        # latency-bound chain per sample); the Gram and the rows then run one after the other
        # on the main stream, each followed by its refinement pass, so each launch's own time
        # is measured.
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)] if record else None
        rec = (lambda q: ev[q].record(stream)) if record else (lambda q: None)
        rec(0)
        side.wait_stream(stream)
        mtr = dualk.mps_build(ctx, x_tr, fm, out=mps_tr, bond=bond_tr, log_norm=ln_tr)
        mte = dualk.mps_build(ctx, x_te, fm, out=mps_te, bond=bond_te, log_norm=ln_te, stream=side)
        rec(1)
        ctx.set_gram_config(cfg_gram)
        dualk.gram_tile(ctx, mtr, mtr, symmetric=True, w=w, out=g_out, ld=n_tr, refine=None)
        rec(2)
        dualk.gram_refine(ctx, mtr, mtr, 0, n_tr, 0, n_tr, g_out, n_tr, 1.0 / d, w, symmetric=True, ws=ref_ws)
        rec(3)
        stream.wait_stream(side)
        ctx.set_gram_config(cfg_rows)
        dualk.dual_kernel_rows(ctx, mte, mtr, w=w, out=r_out, refine=None)
        rec(4)
        dualk.gram_refine(ctx, mte, mtr, 0, n_te, 0, n_tr, r_out, n_tr, 1.0 / d, w, ws=ref_ws)
        rec(5)
        if record:
            phase_events.append(ev)

    # MPS build x 2 (the ln-norms are fused into the build at bond 4), Gram, rows, and the
    # refinement pass after each of the two (dk_gram_refine with a workspace: a scan marking
    # the samples entries with K_q > 0.02 need, their double-word norms, the pass; here scans
    # only, as no off-diagonal K_q of independent 784-qubit samples comes near 0.02): ten
    # libdualk kernels per step
    launches_per_step = 2 + 1 + 1 + 2 * 3

    def barrier():
        if world > 1:
            tdist.barrier()

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    ctx.sync_status()

    sampler = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        flush.zero_()
        step(record=True)
    t1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ms = t0.elapsed_time(t1)
    if world > 1:
        tt = torch.tensor([ms], device=dev)
        tdist.all_reduce(tt, op=tdist.ReduceOp.MAX)
        ms = float(tt.item())
    ctx.sync_status()
    gram_ms = [ev[1].elapsed_time(ev[2]) for ev in phase_events]
    phases = {"mps_build_ms": statistics.mean(ev[0].elapsed_time(ev[1]) for ev in phase_events),
              "gram_ms": statistics.mean(gram_ms),
              "gram_refine_ms": statistics.mean(ev[2].elapsed_time(ev[3]) for ev in phase_events),
              "rows_ms": statistics.mean(ev[3].elapsed_time(ev[4]) for ev in phase_events),
              "rows_refine_ms": statistics.mean(ev[4].elapsed_time(ev[5]) for ev in phase_events)}

    units_step = entries_per_step(n_tr, n_te) * d
    value = world * units_step * args.steps / (ms / 1e3)

    e2e = None
    if not args.no_e2e:
        e2e = end_to_end(torch, tdist, args, world, stream, flush, x_tr, x_te, g_out, r_out, data, step,
                         units_step, barrier, dev)

    tile_gram = dualk.gram_config_info(cfg_gram)
    peaks = measured_peaks()
    props = torch.cuda.get_device_properties(dev)
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_tflops = workload.fp32_peak_tflops(props.multi_processor_count, sm_max)
    gram_flops = workload.gram_entries(n_tr) * workload.flops_per_pair(d, reps)
    gram_avg_ms = statistics.mean(gram_ms)
    achieved = gram_flops / (gram_avg_ms / 1e3) / 1e12

    cpu = cpu_all = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        s_tr, s_te = 48, 16
        rate, secs = oracle_rate(s_tr, s_te, d, reps)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"MPS of {s_tr}+{s_te} samples at n=784 (TEBD), {s_tr * (s_tr + 1) // 2} Gram + "
                         f"{s_tr * s_te} row entries, {secs:.1f} s, FP64 NumPy single thread"}
        procs = os.cpu_count() or 1
        rate_all, secs_all = oracle_rate_all_cores(s_tr, s_te, d, reps, procs)
        cpu_all = {"value": rate_all, "unit": UNIT, "cores": procs, "kind": "oracle",
                   "sample": f"the same sample, MPS builds by sample chunk and pair blocks split over {procs} "
                             f"spawned processes (one BLAS thread each), {secs_all:.1f} s wall"}

    # The other two parts of the metric, measured after the timed region (rank 0, one GPU):
    # the precision form at its stated size (d = 256, 4000 samples) against the stored FP64
    # oracle values of its sampled pairs; the split-BF16 tensor-core Gram against the FP32 one
    # at bond 32 on 512 samples (d = 256, where every off-diagonal K_q is tiny, and d = 16,
    # where many are not); the FP32 against the FP64 QR sweep of the bond-4 build; and the
    # continuous-batching server's latency.
    mixed = serving_stats = svm_stats = block_stats = sweep_stats = None
    if rank == 0 and world == 1 and not args.no_extras:
        from paper_2602_01330_gb300 import blockmap, precision, serving, svm
        from paper_2602_01330_gb300 import sweep as gsweep
        # the feature-dimension sweep: ten 2000-sample Grams, d = 2 .. 784
        sweep_stats = gsweep.run_benchmark(ctx, m=2000, peak_tflops=peak_tflops)
        mixed = {"cfg3_full_size_vs_oracle": precision_vs_oracle(ctx),
                 "d256": precision.compare(m=512, pool=128, n_uniform=40, n_near=20, n_diag=10, ctx=ctx),
                 "d16": precision.compare(m=512, d=16, pool=128, n_uniform=40, n_near=20, n_diag=10, ctx=ctx),
                 "mps_build_qr": precision.compare_build_qr(ctx=ctx)}
        serving_stats = serving.run_benchmark(ctx, m=8000, requests=2000, rho=(0.5, 0.8, 0.95), slots=8)
        # the SVM that consumes this step's Gram and rows: 5-fold CV over C x w, fit, test votes
        svm_stats = svm.run_pipeline(ctx, n_tr, n_te, d, reps,
                                     gram=(g_out["kq"], g_out["kc"], r_out["kq"], r_out["kc"]))
        # the same data through a block-structured map (all-to-all ZZ in blocks of 10 qubits),
        # contracted exactly by per-block statevector overlaps
        block_stats = {"f32": blockmap.run_benchmark(ctx, n_tr, n_te, d, block=10, reps=reps),
                       "bf16x3": blockmap.run_benchmark(ctx, n_tr, n_te, d, block=10, reps=reps,
                                                        prec=dualk.DK_PREC_BF16X3),
                       "bf16x3_mma_sync": blockmap.run_benchmark(ctx, n_tr, n_te, d, block=10, reps=reps,
                                                                 prec=dualk.DK_PREC_BF16X3,
                                                                 form=dualk.DK_BLOCK_MMA_SYNC)}

    if world > 1:
        tdist.destroy_process_group()
    ctx.close()
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (Fashion-MNIST-shaped, seeded; the real data set is not available)",
        "config": {"workload": WL["workload"], "d": d, "n_train": n_tr, "n_test": n_te, "reps": reps, "chi": chi,
                   "w": w, "mps_dtype": "complex64", "parallelism": f"independent problem per GPU x{world}",
                   "l2": "256 MB buffer written before every timed step (inside the timed region)"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                     "frac": achieved / peak_tflops, "traffic": gram_traffic(n_tr, cfg_gram),
                     "kernel": f"gram_kernel<float,chi=4> (symmetric {n_tr}x{n_tr} Gram), "
                               f"{tile_gram[0]}x{tile_gram[1]} tiles, {tile_gram[2]} threads",
                     "tile_shape_ids": {"gram": cfg_gram, "rows": cfg_rows},
                     "peak_source": (f"FP32 FMA peak {props.multi_processor_count} SMs x 128 lanes x 2 x "
                                     f"{sm_max:.0f} MHz"),
                     "avg_launch_ms": gram_avg_ms},
        "e2e": e2e,
        "phases_ms": phases,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        "cpu_baseline": cpu,
        "cpu_baseline_all_cores": cpu_all,
        "mixed_precision": mixed,
        "serving": serving_stats,
        "svm": svm_stats,
        "block_product_map": block_stats,
        "feature_dimension_sweep": sweep_stats,
    }
    print(json.dumps(line), flush=True)


SPLIT_WL = dict(workload="fmnist784_gram8000_rowsplit", d=784, m=8000, reps=2, chi=4, w=0.5)


def run_split(args):
    """Strong scaling over one Gram (§II-D: blocks of one kernel matrix on several GPU workers):
    the 8000-sample symmetric Gram at n = 784 split into balanced row blocks, one per rank
    (shard.gram_row_block: no exchange while computing). value = the Gram's unique entries x
    qubits / the slowest rank's time per step; e2e adds, every step, the host-to-device copy of
    the features and the gather of every rank's K block into each rank's host memory."""
    import torch
    import torch.distributed as tdist

    from paper_2602_01330_gb300 import build as libbuild
    from paper_2602_01330_gb300 import dualk, shard, synthetic, workload

    world, rank, local = dist_setup()
    if world > 1:
        tdist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if not os.path.exists(dualk.LIB_PATH):
        libbuild.build()
    m, d, reps, chi, w = SPLIT_WL["m"], SPLIT_WL["d"], SPLIT_WL["reps"], SPLIT_WL["chi"], SPLIT_WL["w"]
    data = synthetic.fmnist_like(m, 0, d)
    ctx = dualk.Context(local)
    fm = dualk.FeatureMap(reps=reps, chi_max=chi)
    stream = torch.cuda.current_stream()
    x = torch.from_numpy(data["x_train"]).to(dev)
    mps_buf = torch.empty(dualk.mps_bytes(m, d, chi), dtype=torch.uint8, device=dev)
    bond = torch.empty(d + 1, dtype=torch.int32, device=dev)
    ln = torch.empty(m, dtype=torch.float32, device=dev)
    lo, hi = shard.balanced_row_blocks(m, world)[rank]
    block = {k: torch.empty((hi - lo, m - lo), dtype=torch.float32, device=dev) for k in ("k", "kq", "kc", "logkq")}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def barrier():
        if world > 1:
            tdist.barrier()

    def step():
        mp_ = dualk.mps_build(ctx, x, fm, out=mps_buf, bond=bond, log_norm=ln)
        shard.gram_row_block(ctx, mp_, rank, world, w=w, out=block)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    ctx.sync_status()
    sampler = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        flush.zero_()
        step()
    t1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ms = t0.elapsed_time(t1)
    if world > 1:
        tt = torch.tensor([ms], device=dev)
        tdist.all_reduce(tt, op=tdist.ReduceOp.MAX)
        ms = float(tt.item())
    ctx.sync_status()
    units_step = workload.gram_entries(m) * d
    value = units_step * args.steps / (ms / 1e3)
    # end to end: features in from pinned host memory, K blocks gathered to every rank's host
    h_x = torch.from_numpy(data["x_train"]).pin_memory()
    e_steps = max(1, min(args.steps, 3))
    barrier()
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    for _ in range(e_steps):
        x.copy_(h_x, non_blocking=True)
        step()
        if world > 1:
            full = shard.gather_gram({"k": block["k"]}, m, world)
        else:
            full = {"k": shard.assemble([block["k"].cpu()], [(lo, hi)], m)}
    torch.cuda.synchronize()
    barrier()
    e2e_s = (time.perf_counter() - e0) / e_steps
    if world > 1:
        tt = torch.tensor([e2e_s], device=dev)
        tdist.all_reduce(tt, op=tdist.ReduceOp.MAX)
        e2e_s = float(tt.item())
    assert full["k"].shape == (m, m)
    if world > 1:
        tdist.destroy_process_group()
    ctx.close()
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (Fashion-MNIST-shaped, seeded; the real data set is not available)",
        "config": {"workload": SPLIT_WL["workload"], "d": d, "m": m, "reps": reps, "chi": chi, "w": w,
                   "parallelism": f"balanced row blocks of one Gram over {world} GPU(s)",
                   "l2": "256 MB buffer written before every timed step (inside the timed region)"},
        "e2e": {"value": units_step / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h_x.numel() * 4,
                "d2h_bytes_per_step": (hi - lo) * (m - lo) * 4, "gather": "all ranks' K blocks to every host"},
        "gpu_launches": (1 + 2 * (1 if hi < m else 0) + 2) * args.steps,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--tile-shapes", default="", help="G,R: Gram and rows tile-shape ids (default: autotuned)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the mixed-precision and serving measurements after the timed region")
    ap.add_argument("--n-train", type=int, default=WL["n_train"],
                    help="training-set size; smaller cases serve ncu captures, not bench lines")
    ap.add_argument("--n-test", type=int, default=WL["n_test"])
    ap.add_argument("--split", action="store_true",
                    help="strong scaling: one 8000-sample Gram split into row blocks over the ranks")
    args = ap.parse_args()
    if (args.n_train, args.n_test) != (WL["n_train"], WL["n_test"]):
        WL.update(n_train=args.n_train, n_test=args.n_test,
                  workload=f"fmnist784_gram{args.n_train}_rows{args.n_test}")
    if args.impl == "reference":
        run_reference(args)
    elif args.split:
        run_split(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
