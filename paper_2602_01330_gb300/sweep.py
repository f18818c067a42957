"""Feature-dimension sweep: many Gram matrices of uneven qubit counts in persistent,
graph-captured launches with autotuned tile shapes (§III-A: d = 2 .. 784; §II-D: the
kernel matrix is built in blocks).

* ``Autotuner`` times every Gram tile shape the library offers on a slice of the
  caller's workload and keeps the fastest per (dtype, chi, n, m, symmetric) key.
* ``GramSweep`` owns the device buffers of all matrices, records one pass (per matrix:
  MPS build, tile shape, persistent symmetric Gram) into a CUDA graph, and replays it.

Everything here is orchestration: the arithmetic runs in libdualk's kernels.
"""
from __future__ import annotations

import json
import os
import time
from dataclasses import dataclass

import torch

from . import dualk


def _time_ms(fn, reps: int = 3, stream=None) -> float:
    stream = stream or torch.cuda.current_stream()
    fn()
    stream.synchronize()
    best = float("inf")
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


class Autotuner:
    """Picks the fastest Gram tile shape for a workload by timing each one.

    The timing runs the whole sample count (so the number of tiles, and hence how well
    each shape fills the GPU, is the real one) on an MPS of the first ``probe_sites``
    features only: the per-site cost of a shape does not depend on n. Results are cached
    in memory and, if ``path`` is given, in a JSON file.
    """

    def __init__(self, ctx: dualk.Context, path: str | None = None, probe_sites: int = 48, reps: int = 2):
        self.ctx = ctx
        self.path = path
        self.probe_sites = probe_sites
        self.reps = reps
        self.cache: dict[str, int] = {}
        self.timings: dict[str, dict[int, float]] = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.cache = {k: int(v) for k, v in json.load(f).items()}

    @staticmethod
    def key(mps: dualk.MPS, symmetric: bool, cols: dualk.MPS | None = None) -> str:
        m_cols = mps.m if cols is None else cols.m
        return f"dtype{mps.dtype}-chi{mps.chi_max}-n{mps.n}-m{mps.m}-c{m_cols}-sym{int(symmetric)}"

    def _probe(self, mps: dualk.MPS) -> dualk.MPS:
        sites = min(mps.n, self.probe_sites)
        fm = mps.fmap if mps.fmap is not None else dualk.FeatureMap(chi_max=mps.chi_max)
        return dualk.mps_build(self.ctx, mps.x[:, :sites].contiguous(), fm, dtype=mps.dtype)

    def best(self, mps: dualk.MPS, symmetric: bool = True, cols: dualk.MPS | None = None) -> int:
        """Fastest tile shape for the Gram of `mps` (symmetric) or its block against `cols`."""
        k = self.key(mps, symmetric, cols)
        if k in self.cache:
            return self.cache[k]
        count = dualk.gram_config_count(mps.dtype, mps.chi_max)
        if count <= 1:
            self.cache[k] = 0
            return 0
        prow = self._probe(mps)
        pcol = prow if cols is None else self._probe(cols)
        rows, ncols = prow.m, pcol.m
        # the mixed K, as the Gram and row calls produce it: the probe then pays for the
        # RBF epilogue (per-tile feature loads) in proportion, like the real launch
        out = {"k": torch.empty((rows, ncols), dtype=torch.float32, device=mps.data.device)}
        times = {}
        for cid in range(1, count + 1):
            self.ctx.set_gram_config(cid)
            times[cid] = _time_ms(lambda: dualk.gram_tile(self.ctx, prow, pcol, 0, rows, 0, ncols, w=0.5, out=out,
                                                          ld=ncols, symmetric=symmetric), self.reps)
        self.ctx.set_gram_config(0)
        choice = min(times, key=times.get)
        self.cache[k] = choice
        self.timings[k] = times
        if self.path:
            with open(self.path, "w") as f:
                json.dump(self.cache, f, indent=1)
        return choice


@dataclass
class SweepMatrix:
    d: int
    x: torch.Tensor
    mps: torch.Tensor
    bond: torch.Tensor
    log_norm: torch.Tensor
    out: dict
    cfg: int = 0


class GramSweep:
    """All Gram matrices of a feature-dimension sweep, captured as one CUDA graph.

    ``features`` maps d -> (m x d float32 array or tensor). One pass = for every d: MPS
    build, then the symmetric Gram (persistent launch over its tiles) with its autotuned
    tile shape, writing K, K_q, K_c and log K_q.
    """

    def __init__(self, ctx: dualk.Context, features: dict, fmap: dualk.FeatureMap, w: float = 0.5,
                 autotuner: Autotuner | None = None, want=("k", "kq", "kc", "logkq"), device=None,
                 refine: float | None = dualk.REFINE_TAU):
        self.ctx = ctx
        self.refine = refine  # tau of the refinement pass after each Gram (None: none)
        self.fmap = fmap
        self.w = w
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.mats: list[SweepMatrix] = []
        for d, x in sorted(features.items()):
            xt = torch.as_tensor(x, dtype=torch.float32).to(self.device).contiguous()
            m = xt.shape[0]
            buf = torch.empty(dualk.mps_bytes(m, d, fmap.chi_max), dtype=torch.uint8, device=self.device)
            bond = torch.empty(d + 1, dtype=torch.int32, device=self.device)
            ln = torch.empty(m, dtype=torch.float32, device=self.device)
            out = {k: torch.empty((m, m), dtype=torch.float32, device=self.device) for k in want}
            self.mats.append(SweepMatrix(d, xt, buf, bond, ln, out))
        self.graph = None
        m_max = max(mt.x.shape[0] for mt in self.mats)
        self.refine_ws = dualk.refine_workspace(m_max, m_max, self.device)  # reused by every item
        if autotuner is not None:
            for mt in self.mats:
                mps = dualk.mps_build(self.ctx, mt.x, self.fmap, out=mt.mps, bond=mt.bond, log_norm=mt.log_norm)
                mt.cfg = autotuner.best(mps, symmetric=True)
            torch.cuda.synchronize()

    def _pass(self, stream=None):
        for mt in self.mats:
            mps = dualk.mps_build(self.ctx, mt.x, self.fmap, out=mt.mps, bond=mt.bond, log_norm=mt.log_norm,
                                  stream=stream)
            self.ctx.set_gram_config(mt.cfg)
            dualk.gram_tile(self.ctx, mps, mps, symmetric=True, w=self.w, out=mt.out, ld=mt.x.shape[0],
                            stream=stream, refine=self.refine, refine_ws=self.refine_ws)
        self.ctx.set_gram_config(0)

    def run_eager(self):
        self._pass()

    def capture(self):
        """Record one pass into a CUDA graph (after an eager warm-up pass)."""
        self._pass()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream(device=self.device)
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            with torch.cuda.graph(g, stream=side):
                self._pass(stream=side)
        torch.cuda.current_stream().wait_stream(side)
        self.graph = g
        return g

    def replay(self):
        if self.graph is None:
            self.capture()
        self.graph.replay()

    def run_native(self, graph: bool = True, stream=None):
        """One pass through the library's own sweep call: the MPS builds, then every Gram by
        dk_gram_sweep, which with graph=True records its launches once into a CUDA graph kept
        by the context and replays it afterwards (a non-default stream is required)."""
        items = []
        for mt in self.mats:
            mps = dualk.mps_build(self.ctx, mt.x, self.fmap, out=mt.mps, bond=mt.bond, log_norm=mt.log_norm,
                                  stream=stream)
            items.append((mps, mt.out, mt.cfg))
        dualk.gram_sweep(self.ctx, items, w=self.w, graph=graph, stream=stream, ws=self.refine_ws)

    def concentration(self) -> dict:
        """Per qubit count: mean and variance of the off-diagonal K_q and log K_q of the last
        pass (dk_gram_stats), the concentration of the quantum kernel as n grows."""
        res = {}
        for mt in self.mats:
            if "kq" in mt.out and "logkq" in mt.out:
                res[mt.d] = dualk.gram_stats(self.ctx, mt.out["kq"], mt.out["logkq"], symmetric=True)
        return res

    def entries_qubits(self) -> int:
        return sum(mt.x.shape[0] * (mt.x.shape[0] + 1) // 2 * mt.d for mt in self.mats)


DIMS = (2, 4, 8, 16, 32, 64, 128, 256, 512, 784)


def run_benchmark(ctx: dualk.Context, m: int = 2000, dims=DIMS, reps: int = 3, autotune: bool = True,
                  peak_tflops: float | None = None) -> dict:
    """The feature-dimension sweep (Fashion-MNIST-shaped data, m samples per d, reps 2, bond 4):
    one pass = every d's MPS build, symmetric Gram (autotuned tile shape) and refinement pass.
    Timed eagerly, replayed from a torch-captured graph, and through the library's own
    dk_gram_sweep with its cached graph; entry-qubits/s, the Gram flops (block count) per
    second of the whole pass as a fraction of the FP32 peak, and the concentration per d."""
    from . import synthetic, workload

    feats = {d: synthetic.fmnist_like(m, 0, d)["x_train"] for d in dims}
    tuner = Autotuner(ctx) if autotune else None
    sw = GramSweep(ctx, feats, dualk.FeatureMap(reps=2, chi_max=4), autotuner=tuner)
    eager = _time_ms(sw.run_eager, reps)
    sw.capture()
    graph = _time_ms(sw.replay, reps)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())

    def native():
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            sw.run_native(graph=True, stream=side)
        torch.cuda.current_stream().wait_stream(side)
    native_ms = _time_ms(native, reps)
    sw.refine = None  # the same pass without the refinement passes (kernels of the plain FP32 path)
    plain_ms = _time_ms(sw.run_eager, reps)
    sw.refine = dualk.REFINE_TAU
    ctx.sync_status()
    units = sw.entries_qubits()
    flops = sum(workload.gram_entries(mt.x.shape[0]) * workload.flops_per_pair(mt.d, 2) for mt in sw.mats)
    best = min(eager, graph, native_ms)
    gram_only = plain_ms
    res = {
        "workload": f"sweep d={list(dims)} m={m} reps=2 chi=4 (build + Gram + refinement per d)",
        "entry_qubits": units,
        "eager_ms": eager, "graph_ms": graph, "native_sweep_graph_ms": native_ms,
        "eager_entry_qubits_per_s": units / (eager / 1e3), "graph_entry_qubits_per_s": units / (graph / 1e3),
        "native_sweep_entry_qubits_per_s": units / (native_ms / 1e3),
        "eager_without_refinement_ms": plain_ms,
        "eager_without_refinement_entry_qubits_per_s": units / (plain_ms / 1e3),
        "gram_tflops_block_count_best": flops / (best / 1e3) / 1e12,
        "tile_shapes": {mt.d: (mt.cfg, dualk.gram_config_info(mt.cfg) if mt.cfg else None) for mt in sw.mats},
        "concentration": {d: {k: s_[k] for k in ("kq_mean", "kq_var", "logkq_mean", "logkq_var") if k in s_}
                          for d, s_ in sw.concentration().items()},
    }
    res["gram_tflops_block_count_without_refinement"] = flops / (gram_only / 1e3) / 1e12
    if peak_tflops:
        res["fraction_of_fp32_peak_best"] = res["gram_tflops_block_count_best"] / peak_tflops
        res["fraction_of_fp32_peak_without_refinement"] = (res["gram_tflops_block_count_without_refinement"]
                                                           / peak_tflops)
    return res


def main():
    """Time the d in {2, ..., 784} sweep (2000 samples each, reps 2, chi 4): eager vs graph."""
    import argparse

    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--m", type=int, default=2000)
    ap.add_argument("--dims", default=",".join(str(d) for d in DIMS))
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--no-autotune", action="store_true")
    args = ap.parse_args()
    dims = [int(v) for v in args.dims.split(",")]
    ctx = dualk.Context(0)
    print(json.dumps(run_benchmark(ctx, args.m, dims, args.reps, not args.no_autotune), default=str))
    ctx.close()


if __name__ == "__main__":
    main()
