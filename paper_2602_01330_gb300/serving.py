"""Continuous-batching service of dual-kernel rows against resident training sets.

Prediction with the dual-kernel SVM needs, for every test sample x, the kernel values
K(x_i, x) against the training samples (§II-B, Eq. 5). The server keeps one training
set per qubit count resident on the device (its MPS, features and norms) and answers
requests — batches of test samples of one qubit count — with their b x m row block.

Continuous batching: requests arrive over time; each is admitted into a free slot as
soon as one is free and the device has room for its buffers (free HBM from
``torch.cuda.mem_get_info`` minus a reserve), runs on its slot's own stream (test MPS
build, then dual-kernel rows, then the copy of K to pinned host memory), and overlaps on
the device with every other admitted request. A request that could never fit is
rejected. Results do not depend on what else runs: every pair is contracted by the same
arithmetic in the same order whatever tile or launch it lands in.

All device work runs in libdualk's kernels; this module only schedules it.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np
import torch

from . import dualk


@dataclass
class Request:
    rid: int
    n: int
    x: np.ndarray                 # b x n float32 test features
    arrival: float                # seconds (host clock) at which it may be admitted
    admitted: float | None = None
    done: float | None = None
    result: np.ndarray | None = None
    rejected: bool = False


@dataclass
class _Slot:
    stream: torch.cuda.Stream
    req: Request | None = None
    event: torch.cuda.Event | None = None
    host_out: torch.Tensor | None = None
    keep: list = field(default_factory=list)


class TrainingSet:
    """A training set kept resident on the device: features, MPS and ln-norms."""

    def __init__(self, ctx: dualk.Context, x: np.ndarray, fmap: dualk.FeatureMap, device):
        self.x = torch.as_tensor(x, dtype=torch.float32).to(device).contiguous()
        self.mps = dualk.mps_build(ctx, self.x, fmap)
        self.m, self.n = self.x.shape

    def bytes(self) -> int:
        return self.mps.data.numel() + self.x.numel() * 4 + self.m * 4


class KernelServer:
    """Serves K(test, train) row blocks with continuous batching over ``slots`` streams."""

    def __init__(self, ctx: dualk.Context, train: dict, fmap: dualk.FeatureMap, w: float = 0.5,
                 slots: int = 8, reserve_bytes: int = 2 << 30, device=None):
        self.ctx = ctx
        self.fmap = fmap
        self.w = w
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.train = {n: TrainingSet(ctx, x, fmap, self.device) for n, x in train.items()}
        torch.cuda.synchronize()
        self.slots = [_Slot(torch.cuda.Stream(device=self.device)) for _ in range(slots)]
        self.reserve = reserve_bytes
        self.admitted = 0
        self.rejected = 0

    def request_bytes(self, b: int, n: int) -> int:
        m = self.train[n].m
        return dualk.mps_bytes(b, n, self.fmap.chi_max) + b * n * 4 + 2 * b * 4 + b * m * 4 + 4096

    def _mem(self):
        """(free, total) device bytes."""
        return torch.cuda.mem_get_info(self.device)

    def _fits(self, req: Request) -> bool:
        return self.request_bytes(req.x.shape[0], req.n) + self.reserve <= self._mem()[0]

    def _launch(self, slot: _Slot, req: Request):
        ts = self.train[req.n]
        b = req.x.shape[0]
        with torch.cuda.stream(slot.stream):
            hx = torch.from_numpy(np.ascontiguousarray(req.x, dtype=np.float32)).pin_memory()
            x = torch.empty((b, req.n), dtype=torch.float32, device=self.device)
            x.copy_(hx, non_blocking=True)
            test = dualk.mps_build(self.ctx, x, self.fmap, stream=slot.stream)
            out = {"k": torch.empty((b, ts.m), dtype=torch.float32, device=self.device)}
            dualk.dual_kernel_rows(self.ctx, test, ts.mps, w=self.w, want=("k",), out=out, stream=slot.stream)
            host = torch.empty((b, ts.m), dtype=torch.float32).pin_memory()
            host.copy_(out["k"], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(slot.stream)
        slot.req, slot.event, slot.host_out = req, ev, host
        slot.keep = [hx, x, test, out]  # alive until the stream has passed them

    def run(self, requests: list[Request], clock=time.perf_counter, poll_sleep: float = 0.0):
        """Serve every request; arrivals are honoured relative to the start of the call."""
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        waiting: deque[Request] = deque()
        t0 = clock()
        done = 0
        total = len(requests)
        while done < total:
            now = clock() - t0
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            # retire finished requests
            for slot in self.slots:
                if slot.req is not None and slot.event.query():
                    slot.req.result = slot.host_out.numpy()
                    slot.req.done = clock() - t0
                    slot.req, slot.event, slot.host_out, slot.keep = None, None, None, []
                    done += 1
            # admit into free slots while memory allows
            for slot in self.slots:
                if not waiting:
                    break
                if slot.req is not None:
                    continue
                req = waiting[0]
                if self.request_bytes(req.x.shape[0], req.n) + self.reserve > self._mem()[1]:
                    waiting.popleft()
                    req.rejected = True
                    self.rejected += 1
                    done += 1
                    continue
                if not self._fits(req):
                    break
                waiting.popleft()
                req.admitted = clock() - t0
                self.admitted += 1
                self._launch(slot, req)
            if poll_sleep:
                time.sleep(poll_sleep)
        self.ctx.sync_status()
        return requests

    def solve_alone(self, req: Request) -> np.ndarray:
        """The same request with nothing else on the device (for the determinism check)."""
        torch.cuda.synchronize()
        slot = self.slots[0]
        assert slot.req is None
        self._launch(slot, req)
        slot.event.synchronize()
        out = slot.host_out.numpy().copy()
        slot.req, slot.event, slot.host_out, slot.keep = None, None, None, []
        return out


def latency_stats(requests: list[Request]) -> dict:
    served = [r for r in requests if r.done is not None and not r.rejected]
    lat = np.array([r.done - r.arrival for r in served]) * 1e3
    rows = sum(r.x.shape[0] for r in served)
    span = max(r.done for r in served) - min(r.arrival for r in served) if served else 0.0
    return {
        "served": len(served), "rejected": sum(r.rejected for r in requests),
        "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
        "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None,
        "mean_ms": float(lat.mean()) if len(lat) else None,
        "rows_per_s": rows / span if span > 0 else None,
    }


def poisson_requests(rng: np.random.Generator, count: int, rate_per_s: float, dims, features_by_n,
                     b_max: int = 256) -> list[Request]:
    """Requests with exponential inter-arrival times, batch size U{1..b_max}, n uniform over dims."""
    t = 0.0
    reqs = []
    for rid in range(count):
        t += rng.exponential(1.0 / rate_per_s)
        n = int(rng.choice(dims))
        b = int(rng.integers(1, b_max + 1))
        pool = features_by_n[n]
        idx = rng.integers(0, pool.shape[0], size=b)
        reqs.append(Request(rid, n, pool[idx], t))
    return reqs


def run_benchmark(ctx: dualk.Context, m: int = 8000, requests: int = 300, rho: float = 0.8, slots: int = 8,
                  seed: int = 4, dims=(16, 128, 784), b_max: int = 256) -> dict:
    """Resident training sets of m samples per qubit count, a saturating burst to measure the
    peak rows/s, then Poisson arrivals at rho times that rate; p50/p99 latency, rows/s,
    admissions, and whether a few results are bit-identical when run alone."""
    from . import synthetic

    fm = dualk.FeatureMap(reps=2, chi_max=4)
    train = {n: synthetic.fmnist_like(m, 0, n)["x_train"] for n in dims}
    test_pool = {n: synthetic.fmnist_like(16, 512, n)["x_test"] for n in dims}
    srv = KernelServer(ctx, train, fm, slots=slots)
    rng = np.random.Generator(np.random.PCG64(seed))
    burst = poisson_requests(rng, 32, 1e9, dims, test_pool, b_max)
    t0 = time.perf_counter()
    srv.run(burst)
    sat_rows = sum(r.x.shape[0] for r in burst) / (time.perf_counter() - t0)
    rate = rho * sat_rows / ((1 + b_max) / 2)
    reqs = poisson_requests(rng, requests, rate, dims, test_pool, b_max)
    srv.run(reqs)
    stats = latency_stats(reqs)
    same = all(np.array_equal(srv.solve_alone(r), r.result) for r in reqs[:5] if r.result is not None)
    return {"workload": f"serving m={m} n={tuple(dims)} slots={slots} rho={rho} requests={requests}",
            "saturated_rows_per_s": sat_rows, "offered_requests_per_s": rate, **stats,
            "admitted": srv.admitted, "same_alone_and_in_mix": same}


def main():
    """Serving run: 8000-sample training sets at n in {16, 128, 784}, Poisson arrivals."""
    import argparse
    import json

    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--m", type=int, default=8000)
    ap.add_argument("--requests", type=int, default=300)
    ap.add_argument("--rho", type=float, default=0.8, help="offered load as a fraction of the saturated rows/s")
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--seed", type=int, default=4)
    args = ap.parse_args()
    ctx = dualk.Context(0)
    print(json.dumps(run_benchmark(ctx, args.m, args.requests, args.rho, args.slots, args.seed)))
    ctx.close()


if __name__ == "__main__":
    main()
