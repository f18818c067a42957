"""Continuous-batching service of dual-kernel rows against resident training sets.

Prediction with the dual-kernel SVM needs, for every test sample x, the kernel values
K(x_i, x) against the training samples (§II-B, Eq. 5). The server keeps one training
set per qubit count resident on the device (its MPS, features and norms) and answers
requests — batches of test samples of one qubit count — with their b x m row block.

Continuous batching: requests arrive over time; each is admitted into a free slot as
soon as one is free and the device has room for its buffers (free HBM: the driver's free
bytes plus what torch's caching allocator holds unused, minus a reserve), runs on its
slot's own stream (test MPS build, then dual-kernel rows and their refinement pass, then
the copy of K to pinned host memory), and overlaps on the device with every other admitted
request. Waiting requests of the same qubit count are merged into one launch of up to
``merge_rows`` test rows (first come first served; a request is never split), so that
small requests share one pair tile instead of each leaving most of a tile idle. A request
that could never fit is rejected. Results do not depend on what else runs: every pair is
contracted by the same arithmetic in the same order whatever tile, launch or merged batch
it lands in.

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
    reqs: list = field(default_factory=list)   # requests of the launch in flight (one n)
    event: torch.cuda.Event | None = None
    host_out: torch.Tensor | None = None
    keep: list = field(default_factory=list)

    @property
    def busy(self) -> bool:
        return bool(self.reqs)


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
                 slots: int = 8, reserve_bytes: int = 2 << 30, device=None, merge_rows: int = 256):
        self.ctx = ctx
        self.fmap = fmap
        self.w = w
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.train = {n: TrainingSet(ctx, x, fmap, self.device) for n, x in train.items()}
        torch.cuda.synchronize()
        self.slots = [_Slot(torch.cuda.Stream(device=self.device)) for _ in range(slots)]
        self.reserve = reserve_bytes
        self.merge_rows = merge_rows
        self.admitted = 0
        self.rejected = 0
        self.launches = 0
        self.max_in_flight = 0        # most requests on the device at once
        self.max_launches_in_flight = 0

    def request_bytes(self, b: int, n: int) -> int:
        m = self.train[n].m
        return dualk.mps_bytes(b, n, self.fmap.chi_max) + b * n * 4 + 2 * b * 4 + b * m * 4 + 4096

    def _mem(self):
        """(free, total) device bytes; free counts memory that torch's caching allocator has
        reserved but not handed out, which it reuses before asking the driver for more."""
        free, total = torch.cuda.mem_get_info(self.device)
        cached = torch.cuda.memory_reserved(self.device) - torch.cuda.memory_allocated(self.device)
        return free + max(cached, 0), total

    def _fits(self, reqs) -> bool:
        b = sum(r.x.shape[0] for r in reqs)
        return self.request_bytes(b, reqs[0].n) + self.reserve <= self._mem()[0]

    def _launch(self, slot: _Slot, reqs: list):
        ts = self.train[reqs[0].n]
        xs = np.concatenate([np.ascontiguousarray(r.x, dtype=np.float32) for r in reqs])
        b, n = xs.shape
        with torch.cuda.stream(slot.stream):
            hx = torch.from_numpy(xs).pin_memory()
            x = torch.empty((b, n), dtype=torch.float32, device=self.device)
            x.copy_(hx, non_blocking=True)
            test = dualk.mps_build(self.ctx, x, self.fmap, stream=slot.stream)
            out = {"k": torch.empty((b, ts.m), dtype=torch.float32, device=self.device),
                   "kq": torch.empty((b, ts.m), dtype=torch.float32, device=self.device)}
            dualk.dual_kernel_rows(self.ctx, test, ts.mps, w=self.w, want=("k", "kq"), out=out, stream=slot.stream)
            host = torch.empty((b, ts.m), dtype=torch.float32).pin_memory()
            host.copy_(out["k"], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(slot.stream)
        slot.reqs, slot.event, slot.host_out = list(reqs), ev, host
        slot.keep = [hx, x, test, out]  # alive until the stream has passed them
        self.launches += 1

    def _take_batch(self, waiting: deque) -> list:
        """The first waiting request and, after it, waiting requests of the same qubit count
        while the merged batch stays within merge_rows rows (queue order otherwise kept)."""
        first = waiting[0]
        batch, rows = [first], first.x.shape[0]
        for r in list(waiting)[1:]:
            if r.n == first.n and rows + r.x.shape[0] <= self.merge_rows:
                batch.append(r)
                rows += r.x.shape[0]
        return batch

    def _retire(self, slot: _Slot, now: float):
        out = slot.host_out.numpy()
        row = 0
        for r in slot.reqs:
            b = r.x.shape[0]
            r.result = out[row:row + b]
            r.done = now
            row += b
        n = len(slot.reqs)
        slot.reqs, slot.event, slot.host_out, slot.keep = [], None, None, []
        return n

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
            # retire finished launches
            for slot in self.slots:
                if slot.busy and slot.event.query():
                    done += self._retire(slot, clock() - t0)
            # admit into free slots while memory allows
            for slot in self.slots:
                if not waiting:
                    break
                if slot.busy:
                    continue
                req = waiting[0]
                if self.request_bytes(req.x.shape[0], req.n) + self.reserve > self._mem()[1]:
                    waiting.popleft()
                    req.rejected = True
                    self.rejected += 1
                    done += 1
                    continue
                batch = self._take_batch(waiting)
                while len(batch) > 1 and not self._fits(batch):
                    batch.pop()
                if not self._fits(batch):
                    break
                for r in batch:
                    waiting.remove(r)
                    r.admitted = clock() - t0
                self.admitted += len(batch)
                self._launch(slot, batch)
            busy = [s_ for s_ in self.slots if s_.busy]
            self.max_in_flight = max(self.max_in_flight, sum(len(s_.reqs) for s_ in busy))
            self.max_launches_in_flight = max(self.max_launches_in_flight, len(busy))
            if poll_sleep:
                time.sleep(poll_sleep)
        self.ctx.sync_status()
        return requests

    def solve_alone(self, req: Request) -> np.ndarray:
        """The same request with nothing else on the device (for the determinism check)."""
        torch.cuda.synchronize()
        slot = self.slots[0]
        assert not slot.busy
        self._launch(slot, [req])
        slot.event.synchronize()
        out = slot.host_out.numpy().copy()
        slot.reqs, slot.event, slot.host_out, slot.keep = [], None, None, []
        self.launches -= 1
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


def run_benchmark(ctx: dualk.Context, m: int = 8000, requests: int = 300, rho=(0.8,), slots: int = 8,
                  seed: int = 4, dims=(16, 128, 784), b_max: int = 256) -> dict:
    """Resident training sets of m samples per qubit count, a saturating burst to measure the
    peak rows/s, then for each offered load rho a Poisson stream at rho times that rate;
    per load p50/p99 latency, rows/s, admissions, launches, the most requests and launches
    on the device at once, and whether a few results are bit-identical when run alone."""
    from . import synthetic

    fm = dualk.FeatureMap(reps=2, chi_max=4)
    train = {n: synthetic.fmnist_like(m, 0, n)["x_train"] for n in dims}
    test_pool = {n: synthetic.fmnist_like(16, 512, n)["x_test"] for n in dims}
    srv = KernelServer(ctx, train, fm, slots=slots)
    rng = np.random.Generator(np.random.PCG64(seed))
    burst = poisson_requests(rng, 64, 1e9, dims, test_pool, b_max)
    srv.run(burst[:8])  # warm-up: first launches of every kernel
    t0 = time.perf_counter()
    srv.run(burst[8:])
    sat_rows = sum(r.x.shape[0] for r in burst[8:]) / (time.perf_counter() - t0)
    res = {"workload": f"serving m={m} n={tuple(dims)} slots={slots} requests={requests} per load, "
                       f"batch U{{1..{b_max}}}, Poisson arrivals",
           "saturated_rows_per_s": sat_rows, "loads": {}}
    for r_ in (rho if isinstance(rho, (tuple, list)) else (rho,)):
        rate = r_ * sat_rows / ((1 + b_max) / 2)
        reqs = poisson_requests(rng, requests, rate, dims, test_pool, b_max)
        srv.admitted = srv.rejected = srv.launches = srv.max_in_flight = srv.max_launches_in_flight = 0
        srv.run(reqs)
        stats = latency_stats(reqs)
        same = all(np.array_equal(srv.solve_alone(r), r.result) for r in reqs[:5] if r.result is not None)
        res["loads"][f"rho={r_}"] = {"offered_requests_per_s": rate, **stats, "admitted": srv.admitted,
                                     "launches": srv.launches, "max_requests_in_flight": srv.max_in_flight,
                                     "max_launches_in_flight": srv.max_launches_in_flight,
                                     "same_alone_and_in_mix": same}
    return res


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
    print(json.dumps(run_benchmark(ctx, args.m, args.requests, (args.rho,), args.slots, args.seed)))
    ctx.close()


if __name__ == "__main__":
    main()
