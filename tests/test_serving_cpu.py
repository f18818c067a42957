"""Admission logic of the continuous-batching server, on the CPU with a fake device:
no kernel runs; slots complete after a simulated service time and the device memory is a
counter that admitted requests draw from."""
from types import SimpleNamespace

import numpy as np
import torch

from paper_2602_01330_gb300.serving import KernelServer, Request, _Slot, latency_stats, poisson_requests


class _Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1e-3  # every look at the clock advances 1 ms
        return self.t


class _Event:
    def __init__(self, clock, ready_at):
        self.clock, self.ready_at = clock, ready_at

    def query(self):
        return self.clock.t >= self.ready_at


class FakeServer(KernelServer):
    def __init__(self, clock, free_bytes, total_bytes, slots, service_s, merge_rows=1):
        self.clock = clock
        self.slots = [_Slot(stream=None) for _ in range(slots)]
        self.reserve = 0
        self.merge_rows = merge_rows
        self.admitted = 0
        self.rejected = 0
        self.launches = 0
        self.max_in_flight = 0
        self.max_launches_in_flight = 0
        self.batches = []
        self.train = {8: SimpleNamespace(m=10), 32: SimpleNamespace(m=10)}
        self.free_bytes, self.total_bytes = free_bytes, total_bytes
        self.service_s = service_s
        self.ctx = SimpleNamespace(sync_status=lambda: None)
        self.max_inflight = 0
        self.order = []

    def request_bytes(self, b, n):
        return 100 * b

    def _mem(self):
        used = sum(self.request_bytes(r.x.shape[0], r.n) for s in self.slots for r in s.reqs)
        return self.free_bytes - used, self.total_bytes

    def _launch(self, slot, reqs):
        slot.reqs = list(reqs)
        slot.event = _Event(self.clock, self.clock.t + self.service_s)
        slot.host_out = torch.cat([torch.full((r.x.shape[0], 10), float(r.rid)) for r in reqs])
        self.order.extend(r.rid for r in reqs)
        self.batches.append([r.rid for r in reqs])
        self.launches += 1
        self.max_inflight = max(self.max_inflight, sum(len(s.reqs) for s in self.slots))


def _req(rid, b, n=8, t=0.0):
    return Request(rid, n, np.zeros((b, n), np.float32), t)


def test_memory_limits_concurrency_and_fifo_order():
    clk = _Clock()
    srv = FakeServer(clk, free_bytes=2000, total_bytes=10_000, slots=8, service_s=0.01)
    reqs = [_req(i, 10) for i in range(6)]  # 1000 bytes each: two fit at a time
    srv.run(reqs, clock=clk)
    assert srv.max_inflight == 2
    assert srv.order == list(range(6))
    assert all(r.done is not None and not r.rejected for r in reqs)
    assert all(np.all(r.result == r.rid) for r in reqs)


def test_request_larger_than_device_is_rejected_others_served():
    clk = _Clock()
    srv = FakeServer(clk, free_bytes=5000, total_bytes=5000, slots=4, service_s=0.005)
    reqs = [_req(0, 10), _req(1, 80), _req(2, 10)]  # 8000 bytes never fits
    srv.run(reqs, clock=clk)
    assert reqs[1].rejected and reqs[1].result is None
    assert not reqs[0].rejected and not reqs[2].rejected
    assert srv.rejected == 1 and srv.admitted == 2


def test_slots_bound_concurrency_and_arrivals_are_honoured():
    clk = _Clock()
    srv = FakeServer(clk, free_bytes=1 << 30, total_bytes=1 << 30, slots=3, service_s=0.02)
    reqs = [_req(i, 1, t=0.05 * i) for i in range(7)]
    srv.run(reqs, clock=clk)
    assert srv.max_inflight <= 3
    assert all(r.admitted >= r.arrival for r in reqs)
    st = latency_stats(reqs)
    assert st["served"] == 7 and st["p99_ms"] >= st["p50_ms"] > 0


def test_poisson_requests_shape():
    rng = np.random.Generator(np.random.PCG64(4))
    pool = {16: np.zeros((50, 16), np.float32), 128: np.zeros((50, 128), np.float32)}
    reqs = poisson_requests(rng, 200, 100.0, (16, 128), pool, b_max=256)
    arr = np.array([r.arrival for r in reqs])
    assert np.all(np.diff(arr) > 0)
    assert 1.0 < arr[-1] < 3.5  # 200 arrivals at 100/s
    assert all(1 <= r.x.shape[0] <= 256 and r.x.shape[1] == r.n for r in reqs)


def test_waiting_requests_of_one_qubit_count_merge_into_one_launch():
    clk = _Clock()
    srv = FakeServer(clk, free_bytes=1 << 30, total_bytes=1 << 30, slots=1, service_s=0.05, merge_rows=25)
    # r0 occupies the only slot; r1..r5 wait together and are merged by qubit count up to 25 rows
    reqs = [_req(0, 5), _req(1, 10, t=0.01), _req(2, 10, n=32, t=0.01), _req(3, 10, t=0.01),
            _req(4, 10, t=0.01), _req(5, 5, n=32, t=0.01)]
    srv.run(reqs, clock=clk)
    assert srv.batches[0] == [0]
    assert srv.batches[1] == [1, 3]          # n = 8, 20 rows; r4 would make 30
    assert srv.batches[2] == [2, 5]          # n = 32, queue order
    assert srv.batches[3] == [4]
    assert srv.launches == 4 and srv.admitted == 6
    assert all(np.all(r.result == r.rid) and r.result.shape[0] == r.x.shape[0] for r in reqs)


def test_merged_batch_shrinks_to_fit_memory():
    clk = _Clock()
    srv = FakeServer(clk, free_bytes=2500, total_bytes=10_000, slots=2, service_s=0.01, merge_rows=256)
    reqs = [_req(i, 10) for i in range(5)]   # 1000 bytes each: at most two per batch
    srv.run(reqs, clock=clk)
    assert max(len(b) for b in srv.batches) == 2
    assert srv.order == list(range(5))
    assert all(r.done is not None and not r.rejected for r in reqs)


def test_admission_counts_memory_cached_by_the_allocator(monkeypatch):
    srv = KernelServer.__new__(KernelServer)
    srv.device = torch.device("cpu")
    monkeypatch.setattr(torch.cuda, "mem_get_info", lambda dev: (1000, 5000))
    monkeypatch.setattr(torch.cuda, "memory_reserved", lambda dev: 800)
    monkeypatch.setattr(torch.cuda, "memory_allocated", lambda dev: 300)
    assert srv._mem() == (1500, 5000)
