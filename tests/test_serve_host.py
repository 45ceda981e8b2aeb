"""Host-side tests of the continuous-batching request loop (no GPU).

A fake executor stands in for the device: batches finish after a fixed
simulated time, memory is a counter, allocation or completion can be made to
fail.  Checked: every request finishes once, the HBM budget is never
exceeded, requests that arrive while others run are admitted as memory frees
up (batches overlap), FIFO order, oversized requests are rejected, refused
allocations are retried, and a batch past its deadline fails its requests
without blocking the loop.
"""
import pytest

from paper_2302_08251_gb300 import serve, synth


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-5)


class FakeExecutor:
    streams = 3

    def __init__(self, clock, bw=100e9, free=1 << 40, fail_alloc=(), stuck=()):
        self.clock, self.bw, self.free = clock, bw, free
        self.fail_alloc, self.stuck = set(fail_alloc), set(stuck)
        self.live = {}
        self.allocated = 0
        self.launches = []

    def nbytes(self, r):
        return 56 * r.n

    def free_bytes(self):
        return self.free - self.allocated

    def allocate(self, r):
        if r.rid in self.fail_alloc:
            self.fail_alloc.discard(r.rid)      # refuse once
            raise MemoryError("fake")
        self.allocated += r.nbytes
        self.live[r.rid] = r.nbytes

    def launch(self, reqs, stream_index):
        end = self.clock() + sum(r.nbytes for r in reqs) / self.bw + 1e-5
        stuck = any(r.rid in self.stuck for r in reqs)
        self.launches.append([r.rid for r in reqs])
        return (end, stuck)

    def done(self, handle):
        end, stuck = handle
        return not stuck and self.clock() >= end

    def release(self, r):
        self.allocated -= self.live.pop(r.rid)


def make(count=200, rate=2000.0, seed=3):
    return serve.workload(count=count, rate_hz=rate, n_lo=1e3, n_hi=1e6, seed=seed)


def run(reqs, **kw):
    clock = FakeClock()
    ex_kw = {k: kw.pop(k) for k in ("bw", "free", "fail_alloc", "stuck") if k in kw}
    ex = FakeExecutor(clock, **ex_kw)
    srv = serve.Server(ex, clock=clock, sleep=clock.sleep, free_margin=0, **kw)
    return srv.run(reqs), ex


def test_every_request_completes_once_and_memory_is_returned():
    reqs = make()
    stats, ex = run(reqs)
    assert stats.done == len(reqs) and stats.failed == 0 and stats.rejected == 0
    assert all(r.status == "done" for r in reqs)
    assert sorted(sum(ex.launches, [])) == [r.rid for r in reqs]
    assert ex.allocated == 0 and not ex.live
    assert len(stats.latencies_s) == len(reqs)
    assert all(r.done >= r.arrival for r in reqs)


def test_budget_is_never_exceeded_and_batches_overlap():
    reqs = make(count=300, rate=20000.0)
    budget = 3 * max(r.n for r in reqs) * 56
    stats, _ = run(reqs, budget_bytes=budget, bw=20e9)
    assert stats.max_in_flight_bytes <= budget
    assert stats.done == len(reqs)
    assert stats.max_overlap >= 2           # later arrivals ran beside earlier batches
    assert stats.batches > 1


def test_admission_is_fifo():
    reqs = make(count=120, rate=50000.0)
    stats, ex = run(reqs, budget_bytes=2 * max(r.n for r in reqs) * 56, bw=5e9)
    order = sum(ex.launches, [])
    assert order == sorted(order)


def test_request_larger_than_the_budget_is_rejected():
    reqs = make(count=20)
    big = max(reqs, key=lambda r: r.n)
    stats, _ = run(reqs, budget_bytes=56 * big.n - 1)
    assert big.status == "rejected" and stats.rejected >= 1
    assert stats.done + stats.rejected == len(reqs)


def test_refused_allocation_is_retried():
    reqs = make(count=30)
    stats, ex = run(reqs, fail_alloc={3, 7})
    assert stats.done == len(reqs)
    assert reqs[3].status == "done" and reqs[7].status == "done"


def test_free_device_memory_gates_admission():
    reqs = make(count=50, rate=1e5)
    limit = 2 * max(r.n for r in reqs) * 56
    stats, ex = run(reqs, free=limit, budget_bytes=1 << 50)
    assert stats.done == len(reqs)
    assert stats.max_in_flight_bytes <= limit


def test_stuck_batch_fails_after_its_deadline():
    reqs = make(count=40)
    stats, ex = run(reqs, stuck={5}, deadline_s=0.05)
    assert reqs[5].status == "failed"
    assert stats.failed >= 1
    assert stats.done + stats.failed == len(reqs)
    assert ex.allocated == 0


def test_workload_shape():
    reqs = serve.workload(count=4096)
    ns = [r.n for r in reqs]
    assert min(ns) >= 1000 and max(ns) <= 10_000_000
    assert 1.5 < reqs[-1].arrival < 2.6      # ~2.05 s of arrivals at 2000 req/s
    kinds = {(tuple(r.record), str(r.src_map), str(r.dst_map)) for r in reqs}
    assert len(kinds) == len(serve.SERVE_PAIRS)


def test_summary_percentiles():
    s = serve.ServeStats(latencies_s=[i / 1000 for i in range(1, 101)], makespan_s=1.0, bytes=10**9)
    out = s.summary()
    assert out["p50_ms"] == 50.0 and out["p99_ms"] == 99.0 and out["GB/s"] == 1.0
