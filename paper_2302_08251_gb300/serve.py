"""Continuous-batching request loop for re-layout requests.

Requests (a record type, a source and a destination mapping, a record count)
arrive over time.  The loop:

1. moves requests whose arrival time has passed into a FIFO queue;
2. retires finished batches (their device events), records each request's
   latency (arrival -> observed completion) and releases its memory;
3. admits queued requests while the bytes of admitted, unfinished requests
   stay within the HBM budget and the device reports enough free memory;
4. turns the requests admitted in this tick into one batch (one fused launch
   per kernel mode) on the next of k streams -- batches from different ticks
   overlap on the device;
5. fails a batch whose event does not complete within its deadline.

The device work goes through an executor (``GpuExecutor`` uses the CUDA
library; tests substitute a host fake), so admission and queueing are
testable without a GPU.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field

from . import synth

GB = 1 << 30


@dataclass
class Request:
    rid: int
    record: list
    src_map: dict
    dst_map: dict
    n: int
    arrival: float                 # seconds after the start of the run
    nbytes: int = 0                # source + destination blob bytes
    admitted: float | None = None
    done: float | None = None
    status: str = "pending"        # pending, queued, running, done, failed, rejected
    views: tuple | None = None


@dataclass
class ServeStats:
    requests: int = 0
    done: int = 0
    failed: int = 0
    rejected: int = 0
    batches: int = 0
    bytes: int = 0
    makespan_s: float = 0.0
    latencies_s: list = field(default_factory=list)
    max_in_flight_bytes: int = 0
    max_overlap: int = 0

    def summary(self) -> dict:
        lat = sorted(self.latencies_s)

        def pct(p):
            if not lat:
                return None
            k = min(len(lat) - 1, max(0, int(math.ceil(p / 100.0 * len(lat))) - 1))
            return lat[k]
        return {"requests": self.requests, "done": self.done, "failed": self.failed,
                "rejected": self.rejected, "batches": self.batches,
                "GB/s": round(self.bytes / self.makespan_s / 1e9, 2) if self.makespan_s else None,
                "p50_ms": round(pct(50) * 1e3, 3) if lat else None,
                "p99_ms": round(pct(99) * 1e3, 3) if lat else None,
                "makespan_s": round(self.makespan_s, 4),
                "max_in_flight_GB": round(self.max_in_flight_bytes / 1e9, 3),
                "max_overlapping_batches": self.max_overlap}


class Server:
    """The request loop.  `executor` provides nbytes(req), free_bytes(),
    allocate(req), launch(reqs, stream_index) -> handle, done(handle),
    release(req) and streams (k)."""

    def __init__(self, executor, budget_bytes: int = 64 * GB, deadline_s: float = 30.0,
                 max_batch: int = 256, clock=time.perf_counter, sleep=time.sleep,
                 free_margin: int = 1 * GB):
        self.ex = executor
        self.budget = budget_bytes
        self.deadline = deadline_s
        self.max_batch = max_batch
        self.clock = clock
        self.sleep = sleep
        self.free_margin = free_margin

    def run(self, requests) -> ServeStats:
        reqs = sorted(requests, key=lambda r: r.arrival)
        stats = ServeStats(requests=len(reqs))
        for r in reqs:
            r.nbytes = self.ex.nbytes(r)
        pending = collections.deque(reqs)
        queue: collections.deque = collections.deque()
        in_flight = []          # (handle, requests, bytes, launch time)
        used = 0
        next_stream = 0
        t0 = self.clock()
        while pending or queue or in_flight:
            now = self.clock() - t0
            while pending and pending[0].arrival <= now:
                r = pending.popleft()
                if r.nbytes > self.budget:
                    r.status = "rejected"          # can never fit the budget
                    stats.rejected += 1
                    continue
                r.status = "queued"
                queue.append(r)
            still = []
            for handle, batch, nbytes, started in in_flight:
                if self.ex.done(handle):
                    t = self.clock() - t0
                    for r in batch:
                        r.done, r.status = t, "done"
                        stats.latencies_s.append(t - r.arrival)
                        self.ex.release(r)
                    stats.done += len(batch)
                    stats.bytes += nbytes
                    used -= nbytes
                elif self.clock() - started > self.deadline:
                    for r in batch:
                        r.status = "failed"
                        self.ex.release(r)
                    stats.failed += len(batch)
                    used -= nbytes
                else:
                    still.append((handle, batch, nbytes, started))
            in_flight = still
            admitted = []
            free = self.ex.free_bytes()
            while queue and len(admitted) < self.max_batch:
                r = queue[0]
                if used + r.nbytes > self.budget or r.nbytes + self.free_margin > free:
                    break                          # FIFO: wait for memory to free up
                try:
                    self.ex.allocate(r)
                except MemoryError:
                    break                          # device refused: retry next tick
                queue.popleft()
                r.admitted, r.status = self.clock() - t0, "running"
                used += r.nbytes
                free -= r.nbytes
                admitted.append(r)
            if admitted:
                handle = self.ex.launch(admitted, next_stream % self.ex.streams)
                next_stream += 1
                nbytes = sum(r.nbytes for r in admitted)
                in_flight.append((handle, admitted, nbytes, self.clock()))
                stats.batches += 1
            stats.max_in_flight_bytes = max(stats.max_in_flight_bytes, used)
            stats.max_overlap = max(stats.max_overlap, len(in_flight))
            assert used <= self.budget
            if not admitted:
                waits = [pending[0].arrival - (self.clock() - t0)] if pending else []
                self.sleep(max(0.0, min([2e-4] + waits)))
        stats.makespan_s = self.clock() - t0
        return stats


# ---------------------------------------------------------------- device --

class GpuExecutor:
    """Runs request batches through the CUDA library on k streams, each batch
    one llgb_batch_arena_copy (fused launches over descriptor tables allocated
    once).  Source blobs are filled on the request's stream at admission
    (seeded bytes)."""

    def __init__(self, streams: int = 4, device=None, seed: int = 1, keep: bool = False,
                 max_batch: int = 256):
        import torch
        from . import llgb
        self.torch = torch
        self.llgb = llgb
        self.device = device if device is not None else torch.device("cuda")
        self.streams = streams
        self._streams = [torch.cuda.Stream(device=self.device) for _ in range(streams)]
        # descriptor tables for every batch, allocated once: launching a batch
        # then neither allocates nor frees device memory, and nothing in the
        # loop synchronises the device
        with torch.cuda.device(self.device):
            self._arena = llgb.Arena(max_pairs=max_batch, slots=2 * streams + 2)
        self._records = {}
        self._sizes = {}
        self.seed = seed
        self.keep = keep  # keep each finished request's views in r.result (tests)

    def warm(self, pairs, n: int = 1 << 16) -> None:
        """Before serving: plan one batch of n-record views per (record,
        source mapping, destination mapping) in `pairs` and drop it, so that
        the library's cache holds the gather programs of those layouts (the
        arena only looks programs up; it builds none).  Allocates and waits,
        once per layout."""
        import json
        torch = self.torch
        seen = set()
        for record, src_map, dst_map in pairs:
            key = (tuple(record), json.dumps(src_map, sort_keys=True), json.dumps(dst_map, sort_keys=True))
            if key in seen:
                continue
            seen.add(key)
            rec = self._record(record)
            with torch.cuda.device(self.device):
                src = self.llgb.View(rec, src_map, (n,), device=self.device)
                dst = self.llgb.View(rec, dst_map, (n,), device=self.device)
                self.llgb.Batch([(src, dst)]).close()
            del src, dst

    def _record(self, rec):
        key = tuple(rec)
        if key not in self._records:
            self._records[key] = self.llgb.Record(rec)
        return self._records[key]

    def nbytes(self, r: Request) -> int:
        import json
        key = (tuple(r.record), json.dumps(r.src_map, sort_keys=True),
               json.dumps(r.dst_map, sort_keys=True), r.n)
        if key not in self._sizes:
            rec = self._record(r.record)
            self._sizes[key] = (sum(self.llgb.blob_sizes(rec, r.src_map, (r.n,))) +
                                sum(self.llgb.blob_sizes(rec, r.dst_map, (r.n,))))
        return self._sizes[key]

    def free_bytes(self) -> int:
        return int(self.torch.cuda.mem_get_info(self.device)[0])

    def allocate(self, r: Request) -> None:
        torch = self.torch
        rec = self._record(r.record)
        try:
            src = self.llgb.View(rec, r.src_map, (r.n,), device=self.device)
            dst = self.llgb.View(rec, r.dst_map, (r.n,), device=self.device)
        except torch.cuda.OutOfMemoryError as e:
            raise MemoryError(str(e))
        s = self._streams[r.rid % self.streams]
        with torch.cuda.stream(s):
            for k, b in enumerate(src.blobs):
                b.copy_(synth.device_random_bytes(b.numel(), self.seed * 1000003 + r.rid * 64 + k,
                                                  device=self.device))
        r.views = (src, dst, s)

    def launch(self, reqs, stream_index: int):
        torch = self.torch
        s = self._streams[stream_index]
        for r in reqs:                     # sources were filled on their own streams
            s.wait_stream(r.views[2])
        self._arena.copy([(r.views[0], r.views[1]) for r in reqs], stream=s)
        ev = torch.cuda.Event()
        ev.record(s)
        return (ev, s)

    def done(self, handle) -> bool:
        return handle[0].query()

    def release(self, r: Request) -> None:
        if r.views is not None:
            src, dst, s = r.views
            r.views = None
            if self.keep:
                r.result = (src, dst)
                return
            # blobs go back to torch's caching allocator once the stream is past them
            for b in list(src.blobs) + list(dst.blobs):
                b.record_stream(s)


# -------------------------------------------------------------- workload --

SERVE_PAIRS = [
    ("particle", {"kind": "aos"}, {"kind": "soa_mb"}),
    ("particle", {"kind": "soa_mb"}, {"kind": "aos"}),
    ("cfd", {"kind": "soa_mb"}, {"kind": "aosoa", "lanes": 32}),
    ("cfd", {"kind": "aosoa", "lanes": 32}, {"kind": "soa_mb"}),
    ("cfd", {"kind": "aosoa", "lanes": 8}, {"kind": "aosoa", "lanes": 32}),
    ("int6", {"kind": "soa_mb"}, {"kind": "bitpack_int", "bits": 12}),
    ("particle", {"kind": "soa_mb"}, {"kind": "bytesplit", "inner": {"kind": "soa_mb"}}),
]
RECORD = {"particle": synth.PARTICLE, "cfd": synth.CFD, "int6": synth.INT6}


def workload(count: int = 4096, rate_hz: float = 2000.0, n_lo: float = 1e3, n_hi: float = 1e7,
             seed: int = 2302082514):
    """Requests with log-uniform record counts in [n_lo, n_hi], mapping pairs
    drawn uniformly from SERVE_PAIRS, Poisson arrivals at rate_hz."""
    g = synth.rng(seed)
    t = 0.0
    out = []
    for k in range(count):
        t += float(g.exponential(1.0 / rate_hz))
        name, sm, dm = SERVE_PAIRS[int(g.integers(0, len(SERVE_PAIRS)))]
        n = int(round(math.exp(g.uniform(math.log(n_lo), math.log(n_hi)))))
        out.append(Request(rid=k, record=RECORD[name], src_map=sm, dst_map=dm, n=n, arrival=t))
    return out
