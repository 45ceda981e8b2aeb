"""The request loop on the GPU: every request's result equals the oracle's
copy of the same source bytes, byte for byte, and equals the same copy run
alone; the HBM budget holds on the device."""
import numpy as np
import pytest
import torch

import oracle
from paper_2302_08251_gb300 import llgb, serve
from gpu_util import check_windows, ensure_library, sync_and_check_status

pytestmark = pytest.mark.gpu


def oracle_result(r, src):
    """The oracle's copy of request r's source bytes into r's destination mapping."""
    src_o = oracle.OracleView(r.record, r.src_map, r.n, blobs=src.blob_bytes())
    dst_o = oracle.OracleView(r.record, r.dst_map, r.n)
    src_o.copy_to(dst_o)
    return dst_o.blobs


def test_each_result_matches_the_oracle_alone_and_in_the_mix():
    ensure_library()
    reqs = serve.workload(count=80, rate_hz=20000.0, n_lo=1e3, n_hi=3e5, seed=17)
    ex = serve.GpuExecutor(streams=3, seed=5, keep=True)
    srv = serve.Server(ex, budget_bytes=serve.GB, deadline_s=60.0)
    stats = srv.run(reqs)
    sync_and_check_status()
    assert stats.done == len(reqs) and stats.failed == 0
    assert stats.batches > 1
    assert {r.dst_map["kind"] for r in reqs} >= {"soa_mb", "aos", "aosoa", "bitpack_int", "bytesplit"}
    for r in reqs:
        src, dst_mix = r.result
        mixed = dst_mix.blob_bytes()
        # the oracle, from the same source bytes
        for k, (m, e) in enumerate(zip(mixed, oracle_result(r, src))):
            assert np.array_equal(m, e), (r.rid, r.src_map, r.dst_map, r.n, k)
        # the same copy alone
        alone = llgb.View(ex._record(r.record), r.dst_map, (r.n,))
        for b in alone.blobs:
            b.fill_(0x3C)
        llgb.llgb_copy(src, alone)
        torch.cuda.synchronize()
        for a, m in zip(alone.blob_bytes(), mixed):
            assert np.array_equal(a, m), (r.rid, r.src_map, r.dst_map, r.n)


def test_budget_holds_on_the_device():
    ensure_library()
    reqs = serve.workload(count=40, rate_hz=50000.0, n_lo=1e4, n_hi=1e6, seed=3)
    ex = serve.GpuExecutor(streams=2, seed=1)
    budget = 200 * 1000 * 1000
    srv = serve.Server(ex, budget_bytes=budget, deadline_s=60.0)
    stats = srv.run(reqs)
    sync_and_check_status()
    assert stats.max_in_flight_bytes <= budget
    assert stats.done + stats.rejected == len(reqs)


def test_batches_from_different_ticks_overlap_on_the_device():
    # requests arrive faster than large copies finish: later ticks launch
    # their batches while earlier ones still run (no call in the loop
    # synchronises the device), and every result still equals the oracle's
    ensure_library()
    reqs = serve.workload(count=32, rate_hz=100000.0, n_lo=3e6, n_hi=1e7, seed=29)
    ex = serve.GpuExecutor(streams=4, seed=9, keep=True)
    # the arena then takes the gather programs of these pairs from the cache
    ex.warm([(r.record, r.src_map, r.dst_map) for r in reqs])
    srv = serve.Server(ex, budget_bytes=32 * serve.GB, deadline_s=60.0, max_batch=2)
    stats = srv.run(reqs)
    sync_and_check_status()
    assert stats.done == len(reqs) and stats.failed == 0
    assert stats.max_overlap >= 2, stats.summary()
    for r in reqs:
        src, dst = r.result
        check_windows(src, dst, r.record, r.src_map, r.dst_map, r.n, seed=r.rid)


def test_arena_copies_on_several_streams_match_the_oracle():
    ensure_library()
    reqs = serve.workload(count=30, rate_hz=1e6, n_lo=1e3, n_hi=1e5, seed=41)
    ex = serve.GpuExecutor(streams=1, seed=3, keep=True)
    arena = llgb.Arena(max_pairs=8, slots=3)
    streams = [torch.cuda.Stream() for _ in range(3)]
    for r in reqs:
        ex.allocate(r)
    torch.cuda.synchronize()
    for k in range(0, len(reqs), 5):     # 6 calls over 3 streams and 3 slots: slots are reused
        arena.copy([(r.views[0], r.views[1]) for r in reqs[k:k + 5]], stream=streams[(k // 5) % 3])
    torch.cuda.synchronize()
    arena.close()
    sync_and_check_status()
    for r in reqs:
        src, dst, _ = r.views
        for k, (m, e) in enumerate(zip(dst.blob_bytes(), oracle_result(r, src))):
            assert np.array_equal(m, e), (r.rid, r.src_map, r.dst_map, r.n, k)
