"""The request loop on the GPU: every request's result is the same alone and
in the mix (bit-exact: the copies are bit-exact), with batches from
different ticks overlapping on the device."""
import numpy as np
import pytest
import torch

from paper_2302_08251_gb300 import llgb, serve
from gpu_util import ensure_library, sync_and_check_status

pytestmark = pytest.mark.gpu


def test_each_result_is_the_same_alone_and_in_the_mix():
    ensure_library()
    reqs = serve.workload(count=80, rate_hz=20000.0, n_lo=1e3, n_hi=3e5, seed=17)
    ex = serve.GpuExecutor(streams=3, seed=5, keep=True)
    srv = serve.Server(ex, budget_bytes=serve.GB, deadline_s=60.0)
    stats = srv.run(reqs)
    sync_and_check_status()
    assert stats.done == len(reqs) and stats.failed == 0
    assert stats.batches > 1
    for r in reqs:
        src, dst_mix = r.result
        alone = llgb.View(ex._record(r.record), r.dst_map, (r.n,))
        for b in alone.blobs:
            b.fill_(0x3C)
        llgb.llgb_copy(src, alone)
        torch.cuda.synchronize()
        for a, m in zip(alone.blob_bytes(), dst_mix.blob_bytes()):
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
