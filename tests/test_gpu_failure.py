"""Failure detection of the copy kernels on the GPU (bounded waits).

Every wait of a copy kernel on a pipeline barrier is bounded; when one runs
out the kernel records LLGB_ERR_TIMEOUT in the device status word and returns.
The self-test kernel takes that same bounded wait, with a short limit, on a
barrier nothing arrives on: the wait must give up after the limit, the status
word must say TIMEOUT, and the context must stay usable -- a copy right after
is byte-exact against the oracle.  Nothing here faults or hangs: the wait ends
by its limit."""
import pytest
import torch

import oracle
from paper_2302_08251_gb300 import llgb, synth
from helpers import oracle_view
from gpu_util import assert_same_bytes, device_view_of, empty_device_view, ensure_library, sync_and_check_status

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("limit_ns", [1_000_000, 20_000_000])
def test_bounded_wait_gives_up_records_timeout_and_the_context_stays_usable(limit_ns):
    ensure_library()
    sync_and_check_status()
    waited = torch.zeros(1, dtype=torch.int64, device="cuda")
    llgb.llgb_wait_selftest(limit_ns, waited)
    torch.cuda.synchronize()
    assert llgb.llgb_device_status(reset=True) == llgb.ERR_TIMEOUT
    w = int(waited.item())
    assert limit_ns <= w < limit_ns + 200_000_000, w
    # the word was cleared, and the context still runs copies exactly
    assert llgb.llgb_device_status() == 0
    n = 5000
    fields = synth.particles(n, seed=3)
    src_o = oracle_view(synth.PARTICLE, {"kind": "aos"}, fields)
    dst_o = oracle.OracleView(synth.PARTICLE, {"kind": "aosoa", "lanes": 32}, n)
    src_o.copy_to(dst_o)
    dst = empty_device_view(synth.PARTICLE, {"kind": "aosoa", "lanes": 32}, n)
    llgb.llgb_copy(device_view_of(src_o), dst)
    sync_and_check_status()
    assert_same_bytes(dst, dst_o, "copy after a timed-out wait")
