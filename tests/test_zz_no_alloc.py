"""The allocation-free batched copy (llgb_batch_copy_noalloc).

Callers that cannot allocate device memory while they run (cudaMalloc may
synchronise the device; a host framework's allocator may own all free HBM;
some deployments fix device memory at start-up) use this entry point.  It
keeps its descriptor tables in a static device array of the library instead
of cudaMalloc'd memory.  Its output must equal the regular entry point's
(llgb_copy per pair) byte for byte -- the same tolerance as every copy test
-- on two calls in a row, which reuse the shared array.

The file is named to be collected last: the test passes alone in a fresh
process and after the rest of the suite.
"""
import ctypes

import numpy as np
import torch
import pytest

from paper_2302_08251_gb300 import llgb, synth
from helpers import oracle_view
from gpu_util import device_view_of, empty_device_view, ensure_library, sync_and_check_status

pytestmark = pytest.mark.gpu

PAIRS = [
    (synth.PARTICLE, {"kind": "aos"}, {"kind": "soa_mb"}),
    (synth.CFD, {"kind": "soa_mb"}, {"kind": "aosoa", "lanes": 32}),
    (synth.CFD, {"kind": "aosoa", "lanes": 8}, {"kind": "aos"}),
    (synth.INT6, {"kind": "soa_mb"}, {"kind": "bitpack_int", "bits": 12}),
    (synth.INT6, {"kind": "bitpack_int", "bits": 12}, {"kind": "soa_mb"}),
    (synth.MIXED_F, {"kind": "soa_mb"}, {"kind": "bytesplit", "inner": {"kind": "soa_mb"}}),
    (synth.MIXED_F, {"kind": "soa_mb"}, {"kind": "bitpack_float", "exp": 8, "man": 23}),
    (synth.MIXED_F, {"kind": "aos"}, {"kind": "changetype", "ct": [("f64", "f32")],
                                      "inner": {"kind": "soa_mb"}}),
    # bit streams organised as AoSoA: a configured width (kernel mode 3) and
    # another one (the generic loop, mode 1)
    (synth.INT6, {"kind": "soa_mb"}, {"kind": "bitpack_int", "bits": 12, "lanes": 32}),
    (synth.INT6, {"kind": "soa_mb"}, {"kind": "bitpack_int", "bits": 11, "lanes": 32}),
]


def fields_for(rec, n, seed):
    if rec is synth.INT6:
        return synth.int6(n, 12, seed)
    if rec is synth.MIXED_F:
        return synth.mixed_f(n, seed)
    return synth.uniform_fields(rec, n, seed)


def build_pairs(seed):
    g = synth.rng(seed)
    pairs = []
    for k in range(24):
        rec, sm, dm = PAIRS[k % len(PAIRS)]
        n = int(g.choice([1, 129, 4000, 50000 + int(g.integers(0, 999))]))
        src = device_view_of(oracle_view(rec, sm, fields_for(rec, n, seed + k)))
        pairs.append((rec, dm, n, src))
    return pairs


def test_noalloc_batch_matches_the_regular_copy_on_two_calls_in_a_row():
    ensure_library()
    pairs = build_pairs(seed=41)
    ref = []
    for rec, dm, n, src in pairs:
        d = empty_device_view(rec, dm, n, fill=0x11)
        llgb.llgb_copy(src, d)
        ref.append(d)
    sync_and_check_status()
    want = [d.blob_bytes() for d in ref]
    outs = [empty_device_view(rec, dm, n) for rec, dm, n, _ in pairs]
    for call in range(2):
        for d in outs:
            for b in d.blobs:
                b.fill_(0x77 + call)  # stale bytes must not survive a call
        # straight through the C ABI
        n = len(pairs)
        srcs = (ctypes.c_void_p * n)(*[p[3].handle for p in pairs])
        dsts = (ctypes.c_void_p * n)(*[d.handle for d in outs])
        llgb.check(llgb.lib().llgb_batch_copy_noalloc(n, srcs, dsts, llgb._stream_ptr(None)))
        sync_and_check_status()
        for k, d in enumerate(outs):
            for got, exp in zip(d.blob_bytes(), want[k]):
                assert np.array_equal(got, exp), (call, k, pairs[k][1])


def test_noalloc_batch_rejects_more_than_64_pairs():
    ensure_library()
    rec = llgb.Record(synth.PARTICLE)
    views = [(llgb.View(rec, {"kind": "aos"}, (10,)), llgb.View(rec, {"kind": "soa_mb"}, (10,)))
             for _ in range(65)]
    with pytest.raises(llgb.LlgbError) as err:
        llgb.llgb_batch_copy_noalloc(views)
    assert err.value.status == llgb.ERR_INVALID_ARG
    llgb.llgb_batch_copy_noalloc(views[:64])
    sync_and_check_status()


def test_noalloc_batch_of_large_jobs_with_opposite_image_sizes():
    # full-size tiles: a pack (large source image) and an unpack (large
    # destination image) in one call share each kernel's stage sizes
    ensure_library()
    n = 1 << 21
    fields = synth.int6(n, 12, 5)
    jobs = [({"kind": "soa_mb"}, {"kind": "bitpack_int", "bits": 12}),
            ({"kind": "bitpack_int", "bits": 12}, {"kind": "aos"})]
    views, ref = [], []
    for sm, dm in jobs:
        src = device_view_of(oracle_view(synth.INT6, sm, fields))
        r = empty_device_view(synth.INT6, dm, n, fill=0x11)
        llgb.llgb_copy(src, r)
        views.append((src, empty_device_view(synth.INT6, dm, n, fill=0x22)))
        ref.append(r)
    sync_and_check_status()
    llgb.llgb_batch_copy_noalloc(views)
    sync_and_check_status()
    for (_, d), r in zip(views, ref):
        for got, exp in zip(d.blob_bytes(), r.blob_bytes()):
            assert np.array_equal(got, exp)


def test_two_calls_with_different_pairs_queued_back_to_back_on_one_stream():
    # no wait between the calls: the second call's descriptors must reach the
    # shared array only after the first call's kernels have read theirs, so
    # both outputs equal the regular copy
    ensure_library()
    first = build_pairs(seed=7)[:9]
    second = build_pairs(seed=8)[9:20]
    assert [p[1] for p in first] != [p[1] for p in second]
    refs = []
    for group in (first, second):
        ref = []
        for rec, dm, n, src in group:
            d = empty_device_view(rec, dm, n, fill=0x11)
            llgb.llgb_copy(src, d)
            ref.append(d.blob_bytes())
        refs.append(ref)
    sync_and_check_status()
    outs = [[empty_device_view(rec, dm, n, fill=0x5A) for rec, dm, n, _ in group] for group in (first, second)]
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    for group, out in zip((first, second), outs):
        n = len(group)
        srcs = (ctypes.c_void_p * n)(*[p[3].handle for p in group])
        dsts = (ctypes.c_void_p * n)(*[d.handle for d in out])
        llgb.check(llgb.lib().llgb_batch_copy_noalloc(n, srcs, dsts, llgb._stream_ptr(stream)))
    stream.synchronize()
    sync_and_check_status()
    for g, (group, out) in enumerate(zip((first, second), outs)):
        for k, d in enumerate(out):
            for got, exp in zip(d.blob_bytes(), refs[g][k]):
                assert np.array_equal(got, exp), (g, k, group[k][1])
