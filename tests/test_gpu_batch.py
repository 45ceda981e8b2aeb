"""Batched copies and the autotuner, against per-view copies and the oracle.

A batch must move every pair exactly as one llgb_copy per pair does (same
bytes, padding included), with or without a CUDA graph, for mixed mapping
pairs, records and sizes (1 record, ragged tails, empty views).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2302_08251_gb300 import llgb, synth
from helpers import oracle_view
from gpu_util import device_view_of, empty_device_view, ensure_library, sync_and_check_status

pytestmark = pytest.mark.gpu

PAIRS = [
    (synth.PARTICLE, {"kind": "aos"}, {"kind": "soa_mb"}),
    (synth.PARTICLE, {"kind": "soa_mb"}, {"kind": "aos"}),
    (synth.CFD, {"kind": "soa_mb"}, {"kind": "aosoa", "lanes": 32}),
    (synth.CFD, {"kind": "aosoa", "lanes": 32}, {"kind": "soa_mb"}),
    (synth.CFD, {"kind": "aosoa", "lanes": 8}, {"kind": "aosoa", "lanes": 32}),
    (synth.INT6, {"kind": "soa_mb"}, {"kind": "bitpack_int", "bits": 12}),
    (synth.INT6, {"kind": "bitpack_int", "bits": 12}, {"kind": "aos"}),
    (synth.MIXED_F, {"kind": "soa_mb"}, {"kind": "bytesplit", "inner": {"kind": "soa_mb"}}),
    (synth.MIXED_F, {"kind": "soa_mb"}, {"kind": "changetype", "ct": [("f64", "f32")],
                                         "inner": {"kind": "soa_mb"}}),
    (synth.MIXED_F, {"kind": "aos"}, {"kind": "bitpack_float", "exp": 5, "man": 10}),
]


@pytest.fixture(scope="module", autouse=True)
def lib():
    return ensure_library()


def fields_for(rec, n, seed):
    if rec is synth.INT6:
        return synth.int6(n, 12, seed)
    if rec is synth.MIXED_F:
        return synth.mixed_f(n, seed)
    return synth.uniform_fields(rec, n, seed)


def make_requests(count, seed):
    g = synth.rng(seed)
    reqs = []
    for k in range(count):
        rec, sm, dm = PAIRS[k % len(PAIRS)]
        n = int(g.choice([0, 1, 77, 128, 1000, 3001, 20000 + int(g.integers(0, 5000))]))
        src_o = oracle_view(rec, sm, fields_for(rec, n, seed + k), n=n) if n else \
            oracle.OracleView(rec, sm, 0)
        dst_o = oracle.OracleView(rec, dm, n)
        if n:
            src_o.copy_to(dst_o)
        reqs.append((rec, sm, dm, n, src_o, dst_o))
    return reqs


def test_batch_equals_per_view_copies_and_the_oracle():
    reqs = make_requests(40, seed=5)
    pairs, singles = [], []
    for rec, sm, dm, n, src_o, dst_o in reqs:
        src = device_view_of(src_o) if n else empty_device_view(rec, sm, 0)
        pairs.append((src, empty_device_view(rec, dm, n)))
        singles.append((src, empty_device_view(rec, dm, n, fill=0x5A)))
    batch = llgb.Batch(pairs)
    info = batch.info()
    assert 1 <= info["launches"] <= 3
    batch.launch()
    for s, d in singles:
        llgb.llgb_copy(s, d)
    sync_and_check_status()
    for (rec, sm, dm, n, src_o, dst_o), (_, d_batch), (_, d_single) in zip(reqs, pairs, singles):
        got, alone = d_batch.blob_bytes(), d_single.blob_bytes()
        for g_blob, a_blob, e_blob in zip(got, alone, dst_o.blobs):
            assert np.array_equal(g_blob, e_blob), (sm, dm, n)
            assert np.array_equal(a_blob, g_blob), (sm, dm, n)
    batch.close()


def test_graph_replays_give_the_same_bytes():
    reqs = make_requests(12, seed=9)
    pairs = []
    for rec, sm, dm, n, src_o, dst_o in reqs:
        src = device_view_of(src_o) if n else empty_device_view(rec, sm, 0)
        pairs.append((src, empty_device_view(rec, dm, n)))
    batch = llgb.Batch(pairs)
    for _ in range(3):
        for _, d in pairs:
            for b in d.blobs:
                b.fill_(0xC3)
        batch.launch(use_graph=True)
        sync_and_check_status()
        for (rec, sm, dm, n, src_o, dst_o), (_, d) in zip(reqs, pairs):
            for g_blob, e_blob in zip(d.blob_bytes(), dst_o.blobs):
                assert np.array_equal(g_blob, e_blob)
    batch.close()


def test_batch_on_a_side_stream():
    reqs = make_requests(6, seed=2)
    pairs = [(device_view_of(s) if n else empty_device_view(r, sm, 0), empty_device_view(r, dm, n))
             for r, sm, dm, n, s, _ in reqs]
    batch = llgb.Batch(pairs)
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    batch.launch(stream=st, use_graph=True)
    st.synchronize()
    for (r, sm, dm, n, _, dst_o), (_, d) in zip(reqs, pairs):
        for g_blob, e_blob in zip(d.blob_bytes(), dst_o.blobs):
            assert np.array_equal(g_blob, e_blob)
    batch.close()


def test_autotune_picks_a_valid_shape_and_copies_stay_exact():
    n = 200003
    fields = synth.cfd(n, 4)
    src_o = oracle_view(synth.CFD, {"kind": "aos"}, fields)
    dst_o = oracle.OracleView(synth.CFD, {"kind": "soa_mb"}, n)
    src_o.copy_to(dst_o)
    src = device_view_of(src_o)
    dst = empty_device_view(synth.CFD, {"kind": "soa_mb"}, n)
    best = llgb.llgb_autotune(src, dst)
    assert best["tile_records"] % 128 == 0 and best["threads"] in (128, 256, 512)
    assert llgb.llgb_copy_config(src, dst) == best
    for b in dst.blobs:
        b.fill_(0xEE)
    llgb.llgb_copy(src, dst)
    sync_and_check_status()
    for g_blob, e_blob in zip(dst.blob_bytes(), dst_o.blobs):
        assert np.array_equal(g_blob, e_blob)
    llgb.llgb_autotune_clear()


def test_batch_of_large_jobs_with_opposite_image_sizes():
    # a pack (large source image, small destination) and an unpack (small
    # source, large destination) at full-size tiles share one batch kernel,
    # whose stages take the largest image of each side
    n = 1 << 21
    fields = synth.int6(n, 12, 31)
    jobs = [({"kind": "soa_mb"}, {"kind": "bitpack_int", "bits": 12}),
            ({"kind": "bitpack_int", "bits": 12}, {"kind": "aos"}),
            ({"kind": "aos"}, {"kind": "aosoa", "lanes": 32})]
    pairs, expect = [], []
    for sm, dm in jobs:
        src_o = oracle_view(synth.INT6, sm, fields)
        dst_o = oracle.OracleView(synth.INT6, dm, n)
        src_o.copy_to(dst_o)
        pairs.append((device_view_of(src_o), empty_device_view(synth.INT6, dm, n)))
        expect.append(dst_o)
    batch = llgb.Batch(pairs)
    batch.launch(use_graph=True)
    sync_and_check_status()
    for (_, d), dst_o in zip(pairs, expect):
        for g_blob, e_blob in zip(d.blob_bytes(), dst_o.blobs):
            assert np.array_equal(g_blob, e_blob)
    batch.close()


GATHER_PAIRS = [
    (synth.PARTICLE, {"kind": "aos"}, {"kind": "soa_mb"}),
    (synth.PARTICLE, {"kind": "soa_mb"}, {"kind": "aos"}),
    (synth.CFD, {"kind": "soa_mb"}, {"kind": "aosoa", "lanes": 32}),
    (synth.CFD, {"kind": "aosoa", "lanes": 8}, {"kind": "aosoa", "lanes": 32}),
    (synth.CFD, {"kind": "aos", "packed": 1}, {"kind": "soa_sb"}),
]


@pytest.mark.parametrize("pair", range(len(GATHER_PAIRS)))
def test_shared_and_per_cta_gather_programs_give_the_same_bytes(pair):
    # llgb_copy and llgb_batch take the job's gather program from the
    # library's program cache (built once by a small kernel), and a batch
    # arena takes it from there when the cache has it; the allocation-free
    # batch never uses the cache, so every CTA builds its own.  All four must
    # store the oracle's bytes.
    rec, sm, dm = GATHER_PAIRS[pair]
    n = 400_000 + 77  # many tiles per CTA: the copy runs its gather kernel mode
    src_o = oracle_view(rec, sm, fields_for(rec, n, 90 + pair))
    dst_o = oracle.OracleView(rec, dm, n)
    src_o.copy_to(dst_o)
    src = device_view_of(src_o)
    d_copy, d_batch, d_arena, d_free = (empty_device_view(rec, dm, n, fill=f) for f in (0xAB, 0x5A, 0x3C, 0x77))
    assert llgb.llgb_copy_plan(src, d_copy)["kernel_mode"] in (2, 4)
    llgb.llgb_copy(src, d_copy)
    batch = llgb.Batch([(src, d_batch)])
    batch.launch()
    arena = llgb.Arena(max_pairs=4, slots=2)
    arena.copy([(src, d_arena)])
    llgb.llgb_batch_copy_noalloc([(src, d_free)])
    sync_and_check_status()
    for d in (d_copy, d_batch, d_arena, d_free):
        got = d.blob_bytes()
        assert all(np.array_equal(g, e) for g, e in zip(got, dst_o.blobs))
    batch.close()
    arena.close()
