"""Batched copies and the autotuner, against per-view copies and the oracle.

A batch must move every pair exactly as one llgb_copy per pair does (same
bytes, padding included), with or without a CUDA graph, for mixed mapping
pairs, records and sizes (1 record, ragged tails, empty views).
"""
import random

import numpy as np
import pytest
import torch

import oracle
from paper_2302_08251_gb300 import llgb, synth
from helpers import oracle_view
from gpu_util import assert_same_bytes, device_view_of, empty_device_view, ensure_library, sync_and_check_status
from test_gpu_random_pairs import random_field
from test_plan_sweep import leaf_mapping, random_record

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


@pytest.mark.parametrize("seed", range(4))
def test_random_pairs_in_one_batch_arena_and_allocation_free_call(seed):
    # 24 seeded random records and mapping pairs (as in the random single-copy
    # sweep: plain, bit-packed in both organisations, Bytesplit, ChangeType,
    # Split with Null, nested), 0 to 100,007 records each, mixed in one batch
    # (graph and stream launches), one arena copy and one allocation-free
    # call: the jobs of every kernel mode share launch groups and descriptor
    # tables, and every destination must hold the oracle's bytes
    g = random.Random(5000 + seed)
    vals = np.random.default_rng(6000 + seed)
    cases = []
    for _ in range(200):
        if len(cases) == 24:
            break
        leaves = random_record(g)
        types = [t for _, t in leaves]
        n = g.choice([0, 1, 129, 1000, 4097, 20003, 100_007])
        src_map, dst_map = (leaf_mapping(g, types, 0) for _ in range(2))
        try:
            src_o = oracle_view(leaves, src_map, [random_field(t, n, vals) for t in types]) if n else \
                oracle.OracleView(leaves, src_map, 0)
            dst_o = oracle.OracleView(leaves, dst_map, n)
        except ValueError:
            continue  # a mapping the oracle does not take for these leaves
        try:
            src = device_view_of(src_o) if n else empty_device_view(leaves, src_map, 0)
            llgb.llgb_copy_plan(src, empty_device_view(leaves, dst_map, n))
        except llgb.LlgbError as err:
            assert err.status == llgb.ERR_UNSUPPORTED, (src_map, dst_map, err)
            continue
        if n:
            src_o.copy_to(dst_o)
        cases.append((leaves, dst_map, n, src, dst_o))
    assert len(cases) == 24
    outs = [[empty_device_view(leaves, dm, n, fill=f) for leaves, dm, n, _, _ in cases]
            for f in (0xAB, 0x5A, 0x3C, 0x77)]
    pairs = [[(c[3], d) for c, d in zip(cases, out)] for out in outs]
    graph_batch, stream_batch = llgb.Batch(pairs[0]), llgb.Batch(pairs[1])
    graph_batch.launch(use_graph=True)
    stream_batch.launch()
    arena = llgb.Arena(max_pairs=24, slots=2)
    arena.copy(pairs[2])
    llgb.llgb_batch_copy_noalloc(pairs[3])
    sync_and_check_status()
    for how, out in zip(("graph batch", "batch", "arena", "allocation-free"), outs):
        for (leaves, dm, n, _, dst_o), d in zip(cases, out):
            assert_same_bytes(d, dst_o, f"{how}: {leaves} n={n} -> {dm}")
    graph_batch.close()
    stream_batch.close()
    arena.close()
