"""Host-side checks of the C ABI (no GPU needed, no compute calls).

* the library builds, loads and exports every function declared in include/*.h;
* view planning (blob count and sizes) agrees with the oracle for every
  mapping kind, record and size class;
* descriptor validation and the index-type rule of Sec. 2 (a view whose
  record count or largest byte offset does not fit its index type is
  rejected) return the documented status codes.
"""
import ctypes
import glob
import os
import re
import subprocess

import pytest

import oracle
from paper_2302_08251_gb300 import build, llgb, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names.update(re.findall(r"\b(llgb_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported():
    names = declared_functions()
    assert len(names) >= 19
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (llgb_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    L = llgb.lib()
    for n in names:
        assert hasattr(L, n)


def test_binding_covers_the_exports():
    assert set(llgb.EXPORTS) <= set(declared_functions())


def test_version_and_no_error_yet():
    assert b"sm_103a" in llgb.lib().llgb_version()


def host_view(record, mapping, n, index_type="u64", extents=None):
    """Plan a view (host only) and return its blob sizes."""
    rec = llgb.Record(record)
    ext = extents if extents is not None else (n,)
    keep = []
    e = llgb.extents_desc(ext, index_type)
    m = llgb.mapping_desc(mapping, keep)
    h = ctypes.c_void_p()
    llgb.check(llgb.lib().llgb_view_create(rec.handle, ctypes.byref(e), ctypes.byref(m),
                                           ctypes.byref(h)))
    nb = llgb.lib().llgb_view_blob_count(h)
    sizes = [int(llgb.lib().llgb_view_blob_size(h, k)) for k in range(nb)]
    llgb.lib().llgb_view_destroy(h)
    return rec, sizes


MAPPINGS = [
    {"kind": "aos"}, {"kind": "aos", "packed": 1}, {"kind": "soa_mb"}, {"kind": "soa_sb"},
    {"kind": "soa_sb", "subarray_align": 128}, {"kind": "aosoa", "lanes": 8},
    {"kind": "aosoa", "lanes": 32}, {"kind": "aosoa", "lanes": 3},
    {"kind": "bytesplit", "inner": {"kind": "soa_mb"}},
    {"kind": "bytesplit", "inner": {"kind": "aos", "packed": 1}},
    {"kind": "changetype", "ct": [("f64", "f32")], "inner": {"kind": "soa_mb"}},
    {"kind": "changetype", "ct": [("f64", "f32")], "inner": {"kind": "aos"}},
    {"kind": "null"},
    {"kind": "split", "fields": [0], "inner": {"kind": "soa_mb"}, "rest": {"kind": "aos"}},
    {"kind": "split", "fields": [1, 2], "inner": {"kind": "null"}, "rest": {"kind": "aosoa", "lanes": 8}},
    {"kind": "split", "fields": [0, 2], "inner": {"kind": "bytesplit", "inner": {"kind": "soa_mb"}},
     "rest": {"kind": "split", "fields": [0], "inner": {"kind": "soa_sb"}, "rest": {"kind": "aos", "packed": 1}}},
]


@pytest.mark.parametrize("mapping", MAPPINGS, ids=str)
@pytest.mark.parametrize("rec", [synth.MIXED_F, synth.CFD, synth.PARTICLE], ids=["mixed", "cfd", "particle"])
@pytest.mark.parametrize("n", [1, 127, 128, 1000, 65537])
def test_blob_sizes_agree_with_the_oracle(mapping, rec, n):
    _, sizes = host_view(rec, mapping, n)
    assert sizes == oracle.OracleView(rec, mapping, n).blob_sizes


@pytest.mark.parametrize("b", [1, 3, 7, 12, 17, 31, 32])
@pytest.mark.parametrize("n", [1, 33, 4096, 100003])
def test_bitpack_int_blob_sizes(b, n):
    m = {"kind": "bitpack_int", "bits": b}
    _, sizes = host_view(synth.INT6, m, n)
    assert sizes == oracle.OracleView(synth.INT6, m, n).blob_sizes


@pytest.mark.parametrize("e,m", [(5, 2), (5, 10), (8, 23), (11, 52), (11, 23), (8, 52)])
def test_bitpack_float_blob_sizes(e, m):
    mp = {"kind": "bitpack_float", "exp": e, "man": m}
    _, sizes = host_view(synth.MIXED_F, mp, 1001)
    assert sizes == oracle.OracleView(synth.MIXED_F, mp, 1001).blob_sizes


def test_full_size_workloads_fit_u32_indexing():
    _, s = host_view(synth.CFD, {"kind": "aos"}, 0, "u32", extents=(512, 512, 512))
    assert s == [512 ** 3 * 24]
    _, s = host_view(synth.INT6, {"kind": "bitpack_int", "bits": 31}, 1 << 26, "u32")
    assert len(s) == 6
    _, s = host_view(synth.MIXED_F, {"kind": "bitpack_float", "exp": 11, "man": 52}, 1 << 25, "i32")
    assert s == [(1 << 25) * 8] * 4


def expect_status(record, mapping, ext, itype, status):
    rec = llgb.Record(record)
    keep = []
    e = llgb.extents_desc(ext, itype)
    m = llgb.mapping_desc(mapping, keep)
    h = ctypes.c_void_p()
    got = llgb.lib().llgb_view_create(rec.handle, ctypes.byref(e), ctypes.byref(m), ctypes.byref(h))
    if got == 0:
        llgb.lib().llgb_view_destroy(h)
    assert got == status, llgb.lib().llgb_last_error()
    return llgb.lib().llgb_last_error().decode()


def test_index_type_overflow_is_rejected():
    # 2^15 records of 24 bytes: n-1 fits i16? no (32767 is the max index)
    expect_status(synth.CFD, {"kind": "soa_mb"}, (32768,), "i16", llgb.ERR_INDEX_OVERFLOW)
    # 1366 records x 24 B = 32784 bytes: the largest byte offset overflows i16
    expect_status(synth.CFD, {"kind": "aos"}, (1366,), "i16", llgb.ERR_INDEX_OVERFLOW)
    expect_status(synth.CFD, {"kind": "aos"}, (1365,), "i16", llgb.OK)
    # 512^3 x 24 B fits u32 but not i32
    expect_status(synth.CFD, {"kind": "aos"}, (512, 512, 512), "u32", llgb.OK)
    expect_status(synth.CFD, {"kind": "aos"}, (512, 512, 512), "i32", llgb.ERR_INDEX_OVERFLOW)
    expect_status(synth.CFD, {"kind": "aos"}, (512, 512, 700), "u32", llgb.ERR_INDEX_OVERFLOW)


def test_descriptor_validation():
    expect_status(synth.MIXED_F, {"kind": "bitpack_int", "bits": 8}, (10,), "u64",
                  llgb.ERR_INVALID_ARG)
    expect_status(synth.INT6, {"kind": "bitpack_float", "exp": 8, "man": 23}, (10,), "u64",
                  llgb.ERR_INVALID_ARG)
    expect_status(synth.INT6, {"kind": "bitpack_int", "bits": 33}, (10,), "u64",
                  llgb.ERR_INVALID_ARG)
    expect_status(synth.MIXED_F, {"kind": "bitpack_float", "exp": 1, "man": 23}, (10,), "u64",
                  llgb.ERR_INVALID_ARG)
    expect_status(synth.MIXED_F, {"kind": "bytesplit", "inner": {"kind": "bitpack_int", "bits": 3}},
                  (10,), "u64", llgb.ERR_UNSUPPORTED)
    expect_status(synth.MIXED_F, {"kind": "soa_sb", "subarray_align": 24}, (10,), "u64",
                  llgb.ERR_INVALID_ARG)
    expect_status(synth.INT6, {"kind": "changetype", "ct": [("i32", "i16")],
                               "inner": {"kind": "soa_mb"}}, (10,), "u64", llgb.ERR_INVALID_ARG)


def test_record_validation():
    with pytest.raises(llgb.LlgbError):
        llgb.Record([("a", "f32"), ("a", "f32")])
    r = llgb.Record(synth.MIXED_F)
    assert r.size(packed=False) == 32 and r.size(packed=True) == 28


def test_copy_rejects_mismatched_and_unbound_views():
    L = llgb.lib()
    r1, r2 = llgb.Record(synth.MIXED_F), llgb.Record(synth.CFD)
    handles = []
    for rec, n in ((r1, 10), (r1, 11), (r2, 10)):
        keep = []
        e = llgb.extents_desc((n,))
        m = llgb.mapping_desc({"kind": "soa_mb"}, keep)
        h = ctypes.c_void_p()
        llgb.check(L.llgb_view_create(rec.handle, ctypes.byref(e), ctypes.byref(m), ctypes.byref(h)))
        handles.append(h)
    assert L.llgb_copy(handles[0], handles[1], None) == llgb.ERR_MISMATCH
    assert L.llgb_copy(handles[0], handles[2], None) == llgb.ERR_MISMATCH
    assert L.llgb_copy(handles[0], handles[0], None) == llgb.ERR_UNBOUND
    bad = (ctypes.c_void_p * 4)(*[ctypes.c_void_p(8)] * 4)
    assert L.llgb_view_bind(handles[0], bad, 4) == llgb.ERR_INVALID_ARG
    assert L.llgb_view_bind(handles[0], bad, 3) == llgb.ERR_INVALID_ARG
    for h in handles:
        L.llgb_view_destroy(h)


def test_default_launch_shape_fits_the_tile_rules():
    L = llgb.lib()
    rec = llgb.Record(synth.CFD)
    hs = []
    for mp in ({"kind": "aos"}, {"kind": "aosoa", "lanes": 32}):
        keep = []
        e = llgb.extents_desc((1 << 20,))
        m = llgb.mapping_desc(mp, keep)
        h = ctypes.c_void_p()
        llgb.check(L.llgb_view_create(rec.handle, ctypes.byref(e), ctypes.byref(m), ctypes.byref(h)))
        hs.append(h)
    c = llgb.LaunchConfig()
    llgb.check(L.llgb_copy_config(hs[0], hs[1], ctypes.byref(c)))
    assert c.tile_records % 128 == 0 and c.tile_records >= 128
    assert c.threads in (128, 256, 512, 1024)
    for h in hs:
        L.llgb_view_destroy(h)


def test_copy_with_rejects_an_unknown_engine():
    L = llgb.lib()
    rec = llgb.Record(synth.PARTICLE)
    hs = []
    for mp in ({"kind": "aos"}, {"kind": "soa_mb"}):
        keep = []
        e = llgb.extents_desc((1000,))
        m = llgb.mapping_desc(mp, keep)
        h = ctypes.c_void_p()
        llgb.check(L.llgb_view_create(rec.handle, ctypes.byref(e), ctypes.byref(m), ctypes.byref(h)))
        hs.append(h)
    c = llgb.LaunchConfig(tile_records=128, src_stages=2, dst_stages=2, threads=256, ctas_per_sm=1, engine=7)
    assert L.llgb_copy_with(hs[0], hs[1], ctypes.byref(c), None) == llgb.ERR_INVALID_ARG
    c.engine = 1
    c.reserved = 5
    assert L.llgb_copy_with(hs[0], hs[1], ctypes.byref(c), None) == llgb.ERR_INVALID_ARG
    c.reserved = 0
    c.staging = 4
    assert L.llgb_copy_with(hs[0], hs[1], ctypes.byref(c), None) == llgb.ERR_INVALID_ARG
    for h in hs:
        L.llgb_view_destroy(h)


@pytest.mark.parametrize("bad", [
    {"kind": "split", "fields": [], "inner": {"kind": "aos"}, "rest": {"kind": "aos"}},
    {"kind": "split", "fields": [0, 1, 2, 3], "inner": {"kind": "aos"}, "rest": {"kind": "aos"}},
    {"kind": "split", "fields": [9], "inner": {"kind": "aos"}, "rest": {"kind": "aos"}},
])
def test_split_needs_leaves_on_both_sides(bad):
    with pytest.raises(llgb.LlgbError) as err:
        host_view(synth.MIXED_F, bad, 10)
    assert err.value.status == llgb.ERR_INVALID_ARG


def test_split_of_bitpacked_integers_and_plain_floats_plans():
    # reading (15)'s alternative: integer leaves bit-packed, float leaves SoA
    rec = [("x", "f32"), ("n", "u32"), ("y", "f32"), ("k", "i32")]
    m = {"kind": "split", "fields": [1, 3], "inner": {"kind": "bitpack_int", "bits": 12},
         "rest": {"kind": "soa_mb"}}
    _, sizes = host_view(rec, m, 1000)
    assert sizes == oracle.OracleView(rec, m, 1000).blob_sizes == [1500, 1500, 4000, 4000]



@pytest.mark.parametrize("m", [
    {"kind": "bitpack_int", "bits": 12, "lanes": 32},
    {"kind": "bitpack_int", "bits": 0, "field_bits": [1, 3, 7, 12, 17, 31], "lanes": 64},
    {"kind": "bitpack_int", "bits": 32, "lanes": 1024},
])
@pytest.mark.parametrize("n", [1, 31, 32, 33, 1000, 4097])
def test_bitpacked_aosoa_blob_sizes_match_the_oracle(m, n):
    _, sizes = host_view(synth.INT6, m, n)
    assert sizes == oracle.OracleView(synth.INT6, m, n).blob_sizes


def test_bitpacked_float_aosoa_blob_sizes_match_the_oracle():
    m = {"kind": "bitpack_float", "exp": 5, "man": 10, "lanes": 128}
    for n in (1, 127, 128, 129, 5000):
        _, sizes = host_view(synth.MIXED_F, m, n)
        assert sizes == oracle.OracleView(synth.MIXED_F, m, n).blob_sizes


@pytest.mark.parametrize("lanes", [1, 8, 16, 48, 2048])
def test_bitpacked_aosoa_needs_power_of_two_lanes_from_32_to_1024(lanes):
    with pytest.raises(llgb.LlgbError) as err:
        host_view(synth.INT6, {"kind": "bitpack_int", "bits": 12, "lanes": lanes}, 100)
    assert err.value.status == llgb.ERR_UNSUPPORTED


def _handle(record, mapping, n):
    rec = llgb.Record(record)
    keep = []
    e = llgb.extents_desc((n,))
    m = llgb.mapping_desc(mapping, keep)
    h = ctypes.c_void_p()
    llgb.check(llgb.lib().llgb_view_create(rec.handle, ctypes.byref(e), ctypes.byref(m), ctypes.byref(h)))
    return rec, h


def test_nbody_phases_reject_an_unknown_traversal_before_anything_else():
    L = llgb.lib()
    rec, h = _handle(synth.PARTICLE, {"kind": "aos"}, 100)
    assert L.llgb_nbody_move(h, 0.1, 2, None) == llgb.ERR_INVALID_ARG
    assert L.llgb_nbody_update(h, 0.1, 0.1, -1, None) == llgb.ERR_INVALID_ARG
    # a known traversal gets as far as the (unbound) view
    assert L.llgb_nbody_move(h, 0.1, 1, None) == llgb.ERR_UNBOUND
    L.llgb_view_destroy(h)


@pytest.mark.parametrize("lanes", [1, 3, 48, 64])
def test_nbody_takes_aosoa_views_of_any_lane_count(lanes):
    L = llgb.lib()
    rec, h = _handle(synth.PARTICLE, {"kind": "aosoa", "lanes": lanes}, 1000)
    assert L.llgb_nbody_step(h, 0.01, 1e-4, None) == llgb.ERR_UNBOUND  # accepted, then needs memory
    L.llgb_view_destroy(h)


@pytest.mark.parametrize("m", [{"kind": "bitpack_int", "bits": 12},
                               {"kind": "split", "fields": [0], "inner": {"kind": "aos"}, "rest": {"kind": "null"}}])
def test_nbody_rejects_bitpacked_and_split_particle_views(m):
    L = llgb.lib()
    rec = [(f"l{k}", "u32") for k in range(7)] if m["kind"] == "bitpack_int" else synth.PARTICLE
    r, h = _handle(rec, m, 100)
    assert L.llgb_nbody_step(h, 0.01, 1e-4, None) in (llgb.ERR_INVALID_ARG, llgb.ERR_UNSUPPORTED)
    L.llgb_view_destroy(h)


@pytest.mark.parametrize("lanes", [256, 1024])
def test_copy_config_tiles_hold_whole_bit_blocks(lanes):
    L = llgb.lib()
    _, a = _handle(synth.INT6, {"kind": "soa_mb"}, 1 << 20)
    _, b = _handle(synth.INT6, {"kind": "bitpack_int", "bits": 12, "lanes": lanes}, 1 << 20)
    c = llgb.LaunchConfig()
    llgb.check(L.llgb_copy_config(a, b, ctypes.byref(c)))
    assert c.tile_records % lanes == 0 and c.tile_records % 128 == 0
    L.llgb_view_destroy(a)
    L.llgb_view_destroy(b)


def _default_shape(record, src_map, dst_map, n=1 << 26):
    L = llgb.lib()
    _, a = _handle(record, src_map, n)
    _, b = _handle(record, dst_map, n)
    c = llgb.LaunchConfig()
    llgb.check(L.llgb_copy_config(a, b, ctypes.byref(c)))
    L.llgb_view_destroy(a)
    L.llgb_view_destroy(b)
    return c.as_dict()


@pytest.mark.parametrize("dst", [{"kind": "bitpack_int", "bits": 1}, {"kind": "bitpack_int", "bits": 12},
                                 {"kind": "bitpack_int", "bits": 12, "lanes": 32}])
def test_integer_stream_packs_default_to_two_256_thread_ctas(dst):
    c = _default_shape(synth.INT6, {"kind": "soa_mb"}, dst)
    assert (c["threads"], c["ctas_per_sm"], c["src_stages"], c["dst_stages"]) == (256, 2, 2, 2)
    assert 1024 <= c["tile_records"] <= 4096 and c["tile_records"] % 128 == 0


@pytest.mark.parametrize("src, dst", [
    ({"kind": "soa_mb"}, {"kind": "bitpack_float", "exp": 8, "man": 10}),
    ({"kind": "bitpack_float", "exp": 8, "man": 10}, {"kind": "soa_mb"}),
    ({"kind": "soa_mb"}, {"kind": "bytesplit", "inner": {"kind": "soa_mb"}}),
])
def test_float_packs_unpacks_and_bytesplit_keep_one_512_thread_cta(src, dst):
    c = _default_shape(synth.MIXED_F, src, dst, 1 << 25)
    assert (c["threads"], c["ctas_per_sm"]) == (512, 1)


def test_integer_unpacks_keep_one_512_thread_cta():
    c = _default_shape(synth.INT6, {"kind": "bitpack_int", "bits": 12}, {"kind": "soa_mb"})
    assert (c["threads"], c["ctas_per_sm"]) == (512, 1)


# ---- planner decisions, read with llgb_copy_plan (host only) ----

def plan_of(record, src_map, dst_map, n, cfg=None):
    _, a = _handle(record, src_map, n)
    _, b = _handle(record, dst_map, n)
    try:
        return llgb.plan_info(a, b, cfg)
    finally:
        llgb.lib().llgb_view_destroy(a)
        llgb.lib().llgb_view_destroy(b)


def test_plan_affine_pairs_take_gather_programs():
    for src, dst in (({"kind": "aos"}, {"kind": "soa_mb"}), ({"kind": "soa_mb"}, {"kind": "aos"})):
        p = plan_of(synth.CFD, src, dst, 1 << 24)
        assert p["kernel_mode"] in (2, 4), (src, dst)
        assert p["generic_items"] == 0 and p["tiles"] * p["tile_records"] >= 1 << 24
    # as batch entries both keep their gather programs: each runs in CTAs of
    # its own launch shape's size (512 threads for the SoA destination)
    assert plan_of(synth.CFD, {"kind": "soa_mb"}, {"kind": "aos"}, 1 << 24)["batch_kernel_mode"] in (2, 4)
    assert plan_of(synth.CFD, {"kind": "aos"}, {"kind": "soa_mb"}, 1 << 24)["batch_kernel_mode"] in (2, 4)


def test_plan_few_tiles_take_the_value_loops():
    p = plan_of(synth.CFD, {"kind": "aos"}, {"kind": "soa_mb"}, 300)
    assert p["kernel_mode"] == 0 and p["batch_kernel_mode"] == 0


def test_plan_bit_streams_run_specialised_loops():
    # SoA streams in kernel mode 0; AoSoA-organised ones in mode 3 (its loops
    # address runs of a block)
    for m, mode in (({"kind": "bitpack_int", "bits": 12}, 0), ({"kind": "bitpack_int", "bits": 12, "lanes": 256}, 3),
                    ({"kind": "bitpack_int", "bits": 9}, 0)):
        p = plan_of(synth.INT6, {"kind": "soa_mb"}, m, 1 << 20)
        assert p["kernel_mode"] == mode and p["generic_items"] == 0 and p["items"] == 6, m


@pytest.mark.parametrize("n", [1, 100, 1 << 20])
def test_plan_short_bit_runs_take_modes_3_and_1_also_in_batches(n):
    # 32-lane runs hold a quarter of a 128-record super-group, however few the
    # tiles: the compile-time loop of a configured width in kernel mode 3, the
    # generic loop otherwise in mode 1
    p = plan_of(synth.INT6, {"kind": "soa_mb"}, {"kind": "bitpack_int", "bits": 12, "lanes": 32}, n)
    assert p["kernel_mode"] == 3 and p["batch_kernel_mode"] == 3
    assert p["stream_items"] == 6 and p["generic_items"] == 0
    p = plan_of(synth.INT6, {"kind": "soa_mb"}, {"kind": "bitpack_int", "bits": 11, "lanes": 32}, n)
    assert p["kernel_mode"] == 1 and p["batch_kernel_mode"] == 1
    assert p["stream_items"] == 0 and p["generic_items"] == 6


def test_plan_engine_value_keeps_run_addressed_jobs_in_modes_3_and_1():
    cfg = {"tile_records": 1024, "src_stages": 2, "dst_stages": 2, "threads": 512, "ctas_per_sm": 1,
           "engine": "value"}
    p = plan_of(synth.INT6, {"kind": "bitpack_int", "bits": 7, "lanes": 64}, {"kind": "aos"}, 50000, cfg)
    assert p["kernel_mode"] == 3 and p["tile_records"] == 1024
    p = plan_of(synth.INT6, {"kind": "bitpack_int", "bits": 6, "lanes": 64}, {"kind": "aos"}, 50000, cfg)
    assert p["kernel_mode"] == 1 and p["tile_records"] == 1024


def test_plan_of_an_empty_pair_is_zero():
    assert plan_of(synth.INT6, {"kind": "aos"}, {"kind": "soa_mb"}, 0) == {
        "kernel_mode": 0, "batch_kernel_mode": 0, "tile_records": 0, "items": 0, "generic_items": 0,
        "stream_items": 0, "tiles": 0}


@pytest.mark.parametrize("bits", [1, 3, 7, 12, 17, 31])
def test_plan_configured_integer_widths_run_compile_time_stream_loops(bits):
    m = {"kind": "bitpack_int", "bits": bits}
    for src, dst in (({"kind": "soa_mb"}, m), (m, {"kind": "soa_mb"}), ({"kind": "aos"}, m), (m, {"kind": "aos"})):
        p = plan_of(synth.INT6, src, dst, 1 << 20)
        assert p["kernel_mode"] == 0 and p["stream_items"] == 6, (src, dst)


@pytest.mark.parametrize("e,m", [(e, m) for e in (5, 8, 11) for m in (2, 10, 23, 52)])
def test_plan_configured_float_formats_run_compile_time_stream_loops(e, m):
    fmt = {"kind": "bitpack_float", "exp": e, "man": m}
    # x, y, z are f64 and w is f32: f64 as E8M23 / E11M52 and f32 as E8M23 are
    # plain element moves with loops of their own
    want = 3 * ((e, m) not in ((8, 23), (11, 52))) + ((e, m) != (8, 23))
    for src, dst in (({"kind": "soa_mb"}, fmt), (fmt, {"kind": "soa_mb"})):
        p = plan_of(synth.MIXED_F, src, dst, 1 << 20)
        assert p["kernel_mode"] == 0 and p["stream_items"] == want and p["generic_items"] == 0, (src, dst)


def test_plan_other_widths_and_organisations_keep_the_run_time_loops():
    for m in ({"kind": "bitpack_int", "bits": 5}, {"kind": "bitpack_int", "bits": 12, "field_bits": [12, 12, 12, 12, 12, 9]}):
        p = plan_of(synth.INT6, {"kind": "soa_mb"}, m, 1 << 20)
        assert p["stream_items"] == (5 if "field_bits" in m else 0), m
    # the AoSoA organisation of a configured width takes the compile-time loops of mode 1
    p = plan_of(synth.INT6, {"kind": "soa_mb"}, {"kind": "bitpack_int", "bits": 12, "lanes": 256}, 1 << 20)
    assert p["stream_items"] == 6 and p["kernel_mode"] == 3
    # f64 / f32 as E8M23 run the compile-time loops only when organised as AoSoA
    fmt = {"kind": "bitpack_float", "exp": 8, "man": 23}
    assert plan_of(synth.MIXED_F, {"kind": "soa_mb"}, fmt, 1 << 20)["stream_items"] == 0
    p = plan_of(synth.MIXED_F, {"kind": "soa_mb"}, dict(fmt, lanes=32), 1 << 20)
    assert p["stream_items"] == 4 and p["kernel_mode"] == 3 and p["generic_items"] == 0
    p = plan_of(synth.MIXED_F, {"kind": "soa_mb"}, {"kind": "bitpack_float", "exp": 6, "man": 9}, 1 << 20)
    assert p["stream_items"] == 0 and p["generic_items"] == 0


def test_wait_selftest_rejects_limits_out_of_range():
    L = llgb.lib()
    for limit in (0, 999, 10_000_000_001):
        assert L.llgb_wait_selftest(limit, None, None) == llgb.ERR_INVALID_ARG
    assert L.llgb_wait_selftest(1_000_000, ctypes.c_void_p(12), None) == llgb.ERR_INVALID_ARG


def test_batch_arena_rejects_bad_sizes_before_touching_the_device():
    L = llgb.lib()
    h = ctypes.c_void_p()
    for pairs, slots in ((0, 4), (65537, 4), (16, 0), (16, 65)):
        assert L.llgb_batch_arena_create(pairs, slots, ctypes.byref(h)) == llgb.ERR_INVALID_ARG
    assert L.llgb_batch_arena_copy(None, 1, None, None, None) == llgb.ERR_INVALID_ARG


def test_fma_probe_rejects_bad_arguments_before_launching():
    L = llgb.lib()
    fmas = ctypes.c_uint64()
    assert L.llgb_fma_probe(0, ctypes.c_void_p(256), ctypes.byref(fmas), None) == llgb.ERR_INVALID_ARG
    assert L.llgb_fma_probe(10, None, ctypes.byref(fmas), None) == llgb.ERR_INVALID_ARG


def test_autotune_file_round_trip_and_rejects(tmp_path):
    L = llgb.lib()
    llgb.llgb_autotune_clear()
    good = tmp_path / "tune.json"
    good.write_text('{"llgb_autotune": 1, "entries": {\n'
                    '  "w0b2p0:10,10,:x|w0b6p0:10,10,:y|20": [2048, 4, 2, 512, 1, 0, 1],\n'
                    '  "w0b0p0:2,2,:a|w0b2p0:2,2,:b|12": [640, 2, 3, 256, 2, 2, 0]\n}}\n')
    llgb.llgb_autotune_load(str(good))
    out = tmp_path / "again.json"
    llgb.llgb_autotune_save(str(out))
    text = out.read_text()
    assert '"w0b2p0:10,10,:x|w0b6p0:10,10,:y|20": [2048, 4, 2, 512, 1, 0, 1]' in text
    assert '"w0b0p0:2,2,:a|w0b2p0:2,2,:b|12": [640, 2, 3, 256, 2, 2, 0]' in text
    for bad in ('{"something": 1}', '{"llgb_autotune": 1, "entries": {"k": [1, 2]}}',
                '{"llgb_autotune": 1, "entries": {"k": [128, 2, 2, 300, 1, 0, 0]}}',
                '{"llgb_autotune": 1, "entries": {"k": [128, 2, 2, 256, 1, 0, 9]}}'):
        p = tmp_path / "bad.json"
        p.write_text(bad)
        with pytest.raises(llgb.LlgbError) as err:
            llgb.llgb_autotune_load(str(p))
        assert err.value.status == llgb.ERR_INVALID_ARG
    with pytest.raises(llgb.LlgbError):
        llgb.llgb_autotune_load(str(tmp_path / "missing.json"))
    llgb.llgb_autotune_clear()
    llgb.llgb_autotune_save(str(out))
    assert '"entries": {\n}}' in out.read_text()


def test_null_sourced_leaves_leave_a_byte_move_job_on_gather_programs():
    # a Null part loads 0: into a byte-stored destination that is the zero
    # fill of unowned bytes, so the job keeps only byte moves
    null_mass = {"kind": "split", "fields": [6], "inner": {"kind": "null"}, "rest": {"kind": "soa_mb"}}
    p = plan_of(synth.PARTICLE, null_mass, {"kind": "aos"}, 1 << 20)
    assert p["kernel_mode"] in (2, 4) and p["items"] == 6 and p["generic_items"] == 0
    # a bit-packed destination still takes the value loops for every leaf
    p = plan_of(synth.INT6, {"kind": "split", "fields": [5], "inner": {"kind": "null"}, "rest": {"kind": "soa_mb"}},
                {"kind": "bitpack_int", "bits": 12}, 1 << 20)
    assert p["kernel_mode"] == 0 and p["items"] == 6
