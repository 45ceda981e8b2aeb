"""GPU parity of the layout-aware copy against the oracle, byte for byte.

Every destination blob is pre-filled with 0xAB, so padding, AoSoA tail lanes
and bit-stream tail bits written as zero are checked too.  Sizes span several
tiles and a ragged tail; launch shapes are swept.  Bar: bit-exact.
"""
import itertools

import numpy as np
import pytest
import torch

import oracle
from paper_2302_08251_gb300 import llgb, synth
from helpers import AFFINE, oracle_view
from gpu_util import (assert_same_bytes, device_view_of, empty_device_view, ensure_library,
                      sync_and_check_status)

pytestmark = pytest.mark.gpu

PADDED = [("a", "u8"), ("b", "f64"), ("c", "i16"), ("d", "f32"), ("e", "u8")]
RECORDS = {"cfd": synth.CFD, "mixed_f": synth.MIXED_F, "padded": PADDED,
           "particle": synth.PARTICLE}


@pytest.fixture(scope="module", autouse=True)
def lib():
    return ensure_library()


def run_pair(record, fields, src_map, dst_map, cfg=None):
    n = len(fields[0])
    src_o = oracle_view(record, src_map, fields)
    dst_o = oracle.OracleView(record, dst_map, n)
    src_o.copy_to(dst_o)
    src_g = device_view_of(src_o)
    dst_g = empty_device_view(record, dst_map, n)
    if cfg is None:
        llgb.llgb_copy(src_g, dst_g)
    else:
        llgb.llgb_copy_with(src_g, dst_g, cfg)
    sync_and_check_status()
    assert_same_bytes(dst_g, dst_o, f"{src_map} -> {dst_map}")


PAIRS = list(itertools.product(range(len(AFFINE)), repeat=2))


ENGINE_SHAPE = {"tile_records": 384, "src_stages": 4, "dst_stages": 3, "threads": 256, "ctas_per_sm": 2}


@pytest.mark.parametrize("engine", ["auto", "gather", "value"])
@pytest.mark.parametrize("pair", PAIRS, ids=lambda p: f"{p[0]}-{p[1]}")
@pytest.mark.parametrize("name", ["cfd", "padded"])
def test_affine_pairs(pair, name, engine):
    # both tile engines (gather programs, value loops) on every mapping pair;
    # "auto" takes the library's shape and engine choice
    rec = RECORDS[name]
    n = 3001  # several tiles and a ragged tail
    cfg = None if engine == "auto" else dict(ENGINE_SHAPE, engine=engine)
    run_pair(rec, synth.uniform_fields(rec, n, 7), AFFINE[pair[0]], AFFINE[pair[1]], cfg)


@pytest.mark.parametrize("n", [1, 2, 31, 127, 128, 129, 1000, 4096, 65536, 65537])
def test_particle_aos_to_soa_sizes(n):
    run_pair(synth.PARTICLE, synth.particles(n, n), {"kind": "aos"}, {"kind": "soa_mb"})
    run_pair(synth.PARTICLE, synth.particles(n, n), {"kind": "aos"}, {"kind": "soa_mb"},
             dict(ENGINE_SHAPE, tile_records=128, engine="gather"))


@pytest.mark.parametrize("b", [1, 3, 7, 12, 17, 31, 32])
@pytest.mark.parametrize("n", [1, 100, 5000])
def test_bitpack_int_pack_and_unpack(b, n):
    fields = synth.int6(n, b, seed=b + n)
    packed = {"kind": "bitpack_int", "bits": b}
    run_pair(synth.INT6, fields, {"kind": "soa_mb"}, packed)
    run_pair(synth.INT6, fields, packed, {"kind": "soa_mb"})
    run_pair(synth.INT6, fields, {"kind": "aos"}, packed)
    run_pair(synth.INT6, fields, packed, {"kind": "aosoa", "lanes": 32})


def test_bitpack_int_wraps_out_of_range_values():
    n = 2000
    fields = synth.uniform_fields(synth.INT6, n, 3)  # full 32-bit range
    for b in (1, 5, 12, 31):
        run_pair(synth.INT6, fields, {"kind": "soa_mb"}, {"kind": "bitpack_int", "bits": b})


def test_bitpack_int_mixed_widths_and_types():
    rec = [("a", "u8"), ("b", "i16"), ("c", "u64"), ("d", "i64"), ("e", "i8")]
    n = 999
    fields = synth.uniform_fields(rec, n, 5)
    m = {"kind": "bitpack_int", "bits": 0, "field_bits": [3, 9, 64, 33, 1]}
    run_pair(rec, fields, {"kind": "soa_mb"}, m)
    run_pair(rec, fields, m, {"kind": "aos"})


EM = [(5, 2), (5, 10), (5, 23), (5, 52), (8, 2), (8, 10), (8, 23), (8, 52),
      (11, 2), (11, 10), (11, 23), (11, 52)]


@pytest.mark.parametrize("em", EM, ids=lambda x: f"E{x[0]}M{x[1]}")
def test_bitpack_float_pack_and_unpack(em):
    e, m = em
    n = 3000
    fields = synth.mixed_f(n, seed=e * 64 + m)
    special = synth.special_f64(n, seed=e + m)[:n]
    fields[0] = special
    fields[3] = synth.special_f32(n, seed=m)[:n]
    packed = {"kind": "bitpack_float", "exp": e, "man": m}
    run_pair(synth.MIXED_F, fields, {"kind": "soa_mb"}, packed)
    run_pair(synth.MIXED_F, fields, packed, {"kind": "soa_mb"})
    run_pair(synth.MIXED_F, fields, {"kind": "aos"}, packed)


def test_bitpack_float_to_bitpack_float():
    n = 1500
    fields = synth.mixed_f(n, seed=1)
    run_pair(synth.MIXED_F, fields, {"kind": "bitpack_float", "exp": 8, "man": 23},
             {"kind": "bitpack_float", "exp": 5, "man": 2})


@pytest.mark.parametrize("engine", ["auto", "gather"])
@pytest.mark.parametrize("inner", [{"kind": "soa_mb"}, {"kind": "aos", "packed": 1},
                                   {"kind": "aosoa", "lanes": 32}, {"kind": "soa_sb"}], ids=str)
def test_bytesplit(inner, engine):
    # "gather": the byte-move form (one move per byte plane) where a leaf
    # does not take the transpose loops
    n = 2500
    cfg = None if engine == "auto" else dict(ENGINE_SHAPE, tile_records=128, engine=engine)
    fields = synth.mixed_f(n, seed=4)
    bs = {"kind": "bytesplit", "inner": inner}
    run_pair(synth.MIXED_F, fields, {"kind": "soa_mb"}, bs, cfg)
    run_pair(synth.MIXED_F, fields, bs, {"kind": "aos"}, cfg)
    run_pair(synth.CFD, synth.cfd(n, 2), {"kind": "aos"}, bs, cfg)


@pytest.mark.parametrize("inner", [{"kind": "soa_mb"}, {"kind": "aos"},
                                   {"kind": "aosoa", "lanes": 8}], ids=str)
def test_changetype_f64_to_f32(inner):
    n = 3000
    fields = synth.mixed_f(n, seed=6)
    fields[1] = synth.special_f64(n, seed=9)[:n]
    ct = {"kind": "changetype", "ct": [("f64", "f32")], "inner": inner}
    run_pair(synth.MIXED_F, fields, {"kind": "soa_mb"}, ct)
    run_pair(synth.MIXED_F, fields, ct, {"kind": "soa_mb"})
    run_pair(synth.MIXED_F, fields, {"kind": "aos"}, ct)


@pytest.mark.parametrize("to", ["f16", "bf16"])
def test_changetype_f32_to_half_types(to):
    rec = [("a", "f32"), ("b", "f32"), ("c", "i32")]
    n = 4000
    fields = [synth.special_f32(n, seed=1)[:n], synth.particles(n, 2)[0],
              synth.uniform_fields([("c", "i32")], n, 3)[0]]
    ct = {"kind": "changetype", "ct": [("f32", to)], "inner": {"kind": "soa_mb"}}
    run_pair(rec, fields, {"kind": "aos"}, ct)
    run_pair(rec, fields, ct, {"kind": "aos"})


def test_changetype_to_bytesplit_pair():
    n = 1000
    fields = synth.mixed_f(n, seed=3)
    ct = {"kind": "changetype", "ct": [("f64", "f32")], "inner": {"kind": "aos", "packed": 1}}
    bs = {"kind": "bytesplit", "inner": {"kind": "soa_mb"}}
    run_pair(synth.MIXED_F, fields, ct, bs)
    run_pair(synth.MIXED_F, fields, bs, ct)


CONFIGS = [
    {"tile_records": 128, "src_stages": 1, "dst_stages": 1, "threads": 128, "ctas_per_sm": 1},
    {"tile_records": 256, "src_stages": 2, "dst_stages": 1, "threads": 256, "ctas_per_sm": 2},
    {"tile_records": 1024, "src_stages": 4, "dst_stages": 2, "threads": 512, "ctas_per_sm": 1},
    {"tile_records": 2048, "src_stages": 2, "dst_stages": 1, "threads": 512, "ctas_per_sm": 1},
    {"tile_records": 512, "src_stages": 8, "dst_stages": 4, "threads": 256, "ctas_per_sm": 1},
    {"tile_records": 384, "src_stages": 3, "dst_stages": 2, "threads": 256, "ctas_per_sm": 3},
]


@pytest.mark.parametrize("cfg", CONFIGS, ids=lambda c: f"t{c['tile_records']}s{c['src_stages']}d{c['dst_stages']}")
@pytest.mark.parametrize("maps", [({"kind": "aos"}, {"kind": "soa_mb"}),
                                  ({"kind": "soa_mb"}, {"kind": "aosoa", "lanes": 32}),
                                  ({"kind": "aosoa", "lanes": 8}, {"kind": "aosoa", "lanes": 32}),
                                  ({"kind": "soa_mb"}, {"kind": "bitpack_int", "bits": 12})],
                         ids=["aos-soa", "soa-aosoa32", "aosoa8-aosoa32", "pack12"])
@pytest.mark.parametrize("engine", ["auto", "gather"])
def test_launch_shapes(cfg, maps, engine):
    n = 40000 + 77
    if maps[1]["kind"] == "bitpack_int":
        rec, fields = synth.INT6, synth.int6(n, 12, 5)
    else:
        rec, fields = synth.CFD, synth.cfd(n, 5)
    run_pair(rec, fields, maps[0], maps[1], dict(cfg, engine=engine))


def test_single_blob_with_wide_subarray_alignment_zeroes_the_gaps():
    n = 1001  # 4004-byte sub-arrays, each followed by a 92-byte gap at align 4096
    rec = synth.CFD
    fields = synth.cfd(n, 6)
    run_pair(rec, fields, {"kind": "aos"}, {"kind": "soa_sb", "subarray_align": 4096})
    run_pair(rec, fields, {"kind": "soa_sb", "subarray_align": 4096}, {"kind": "aosoa", "lanes": 8})


def test_too_large_launch_shape_is_rejected():
    n = 10000
    src = empty_device_view(synth.CFD, {"kind": "aos"}, n)
    dst = empty_device_view(synth.CFD, {"kind": "soa_mb"}, n)
    with pytest.raises(llgb.LlgbError):
        llgb.llgb_copy_with(src, dst, {"tile_records": 4096, "src_stages": 8, "dst_stages": 4,
                                       "threads": 256, "ctas_per_sm": 1})
    with pytest.raises(llgb.LlgbError):
        llgb.llgb_copy_with(src, dst, {"tile_records": 100, "src_stages": 2, "dst_stages": 1,
                                       "threads": 256, "ctas_per_sm": 1})


def test_unaligned_single_blob_uses_the_plain_path():
    # sub-arrays of 7 i16 / u8 values are not 16-byte aligned: no TMA, same bytes
    rec = [("a", "u8"), ("b", "i16"), ("c", "f32"), ("d", "u8")]
    n = 20001
    fields = synth.uniform_fields(rec, n, 8)
    run_pair(rec, fields, {"kind": "soa_sb"}, {"kind": "aos"})
    run_pair(rec, fields, {"kind": "aos"}, {"kind": "soa_sb"})


def test_empty_view_is_a_no_op():
    src = empty_device_view(synth.CFD, {"kind": "aos"}, 0)
    dst = empty_device_view(synth.CFD, {"kind": "soa_mb"}, 0)
    llgb.llgb_copy(src, dst)
    sync_and_check_status()


def test_multidimensional_extents_with_u32_index_and_static_inner_extents():
    n = 8 * 16 * 16
    fields = synth.cfd(n, 12)
    src_o = oracle_view(synth.CFD, {"kind": "aos"}, fields)
    dst_o = oracle.OracleView(synth.CFD, {"kind": "aosoa", "lanes": 32}, n)
    src_o.copy_to(dst_o)
    rec = llgb.Record(synth.CFD)
    src_g = llgb.View(rec, {"kind": "aos"}, (8, 16, 16), index_type="u32",
                      static=(False, True, True))
    src_g.blobs[0][:src_o.blobs[0].size].copy_(torch.from_numpy(src_o.blobs[0]))
    dst_g = empty_device_view(synth.CFD, {"kind": "aosoa", "lanes": 32}, n, extents=(8, 16, 16),
                              index_type="u16", static=(False, True, True))
    llgb.llgb_copy(src_g, dst_g)
    sync_and_check_status()
    assert_same_bytes(dst_g, dst_o)


def test_pack_and_unpack_check_kinds():
    n = 300
    fields = synth.int6(n, 7, 1)
    plain = device_view_of(oracle_view(synth.INT6, {"kind": "soa_mb"}, fields))
    packed = empty_device_view(synth.INT6, {"kind": "bitpack_int", "bits": 7}, n)
    llgb.llgb_pack(plain, packed)
    back = empty_device_view(synth.INT6, {"kind": "soa_mb"}, n)
    llgb.llgb_unpack(packed, back)
    sync_and_check_status()
    for a, b in zip(back.blob_bytes(), plain.blob_bytes()):
        assert np.array_equal(a, b)
    with pytest.raises(llgb.LlgbError):
        llgb.llgb_pack(packed, back)
    with pytest.raises(llgb.LlgbError):
        llgb.llgb_unpack(plain, back)


def test_stream_argument_is_honoured():
    n = 50000
    fields = synth.cfd(n, 4)
    src_o = oracle_view(synth.CFD, {"kind": "soa_mb"}, fields)
    dst_o = oracle.OracleView(synth.CFD, {"kind": "aos"}, n)
    src_o.copy_to(dst_o)
    src_g = device_view_of(src_o)
    dst_g = empty_device_view(synth.CFD, {"kind": "aos"}, n)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    llgb.llgb_copy(src_g, dst_g, stream=s)
    s.synchronize()
    assert_same_bytes(dst_g, dst_o)


@pytest.mark.parametrize("em", [(5, 2), (2, 5), (5, 10), (8, 23), (11, 52), (3, 4)],
                         ids=lambda x: f"E{x[0]}M{x[1]}")
def test_bitpack_float_many_tiles_per_cta(em):
    # more tiles than CTAs, so every stage is reused: stale stage bytes must
    # never leak into a stream (whole-byte widths included)
    e, m = em
    n = 400000 + 3
    fields = synth.mixed_f(n, seed=e + 7 * m)
    packed = {"kind": "bitpack_float", "exp": e, "man": m}
    cfg = {"tile_records": 128, "src_stages": 2, "dst_stages": 2, "threads": 128, "ctas_per_sm": 1}
    run_pair(synth.MIXED_F, fields, {"kind": "soa_mb"}, packed, cfg)
    run_pair(synth.MIXED_F, fields, packed, {"kind": "aos"}, cfg)


@pytest.mark.parametrize("b", [1, 7, 8, 16, 31])
def test_bitpack_int_many_tiles_per_cta(b):
    n = 300000 + 5
    fields = synth.int6(n, b, seed=b)
    cfg = {"tile_records": 128, "src_stages": 2, "dst_stages": 2, "threads": 128, "ctas_per_sm": 1}
    run_pair(synth.INT6, fields, {"kind": "soa_mb"}, {"kind": "bitpack_int", "bits": b}, cfg)
    run_pair(synth.INT6, fields, {"kind": "bitpack_int", "bits": b}, {"kind": "aos"}, cfg)


# ---- the specialised value loops: lane-constant addressing of 32-record
# groups, shuffle-assembled stream words, integer f64 <-> f32 conversion ----

SHAPES = [
    {"tile_records": 128, "src_stages": 2, "dst_stages": 2, "threads": 128, "ctas_per_sm": 1},
    {"tile_records": 384, "src_stages": 2, "dst_stages": 3, "threads": 512, "ctas_per_sm": 1},
    {"tile_records": 1152, "src_stages": 2, "dst_stages": 2, "threads": 256, "ctas_per_sm": 1},
]


@pytest.mark.parametrize("cfg", SHAPES, ids=lambda c: f"t{c['tile_records']}x{c['threads']}")
@pytest.mark.parametrize("b", [8, 16, 32])
def test_bitpack_int_whole_byte_widths(b, cfg):
    n = 200000 + 77
    fields = synth.int6(n, b, seed=3 * b)
    packed = {"kind": "bitpack_int", "bits": b}
    for other in ({"kind": "soa_mb"}, {"kind": "aosoa", "lanes": 8}, {"kind": "aosoa", "lanes": 64}):
        run_pair(synth.INT6, fields, other, packed, cfg)
        run_pair(synth.INT6, fields, packed, other, cfg)


@pytest.mark.parametrize("cfg", SHAPES, ids=lambda c: f"t{c['tile_records']}x{c['threads']}")
@pytest.mark.parametrize("b", [1, 2, 5, 12, 13, 24, 31])
def test_bitpack_int_group_boundaries(b, cfg):
    # tiles of 4, 12 and 36 groups over 3, 15 and 7 consumer warps: item
    # shares start and end inside items
    n = 150000 + 31
    fields = synth.int6(n, b, seed=b)
    packed = {"kind": "bitpack_int", "bits": b}
    run_pair(synth.INT6, fields, {"kind": "aosoa", "lanes": 16}, packed, cfg)
    run_pair(synth.INT6, fields, packed, {"kind": "aosoa", "lanes": 4}, cfg)


@pytest.mark.parametrize("em", [(11, 40), (8, 40), (10, 30), (11, 51), (9, 24)],
                         ids=lambda x: f"E{x[0]}M{x[1]}")
def test_bitpack_float_codes_wider_than_32_bits(em):
    e, m = em
    n = 90000 + 5
    fields = synth.mixed_f(n, seed=e * m)
    fields[1] = synth.special_f64(n, seed=e)[:n]
    fields[3] = synth.special_f32(n, seed=m)[:n]
    packed = {"kind": "bitpack_float", "exp": e, "man": m}
    for cfg in SHAPES[:2]:
        run_pair(synth.MIXED_F, fields, {"kind": "soa_mb"}, packed, cfg)
        run_pair(synth.MIXED_F, fields, packed, {"kind": "aos"}, cfg)


def test_f64_to_f32_rounding_ties_and_range_edges():
    n = 300000 + 9
    fields = synth.mixed_f(n, seed=8)
    for k in range(3):
        fields[k] = synth.f32_range_f64(n, seed=20 + k)
    f32 = {"kind": "bitpack_float", "exp": 8, "man": 23}
    ct = {"kind": "changetype", "ct": [("f64", "f32")], "inner": {"kind": "soa_mb"}}
    for cfg in (None, SHAPES[1]):
        run_pair(synth.MIXED_F, fields, {"kind": "soa_mb"}, f32, cfg)
        run_pair(synth.MIXED_F, fields, {"kind": "soa_mb"}, ct, cfg)
        run_pair(synth.MIXED_F, fields, ct, {"kind": "aos"}, cfg)
        run_pair(synth.MIXED_F, fields, f32, {"kind": "soa_mb"}, cfg)


BYTES_REC = [("a", "u8"), ("b", "i16"), ("c", "f32"), ("d", "f64"), ("e", "u64"), ("f", "u16")]


@pytest.mark.parametrize("cfg", SHAPES, ids=lambda c: f"t{c['tile_records']}x{c['threads']}")
@pytest.mark.parametrize("inner", [{"kind": "soa_mb"}, {"kind": "aos"}, {"kind": "aosoa", "lanes": 8},
                                   {"kind": "aosoa", "lanes": 64}, {"kind": "soa_sb"}], ids=str)
def test_bytesplit_planes_many_tiles(inner, cfg):
    # 2-, 4- and 8-byte leaves to byte planes and back through 4 x 4 byte
    # transposes; 1-byte leaves stay plain moves; a ragged last tile
    n = 100000 + 45
    fields = synth.uniform_fields(BYTES_REC, n, 12)
    bs = {"kind": "bytesplit", "inner": inner}
    run_pair(BYTES_REC, fields, {"kind": "soa_mb"}, bs, cfg)
    run_pair(BYTES_REC, fields, {"kind": "aos"}, bs, cfg)
    run_pair(BYTES_REC, fields, bs, {"kind": "soa_mb"}, cfg)
    run_pair(BYTES_REC, fields, bs, {"kind": "aosoa", "lanes": 16}, cfg)


@pytest.mark.parametrize("cfg", SHAPES, ids=lambda c: f"t{c['tile_records']}x{c['threads']}")
@pytest.mark.parametrize("inner", [{"kind": "soa_mb"}, {"kind": "aos"}, {"kind": "aosoa", "lanes": 8},
                                   {"kind": "aosoa", "lanes": 64}], ids=str)
def test_moves_beside_conversions(inner, cfg):
    # one f64 leaf changes type, so the job converts values and its 1-, 2-,
    # 4- and 8-byte leaves run as whole-element moves in the value loops
    n = 120000 + 13
    fields = synth.uniform_fields(BYTES_REC, n, 21)
    ct = {"kind": "changetype", "ct": [("f64", "f32")], "inner": inner}
    for other in ({"kind": "soa_mb"}, {"kind": "aos"}, {"kind": "aosoa", "lanes": 32}):
        run_pair(BYTES_REC, fields, other, ct, cfg)
        run_pair(BYTES_REC, fields, ct, other, cfg)
