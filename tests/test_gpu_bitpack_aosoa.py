"""GPU parity of bit-packed mappings organised as AoSoA against the oracle,
byte for byte (destination blobs pre-filled with 0xAB): packing from plain
layouts, unpacking back, between the SoA and AoSoA organisations, inside a
Split, at ragged record counts and over many tiles.
"""
import numpy as np
import pytest

import oracle
from paper_2302_08251_gb300 import llgb, synth
from helpers import oracle_view
from gpu_util import assert_same_bytes, device_view_of, empty_device_view, ensure_library, sync_and_check_status

pytestmark = pytest.mark.gpu

INT_MAPS = [
    {"kind": "bitpack_int", "bits": 12, "lanes": 32},
    {"kind": "bitpack_int", "bits": 0, "field_bits": [1, 3, 7, 12, 17, 31], "lanes": 64},
    {"kind": "bitpack_int", "bits": 0, "field_bits": [32, 5, 9, 1, 30, 2], "lanes": 128},
    {"kind": "bitpack_int", "bits": 8, "lanes": 1024},
    {"kind": "bitpack_int", "bits": 16, "lanes": 32},
]
FLOAT_MAPS = [
    {"kind": "bitpack_float", "exp": 8, "man": 23, "lanes": 32},
    {"kind": "bitpack_float", "exp": 5, "man": 10, "lanes": 128},
    {"kind": "bitpack_float", "exp": 0, "man": 0, "field_exp": [11, 6, 4, 8], "field_man": [52, 9, 3, 7],
     "lanes": 64},
    # a 9-bit leaf first: the 64- and 32-bit codes after it sit on 4-byte, not 8-byte, boundaries
    {"kind": "bitpack_float", "exp": 0, "man": 0, "field_exp": [4, 11, 8, 8], "field_man": [4, 52, 23, 23],
     "lanes": 32},
]
PLAIN = [{"kind": "soa_mb"}, {"kind": "aos"}, {"kind": "aosoa", "lanes": 32}]
SIZES = [1, 33, 1000, 5007]


@pytest.fixture(scope="module", autouse=True)
def lib():
    return ensure_library()


def run_pair(rec, fields, src_map, dst_map, cfg=None):
    n = len(fields[0])
    src_o = oracle_view(rec, src_map, fields)
    dst_o = oracle.OracleView(rec, dst_map, n)
    src_o.copy_to(dst_o)
    src_g = device_view_of(src_o)
    dst_g = empty_device_view(rec, dst_map, n)
    if cfg is None:
        llgb.llgb_copy(src_g, dst_g)
    else:
        llgb.llgb_copy_with(src_g, dst_g, cfg)
    sync_and_check_status()
    assert_same_bytes(dst_g, dst_o, f"{src_map} -> {dst_map}")


def int_fields(n, seed, in_range=True):
    if in_range:
        return synth.int6(n, 12, seed)
    return synth.uniform_fields(synth.INT6, n, seed)  # wrap and sign-extend


def float_fields(n, seed):
    cols = synth.mixed_f(n, seed)
    sp = synth.special_f64(max(0, n - 24), seed)[:n]
    cols[0] = np.where(np.arange(n) % 3 == 0, sp, cols[0])
    return cols


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("plain", range(len(PLAIN)))
@pytest.mark.parametrize("m", range(len(INT_MAPS)))
def test_int_pack_and_unpack(m, plain, n):
    for in_range in (True, False):
        f = int_fields(n, n + m, in_range)
        run_pair(synth.INT6, f, PLAIN[plain], INT_MAPS[m])
        run_pair(synth.INT6, f, INT_MAPS[m], PLAIN[plain])


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("plain", range(len(PLAIN)))
@pytest.mark.parametrize("m", range(len(FLOAT_MAPS)))
def test_float_pack_and_unpack(m, plain, n):
    f = float_fields(n, n + 7 * m)
    run_pair(synth.MIXED_F, f, PLAIN[plain], FLOAT_MAPS[m])
    run_pair(synth.MIXED_F, f, FLOAT_MAPS[m], PLAIN[plain])


@pytest.mark.parametrize("lanes", [32, 256])
def test_between_the_soa_and_aosoa_organisations(lanes):
    n = 3000 + 11
    f = int_fields(n, 5, in_range=False)
    soa = {"kind": "bitpack_int", "bits": 0, "field_bits": [1, 3, 7, 12, 17, 31]}
    aosoa = dict(soa, lanes=lanes)
    run_pair(synth.INT6, f, soa, aosoa)
    run_pair(synth.INT6, f, aosoa, soa)
    g = float_fields(n, 6)
    fs = {"kind": "bitpack_float", "exp": 8, "man": 12}
    run_pair(synth.MIXED_F, g, fs, dict(fs, lanes=lanes))
    run_pair(synth.MIXED_F, g, dict(fs, lanes=lanes), fs)


def test_inside_a_split():
    n = 4000 + 3
    f = int_fields(n, 9)
    m = {"kind": "split", "fields": [0, 2, 4], "inner": {"kind": "bitpack_int", "bits": 12, "lanes": 64},
         "rest": {"kind": "soa_mb"}}
    run_pair(synth.INT6, f, {"kind": "aos"}, m)
    run_pair(synth.INT6, f, m, {"kind": "aos"})


@pytest.mark.parametrize("tile,threads", [(128, 128), (1024, 256), (2048, 512)])
def test_launch_shapes(tile, threads):
    n = 20000 + 5
    f = int_fields(n, 2, in_range=False)
    m = {"kind": "bitpack_int", "bits": 0, "field_bits": [1, 3, 7, 12, 17, 31], "lanes": 128}
    cfg = {"tile_records": tile, "src_stages": 2, "dst_stages": 2, "threads": threads, "ctas_per_sm": 1,
           "engine": "value"}
    run_pair(synth.INT6, f, {"kind": "soa_mb"}, m, cfg)
    run_pair(synth.INT6, f, m, {"kind": "soa_mb"}, cfg)


@pytest.mark.parametrize("lanes", [32, 256])
def test_many_tiles(lanes):
    # lanes 32: the generic loop (a 128-record super-group spans runs); 256:
    # the word-assembling loops, two super-groups per run
    n = (1 << 20) + 3
    f = int_fields(n, 4)
    m = {"kind": "bitpack_int", "bits": 12, "lanes": lanes}
    run_pair(synth.INT6, f, {"kind": "soa_mb"}, m)
    run_pair(synth.INT6, f, m, {"kind": "aos"})
    g = float_fields(n // 4, 5)
    fm = {"kind": "bitpack_float", "exp": 8, "man": 23, "lanes": lanes}
    run_pair(synth.MIXED_F, g, {"kind": "soa_mb"}, fm)
    run_pair(synth.MIXED_F, g, fm, {"kind": "soa_mb"})


@pytest.mark.parametrize("noalloc", [False, True])
def test_batched_with_plain_pairs(noalloc):
    # AoSoA-organised bit jobs (kernel mode 1, and mode 0 where the fast
    # loops cover them) batched beside plain re-layouts (modes 0 and 2/4)
    cases = []
    # the 1- and 100-record jobs are few-tile jobs (planned straight into the value loops)
    for k, (m, n) in enumerate([(INT_MAPS[0], 3001), (INT_MAPS[2], 777), ({"kind": "aos"}, 5000),
                                ({"kind": "bitpack_int", "bits": 12, "lanes": 256}, 4099),
                                ({"kind": "aosoa", "lanes": 32}, 1200), (INT_MAPS[0], 100), (INT_MAPS[4], 1),
                                (FLOAT_MAPS[3], 0)]):
        if m["kind"] == "bitpack_float":
            f = float_fields(max(n, 1), 40)
            f = [c[:n] for c in f]
            src_o = oracle_view(synth.MIXED_F, {"kind": "soa_mb"}, f)
            dst_o = oracle.OracleView(synth.MIXED_F, m, n)
            src_o.copy_to(dst_o)
            src = device_view_of(src_o) if n else empty_device_view(synth.MIXED_F, {"kind": "soa_mb"}, 0)
            cases.append((src, empty_device_view(synth.MIXED_F, m, n), dst_o, m))
            continue
        f = int_fields(n, 30 + k, in_range=False)
        src_o = oracle_view(synth.INT6, {"kind": "soa_mb"}, f)
        dst_o = oracle.OracleView(synth.INT6, m, n)
        src_o.copy_to(dst_o)
        cases.append((device_view_of(src_o), empty_device_view(synth.INT6, m, n), dst_o, m))
    pairs = [(s, d) for s, d, _, _ in cases]
    if noalloc:
        llgb.llgb_batch_copy_noalloc(pairs)
    else:
        batch = llgb.Batch(pairs)
        assert 1 <= batch.info()["launches"] <= 4
        batch.launch()
    sync_and_check_status()
    for _, d, want, m in cases:
        assert_same_bytes(d, want, str(m))
    if not noalloc:
        batch.close()


# ---- the compile-time stream loops on AoSoA-organised streams (kernel mode 3):
# every configured width and float format, runs shorter than a super-group
# (32 lanes), one run per super-group (64 or 128) and several super-groups per
# run (256); ragged counts over several tiles ----

@pytest.mark.parametrize("lanes", [32, 64, 256])
@pytest.mark.parametrize("bits", [1, 3, 7, 12, 17, 31])
def test_configured_integer_widths_in_aosoa_streams(bits, lanes):
    m = {"kind": "bitpack_int", "bits": bits, "lanes": lanes}
    n = 70001
    fields = synth.uniform_fields(synth.INT6, n, bits * 7 + lanes)  # wrap and sign-extend
    src = oracle_view(synth.INT6, {"kind": "soa_mb"}, fields)
    packed = oracle.OracleView(synth.INT6, m, n)
    src.copy_to(packed)
    for s, d in (({"kind": "soa_mb"}, m), (m, {"kind": "soa_mb"}), (m, {"kind": "aos"})):
        rec = llgb.Record(synth.INT6)
        views = [llgb.View(rec, x, (n,)) for x in (s, d)]
        p = llgb.llgb_copy_plan(*views)
        assert p["stream_items"] == 6 and p["kernel_mode"] == 3, (s, d)
        del views
        run_pair(synth.INT6, fields, s, d)


@pytest.mark.parametrize("lanes", [32, 64, 256])
@pytest.mark.parametrize("em", [(e, m) for e in (5, 8, 11) for m in (2, 10, 23, 52)], ids=lambda x: f"E{x[0]}M{x[1]}")
def test_configured_float_formats_in_aosoa_streams(em, lanes):
    m = {"kind": "bitpack_float", "exp": em[0], "man": em[1], "lanes": lanes}
    n = 40003
    fields = synth.mixed_f(n, em[0] * 100 + em[1] + lanes)
    fields[0][:64] = synth.special_f64(64, 3)[:64]  # zeros, subnormals, INF, NaN: the general routine
    for s, d in (({"kind": "soa_mb"}, m), (m, {"kind": "soa_mb"})):
        run_pair(synth.MIXED_F, fields, s, d)
