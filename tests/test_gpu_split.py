"""GPU parity of copies through Null and Split views (Sec. 3) against the
oracle, byte for byte (every destination blob pre-filled with 0xAB).
"""
import numpy as np
import pytest

import oracle
from paper_2302_08251_gb300 import llgb, synth
from helpers import oracle_view
from gpu_util import assert_same_bytes, device_view_of, empty_device_view, ensure_library, sync_and_check_status

pytestmark = pytest.mark.gpu

REC = [("x", "f32"), ("n", "u32"), ("y", "f64"), ("k", "i32"), ("c", "u8"), ("z", "f32")]
INT_FLOAT = {"kind": "split", "fields": [1, 3], "inner": {"kind": "bitpack_int", "bits": 12},
             "rest": {"kind": "soa_mb"}}
SPLITS = [
    INT_FLOAT,
    {"kind": "split", "fields": [0, 5], "inner": {"kind": "aosoa", "lanes": 32}, "rest": {"kind": "aos"}},
    {"kind": "split", "fields": [2], "inner": {"kind": "changetype", "ct": [("f64", "f32")],
                                              "inner": {"kind": "soa_mb"}},
     "rest": {"kind": "bytesplit", "inner": {"kind": "soa_mb"}}},
    {"kind": "split", "fields": [0, 1, 2], "inner": {"kind": "split", "fields": [2], "inner": {"kind": "soa_sb"},
                                                     "rest": {"kind": "aos", "packed": 1}},
     "rest": {"kind": "aosoa", "lanes": 8}},
    {"kind": "split", "fields": [4], "inner": {"kind": "null"}, "rest": {"kind": "soa_mb"}},
]
PLAIN = [{"kind": "soa_mb"}, {"kind": "aos"}, {"kind": "aosoa", "lanes": 16}]
SHAPE = {"tile_records": 256, "src_stages": 2, "dst_stages": 2, "threads": 256, "ctas_per_sm": 1}


@pytest.fixture(scope="module", autouse=True)
def lib():
    return ensure_library()


def fields(n, seed):
    cols = synth.uniform_fields(REC, n, seed)
    cols[1] = cols[1] % (1 << 12)          # in range for 12 bits (unsigned)
    cols[3] = cols[3] % (1 << 11) - 1024   # in range for 12 bits (signed)
    return cols


def run_pair(src_map, dst_map, n, cfg=None, seed=1):
    src_o = oracle_view(REC, src_map, fields(n, seed))
    dst_o = oracle.OracleView(REC, dst_map, n)
    src_o.copy_to(dst_o)
    src_g = device_view_of(src_o)
    dst_g = empty_device_view(REC, dst_map, n)
    if cfg is None:
        llgb.llgb_copy(src_g, dst_g)
    else:
        llgb.llgb_copy_with(src_g, dst_g, cfg)
    sync_and_check_status()
    assert_same_bytes(dst_g, dst_o, f"{src_map} -> {dst_map}")


@pytest.mark.parametrize("engine", ["auto", "value", "gather"])
@pytest.mark.parametrize("split", range(len(SPLITS)))
@pytest.mark.parametrize("plain", range(len(PLAIN)))
def test_plain_to_split_and_back(split, plain, engine):
    n = 5000 + 17
    cfg = None if engine == "auto" else dict(SHAPE, engine=engine)
    run_pair(PLAIN[plain], SPLITS[split], n, cfg)
    run_pair(SPLITS[split], PLAIN[plain], n, cfg)


@pytest.mark.parametrize("a,b", [(0, 1), (1, 3), (2, 4), (3, 0), (4, 2)])
def test_split_to_split(a, b):
    run_pair(SPLITS[a], SPLITS[b], 3000 + 5)


def test_null_view_on_either_side():
    n = 2048 + 3
    run_pair({"kind": "null"}, {"kind": "aos"}, n)   # loads zeros
    run_pair({"kind": "soa_mb"}, {"kind": "split", "fields": [0, 2], "inner": {"kind": "soa_mb"},
                                  "rest": {"kind": "null"}}, n)


def test_int_bitpack_float_soa_split_many_tiles():
    # many tiles per CTA at full-size-like tiles: bit streams beside plain arrays
    run_pair({"kind": "soa_mb"}, INT_FLOAT, 400000 + 11)
    run_pair(INT_FLOAT, {"kind": "aos"}, 400000 + 11)


def test_particle_cache_view_on_the_gpu():
    # the subset-field cache view of the n-body consumer, filled by the copy
    # kernel from a SoA particle view: {x, y, z, m} records, no velocities
    n = 65536 + 5
    cols = synth.particles(n, 12)
    cache = {"kind": "split", "fields": [0, 1, 2, 6], "inner": {"kind": "aos"}, "rest": {"kind": "null"}}
    src = device_view_of(oracle_view(synth.PARTICLE, {"kind": "soa_mb"}, cols))
    dst = empty_device_view(synth.PARTICLE, cache, n)
    llgb.llgb_copy(src, dst)
    sync_and_check_status()
    want = np.stack([cols[0], cols[1], cols[2], cols[6]], axis=1).astype(np.float32)
    assert dst.blob_bytes()[0].tobytes() == want.tobytes()
