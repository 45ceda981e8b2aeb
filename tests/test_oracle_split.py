"""Oracle pins for the Null and Split mappings (Sec. 3).

Split{fields -> inner, rest -> rest} must store exactly what two ordinary
views store: one of the selected leaves (in leaf order) under `inner`, one
of the other leaves under `rest`, blobs in that order.  Null stores nothing
and loads zeros.  The ordinary views are pinned elsewhere; these tests pin
the composition (leaf order, blob order, field routing) against them.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2302_08251_gb300 import synth
from helpers import oracle_view

REC = [("a", "u8"), ("b", "f64"), ("c", "i16"), ("d", "f32"), ("e", "u32"), ("f", "f64")]
PLAIN = [{"kind": "aos"}, {"kind": "aos", "packed": 1}, {"kind": "soa_mb"}, {"kind": "soa_sb"},
         {"kind": "aosoa", "lanes": 8}]


def sub_record(fields):
    return [REC[f] for f in fields]


def fill(view_rec, n, seed):
    return synth.uniform_fields(view_rec, n, seed)


@pytest.mark.parametrize("sel", [[0], [1, 3], [0, 2, 4], [5], [1, 2, 3, 4, 5]])
@pytest.mark.parametrize("pair", list(itertools.product(range(len(PLAIN)), repeat=2))[::3])
def test_split_stores_what_two_plain_views_store(sel, pair):
    n = 77
    rest = [f for f in range(len(REC)) if f not in sel]
    m_sel, m_rest = PLAIN[pair[0]], PLAIN[pair[1]]
    split = {"kind": "split", "fields": sel, "inner": m_sel, "rest": m_rest}
    cols = fill(REC, n, 3)
    v = oracle_view(REC, split, cols)
    a = oracle_view(sub_record(sel), m_sel, [cols[f] for f in sel])
    b = oracle_view(sub_record(rest), m_rest, [cols[f] for f in rest])
    assert v.blob_sizes == a.blob_sizes + b.blob_sizes
    for got, want in zip(v.blobs, a.blobs + b.blobs):
        assert np.array_equal(got, want)
    # and every leaf reads back through the split
    for f in range(len(REC)):
        assert np.array_equal(v.field_values(f), oracle_view(REC, {"kind": "soa_mb"}, cols).field_values(f))


def test_null_stores_nothing_and_loads_zeros():
    n = 50
    cols = fill(REC, n, 5)
    src = oracle_view(REC, {"kind": "soa_mb"}, cols)
    split = {"kind": "split", "fields": [1, 4], "inner": {"kind": "null"}, "rest": {"kind": "aos"}}
    dst = oracle.OracleView(REC, split, n)
    src.copy_to(dst)
    rest = [0, 2, 3, 5]
    only_rest = oracle_view(sub_record(rest), {"kind": "aos"}, [cols[f] for f in rest])
    assert dst.blob_sizes == only_rest.blob_sizes  # the null part has no blob
    assert np.array_equal(dst.blobs[0], only_rest.blobs[0])
    for f in range(len(REC)):
        vals = dst.field_values(f)
        if f in (1, 4):
            assert not vals.any()
        else:
            assert np.array_equal(vals, src.field_values(f))


def test_nested_split_and_wrapped_parts():
    n = 40
    cols = fill(REC, n, 8)
    inner = {"kind": "split", "fields": [0], "inner": {"kind": "soa_mb"},
             "rest": {"kind": "changetype", "ct": [("f64", "f32")], "inner": {"kind": "aos"}}}
    nested = {"kind": "split", "fields": [0, 1, 2], "inner": inner,
              "rest": {"kind": "bytesplit", "inner": {"kind": "soa_mb"}}}
    v = oracle_view(REC, nested, cols)
    # leaf 1 (f64) went through ChangeType f64 -> f32 inside the nested split
    want_b = np.array(cols[1], dtype=np.float64).astype(np.float32).astype(np.float64).view(np.uint64)
    assert np.array_equal(v.field_values(1), want_b)
    for f in (0, 2, 3, 4, 5):
        assert np.array_equal(v.field_values(f), oracle_view(REC, {"kind": "soa_mb"}, cols).field_values(f))


@pytest.mark.parametrize("bad", [
    {"kind": "split", "fields": [], "inner": {"kind": "aos"}, "rest": {"kind": "aos"}},
    {"kind": "split", "fields": list(range(6)), "inner": {"kind": "aos"}, "rest": {"kind": "aos"}},
    {"kind": "split", "fields": [7], "inner": {"kind": "aos"}, "rest": {"kind": "aos"}},
])
def test_split_needs_leaves_on_both_sides(bad):
    with pytest.raises(ValueError):
        oracle.OracleView(REC, bad, 4)


def test_particle_cache_view_holds_position_and_mass_records():
    # A subset-field cache view (Sec. 3, Null with Split): pos and mass as
    # AoS records, velocities dropped.  Its blob is the array of {x, y, z, m}
    # records the n-body consumer stages per tile.
    n = 130
    cols = synth.particles(n, 4)
    cache = {"kind": "split", "fields": [0, 1, 2, 6], "inner": {"kind": "aos"}, "rest": {"kind": "null"}}
    v = oracle_view(synth.PARTICLE, cache, cols)
    want = np.stack([cols[0], cols[1], cols[2], cols[6]], axis=1).astype(np.float32)
    assert v.blob_sizes == [16 * n]
    assert bytes(v.blobs[0]) == want.tobytes()
    for f in (3, 4, 5):
        assert not v.field_values(f).any()
