"""Pins of the oracle's affine mappings (AoS, SoA single/multi blob, AoSoA).

The paper names these layouts (Sec. 5, Fig. 3 text: AoS, SoA multi-blob,
AoSoA) without formulas, so the oracle is pinned against things defined
outside it: numpy structured arrays (C struct layout), plain numpy reshapes and
transposes, equivalences between mappings that the oracle computes along
different code paths, and brute-force ownership of every byte.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2302_08251_gb300 import synth
from helpers import AFFINE, bits_of, oracle_view

# a record with padding inside it (u8 then f64) as well as at its end
PADDED = [("a", "u8"), ("b", "f64"), ("c", "i16"), ("d", "f32"), ("e", "u8")]
RECORDS = {"particle": synth.PARTICLE, "int6": synth.INT6,
           "mixed_f": synth.MIXED_F, "cfd": synth.CFD, "padded": PADDED}


def numpy_dtype(record, align):
    return np.dtype({"names": [f"f{k}" for k in range(len(record))],
                     "formats": [synth.NP_DTYPE[t] for _, t in record]},
                    align=align)


@pytest.mark.parametrize("name", RECORDS)
@pytest.mark.parametrize("packed", [0, 1])
def test_record_size_and_offsets_follow_c_struct_rules(name, packed):
    rec = RECORDS[name]
    dt = numpy_dtype(rec, align=not packed)
    v = oracle.OracleView(rec, {"kind": "aos", "packed": packed}, 1)
    assert v.blob_sizes == [dt.itemsize]
    for f, (_, t) in enumerate(rec):
        v.blobs[0][:] = 0
        v.store(0, f, (1 << (8 * oracle.TYPE_SIZE[t])) - 1)
        owned = np.flatnonzero(v.blobs[0])
        off = dt.fields[f"f{f}"][1]
        assert owned.tolist() == list(range(off, off + oracle.TYPE_SIZE[t]))


def test_config_record_sizes():
    sizes = {k: (oracle.OracleView(r, {"kind": "aos"}, 1).blob_sizes[0],
                 oracle.OracleView(r, {"kind": "aos", "packed": 1}, 1).blob_sizes[0])
             for k, r in RECORDS.items()}
    assert sizes == {"particle": (28, 28), "int6": (24, 24),
                     "mixed_f": (32, 28), "cfd": (24, 24), "padded": (32, 16)}


def _fields(rec, n, seed):
    return synth.uniform_fields(rec, n, seed)


@pytest.mark.parametrize("name", RECORDS)
@pytest.mark.parametrize("packed", [0, 1])
@pytest.mark.parametrize("n", [1, 37, 256])
def test_aos_equals_numpy_structured_array(name, packed, n):
    rec = RECORDS[name]
    fields = _fields(rec, n, 11 + n)
    arr = np.zeros(n, dtype=numpy_dtype(rec, align=not packed))
    for f, col in enumerate(fields):
        arr[f"f{f}"] = col
    v = oracle_view(rec, {"kind": "aos", "packed": packed}, fields)
    assert bytes(v.blobs[0]) == arr.tobytes()


@pytest.mark.parametrize("name", RECORDS)
def test_soa_multi_blob_is_one_plain_array_per_leaf(name):
    rec = RECORDS[name]
    fields = _fields(rec, 45, 3)
    v = oracle_view(rec, {"kind": "soa_mb"}, fields)
    assert [bytes(b) for b in v.blobs] == [c.tobytes() for c in fields]


def test_particle_aos_is_the_transpose_of_soa():
    n = 300
    fields = synth.particles(n, 5)
    src = oracle_view(synth.PARTICLE, {"kind": "soa_mb"}, fields)
    dst = oracle.OracleView(synth.PARTICLE, {"kind": "aos"}, n)
    src.copy_to(dst)
    expect = np.stack(fields, axis=1)  # (n, 7)
    assert np.array_equal(dst.blobs[0].view(np.float32).reshape(n, 7), expect)


@pytest.mark.parametrize("lanes", [1, 2, 8, 32, 5])
@pytest.mark.parametrize("n", [1, 31, 64, 100])
def test_particle_aosoa_is_a_blocked_transpose(lanes, n):
    fields = synth.particles(n, 9)
    v = oracle_view(synth.PARTICLE, {"kind": "aosoa", "lanes": lanes}, fields)
    blocks = -(-n // lanes)
    a = np.zeros((blocks * lanes, 7), dtype=np.float32)
    a[:n] = np.stack(fields, axis=1)
    expect = a.reshape(blocks, lanes, 7).transpose(0, 2, 1)
    assert bytes(v.blobs[0]) == np.ascontiguousarray(expect).tobytes()


@pytest.mark.parametrize("name", RECORDS)
@pytest.mark.parametrize("n", [1, 7, 33])
def test_aosoa_limits_are_aos_packed_and_soa_single_blob(name, n):
    rec = RECORDS[name]
    fields = _fields(rec, n, 21)
    aos = oracle_view(rec, {"kind": "aos", "packed": 1}, fields)
    aosoa1 = oracle_view(rec, {"kind": "aosoa", "lanes": 1}, fields)
    assert bytes(aosoa1.blobs[0]) == bytes(aos.blobs[0])
    soa = oracle_view(rec, {"kind": "soa_sb", "subarray_align": 1}, fields)
    aosoan = oracle_view(rec, {"kind": "aosoa", "lanes": n}, fields)
    assert bytes(aosoan.blobs[0]) == bytes(soa.blobs[0])


@pytest.mark.parametrize("name", RECORDS)
def test_soa_single_blob_is_the_multi_blob_arrays_back_to_back(name):
    rec = RECORDS[name]
    n = 64  # every sub-array then ends on an 8-byte boundary
    fields = _fields(rec, n, 4)
    sb = oracle_view(rec, {"kind": "soa_sb"}, fields)
    mb = oracle_view(rec, {"kind": "soa_mb"}, fields)
    assert bytes(sb.blobs[0]) == b"".join(bytes(b) for b in mb.blobs)


def _ownership(view):
    """Brute force: which bytes does each (record, leaf) own?"""
    own = {}
    for i in range(view.n):
        for f, t in enumerate(view.types):
            for b in view.blobs:
                b[:] = 0
            view.store(i, f, (1 << (8 * oracle.TYPE_SIZE[t])) - 1)
            hits = [(k, int(x)) for k, b in enumerate(view.blobs)
                    for x in np.flatnonzero(b)]
            own[(i, f)] = hits
    return own


@pytest.mark.parametrize("mapping", AFFINE, ids=lambda m: str(m))
@pytest.mark.parametrize("name", ["mixed_f", "cfd", "padded"])
@pytest.mark.parametrize("n", [1, 2, 5, 9])
def test_every_byte_has_at_most_one_owner(mapping, name, n):
    rec = RECORDS[name]
    v = oracle.OracleView(rec, mapping, n)
    own = _ownership(v)
    seen = set()
    for (i, f), hits in own.items():
        size = oracle.TYPE_SIZE[rec[f][1]]
        assert len(hits) == size
        blob = hits[0][0]
        offs = [x for _, x in hits]
        assert all(k == blob for k, _ in hits)
        assert offs == list(range(offs[0], offs[0] + size))  # contiguous
        assert offs[0] % size == 0 or mapping.get("packed") or \
            mapping["kind"] == "aosoa" or mapping.get("subarray_align") == 1
        for h in hits:
            assert h not in seen
            seen.add(h)
    owned = len(seen)
    total = sum(v.blob_sizes)
    assert owned == n * sum(oracle.TYPE_SIZE[t] for _, t in rec)
    assert owned <= total


@pytest.mark.parametrize("name", ["mixed_f", "cfd"])
@pytest.mark.parametrize("n", [3, 10])
def test_soa_single_blob_subarrays_are_ordered_aligned_and_tight(name, n):
    rec = RECORDS[name]
    v = oracle.OracleView(rec, {"kind": "soa_sb"}, n)
    own = _ownership(v)
    end_prev = 0
    for f, (_, t) in enumerate(rec):
        s = oracle.TYPE_SIZE[t]
        starts = [own[(i, f)][0][1] for i in range(n)]
        assert starts == [starts[0] + i * s for i in range(n)]
        assert starts[0] % s == 0
        assert end_prev <= starts[0] < end_prev + s
        end_prev = starts[-1] + s
    assert end_prev == v.blob_sizes[0]


@pytest.mark.parametrize("name", ["mixed_f", "cfd", "padded"])
@pytest.mark.parametrize("lanes", [2, 3, 8])
def test_aosoa_lanes_are_contiguous_and_blocks_follow_each_other(name, lanes):
    rec = RECORDS[name]
    n = 2 * lanes + 1
    v = oracle.OracleView(rec, {"kind": "aosoa", "lanes": lanes}, n)
    own = _ownership(v)
    packed = sum(oracle.TYPE_SIZE[t] for _, t in rec)
    for f, (_, t) in enumerate(rec):
        s = oracle.TYPE_SIZE[t]
        for i in range(1, n):
            d = own[(i, f)][0][1] - own[(i - 1, f)][0][1]
            assert d == (s if i % lanes else lanes * packed - (lanes - 1) * s)
    assert v.blob_sizes[0] == 3 * lanes * packed  # tail block is whole


PAIRS = list(itertools.product(range(len(AFFINE)), repeat=2))


@pytest.mark.parametrize("pair", PAIRS, ids=lambda p: f"{p[0]}->{p[1]}")
@pytest.mark.parametrize("name", ["cfd", "padded"])
def test_round_trip_between_affine_mappings(pair, name):
    a, b = AFFINE[pair[0]], AFFINE[pair[1]]
    rec = RECORDS[name]
    n = 41
    fields = _fields(rec, n, 77)
    va = oracle_view(rec, a, fields)
    vb = oracle.OracleView(rec, b, n)
    va.copy_to(vb)
    for f, col in enumerate(fields):
        assert np.array_equal(vb.field_values(f), bits_of(col))
    back = oracle.OracleView(rec, a, n)
    vb.copy_to(back)
    assert [bytes(x) for x in back.blobs] == [bytes(x) for x in va.blobs]


def test_copy_zeroes_bytes_no_leaf_owns():
    rec = synth.MIXED_F
    n = 19
    fields = _fields(rec, n, 8)
    src = oracle_view(rec, {"kind": "soa_mb"}, fields)
    dst = oracle.OracleView(rec, {"kind": "aos"}, n)
    dst.blobs[0][:] = 0xAB
    src.copy_to(dst)
    pad = dst.blobs[0].reshape(n, 32)[:, 28:]
    assert not pad.any()
    dst2 = oracle.OracleView(rec, {"kind": "aosoa", "lanes": 8}, n)
    dst2.blobs[0][:] = 0xCD
    src.copy_to(dst2)
    tail = dst2.blobs[0].reshape(3, 8 * 28)  # third block holds 3 records
    for f, (_, t) in enumerate(rec):
        s = oracle.TYPE_SIZE[t]
        lane_base = 8 * sum(oracle.TYPE_SIZE[u] for _, u in rec[:f])
        assert not tail[2, lane_base + 3 * s: lane_base + 8 * s].any()
