"""Pins of the oracle's BitpackIntSoA (arXiv 2302.08251, Sec. 3).

The paper fixes that integral leaves are stored with a user-chosen bit count,
packed on store and unpacked on load, organised as SoA.  The bit order and the
sign rule are readings (LSB-first stream, two's-complement low bits, sign
extension on load).  Pinned against numpy's own bit packing, plain integer
arithmetic on Python ints, the multi-blob SoA limit and a hand-worked stream.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2302_08251_gb300 import synth
from helpers import bits_of, oracle_view

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def numpy_stream(values_u64: np.ndarray, b: int, nbytes: int) -> bytes:
    """LSB-first bit stream built with numpy.packbits (independent of the oracle)."""
    bits = ((values_u64[:, None] >> np.arange(b, dtype=np.uint64)) & np.uint64(1))
    packed = np.packbits(bits.astype(np.uint8).ravel(), bitorder="little")
    out = np.zeros(nbytes, dtype=np.uint8)
    out[:packed.size] = packed
    return out.tobytes()


@pytest.mark.parametrize("b", [1, 3, 7, 12, 17, 31, 32])
@pytest.mark.parametrize("n", [1, 31, 32, 33, 200])
def test_stream_equals_numpy_packbits(b, n):
    fields = synth.int6(n, b, seed=100 + b)
    v = oracle_view(synth.INT6, {"kind": "bitpack_int", "bits": b}, fields)
    mask = np.uint64((1 << b) - 1)
    for f, col in enumerate(fields):
        nbytes = 4 * (-(-n * b // 32))
        assert v.blob_sizes[f] == nbytes
        assert bytes(v.blobs[f]) == numpy_stream(bits_of(col) & mask, b, nbytes)


@pytest.mark.parametrize("b", [1, 3, 7, 12, 17, 31, 32])
def test_round_trip_in_range(b):
    n = 257
    fields = synth.int6(n, b, seed=b)
    v = oracle_view(synth.INT6, {"kind": "bitpack_int", "bits": b}, fields)
    for f, col in enumerate(fields):
        assert np.array_equal(v.field_values(f), bits_of(col))


@pytest.mark.parametrize("t", ["u8", "u16", "u32", "u64", "i8", "i16", "i32", "i64"])
@pytest.mark.parametrize("b", [1, 2, 5, 8, 13, 33, 63, 64])
def test_out_of_range_values_wrap_modulo_2_to_the_b(t, b):
    size = oracle.TYPE_SIZE[t]
    if b > 8 * size:
        pytest.skip("b larger than the type")
    g = synth.rng(b * 31 + size)
    width = 8 * size
    raw = [int(x) for x in g.integers(0, 2**63, 64, dtype=np.uint64)]
    raw += [0, 1, (1 << width) - 1, 1 << (width - 1), (1 << (width - 1)) - 1]
    raw = [x % (1 << width) for x in raw]
    rec = [("v", t)]
    v = oracle.OracleView(rec, {"kind": "bitpack_int", "bits": b}, len(raw))
    for i, x in enumerate(raw):
        v.store(i, 0, x)
    for i, x in enumerate(raw):
        low = x % (1 << b)
        if t.startswith("i"):
            value = low - (1 << b) if low >= (1 << (b - 1)) else low
            expect = value % (1 << width)   # two's complement in the type
        else:
            expect = low
        assert v.load(i, 0) == expect


def test_signed_one_bit_holds_minus_one_and_zero():
    rec = [("s", "i8")]
    v = oracle.OracleView(rec, {"kind": "bitpack_int", "bits": 1}, 4)
    for i, x in enumerate([0, 0xFF, 2, 3]):  # 0, -1, 2 -> 0, 3 -> -1
        v.store(i, 0, x)
    assert [v.load(i, 0) for i in range(4)] == [0, 0xFF, 0, 0xFF]


@pytest.mark.parametrize("name,rec", [("int6", synth.INT6),
                                      ("mixed", [("a", "u8"), ("b", "i16"),
                                                 ("c", "u64"), ("d", "i32")])])
def test_full_width_equals_soa_multi_blob(name, rec):
    n = 77
    fields = synth.uniform_fields(rec, n, 5)
    bits = [8 * oracle.TYPE_SIZE[t] for _, t in rec]
    bp = oracle_view(rec, {"kind": "bitpack_int", "bits": 0, "field_bits": bits}, fields)
    mb = oracle_view(rec, {"kind": "soa_mb"}, fields)
    for k in range(len(rec)):
        nb = len(mb.blobs[k])
        assert bytes(bp.blobs[k][:nb]) == bytes(mb.blobs[k])
        assert not bp.blobs[k][nb:].any()


@pytest.mark.parametrize("b", [1, 3, 7, 12, 17, 31])
def test_thirty_two_values_fill_exactly_b_words(b):
    v = oracle.OracleView(synth.INT6, {"kind": "bitpack_int", "bits": b}, 32)
    assert v.blob_sizes == [4 * b] * 6


def test_per_field_bit_counts():
    rec = synth.INT6
    n = 50
    widths = [1, 3, 7, 12, 17, 31]
    fields = [synth.int6(n, w, seed=w)[k] for k, w in enumerate(widths)]
    v = oracle_view(rec, {"kind": "bitpack_int", "bits": 0, "field_bits": widths}, fields)
    for k, (w, col) in enumerate(zip(widths, fields)):
        nbytes = 4 * (-(-n * w // 32))
        assert v.blob_sizes[k] == nbytes
        assert bytes(v.blobs[k]) == numpy_stream(bits_of(col) & np.uint64((1 << w) - 1),
                                                 w, nbytes)


def test_hand_worked_stream():
    spec = {}
    for line in open(os.path.join(GOLDEN, "bitpack_int_hand.txt")):
        if line.startswith("#") or not line.strip():
            continue
        key, *vals = line.split()
        spec[key] = vals
    b = int(spec["bits"][0])
    values = [int(x) for x in spec["values"]]
    expect = bytes(int(x, 16) for x in spec["bytes"])
    v = oracle.OracleView([("v", "u32")], {"kind": "bitpack_int", "bits": b}, len(values))
    for i, x in enumerate(values):
        v.store(i, 0, x)
    assert bytes(v.blobs[0]) == expect


def test_rejects_non_integral_and_oversized():
    with pytest.raises(ValueError):
        oracle.OracleView([("x", "f32")], {"kind": "bitpack_int", "bits": 8}, 4)
    with pytest.raises(ValueError):
        oracle.OracleView([("x", "u16")], {"kind": "bitpack_int", "bits": 17}, 4)
    with pytest.raises(ValueError):
        oracle.OracleView([("x", "u16")], {"kind": "bitpack_int", "bits": 0}, 4)
