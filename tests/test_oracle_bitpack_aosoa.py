"""Pins of the oracle's bit-packed mappings organised as AoSoA.

Sec. 3 stores bit-packed leaves as SoA and announces the organisation as a
point to generalise.  Read here as: one blob of blocks of L records, each block
holding leaf 0's L codes, then leaf 1's, and so on; a record is lane i % L of
block i / L; LSB-first 32-bit words as in the SoA streams.  Pinned against a
hand-worked stream, a numpy construction of the blocks, the byte AoSoA mapping
(full-width codes are the values' own bytes), the SoA streams (one block of
whole words is their concatenation) and the values the SoA organisation loads.
"""
import os

import numpy as np
import pytest

from paper_2302_08251_gb300 import synth
from helpers import bits_of, oracle_view

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden():
    spec = {}
    for line in open(os.path.join(GOLDEN, "bitpack_aosoa_hand.txt")):
        if line.startswith("#") or not line.strip():
            continue
        key, *vals = line.split()
        spec[key] = vals
    return spec


@pytest.mark.parametrize("lanes", [1, 2])
def test_hand_worked_blocks(lanes):
    g = golden()
    rec = [("a", "u8"), ("b", "u8")]
    cols = [np.array([int(x) for x in g["a"]], np.uint8), np.array([int(x) for x in g["b"]], np.uint8)]
    v = oracle_view(rec, {"kind": "bitpack_int", "bits": 0, "field_bits": [3, 5], "lanes": lanes}, cols)
    assert v.blob_sizes == [4]
    assert bytes(v.blobs[0]) == bytes(int(x, 16) for x in g[f"lanes{lanes}"])


def numpy_blocks(codes, widths, L):
    """The AoSoA bit blob built with numpy.packbits, block by block."""
    n = len(codes[0])
    nb = -(-n // L)
    bits = []
    for k in range(nb):
        for c, w in zip(codes, widths):
            lane_codes = np.zeros(L, np.uint64)
            part = c[k * L:(k + 1) * L]
            lane_codes[:len(part)] = part
            bits.append(((lane_codes[:, None] >> np.arange(w, dtype=np.uint64)) & np.uint64(1)).ravel())
    flat = np.concatenate(bits).astype(np.uint8)
    packed = np.packbits(flat, bitorder="little")
    out = np.zeros(4 * (-(-flat.size // 32)), np.uint8)
    out[:packed.size] = packed
    return out


@pytest.mark.parametrize("L", [1, 3, 8, 32, 64])
@pytest.mark.parametrize("widths", [[1, 3, 7, 12, 17, 31], [12] * 6, [32, 5, 9, 1, 30, 2]])
def test_blocks_equal_a_numpy_construction(L, widths):
    n = 100
    fields = [synth.int6(n, w, seed=w + 1)[k] for k, w in enumerate(widths)]
    v = oracle_view(synth.INT6, {"kind": "bitpack_int", "bits": 0, "field_bits": widths, "lanes": L}, fields)
    codes = [bits_of(c) & np.uint64((1 << w) - 1) for c, w in zip(fields, widths)]
    want = numpy_blocks(codes, widths, L)
    assert v.blob_sizes == [want.size]
    assert np.array_equal(v.blobs[0], want)


@pytest.mark.parametrize("L", [1, 3, 8, 32])
def test_full_width_integers_are_the_byte_aosoa(L):
    n = 77
    fields = synth.uniform_fields(synth.INT6, n, 3)
    bp = oracle_view(synth.INT6, {"kind": "bitpack_int", "bits": 32, "lanes": L}, fields)
    ref = oracle_view(synth.INT6, {"kind": "aosoa", "lanes": L}, fields)
    assert bytes(bp.blobs[0]) == bytes(ref.blobs[0])


@pytest.mark.parametrize("L", [1, 4, 32])
def test_full_width_floats_are_the_byte_aosoa(L):
    rec = [("x", "f64"), ("y", "f64"), ("z", "f64")]
    n = 45
    fields = synth.uniform_fields(rec, n, 9)
    bp = oracle_view(rec, {"kind": "bitpack_float", "exp": 11, "man": 52, "lanes": L}, fields)
    ref = oracle_view(rec, {"kind": "aosoa", "lanes": L}, fields)
    assert bytes(bp.blobs[0]) == bytes(ref.blobs[0])


@pytest.mark.parametrize("b", [1, 3, 7, 12, 17, 31])
def test_one_block_of_whole_words_is_the_soa_streams_back_to_back(b):
    n = 32  # 32 codes of any width fill whole words
    fields = synth.int6(n, b, seed=b)
    aosoa = oracle_view(synth.INT6, {"kind": "bitpack_int", "bits": b, "lanes": 32}, fields)
    soa = oracle_view(synth.INT6, {"kind": "bitpack_int", "bits": b}, fields)
    assert bytes(aosoa.blobs[0]) == b"".join(bytes(s) for s in soa.blobs)


@pytest.mark.parametrize("kind", ["int", "float"])
@pytest.mark.parametrize("L", [2, 32, 128])
def test_values_load_as_through_the_soa_organisation(kind, L):
    n = 300
    if kind == "int":
        rec = synth.INT6
        fields = synth.uniform_fields(rec, n, 4)  # out of range: wraps, sign-extends
        m = {"kind": "bitpack_int", "bits": 9}
    else:
        rec = synth.MIXED_F
        fields = synth.mixed_f(n, 4)
        fields[0] = synth.special_f64(n - 24, 4)
        m = {"kind": "bitpack_float", "exp": 5, "man": 10}
    soa = oracle_view(rec, m, fields)
    aosoa = oracle_view(rec, dict(m, lanes=L), fields)
    for f in range(len(rec)):
        assert np.array_equal(aosoa.field_values(f), soa.field_values(f)), f
