"""Pins of the oracle's Bytesplit and ChangeType (arXiv 2302.08251, Sec. 3).

Bytesplit splits every leaf into its bytes and forwards the byte record to an
inner mapping (Parquet's BYTE_STREAM_SPLIT when the inner mapping is SoA);
ChangeType stores a leaf as another type and forwards to an inner mapping.
Pinned against numpy byte views and numpy/torch casts.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2302_08251_gb300 import synth
from helpers import AFFINE, bits_of, oracle_view


@pytest.mark.parametrize("rec_name,rec", [("mixed_f", synth.MIXED_F),
                                          ("cfd", synth.CFD),
                                          ("particle", synth.PARTICLE)])
def test_bytesplit_soa_is_parquet_byte_stream_split(rec_name, rec):
    n = 53
    fields = synth.uniform_fields(rec, n, 31)
    v = oracle_view(rec, {"kind": "bytesplit", "inner": {"kind": "soa_mb"}}, fields)
    expect = []
    for col in fields:
        s = col.dtype.itemsize
        planes = col.view(np.uint8).reshape(n, s).T  # byte j of every value
        expect += [planes[j].tobytes() for j in range(s)]
    assert [bytes(b) for b in v.blobs] == expect


@pytest.mark.parametrize("rec", [synth.MIXED_F, synth.CFD])
def test_bytesplit_over_packed_aos_is_packed_aos(rec):
    n = 29
    fields = synth.uniform_fields(rec, n, 2)
    a = oracle_view(rec, {"kind": "aos", "packed": 1}, fields)
    b = oracle_view(rec, {"kind": "bytesplit",
                          "inner": {"kind": "aos", "packed": 1}}, fields)
    assert bytes(a.blobs[0]) == bytes(b.blobs[0])


@pytest.mark.parametrize("inner", AFFINE, ids=str)
def test_bytesplit_round_trip_over_any_inner_mapping(inner):
    rec = synth.MIXED_F
    n = 40
    fields = synth.mixed_f(n, seed=9)
    v = oracle_view(rec, {"kind": "bytesplit", "inner": inner}, fields)
    for f, col in enumerate(fields):
        assert np.array_equal(v.field_values(f), bits_of(col))


def test_changetype_f64_to_f32_matches_numpy_cast():
    n = 5000
    fields = synth.mixed_f(n, seed=3)
    fields[0] = synth.special_f64(n - 24, seed=1)[:n]
    m = {"kind": "changetype", "ct": [("f64", "f32")], "inner": {"kind": "soa_mb"}}
    v = oracle_view(synth.MIXED_F, m, fields)
    assert v.blob_sizes == [4 * n] * 4
    for f in range(3):
        with np.errstate(over="ignore", invalid="ignore"):
            want = fields[f].astype(np.float32)
        got = v.blobs[f].view(np.float32)
        ok = ~np.isnan(fields[f])
        assert np.array_equal(got.view(np.uint32)[ok], want.view(np.uint32)[ok])
        assert np.isnan(got[~ok]).all()
        # loading widens exactly
        back = v.field_values(f).view(np.float64)
        assert np.array_equal(back[ok], want[ok].astype(np.float64))
    assert bytes(v.blobs[3]) == fields[3].tobytes()  # w is f32 already


def test_changetype_f32_to_f16_and_bf16_match_numpy_and_torch():
    n = 4096
    x = synth.special_f32(n - 22, seed=5)[:n]
    rec = [("a", "f32")]
    h = oracle_view(rec, {"kind": "changetype", "ct": [("f32", "f16")],
                          "inner": {"kind": "soa_mb"}}, [x])
    with np.errstate(over="ignore", invalid="ignore"):
        want = x.astype(np.float16).view(np.uint16)
    ok = ~np.isnan(x)
    assert np.array_equal(h.blobs[0].view(np.uint16)[ok], want[ok])
    b = oracle_view(rec, {"kind": "changetype", "ct": [("f32", "bf16")],
                          "inner": {"kind": "soa_mb"}}, [x])
    want_b = torch.from_numpy(x.copy()).to(torch.bfloat16).view(torch.int16).numpy()
    assert np.array_equal(b.blobs[0].view(np.uint16)[ok], want_b.view(np.uint16)[ok])


@pytest.mark.parametrize("inner", [{"kind": "aos", "packed": 0}, {"kind": "aos", "packed": 1},
                                   {"kind": "aosoa", "lanes": 8}], ids=str)
def test_changetype_over_aos_shrinks_the_record(inner):
    n = 33
    fields = synth.mixed_f(n, seed=4)
    m = {"kind": "changetype", "ct": [("f64", "f32")], "inner": inner}
    v = oracle_view(synth.MIXED_F, m, fields)
    lanes = inner.get("lanes", 1)
    assert v.blob_sizes == [16 * (-(-n // lanes)) * lanes]
    with np.errstate(over="ignore"):
        for f in range(3):
            want = fields[f].astype(np.float32).astype(np.float64)
            assert np.array_equal(v.field_values(f).view(np.float64), want)


def test_changetype_rejects_integer_pairs():
    with pytest.raises(ValueError):
        oracle.OracleView([("a", "i32")], {"kind": "changetype", "ct": [("i32", "i16")],
                                           "inner": {"kind": "soa_mb"}}, 4)
