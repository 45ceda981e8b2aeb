"""Parity at the full benchmark sizes, in the launch shape the benchmark uses.

The oracle cannot copy 2^27 records in seconds, so it checks sampled windows:
records [a, a + w) with a and w multiples of 256 occupy, in every blob of
every mapping here, the byte range [size(a), size(a + w)) where size(m) is the
blob size of m records -- itself taken from the oracle.  Each window of the
source is handed to the oracle as a view of w records and its copy compared
with the same window of the GPU result, byte for byte.  Whole-size
properties are checked on the device: round trips return the source bits.

Sources are drawn by the seeded generators: leaf arrays with the benchmark's
value distributions, or raw random bytes for whole blobs (so padding and
NaN/INF codes occur too).
"""
import pytest
import torch

import oracle
from paper_2302_08251_gb300 import llgb, synth
from gpu_util import check_windows, empty_device_view, ensure_library, sync_and_check_status

pytestmark = pytest.mark.gpu

@pytest.fixture(scope="module", autouse=True)
def lib():
    return ensure_library()


def random_view(record, mapping, extents, seed, **kw):
    rec = llgb.Record(record)
    v = llgb.View(rec, mapping, extents, **kw)
    for k, b in enumerate(v.blobs):
        b.copy_(synth.device_random_bytes(b.numel(), seed * 100 + k))
    return v


def field_view(record, fields, n):
    """SoA multi-blob view whose blob k is leaf k's array."""
    rec = llgb.Record(record)
    return llgb.View(rec, {"kind": "soa_mb"}, (n,),
                     blobs=[f.contiguous().view(torch.uint8) for f in fields])


CFD_PAIRS = [({"kind": "aos"}, {"kind": "soa_mb"}),
             ({"kind": "soa_mb"}, {"kind": "aos"}),
             ({"kind": "soa_mb"}, {"kind": "aosoa", "lanes": 32}),
             ({"kind": "aosoa", "lanes": 32}, {"kind": "soa_mb"}),
             ({"kind": "aosoa", "lanes": 8}, {"kind": "aosoa", "lanes": 32})]


@pytest.mark.parametrize("maps", CFD_PAIRS, ids=["aos-soa", "soa-aos", "soa-aosoa32",
                                                 "aosoa32-soa", "aosoa8-aosoa32"])
def test_cfd_512_cubed_relayouts(maps):
    ext = (512, 512, 512)
    n = 512 ** 3
    kw = dict(index_type="u32", static=(False, True, True))
    src = random_view(synth.CFD, maps[0], ext, seed=31, **kw)
    dst = empty_device_view(synth.CFD, maps[1], n, extents=ext, **kw)
    llgb.llgb_copy(src, dst)
    back = empty_device_view(synth.CFD, maps[0], n, extents=ext, **kw)
    llgb.llgb_copy(dst, back)
    sync_and_check_status()
    for a, b in zip(src.blobs, back.blobs):
        assert torch.equal(a, b)
    check_windows(src, dst, synth.CFD, maps[0], maps[1], n, seed=1)
    del src, dst, back
    torch.cuda.empty_cache()


@pytest.mark.parametrize("b", [1, 3, 7, 12, 17, 31])
def test_int6_2_to_26_pack_and_unpack(b):
    n = 1 << 26
    fields = synth.device_fields("int6", n, seed=b, bits=b)
    src = field_view(synth.INT6, fields, n)
    packed_map = {"kind": "bitpack_int", "bits": b}
    packed = empty_device_view(synth.INT6, packed_map, n, index_type="u32")
    llgb.llgb_pack(src, packed)
    back = empty_device_view(synth.INT6, {"kind": "soa_mb"}, n)
    llgb.llgb_unpack(packed, back)
    sync_and_check_status()
    for f, blob in zip(fields, back.blobs):
        assert torch.equal(f.view(torch.uint8), blob)
    check_windows(src, packed, synth.INT6, {"kind": "soa_mb"}, packed_map, n, seed=b)
    rnd = random_view(synth.INT6, packed_map, (n,), seed=b)
    out = empty_device_view(synth.INT6, {"kind": "aos"}, n)
    llgb.llgb_unpack(rnd, out)
    sync_and_check_status()
    check_windows(rnd, out, synth.INT6, packed_map, {"kind": "aos"}, n, seed=b + 1)


@pytest.mark.parametrize("em", [(e, m) for e in (5, 8, 11) for m in (2, 10, 23, 52)],
                         ids=lambda x: f"E{x[0]}M{x[1]}")
def test_mixed_f_2_to_25_float_pack(em):
    n = 1 << 25
    fields = synth.device_fields("mixed_f", n, seed=em[0] * 64 + em[1])
    src = field_view(synth.MIXED_F, fields, n)
    m = {"kind": "bitpack_float", "exp": em[0], "man": em[1]}
    dst = empty_device_view(synth.MIXED_F, m, n)
    llgb.llgb_pack(src, dst)
    sync_and_check_status()
    check_windows(src, dst, synth.MIXED_F, {"kind": "soa_mb"}, m, n, seed=em[1])
    # unpacking the packed values gives the oracle's loads of them
    back = empty_device_view(synth.MIXED_F, {"kind": "soa_mb"}, n)
    llgb.llgb_unpack(dst, back)
    sync_and_check_status()
    check_windows(dst, back, synth.MIXED_F, m, {"kind": "soa_mb"}, n, seed=em[0] * 7)
    del back
    rnd = random_view(synth.MIXED_F, m, (n,), seed=em[0])
    out = empty_device_view(synth.MIXED_F, {"kind": "soa_mb"}, n)
    llgb.llgb_unpack(rnd, out)
    sync_and_check_status()
    check_windows(rnd, out, synth.MIXED_F, m, {"kind": "soa_mb"}, n, seed=em[0] + 1)


@pytest.mark.parametrize("dst_map", [
    {"kind": "bytesplit", "inner": {"kind": "soa_mb"}},
    {"kind": "changetype", "ct": [("f64", "f32")], "inner": {"kind": "soa_mb"}},
    {"kind": "changetype", "ct": [("f64", "f32")], "inner": {"kind": "aos"}},
], ids=["bytesplit", "changetype-soa", "changetype-aos"])
def test_mixed_f_2_to_25_bytesplit_and_changetype(dst_map):
    n = 1 << 25
    fields = synth.device_fields("mixed_f", n, seed=3)
    src = field_view(synth.MIXED_F, fields, n)
    dst = empty_device_view(synth.MIXED_F, dst_map, n)
    llgb.llgb_copy(src, dst)
    back = empty_device_view(synth.MIXED_F, {"kind": "soa_mb"}, n)
    llgb.llgb_copy(dst, back)
    sync_and_check_status()
    if dst_map["kind"] == "bytesplit":
        for f, blob in zip(fields, back.blobs):
            assert torch.equal(f.contiguous().view(torch.uint8), blob)
    else:
        for f, blob in zip(fields[:3], back.blobs[:3]):
            assert torch.equal(f.float().double().view(torch.uint8), blob)
    check_windows(src, dst, synth.MIXED_F, {"kind": "soa_mb"}, dst_map, n, seed=4)


def test_particle_65536_aos_to_soa_whole():
    n = 65536
    fields = synth.particles(n, seed=0)
    from helpers import oracle_view
    src_o = oracle_view(synth.PARTICLE, {"kind": "aos"}, fields)
    dst_o = oracle.OracleView(synth.PARTICLE, {"kind": "soa_mb"}, n)
    src_o.copy_to(dst_o)
    from gpu_util import assert_same_bytes, device_view_of
    src = device_view_of(src_o)
    dst = empty_device_view(synth.PARTICLE, {"kind": "soa_mb"}, n)
    llgb.llgb_copy(src, dst)
    sync_and_check_status()
    assert_same_bytes(dst, dst_o)
