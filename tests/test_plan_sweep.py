"""Seeded random sweep of the host planner (no GPU): for random records,
mapping pairs (plain, bit-packed in both organisations, Bytesplit,
ChangeType, Split with Null, nested) and record counts, the planner's blob
sizes equal the oracle's and the copy plan is well formed -- the tiles cover
the records in multiples of 128 and of every lane count, the kernel modes are
ones the library has, and generic items are a subset of the items."""
import ctypes
import random

import pytest

import oracle
from paper_2302_08251_gb300 import llgb

INTS = ["u8", "u16", "u32", "i8", "i16", "i32", "u64", "i64"]
FLOATS = ["f32", "f64"]


def random_record(g):
    return [(f"l{k}", g.choice(INTS + FLOATS)) for k in range(g.randint(2, 6))]


def leaf_mapping(g, types, depth):
    """A mapping that can hold leaves of `types` (possibly a Split)."""
    ints = all(t in INTS for t in types)
    floats = all(t in FLOATS for t in types)
    choices = ["aos", "aos_p", "soa_mb", "soa_sb", "aosoa", "bytesplit"]
    if ints:
        choices += ["bitpack_int", "bitpack_int_aosoa"]
    if floats:
        choices += ["bitpack_float", "bitpack_float_aosoa", "changetype"]
    if depth < 2 and len(types) >= 2:
        choices += ["split", "split"]
    k = g.choice(choices)
    if k == "aos":
        return {"kind": "aos"}
    if k == "aos_p":
        return {"kind": "aos", "packed": 1}
    if k == "soa_mb":
        return {"kind": "soa_mb"}
    if k == "soa_sb":
        return {"kind": "soa_sb"}
    if k == "aosoa":
        return {"kind": "aosoa", "lanes": g.choice([1, 4, 8, 32, 64])}
    if k == "bytesplit":
        return {"kind": "bytesplit", "inner": {"kind": g.choice(["soa_mb", "aos"])}}
    if k.startswith("bitpack_int"):
        widths = [g.randint(1, 8 * oracle.TYPE_SIZE[t]) for t in types]
        m = {"kind": "bitpack_int", "bits": 0, "field_bits": widths}
    elif k.startswith("bitpack_float"):
        m = {"kind": "bitpack_float", "exp": g.randint(2, 8), "man": g.randint(1, 23)}
    elif k == "changetype":
        return {"kind": "changetype", "ct": [("f64", "f32")], "inner": {"kind": g.choice(["soa_mb", "aos"])}}
    else:  # split
        sel = sorted(g.sample(range(len(types)), g.randint(1, len(types) - 1)))
        rest = [t for f, t in enumerate(types) if f not in sel]
        inner = {"kind": "null"} if g.random() < 0.2 else leaf_mapping(g, [types[f] for f in sel], depth + 1)
        return {"kind": "split", "fields": sel, "inner": inner, "rest": leaf_mapping(g, rest, depth + 1)}
    if k.endswith("aosoa"):
        m["lanes"] = g.choice([32, 64, 128, 256])
    return m


def lane_counts(m):
    out = []
    if m["kind"] == "aosoa":
        out.append(m["lanes"])
    if m["kind"].startswith("bitpack") and m.get("lanes"):
        out.append(m["lanes"])
    for key in ("inner", "rest"):
        if m.get(key):
            out += lane_counts(m[key])
    return out


def handle(rec, m, n):
    keep = []
    e = llgb.extents_desc((n,))
    d = llgb.mapping_desc(m, keep)
    h = ctypes.c_void_p()
    st = llgb.lib().llgb_view_create(rec.handle, ctypes.byref(e), ctypes.byref(d), ctypes.byref(h))
    return st, h


@pytest.mark.parametrize("seed", range(12))
def test_random_mapping_pairs_plan_like_the_oracle(seed):
    g = random.Random(seed)
    L = llgb.lib()
    planned = 0
    for _ in range(25):
        leaves = random_record(g)
        types = [t for _, t in leaves]
        rec = llgb.Record(leaves)
        n = g.choice([0, 1, 127, 128, 129, 1000, 4097, 65536 + 3])
        maps = [leaf_mapping(g, types, 0) for _ in range(2)]
        hs = []
        for m in maps:
            st, h = handle(rec, m, n)
            assert st in (llgb.OK, llgb.ERR_UNSUPPORTED), (m, st)
            if st != llgb.OK:
                break
            nb = L.llgb_view_blob_count(h)
            sizes = [int(L.llgb_view_blob_size(h, k)) for k in range(nb)]
            assert sizes == oracle.OracleView(leaves, m, n).blob_sizes, m
            hs.append(h)
        if len(hs) == 2:
            try:
                p = llgb.plan_info(hs[0], hs[1])
            except llgb.LlgbError as err:
                assert err.status == llgb.ERR_UNSUPPORTED, (maps, err)
            else:
                planned += 1
                if n == 0:
                    assert p["tiles"] == 0
                else:
                    q = 128
                    for lanes in lane_counts(maps[0]) + lane_counts(maps[1]):
                        assert p["tile_records"] % lanes == 0, (maps, p)
                    assert p["tile_records"] % q == 0 and p["tiles"] * p["tile_records"] >= n > (p["tiles"] - 1) * p["tile_records"]
                    assert p["kernel_mode"] in (0, 1, 2, 3, 4) and p["batch_kernel_mode"] in (0, 1, 2, 3, 4)
                    assert 0 <= p["generic_items"] <= p["items"]
        for h in hs:
            L.llgb_view_destroy(h)
    assert planned > 0
