"""GPU parity across launch shapes and staging schemes.

The autotuner may run any pair under another tile, thread count, CTAs per SM,
stage counts, engine or staging scheme (TMA, plain stores, plain loads, plain
both), so every such shape must store the oracle's bytes.  Fixed pairs cover
the kernel modes: gather re-layouts, value loops, integer and float bit
streams in both directions, Bytesplit, ChangeType and Split.  Each runs under
every staging scheme and engine on a many-tile shape.  Then seeded random
pairs run under random launch shapes.  Shapes the library declines are
skipped and counted: LLGB_ERR_INVALID_ARG when the stages do not fit in
shared memory or the tile is not a multiple of a lane count, and
LLGB_ERR_UNSUPPORTED.  Destinations are pre-filled with 0xAB.
Bar: bit-exact against the oracle."""
import random

import numpy as np
import pytest

import oracle
from paper_2302_08251_gb300 import llgb, synth
from helpers import oracle_view
from gpu_util import assert_same_bytes, device_view_of, empty_device_view, ensure_library, sync_and_check_status
from test_gpu_random_pairs import random_field
from test_plan_sweep import leaf_mapping, random_record

pytestmark = pytest.mark.gpu

SOA = {"kind": "soa_mb"}
PAIRS = [
    ("cfd", {"kind": "aos"}, SOA),
    ("cfd", SOA, {"kind": "aos"}),
    ("cfd", SOA, {"kind": "aosoa", "lanes": 32}),
    ("int6_12", SOA, {"kind": "bitpack_int", "bits": 12}),
    ("int6_12", {"kind": "bitpack_int", "bits": 12}, SOA),
    ("int6_3", SOA, {"kind": "bitpack_int", "bits": 3}),
    ("int6_3", {"kind": "bitpack_int", "bits": 3}, {"kind": "aos"}),
    ("mixed_f", SOA, {"kind": "bitpack_float", "exp": 8, "man": 10}),
    ("mixed_f", {"kind": "bitpack_float", "exp": 8, "man": 10}, SOA),
    ("mixed_f", SOA, {"kind": "bytesplit", "inner": SOA}),
    ("mixed_f", {"kind": "aos"}, {"kind": "changetype", "ct": [("f64", "f32")], "inner": SOA}),
    ("particle", {"kind": "aos"},
     {"kind": "split", "fields": [0, 1, 2], "inner": SOA, "rest": {"kind": "aosoa", "lanes": 32}}),
]
# many tiles per CTA on few CTAs, so that the stages cycle several times
SHAPE = {"tile_records": 512, "src_stages": 3, "dst_stages": 2, "threads": 256, "ctas_per_sm": 2}


@pytest.fixture(scope="module", autouse=True)
def lib():
    return ensure_library()


def record_and_fields(kind, n, seed):
    if kind == "cfd":
        return synth.CFD, synth.cfd(n, seed)
    if kind == "int6_12":
        return synth.INT6, synth.int6(n, 12, seed)
    if kind == "int6_3":
        return synth.INT6, synth.int6(n, 3, seed)
    if kind == "mixed_f":
        return synth.MIXED_F, synth.mixed_f(n, seed)
    return synth.PARTICLE, synth.uniform_fields(synth.PARTICLE, n, seed)


def copy_with_shape(rec, fields, src_map, dst_map, cfg):
    """"ran" when the library ran the copy under cfg (and it matched the
    oracle), else what declined it: the oracle (a mapping it does not take for
    these leaves) or the library (a view, plan or shape it does not take)."""
    n = len(fields[0])
    try:
        src_o = oracle_view(rec, src_map, fields)
        dst_o = oracle.OracleView(rec, dst_map, n)
    except ValueError:
        return "oracle"
    try:
        src_g = device_view_of(src_o)
        dst_g = empty_device_view(rec, dst_map, n)
        llgb.llgb_copy_with(src_g, dst_g, cfg)
    except llgb.LlgbError as err:
        assert err.status in (llgb.ERR_INVALID_ARG, llgb.ERR_UNSUPPORTED), (src_map, dst_map, cfg, err)
        return "library"
    src_o.copy_to(dst_o)
    sync_and_check_status()
    assert_same_bytes(dst_g, dst_o, f"{src_map} -> {dst_map} under {cfg}")
    return "ran"


@pytest.mark.parametrize("engine", ["auto", "value", "gather"])
@pytest.mark.parametrize("staging", ["tma", "plain_store", "plain_load", "plain"])
@pytest.mark.parametrize("pair", range(len(PAIRS)))
def test_every_staging_scheme_and_engine_stores_the_oracle_bytes(pair, staging, engine):
    kind, sm, dm = PAIRS[pair]
    n = 40_000 + 77  # 79 tiles of 512 records and a ragged tail
    rec, fields = record_and_fields(kind, n, 60 + pair)
    assert copy_with_shape(rec, fields, sm, dm, dict(SHAPE, staging=staging, engine=engine)) == "ran"


def random_shape(g):
    return {"tile_records": 128 * g.choice([1, 2, 3, 4, 6, 8, 12, 16, 24, 32]),
            "src_stages": g.randint(1, 8), "dst_stages": g.randint(1, 4),
            "threads": g.choice([128, 256, 512]), "ctas_per_sm": g.randint(1, 3),
            "engine": g.choice(["auto", "value", "gather"]),
            "staging": g.choice(["tma", "plain_store", "plain_load", "plain"])}


@pytest.mark.parametrize("seed", range(6))
def test_random_pairs_under_random_launch_shapes(seed):
    g = random.Random(3000 + seed)
    vals = np.random.default_rng(4000 + seed)
    outcome = {"ran": 0, "oracle": 0, "library": 0}
    for _ in range(12):
        leaves = random_record(g)
        types = [t for _, t in leaves]
        n = g.choice([129, 1000, 4097, 20000 + 3])
        src_map, dst_map = (leaf_mapping(g, types, 0) for _ in range(2))
        fields = [random_field(t, n, vals) for t in types]
        outcome[copy_with_shape(leaves, fields, src_map, dst_map, random_shape(g))] += 1
    assert outcome["ran"] >= 5, outcome
