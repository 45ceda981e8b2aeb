"""GPU parity on a seeded random sweep of mapping pairs: random records of
integer and float leaves, random source and destination mappings (AoS aligned
or packed, SoA single- and multi-blob, AoSoA, BitpackInt/Float in both
organisations with per-field widths or random (E, M), Bytesplit, ChangeType,
Split with Null, nested), random record counts around tile and lane
boundaries.  The source is filled by the oracle from random values (special
floats included), copied by the library on the GPU into a destination
pre-filled with 0xAB, and compared with the oracle's copy byte for byte.
Pairs the library declines (LLGB_ERR_UNSUPPORTED when a view is created or a
copy planned) are skipped and counted; the sweep must copy most pairs.
Bar: bit-exact."""
import random

import numpy as np
import pytest

import oracle
from paper_2302_08251_gb300 import llgb
from helpers import oracle_view
from gpu_util import assert_same_bytes, device_view_of, empty_device_view, ensure_library, sync_and_check_status
from test_plan_sweep import leaf_mapping, random_record

pytestmark = pytest.mark.gpu

NP = {"u8": np.uint8, "u16": np.uint16, "u32": np.uint32, "u64": np.uint64,
      "i8": np.int8, "i16": np.int16, "i32": np.int32, "i64": np.int64,
      "f32": np.float32, "f64": np.float64}


@pytest.fixture(scope="module", autouse=True)
def lib():
    return ensure_library()


def random_field(t, n, g):
    """n values of type t: random bit patterns for integers; for floats a mix
    of normal values over a wide exponent range, zeros, INF, NaN and
    subnormals."""
    if t.startswith(("u", "i")):
        raw = g.integers(0, 256, n * np.dtype(NP[t]).itemsize, dtype=np.uint8)
        return raw.view(NP[t]).copy()
    ft = NP[t]
    x = (g.standard_normal(n) * np.exp2(g.integers(-40, 40, n))).astype(ft)
    specials = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, np.finfo(ft).tiny / 4, -np.finfo(ft).tiny,
                         np.finfo(ft).max, 1.0, -1.5], dtype=ft)
    pick = g.random(n) < 0.05
    x[pick] = specials[g.integers(0, specials.size, int(pick.sum()))]
    return x


@pytest.mark.parametrize("seed", range(8))
def test_random_mapping_pairs_copy_like_the_oracle(seed):
    g = random.Random(1000 + seed)
    vals = np.random.default_rng(2000 + seed)
    copied = declined = 0
    for _ in range(16):
        leaves = random_record(g)
        types = [t for _, t in leaves]
        n = g.choice([1, 127, 129, 1000, 4097, 20000 + 3])
        src_map, dst_map = (leaf_mapping(g, types, 0) for _ in range(2))
        fields = [random_field(t, n, vals) for t in types]
        try:
            src_o = oracle_view(leaves, src_map, fields)
            dst_o = oracle.OracleView(leaves, dst_map, n)
        except ValueError:
            declined += 1  # a mapping the oracle does not take for these leaves
            continue
        try:
            src_g = device_view_of(src_o)
            dst_g = empty_device_view(leaves, dst_map, n)
            llgb.llgb_copy(src_g, dst_g)
        except llgb.LlgbError as err:
            assert err.status == llgb.ERR_UNSUPPORTED, (src_map, dst_map, err)
            declined += 1
            continue
        src_o.copy_to(dst_o)
        sync_and_check_status()
        assert_same_bytes(dst_g, dst_o, f"{leaves} n={n}: {src_map} -> {dst_map}")
        copied += 1
    assert copied >= 10, (copied, declined)
