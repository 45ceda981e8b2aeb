"""The n-body phases under both traversals (Sec. 5: a single loop over the
flat record index against loops nested the way the mapping lays records out)
against the FP64 oracle.

Bars: the two traversals give the same result bits; update followed by move
gives the bits of the full step; the move is within one f32 ulp of the
oracle's exact p + dt v (the kernel rounds it once, with a fused multiply-add;
the oracle's double may round once more) and changes no byte outside the pos
leaves; the update's velocities are within 1e-5 of the oracle's, relative to
the largest.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2302_08251_gb300 import llgb, synth
from helpers import oracle_view
from gpu_util import device_view_of, ensure_library, sync_and_check_status

pytestmark = pytest.mark.gpu

EPS, DT = np.float32(0.01), np.float32(1e-4)
MAPS = [{"kind": "aos"}, {"kind": "aos", "packed": 1}, {"kind": "soa_mb"}, {"kind": "soa_sb"},
        {"kind": "aosoa", "lanes": 4}, {"kind": "aosoa", "lanes": 8}, {"kind": "aosoa", "lanes": 32},
        {"kind": "aosoa", "lanes": 48}, {"kind": "aosoa", "lanes": 3}, {"kind": "aosoa", "lanes": 6},
        {"kind": "aosoa", "lanes": 64}, {"kind": "aosoa", "lanes": 1}]
IDS = [m["kind"] + str(m.get("lanes", "")) + ("p" if m.get("packed") else "") for m in MAPS]
SIZES = [1, 3, 31, 33, 1000, 4097]


@pytest.fixture(scope="module", autouse=True)
def lib():
    return ensure_library()


def leaves(dv, mapping, n):
    ov = oracle.OracleView(synth.PARTICLE, mapping, n, blobs=dv.blob_bytes())
    return [ov.field_values(f).astype(np.uint32).view(np.float32) for f in range(7)]


def pos_byte_mask(mapping, n):
    """Per blob, True at the bytes of the pos leaves."""
    ones = np.full(n, 0xFFFFFFFF, np.uint32).view(np.float32)
    cols = [ones if f < 3 else np.zeros(n, np.float32) for f in range(7)]
    return [b != 0 for b in oracle_view(synth.PARTICLE, mapping, cols).blobs]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("mapping", MAPS, ids=IDS)
def test_move_both_traversals_against_the_oracle(mapping, n):
    fields = synth.particles(n, seed=n + 5)
    ov = oracle_view(synth.PARTICLE, mapping, fields)
    ref = ov.nbody_move(float(DT))
    before = ov.blobs
    mask = pos_byte_mask(mapping, n)
    got = {}
    for trav in ("index", "blocks"):
        dv = device_view_of(ov)
        llgb.llgb_nbody_move(dv, float(DT), trav)
        sync_and_check_status()
        after = dv.blob_bytes()
        for b, a, m in zip(before, after, mask):
            assert np.array_equal(a[~m], b[~m]), trav  # vel, mass and padding untouched
        got[trav] = leaves(dv, mapping, n)
    for k in range(3):
        assert np.array_equal(got["index"][k].view(np.uint32), got["blocks"][k].view(np.uint32))
        g = got["blocks"][k]
        ulp = np.spacing(np.abs(g)).astype(np.float64)
        assert np.all(np.abs(g.astype(np.float64) - ref[:, k]) <= ulp), k


@pytest.mark.parametrize("n", [1, 65, 1000, 4097])
@pytest.mark.parametrize("mapping", MAPS, ids=IDS)
def test_update_both_traversals_against_the_oracle(mapping, n):
    fields = synth.particles(n, seed=n + 9)
    ov = oracle_view(synth.PARTICLE, mapping, fields)
    _, ref_vel = ov.nbody_step(float(EPS), float(DT))
    got = {}
    for trav in ("index", "blocks"):
        dv = device_view_of(ov)
        llgb.llgb_nbody_update(dv, float(EPS), float(DT), trav)
        sync_and_check_status()
        got[trav] = leaves(dv, mapping, n)
    for f in range(7):
        assert np.array_equal(got["index"][f].view(np.uint32), got["blocks"][f].view(np.uint32)), f
    for f in (0, 1, 2, 6):  # the update writes velocities only
        assert np.array_equal(got["blocks"][f], fields[f])
    for k in range(3):
        r = ref_vel[:, k]
        scale = np.max(np.abs(r))
        err = np.max(np.abs(got["blocks"][3 + k].astype(np.float64) - r)) / scale
        assert err <= 1e-5, (k, err)


@pytest.mark.parametrize("mapping", MAPS, ids=IDS)
def test_update_then_move_is_the_step(mapping):
    n = 2000 + 21
    fields = synth.particles(n, seed=41)
    ov = oracle_view(synth.PARTICLE, mapping, fields)
    step = device_view_of(ov)
    llgb.llgb_nbody_step(step, float(EPS), float(DT))
    for trav in ("index", "blocks"):
        phases = device_view_of(ov)
        llgb.llgb_nbody_update(phases, float(EPS), float(DT), trav)
        llgb.llgb_nbody_move(phases, float(DT), trav)
        sync_and_check_status()
        for a, b in zip(step.blob_bytes(), phases.blob_bytes()):
            assert np.array_equal(a, b), trav


def test_step_on_lane_counts_that_are_not_powers_of_two():
    n = 3001
    fields = synth.particles(n, seed=13)
    ref = None
    for mapping in ({"kind": "soa_mb"}, {"kind": "aosoa", "lanes": 48}, {"kind": "aosoa", "lanes": 3}):
        dv = device_view_of(oracle_view(synth.PARTICLE, mapping, fields))
        llgb.llgb_nbody_step(dv, float(EPS), float(DT))
        sync_and_check_status()
        cols = leaves(dv, mapping, n)
        if ref is None:
            ref = cols
        for f in range(7):
            assert np.array_equal(cols[f].view(np.uint32), ref[f].view(np.uint32)), (mapping, f)


def test_large_move_sampled():
    # 2^22 + 5 particles: many CTAs in both traversals, ragged last AoSoA block
    n = (1 << 22) + 5
    fields = synth.particles(n, seed=3)
    for mapping in ({"kind": "aosoa", "lanes": 32}, {"kind": "soa_mb"}, {"kind": "aosoa", "lanes": 48}):
        ov = oracle_view(synth.PARTICLE, mapping, fields)
        g = synth.rng(8)
        idx = np.unique(np.concatenate([g.integers(0, n, 2000), np.arange(n - 40, n)]))
        res = {}
        for trav in ("index", "blocks"):
            dv = device_view_of(ov)
            llgb.llgb_nbody_move(dv, float(DT), trav)
            sync_and_check_status()
            res[trav] = leaves(dv, mapping, n)
        for k in range(3):
            assert np.array_equal(res["index"][k].view(np.uint32), res["blocks"][k].view(np.uint32))
        want = ov.nbody_move(float(DT))
        for k in range(3):
            g32 = res["blocks"][k][idx]
            assert np.all(np.abs(g32.astype(np.float64) - want[idx, k]) <= np.spacing(np.abs(g32)))
        del ov
        torch.cuda.empty_cache()


def test_unknown_traversal_is_rejected():
    dv = device_view_of(oracle_view(synth.PARTICLE, {"kind": "aos"}, synth.particles(10, 1)))
    for call in (lambda: llgb.check(llgb.lib().llgb_nbody_move(dv.handle, 0.1, 2, None)),
                 lambda: llgb.check(llgb.lib().llgb_nbody_update(dv.handle, 0.1, 0.1, -1, None))):
        with pytest.raises(llgb.LlgbError) as err:
            call()
        assert err.value.status == llgb.ERR_INVALID_ARG
    sync_and_check_status()
