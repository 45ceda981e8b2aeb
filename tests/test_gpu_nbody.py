"""GPU n-body step (Sec. 5, Fig. 2) against the FP64 oracle.

Tolerance: for each of the 7 leaves, max |gpu - oracle| / max |oracle| <= 1e-5
(the FP32 kernel against FP64 arithmetic on the same FP32 inputs).  The
result bits must not depend on the mapping the particles are read through.
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
TOL = 1e-5
MAPS = [{"kind": "aos"}, {"kind": "soa_mb"}, {"kind": "soa_sb"}, {"kind": "aosoa", "lanes": 32},
        {"kind": "aosoa", "lanes": 8}, {"kind": "aos", "packed": 1}]


@pytest.fixture(scope="module", autouse=True)
def lib():
    return ensure_library()


def gpu_step(fields, mapping):
    ov = oracle_view(synth.PARTICLE, mapping, fields)
    dv = device_view_of(ov)
    llgb.llgb_nbody_step(dv, float(EPS), float(DT))
    sync_and_check_status()
    out = oracle.OracleView(synth.PARTICLE, mapping, len(fields[0]), blobs=dv.blob_bytes())
    cols = [out.field_values(f).astype(np.uint32).view(np.float32) for f in range(7)]
    return cols


def check_against_oracle(fields, cols, sample=None):
    ov = oracle_view(synth.PARTICLE, {"kind": "soa_mb"}, fields)
    n = len(fields[0])
    idx = np.arange(n) if sample is None else sample
    worst = 0.0
    ref_pos = np.zeros((len(idx), 3))
    ref_vel = np.zeros((len(idx), 3))
    # contiguous runs keep the oracle calls few
    runs = np.split(idx, np.flatnonzero(np.diff(idx) != 1) + 1)
    at = 0
    for r in runs:
        p, v = ov.nbody_step(float(EPS), float(DT), int(r[0]), int(r[-1]) + 1)
        ref_pos[at:at + len(r)] = p
        ref_vel[at:at + len(r)] = v
        at += len(r)
    ref = [ref_pos[:, 0], ref_pos[:, 1], ref_pos[:, 2], ref_vel[:, 0], ref_vel[:, 1],
           ref_vel[:, 2], fields[6][idx].astype(np.float64)]
    for f in range(7):
        got = cols[f][idx].astype(np.float64)
        scale = np.max(np.abs(ref[f]))
        diff = np.max(np.abs(got - ref[f]))
        err = diff / scale if scale > 0 else diff
        worst = max(worst, err)
        assert err <= TOL, (f, err)
    return worst


@pytest.mark.parametrize("n", [1, 2, 3, 64, 65, 1000, 4097])
def test_small_systems_match_the_fp64_oracle(n):
    fields = synth.particles(n, seed=n)
    cols = gpu_step(fields, {"kind": "aos"})
    check_against_oracle(fields, cols)
    assert np.array_equal(cols[6], fields[6])  # mass untouched


def test_full_size_sampled_particles():
    n = 65536
    fields = synth.particles(n, seed=2302)
    cols = gpu_step(fields, {"kind": "soa_mb"})
    g = synth.rng(5)
    starts = sorted(set(g.integers(0, n - 64, 6).tolist()))
    sample = np.unique(np.concatenate([np.arange(s, s + 64) for s in starts] +
                                      [np.arange(0, 32), np.arange(n - 32, n)]))
    check_against_oracle(fields, cols, sample)


def test_result_bits_do_not_depend_on_the_mapping():
    n = 3000
    fields = synth.particles(n, seed=77)
    ref = gpu_step(fields, MAPS[0])
    for m in MAPS[1:]:
        got = gpu_step(fields, m)
        for f in range(7):
            assert np.array_equal(got[f].view(np.uint32), ref[f].view(np.uint32)), (m, f)


def test_two_bodies_attract_and_single_body_drifts():
    f1 = [np.array([x], np.float32) for x in (0.5, 0.25, -0.5, 1.0, 2.0, -3.0, 0.7)]
    cols = gpu_step(f1, {"kind": "aos"})
    assert cols[3][0] == 1.0 and cols[4][0] == 2.0 and cols[5][0] == -3.0
    f2 = [np.array(x, np.float32) for x in ([-0.5, 0.5], [0, 0], [0, 0], [0, 0], [0, 0], [0, 0], [1, 1])]
    cols = gpu_step(f2, {"kind": "soa_mb"})
    assert cols[3][0] > 0 > cols[3][1]
    check_against_oracle(f2, cols)


def test_rejects_other_records_and_packed_views():
    rec = llgb.Record(synth.CFD)
    v = llgb.View(rec, {"kind": "aos"}, (10,))
    with pytest.raises(llgb.LlgbError):
        llgb.llgb_nbody_step(v, 0.01, 1e-4)
    rec = llgb.Record(synth.PARTICLE)
    v = llgb.View(rec, {"kind": "bytesplit", "inner": {"kind": "soa_mb"}}, (10,))
    with pytest.raises(llgb.LlgbError):
        llgb.llgb_nbody_step(v, 0.01, 1e-4)
    torch.cuda.synchronize()
