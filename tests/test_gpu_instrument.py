"""FieldAccessCount and Heatmap of the n-body consumer (Sec. 4) against the
oracle's counts of the same access schedule.  Bar: every counter exact; the
instrumented step's result bits equal the plain step's.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2302_08251_gb300 import llgb, synth
from helpers import oracle_view
from gpu_util import device_view_of, ensure_library, sync_and_check_status

pytestmark = pytest.mark.gpu

MAPS = [{"kind": "aos"}, {"kind": "soa_mb"}, {"kind": "soa_sb"}, {"kind": "aosoa", "lanes": 8},
        {"kind": "aosoa", "lanes": 32}, {"kind": "aosoa", "lanes": 64}, {"kind": "aosoa", "lanes": 48}]
EPS, DT = 0.01, 1e-4


@pytest.fixture(scope="module", autouse=True)
def lib():
    return ensure_library()


def particle_view(mapping, n, seed):
    return device_view_of(oracle_view(synth.PARTICLE, mapping, synth.particles(n, seed)))


@pytest.mark.parametrize("mapping", MAPS, ids=lambda m: m["kind"] + str(m.get("lanes", "")))
@pytest.mark.parametrize("n", [1, 63, 64, 65, 1000, 4097])
@pytest.mark.parametrize("mode", ["atomic", "block"])
def test_field_counts_are_exact(mapping, n, mode):
    v = particle_view(mapping, n, n)
    counts = torch.zeros(14, dtype=torch.int64, device="cuda")
    llgb.llgb_nbody_step_instrumented(v, EPS, DT, field_counts=counts, count_mode=mode)
    llgb.llgb_nbody_step_instrumented(v, EPS, DT, field_counts=counts, count_mode=mode)
    sync_and_check_status()
    want = 2 * oracle.nbody_access_counts(n).astype(np.int64)  # counters accumulate
    assert np.array_equal(counts.cpu().numpy(), want)


@pytest.mark.parametrize("mapping", MAPS, ids=lambda m: m["kind"] + str(m.get("lanes", "")))
@pytest.mark.parametrize("g", [1, 4, 64, 4096])
def test_heatmap_is_exact(mapping, g):
    n = 1000 + 37
    v = particle_view(mapping, n, 3)
    size = llgb.llgb_heatmap_counters(v, g)
    assert size == len(oracle.nbody_heatmap(mapping, n, g))
    heat = torch.zeros(size, dtype=torch.int64, device="cuda")
    counts = torch.zeros(14, dtype=torch.int64, device="cuda")
    llgb.llgb_nbody_step_instrumented(v, EPS, DT, field_counts=counts, count_mode="block", heat=heat,
                                      granularity=g)
    sync_and_check_status()
    assert np.array_equal(heat.cpu().numpy(), oracle.nbody_heatmap(mapping, n, g).astype(np.int64))
    assert np.array_equal(counts.cpu().numpy(), oracle.nbody_access_counts(n).astype(np.int64))


@pytest.mark.parametrize("mapping", MAPS[:2] + MAPS[4:5], ids=lambda m: m["kind"] + str(m.get("lanes", "")))
def test_instrumented_step_gives_the_plain_step_bits(mapping):
    n = 3001
    plain = particle_view(mapping, n, 9)
    counted = particle_view(mapping, n, 9)
    llgb.llgb_nbody_step(plain, EPS, DT)
    heat = torch.zeros(llgb.llgb_heatmap_counters(counted, 64), dtype=torch.int64, device="cuda")
    counts = torch.zeros(14, dtype=torch.int64, device="cuda")
    llgb.llgb_nbody_step_instrumented(counted, EPS, DT, field_counts=counts, count_mode="atomic", heat=heat,
                                      granularity=64)
    sync_and_check_status()
    for a, b in zip(plain.blob_bytes(), counted.blob_bytes()):
        assert np.array_equal(a, b)


def test_bad_arguments_are_rejected():
    v = particle_view({"kind": "soa_mb"}, 100, 1)
    counts = torch.zeros(14, dtype=torch.int64, device="cuda")
    with pytest.raises(llgb.LlgbError) as err:
        llgb.llgb_heatmap_counters(v, 3)
    assert err.value.status == llgb.ERR_INVALID_ARG
    heat = torch.zeros(1000, dtype=torch.int64, device="cuda")
    with pytest.raises(llgb.LlgbError) as err:
        llgb.llgb_nbody_step_instrumented(v, EPS, DT, heat=heat, granularity=12)
    assert err.value.status == llgb.ERR_INVALID_ARG
    bad = counts[1:]  # 8-byte aligned, fine; a byte offset is not
    llgb.llgb_nbody_step_instrumented(v, EPS, DT, field_counts=counts, count_mode="block")
    with pytest.raises(llgb.LlgbError) as err:
        llgb.check(llgb.lib().llgb_nbody_step_instrumented(v.handle, EPS, DT, llgb.ctypes.c_void_p(counts.data_ptr()),
                                                           7, None, 1, None))
    assert err.value.status == llgb.ERR_INVALID_ARG
    del bad
    sync_and_check_status()
