"""Pins of the oracle's n-body step (arXiv 2302.08251, Sec. 5, Fig. 2).

The paper shows the loop structure of the update (all j for each i, then store
the velocity) and names the move phase; the interaction is the softened
Newtonian one of the original LLAMA n-body (a reading, G = 1).  Pinned by
physics that holds whatever way the sum is written: the inverse-square law far
from the softening length, the linear core inside it, attraction, momentum
conservation, symmetry, the move using the new velocity, and independence from
the mapping the particles are read through.
"""
import numpy as np
import pytest

import oracle
from paper_2302_08251_gb300 import synth
from helpers import AFFINE, oracle_view

EPS, DT = 0.01, 1e-4


def particles_from(pos, vel, mass):
    pos = np.asarray(pos, np.float32).reshape(-1, 3)
    vel = np.asarray(vel, np.float32).reshape(-1, 3)
    mass = np.asarray(mass, np.float32)
    return [pos[:, 0], pos[:, 1], pos[:, 2], vel[:, 0], vel[:, 1], vel[:, 2], mass]


def step(fields, mapping={"kind": "soa_mb"}, eps=EPS, dt=DT):
    v = oracle_view(synth.PARTICLE, mapping, fields)
    return v.nbody_step(eps, dt)


def test_single_particle_keeps_its_velocity_and_drifts():
    f = particles_from([0.25, -0.5, 0.125], [1.0, 2.0, -4.0], [0.75])
    pos, vel = step(f)
    assert np.array_equal(vel[0], [1.0, 2.0, -4.0])
    np.testing.assert_allclose(pos[0], [0.25 + DT, -0.5 + 2 * DT, 0.125 - 4 * DT],
                               rtol=0, atol=1e-15)


@pytest.mark.parametrize("r", [1.0, 2.0, 16.0])
def test_far_field_is_the_inverse_square_law(r):
    # two bodies at rest, distance r >> eps: |dv| = dt * m_other / r^2
    eps = 1e-6
    m = np.float32(0.5)
    f = particles_from([0, 0, 0, r, 0, 0], [0] * 6, [1.0, m])
    pos, vel = step(f, eps=eps, dt=1.0)
    np.testing.assert_allclose(vel[0], [m / r**2, 0, 0], rtol=1e-9)
    np.testing.assert_allclose(vel[1], [-1.0 / r**2, 0, 0], rtol=1e-9)


def test_inside_the_softening_length_the_pull_grows_linearly():
    # Plummer softening: for r << eps the pull tends to m r / eps^3
    eps = 1.0
    for r in [1e-3, 2e-3]:
        f = particles_from([0, 0, 0, 0, r, 0], [0] * 6, [1.0, 1.0])
        _, vel = step(f, eps=eps, dt=1.0)
        assert vel[0][1] == pytest.approx(r, rel=1e-5)


def test_bodies_attract():
    f = particles_from([-0.5, 0.1, 0, 0.5, 0.1, 0], [0] * 6, [1.0, 1.0])
    pos, vel = step(f)
    assert vel[0][0] > 0 and vel[1][0] < 0
    assert pos[0][0] > -0.5 and pos[1][0] < 0.5


def test_momentum_is_conserved():
    n = 200
    f = synth.particles(n, seed=13)
    _, vel = step(f)
    m = f[6].astype(np.float64)
    v0 = np.stack(f[3:6], axis=1).astype(np.float64)
    dp = (m[:, None] * (vel - v0)).sum(axis=0)
    scale = (m[:, None] * np.abs(vel - v0)).sum(axis=0)
    assert np.all(np.abs(dp) <= 1e-12 * scale)


def test_symmetric_neighbours_cancel():
    pts = [0, 0, 0]
    for axis in range(3):
        for s in (1, -1):
            p = [0.0, 0.0, 0.0]
            p[axis] = 0.5 * s
            pts += p
    f = particles_from(pts, [0.0] * 21, [1.0] * 7)
    _, vel = step(f)
    assert np.all(vel[0] == 0.0)


def test_move_uses_the_updated_velocity():
    n = 50
    f = synth.particles(n, seed=21)
    pos, vel = step(f)
    p0 = np.stack(f[0:3], axis=1).astype(np.float64)
    np.testing.assert_allclose(pos, p0 + DT * vel, rtol=0, atol=1e-15)


@pytest.mark.parametrize("mapping", AFFINE, ids=str)
def test_result_does_not_depend_on_the_mapping(mapping):
    n = 37
    f = synth.particles(n, seed=2)
    ref = step(f)
    got = step(f, mapping)
    assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1])


def test_partial_range_equals_the_slice_of_the_full_step():
    n = 64
    f = synth.particles(n, seed=8)
    v = oracle_view(synth.PARTICLE, {"kind": "aos"}, f)
    full = v.nbody_step(EPS, DT)
    part = v.nbody_step(EPS, DT, 10, 20)
    assert np.array_equal(full[0][10:20], part[0])
    assert np.array_equal(full[1][10:20], part[1])


# ---- access instrumentation of the tiled step (Sec. 4: FieldAccessCount,
# Heatmap): pinned against a direct enumeration of the access events and
# against what every mapping must agree on ----

def enumerate_accesses(n, block=64):
    """Every access of one tiled step as (record, leaf, is_write), listed
    event by event from the schedule: blocks of `block` particles each read
    their own positions, every record's position and mass, then read and
    write their velocities; the move reads pos and vel and writes pos."""
    ev = []
    for b in range(0, n, block):
        mine = range(b, min(n, b + block))
        for i in mine:
            ev += [(i, f, False) for f in (0, 1, 2)]
        for j in range(n):
            ev += [(j, f, False) for f in (0, 1, 2, 6)]
        for i in mine:
            ev += [(i, f, False) for f in (3, 4, 5)] + [(i, f, True) for f in (3, 4, 5)]
    for i in range(n):
        ev += [(i, f, False) for f in range(6)] + [(i, f, True) for f in (0, 1, 2)]
    return ev


@pytest.mark.parametrize("n", [0, 1, 63, 64, 65, 200])
def test_access_counts_match_the_enumerated_schedule(n):
    want = np.zeros(14, dtype=np.uint64)
    for _, f, w in enumerate_accesses(n):
        want[f + (7 if w else 0)] += 1
    assert np.array_equal(oracle.nbody_access_counts(n), want)


def plain_loop_accesses(n):
    """Every access of the paper's plain update loop (Sec. 5, Fig. 2: for each
    particle i, its position, then every particle j's position and mass, then
    i's velocity loaded, updated and stored) followed by the move (each
    particle's position and velocity loaded, its position stored).  Written
    as the nested i / j loop itself, with no notion of a tile or block."""
    ev = []
    for i in range(n):
        ev += [(i, f, False) for f in (0, 1, 2)]
        for j in range(n):
            ev += [(j, f, False) for f in (0, 1, 2, 6)]
        ev += [(i, f, False) for f in (3, 4, 5)] + [(i, f, True) for f in (3, 4, 5)]
    for i in range(n):
        ev += [(i, f, False) for f in range(6)] + [(i, f, True) for f in (0, 1, 2)]
    return ev


@pytest.mark.parametrize("n", [0, 1, 2, 5, 17])
def test_one_particle_blocks_count_the_plain_fig2_loop(n):
    # a block of one particle is the untiled loop: j runs over all particles
    # once per i, so positions are read n + n^2 + n times and masses n^2
    want = np.zeros(14, dtype=np.uint64)
    for _, f, w in plain_loop_accesses(n):
        want[f + (7 if w else 0)] += 1
    assert np.array_equal(oracle.nbody_access_counts(n, block=1), want)
    assert int(want[0]) == 2 * n + n * n and int(want[6]) == n * n


@pytest.mark.parametrize("block", [1, 2, 7, 64, 100, 1000])
@pytest.mark.parametrize("n", [1, 63, 100, 257])
def test_counts_that_every_schedule_shares(n, block):
    # whatever the tiling: each velocity leaf is read in the update and in the
    # move and written once; each position leaf is written once (by the move);
    # mass is never written; the j loop reads positions and mass equally often
    c = oracle.nbody_access_counts(n, block=block).astype(np.int64)
    reads, writes = c[:7], c[7:]
    assert np.all(reads[3:6] == 2 * n)
    assert np.all(writes[3:6] == n) and np.all(writes[0:3] == n) and writes[6] == 0
    assert np.all(reads[0:3] == reads[0]) and reads[0] == reads[6] + 2 * n
    # the j loop runs once per block of the update: ceil(n / block) passes of n
    assert reads[6] == -(-n // block) * n
    # fewer, larger blocks never read more
    if block > 1:
        assert np.all(c <= oracle.nbody_access_counts(n, block=block - 1).astype(np.int64))


@pytest.mark.parametrize("block", [1, 3, 64])
@pytest.mark.parametrize("mapping", [{"kind": "aos"}, {"kind": "soa_mb"}, {"kind": "aosoa", "lanes": 8}],
                         ids=lambda m: m["kind"])
def test_byte_heatmap_holds_four_counts_per_access_for_any_block(mapping, block):
    n = 45
    heat = oracle.nbody_heatmap(mapping, n, 1, block=block)
    counts = oracle.nbody_access_counts(n, block=block)
    assert int(heat.sum()) == 4 * int(counts.sum())
    # per leaf: its bytes' counters add up to 4 x (its reads + writes)
    sizes = oracle.blob_sizes(synth.PARTICLE, mapping, n)
    start = np.cumsum([0] + sizes)
    per_leaf = np.zeros(7, dtype=np.int64)
    for i in range(n):
        for f in range(7):
            b, off = element_offset(mapping, n, i, f)
            per_leaf[f] += int(heat[start[b] + off:start[b] + off + 4].sum())
    assert np.array_equal(per_leaf, 4 * n * ((counts[:7] + counts[7:]) // n).astype(np.int64))


def test_heatmap_of_one_particle_blocks_matches_the_plain_loop():
    n, g = 23, 4
    mapping = {"kind": "aosoa", "lanes": 8}
    sizes = oracle.blob_sizes(synth.PARTICLE, mapping, n)
    start = np.cumsum([0] + [(s + g - 1) // g for s in sizes])
    want = np.zeros(start[-1], dtype=np.uint64)
    for i, f, _ in plain_loop_accesses(n):
        b, off = element_offset(mapping, n, i, f)
        for k in range(off // g, (off + 3) // g + 1):
            want[start[b] + k] += 1
    assert np.array_equal(oracle.nbody_heatmap(mapping, n, g, block=1), want)


def element_offset(mapping, n, i, f):
    """(blob, byte) of leaf f of record i for the particle record, from the
    mapping formulas (28-byte record of 7 f32 leaves)."""
    k = mapping["kind"]
    if k == "aos":
        return 0, 28 * i + 4 * f
    if k == "soa_mb":
        return f, 4 * i
    if k == "soa_sb":
        return 0, 4 * n * f + 4 * i
    L = mapping["lanes"]
    return 0, (i // L) * 28 * L + 4 * L * f + 4 * (i % L)


MAPS = [{"kind": "aos"}, {"kind": "soa_mb"}, {"kind": "soa_sb"}, {"kind": "aosoa", "lanes": 8},
        {"kind": "aosoa", "lanes": 32}]


@pytest.mark.parametrize("mapping", MAPS, ids=lambda m: m["kind"] + str(m.get("lanes", "")))
@pytest.mark.parametrize("g", [1, 2, 4, 8, 64])
def test_heatmap_matches_the_enumerated_accesses(mapping, g):
    n = 70
    sizes = oracle.blob_sizes(synth.PARTICLE, mapping, n)
    start = np.cumsum([0] + [(s + g - 1) // g for s in sizes])
    want = np.zeros(start[-1], dtype=np.uint64)
    for i, f, _ in enumerate_accesses(n):
        b, off = element_offset(mapping, n, i, f)
        for k in range(off // g, (off + 3) // g + 1):
            want[start[b] + k] += 1
    got = oracle.nbody_heatmap(mapping, n, g)
    assert np.array_equal(got, want)
    # every access of a 4-byte element touches 4 byte counters
    if g == 1:
        assert int(got.sum()) == 4 * int(oracle.nbody_access_counts(n).sum())


def test_heatmap_per_element_counts_agree_across_mappings():
    n = 100
    per = [np.sort(oracle.nbody_heatmap(m, n, 4)[np.nonzero(oracle.nbody_heatmap(m, n, 4))])
           for m in MAPS]
    for p in per[1:]:
        assert np.array_equal(p, per[0])


# ---- the move phase alone (Sec. 5): p + dt v ----

def test_move_worked_example_uses_leaves_0_to_5():
    # distinct values in every leaf: a wrong leaf index or sign shows
    f = particles_from([1.0, 2.0, 3.0], [0.5, -1.0, 4.0], [7.0])
    v = oracle_view(synth.PARTICLE, {"kind": "aos"}, f)
    assert np.array_equal(v.nbody_move(0.25), [[1.125, 1.75, 4.0]])
    assert np.array_equal(v.nbody_move(0.0), [[1.0, 2.0, 3.0]])


def test_move_is_the_step_when_no_mass_pulls():
    # massless particles feel no force, so the step's move is the move alone
    n = 40
    f = synth.particles(n, seed=31)
    f[6] = np.zeros(n, np.float32)
    v = oracle_view(synth.PARTICLE, {"kind": "soa_mb"}, f)
    pos, vel = v.nbody_step(EPS, DT)
    assert np.array_equal(vel, np.stack(f[3:6], axis=1).astype(np.float64))
    assert np.array_equal(pos, v.nbody_move(DT))


@pytest.mark.parametrize("mapping", AFFINE + [{"kind": "aosoa", "lanes": 3}, {"kind": "aosoa", "lanes": 48}],
                         ids=str)
def test_move_does_not_depend_on_the_mapping(mapping):
    n = 101
    f = synth.particles(n, seed=4)
    ref = oracle_view(synth.PARTICLE, {"kind": "soa_mb"}, f).nbody_move(DT)
    v = oracle_view(synth.PARTICLE, mapping, f)
    assert np.array_equal(v.nbody_move(DT), ref)
    assert np.array_equal(v.nbody_move(DT, 50, 99), ref[50:99])
