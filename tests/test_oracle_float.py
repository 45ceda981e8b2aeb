"""Pins of the oracle's float conversion (BitpackFloatSoA and ChangeType).

arXiv 2302.08251, Sec. 3: BitpackFloatSoA stores floats with chosen exponent
and mantissa bit counts, keeps NaN and INF, and maps values that overflow on
packing to INF; ChangeType stores a leaf in another floating-point type.
Readings: IEEE-style layout and round to nearest, ties to even.

The oracle converts in the bit domain.  It is pinned here against
  * an exact value-domain rounding written with Python Fractions,
  * brute force over every code of small formats,
  * numpy's float32 / float16 casts and torch's bfloat16 cast,
  * closed-form decoding of every code of small formats,
  * hand-derived codes (tests/golden/bitpack_float_hand.txt).
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle
from paper_2302_08251_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
F64 = (11, 52)
F32 = (8, 23)


# ------------------------------------------------ value-domain reference --

def decode(code: int, e: int, m: int):
    """Exact value of a code: Fraction, or +-inf / nan as floats."""
    sign = (code >> (e + m)) & 1
    ex = (code >> m) & ((1 << e) - 1)
    man = code & ((1 << m) - 1)
    bias = (1 << (e - 1)) - 1
    if ex == (1 << e) - 1:
        return math.nan if man else (-math.inf if sign else math.inf)
    if ex == 0:
        val = Fraction(man, 1 << m) * Fraction(2) ** (1 - bias)
    else:
        val = (1 + Fraction(man, 1 << m)) * Fraction(2) ** (ex - bias)
    return -val if sign else val


def rne_value(x: Fraction, e: int, m: int):
    """Round |x| to the (e, m) grid by exact arithmetic; inf on overflow."""
    bias = (1 << (e - 1)) - 1
    emin = 1 - bias
    ax = abs(x)
    if ax == 0:
        return Fraction(0)
    k = ax.numerator.bit_length() - ax.denominator.bit_length()
    while Fraction(2) ** k > ax:
        k -= 1
    while Fraction(2) ** (k + 1) <= ax:
        k += 1
    k = max(k, emin)
    quantum = Fraction(2) ** (k - m)
    lo = (ax / quantum).__floor__()
    rem = ax / quantum - lo
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and lo % 2 == 1):
        lo += 1
    r = lo * quantum
    max_finite = (2 - Fraction(1, 1 << m)) * Fraction(2) ** bias
    if r > max_finite:
        return math.inf
    return r


def encode(val, sign: int, e: int, m: int) -> int:
    """Code of a representable value (Fraction >= 0, or inf)."""
    if val == math.inf:
        return (sign << (e + m)) | (((1 << e) - 1) << m)
    bias = (1 << (e - 1)) - 1
    if val == 0:
        return sign << (e + m)
    k = val.numerator.bit_length() - val.denominator.bit_length()
    while Fraction(2) ** k > val:
        k -= 1
    while Fraction(2) ** (k + 1) <= val:
        k += 1
    if k < 1 - bias:
        man = val / Fraction(2) ** (1 - bias - m)
        assert man.denominator == 1
        return (sign << (e + m)) | int(man)
    frac = val / Fraction(2) ** k - 1
    man = frac * (1 << m)
    assert man.denominator == 1
    return (sign << (e + m)) | ((k + bias) << m) | int(man)


def expected_code(x: float, e: int, m: int) -> int:
    sign = 1 if math.copysign(1.0, x) < 0 else 0
    if math.isinf(x):
        return encode(math.inf, sign, e, m)
    return encode(rne_value(Fraction(x), e, m), sign, e, m)


def f64_bits(x: float) -> int:
    return int(np.array([x], dtype=np.float64).view(np.uint64)[0])


def f64_of(bits: int) -> float:
    return float(np.array([bits], dtype=np.uint64).view(np.float64)[0])


# --------------------------------------------------------------- tests ----

SMALL = [(2, 1), (3, 2), (4, 3), (5, 2)]


def _probe_values(e, m, seed):
    """Every code value, the midpoints between neighbours (ties), values just
    off the midpoints, random values, and values past overflow."""
    codes = range(0, ((1 << e) - 1) << m)  # every finite non-negative code
    vals = [decode(c, e, m) for c in codes]
    probes = set()
    for a, b in zip(vals, vals[1:]):
        mid = (a + b) / 2
        probes.update([float(a), float(mid)])
        probes.add(float(np.nextafter(float(mid), 0.0)))
        probes.add(float(np.nextafter(float(mid), np.inf)))
    top = vals[-1]
    ulp_top = top - vals[-2]
    for t in [top + ulp_top / 2, top + ulp_top / 4, top * 2, top * 1e6]:
        probes.add(float(t))
        probes.add(float(np.nextafter(float(t), 0.0)))
    g = synth.rng(seed)
    probes.update(float(x) for x in g.uniform(0, float(top) * 1.2, 300))
    probes.update(float(x) for x in g.uniform(0, float(vals[1 << m]) * 1.5, 100))
    probes = sorted(probes)
    return probes + [-x for x in probes]


@pytest.mark.parametrize("fmt", SMALL)
def test_small_formats_brute_force_nearest_even(fmt):
    e, m = fmt
    probes = _probe_values(e, m, seed=e * 10 + m)
    codes = list(range(0, ((1 << e) - 1) << m))
    grid = [decode(c, e, m) for c in codes]
    max_finite = grid[-1]
    half_ulp_top = (grid[-1] - grid[-2]) / 2
    got = oracle.convert_array(np.array([f64_bits(x) for x in probes], dtype=np.uint64),
                               *F64, e, m)
    for x, code in zip(probes, got):
        ax = Fraction(abs(x))
        sign = 1 if math.copysign(1.0, x) < 0 else 0
        if ax >= max_finite + half_ulp_top:
            want = encode(math.inf, sign, e, m)
        else:
            dists = [abs(g - ax) for g in grid]
            best = min(dists)
            cands = [c for c, d in zip(codes, dists) if d == best]
            cands = [c for c in cands if c % 2 == 0] or cands
            want = (sign << (e + m)) | cands[0]
        assert int(code) == want, (x, fmt, hex(int(code)), hex(want))


@pytest.mark.parametrize("fmt", [(2, 1), (4, 3), (5, 2), (5, 10), (8, 7), (8, 2)])
def test_every_code_decodes_to_its_closed_form_value(fmt):
    e, m = fmt
    codes = np.arange(0, 1 << (1 + e + m), dtype=np.uint64)
    out = oracle.convert_array(codes, e, m, *F64)
    for c, o in zip(codes.tolist(), out.tolist()):
        want = decode(c, e, m)
        got = f64_of(o)
        if isinstance(want, float) and math.isnan(want):
            assert math.isnan(got)
            assert (o >> 63) == (c >> (e + m))
        else:
            assert got == want, (fmt, c)


WIDE = [(5, 23), (5, 52), (8, 10), (8, 52), (11, 2), (11, 10), (11, 23),
        (8, 23), (5, 10), (8, 7), (11, 51)]


@pytest.mark.parametrize("fmt", WIDE)
def test_wide_formats_match_exact_rounding(fmt):
    e, m = fmt
    xs = synth.special_f64(3000, seed=e * 100 + m)
    xs = np.concatenate([xs, synth.mixed_f(2000, seed=m)[0]])
    got = oracle.convert_array(xs.view(np.uint64), *F64, e, m)
    for x, code in zip(xs.tolist(), got.tolist()):
        if math.isnan(x):
            continue
        assert code == expected_code(x, e, m), (fmt, x)


@pytest.mark.parametrize("fmt", [(5, 2), (5, 10), (8, 23), (11, 10)])
def test_unpack_of_pack_is_within_half_an_ulp(fmt):
    e, m = fmt
    bias = (1 << (e - 1)) - 1
    xs = synth.mixed_f(500, seed=3)[0]
    codes = oracle.convert_array(xs.view(np.uint64), *F64, e, m)
    back = oracle.convert_array(codes, e, m, *F64).view(np.float64)
    for x, y in zip(xs.tolist(), back.tolist()):
        if math.isinf(y):
            continue
        ax = abs(Fraction(x))
        k = max(math.frexp(abs(x))[1] - 1, 1 - bias)
        ulp = Fraction(2) ** (k - m)
        assert abs(Fraction(y) - Fraction(x)) <= ulp / 2
        assert ax == 0 or math.copysign(1, x) == math.copysign(1, y)


def test_f64_to_f32_matches_numpy_cast():
    xs = np.concatenate([synth.special_f64(200000, seed=1), synth.mixed_f(100000, 2)[0]])
    got = oracle.convert_array(xs.view(np.uint64), *F64, *F32).astype(np.uint32)
    with np.errstate(over="ignore"):
        want = xs.astype(np.float32).view(np.uint32)
    ok = ~np.isnan(xs)
    assert np.array_equal(got[ok], want[ok])


def test_f64_to_f32_ties_and_range_edges_match_numpy_cast():
    # exact ties, one unit either side, mantissa carries into the exponent,
    # overflow to INF and results in the f32 subnormal range
    xs = synth.f32_range_f64(400000, seed=11)
    got = oracle.convert_array(xs.view(np.uint64), *F64, *F32).astype(np.uint32)
    with np.errstate(over="ignore"):
        want = xs.astype(np.float32).view(np.uint32)
    assert np.array_equal(got, want)
    widened = oracle.convert_array(want.astype(np.uint64), *F32, *F64)
    assert np.array_equal(widened, want.view(np.float32).astype(np.float64).view(np.uint64))


def test_f32_to_f16_matches_numpy_cast():
    g = synth.rng(7)
    xs = synth.special_f32(1 << 20, seed=2)
    # every half-way point between neighbouring f16 values, and its neighbours
    h = np.arange(0, 0x7C00, dtype=np.uint16).view(np.float16).astype(np.float32)
    mids = ((h[:-1].astype(np.float64) + h[1:].astype(np.float64)) / 2).astype(np.float32)
    up = np.nextafter(mids, np.float32(np.inf))
    down = np.nextafter(mids, np.float32(0))
    xs = np.concatenate([xs, mids, up, down, -mids, -up,
                         g.normal(0, 1e4, 1 << 16).astype(np.float32)])
    got = oracle.convert_array(xs.view(np.uint32).astype(np.uint64), *F32, 5, 10)
    with np.errstate(over="ignore"):
        want = xs.astype(np.float16).view(np.uint16)
    ok = ~np.isnan(xs)
    assert np.array_equal(got[ok].astype(np.uint16), want[ok])


def test_every_f16_code_widens_like_numpy():
    codes = np.arange(1 << 16, dtype=np.uint64)
    got = oracle.convert_array(codes, 5, 10, *F32).astype(np.uint32)
    halfs = codes.astype(np.uint16).view(np.float16)
    want = halfs.astype(np.float32).view(np.uint32)
    ok = ~np.isnan(halfs)
    assert np.array_equal(got[ok], want[ok])


def test_f32_to_bf16_matches_torch_cast():
    xs = synth.special_f32(1 << 20, seed=4)
    got = oracle.convert_array(xs.view(np.uint32).astype(np.uint64), *F32, 8, 7)
    want = torch.from_numpy(xs.copy()).to(torch.bfloat16).view(torch.int16).numpy()
    ok = ~np.isnan(xs)
    assert np.array_equal(got[ok].astype(np.uint16), want.view(np.uint16)[ok])


def test_same_format_is_the_identity_and_widening_is_exact():
    xs = synth.special_f64(100000, seed=5)
    bits = xs.view(np.uint64)
    got = oracle.convert_array(bits, *F64, *F64)
    ok = ~np.isnan(xs)
    assert np.array_equal(got[ok], bits[ok])
    ys = synth.special_f32(100000, seed=6)
    wide = oracle.convert_array(ys.view(np.uint32).astype(np.uint64), *F32, *F64)
    ok = ~np.isnan(ys)
    assert np.array_equal(wide[ok], ys.astype(np.float64).view(np.uint64)[ok])
    same = oracle.convert_array(ys.view(np.uint32).astype(np.uint64), *F32, *F32)
    assert np.array_equal(same[ok], ys.view(np.uint32).astype(np.uint64)[ok])


@pytest.mark.parametrize("e,m", [(5, 2), (5, 10), (8, 2), (8, 23), (11, 2), (11, 23)])
def test_overflow_threshold_is_max_plus_half_ulp(e, m):
    bias = (1 << (e - 1)) - 1
    threshold = (2 - 2.0 ** (-m - 1)) * 2.0 ** bias
    inf = ((1 << e) - 1) << m
    max_code = inf - 1
    for x, want in [(threshold, inf), (np.nextafter(threshold, 0), max_code),
                    (-threshold, inf | (1 << (e + m))), (threshold * 4, inf)]:
        assert oracle.convert(f64_bits(float(x)), *F64, e, m) == want


@pytest.mark.parametrize("e,m", [(5, 2), (5, 10), (8, 23), (11, 52), (8, 52)])
def test_nan_keeps_sign_top_payload_and_becomes_quiet(e, m):
    for bits in [0x7FF8000000000000, 0xFFF0000000000001, 0x7FF4000000000000,
                 0x7FFFFFFFFFFFFFFF, 0xFFFABCDEF0123456]:
        code = oracle.convert(bits, *F64, e, m)
        assert (code >> (e + m)) == bits >> 63
        assert (code >> m) & ((1 << e) - 1) == (1 << e) - 1
        payload = code & ((1 << m) - 1)
        assert payload >> (m - 1) == 1  # quiet
        src_payload = bits & ((1 << 52) - 1)
        keep = min(m, 52) - 1
        assert (payload & ((1 << (m - 1)) - 1)) >> (m - 1 - keep) == \
            (src_payload & ((1 << 51) - 1)) >> (51 - keep)


def test_hand_derived_codes():
    n = 0
    for line in open(os.path.join(GOLDEN, "bitpack_float_hand.txt")):
        if line.startswith("#") or not line.strip():
            continue
        val, e, m, code = line.split()[:4]
        got = oracle.convert(f64_bits(float(val)), *F64, int(e), int(m))
        assert got == int(code, 16), line
        n += 1
    assert n >= 10


def test_bitpack_float_view_stream_and_round_trip():
    n = 70
    fields = synth.mixed_f(n, seed=12)
    from helpers import oracle_view
    for e, m in [(5, 2), (8, 23), (11, 52), (5, 10)]:
        v = oracle_view(synth.MIXED_F, {"kind": "bitpack_float", "exp": e, "man": m}, fields)
        w = 1 + e + m
        assert v.blob_sizes == [4 * (-(-n * w // 32))] * 4
        for f, col in enumerate(fields):
            src = (11, 52) if col.dtype == np.float64 else (8, 23)
            bits = col.view(np.uint64 if col.dtype == np.float64 else np.uint32)
            codes = oracle.convert_array(bits.astype(np.uint64), *src, e, m)
            stream = ((codes[:, None] >> np.arange(w, dtype=np.uint64)) & np.uint64(1))
            packed = np.packbits(stream.astype(np.uint8).ravel(), bitorder="little")
            assert bytes(v.blobs[f][:packed.size]) == packed.tobytes()
            assert not v.blobs[f][packed.size:].any()
            back = oracle.convert_array(codes, e, m, *src)
            assert np.array_equal(v.field_values(f), back)
