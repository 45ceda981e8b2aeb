"""Seeded synthetic records for tests, the smoke check and the benchmark.

This module only draws numbers: it holds none of the layout or conversion
arithmetic.  It is the one piece shared by the CUDA path's tests and the oracle
tests.  Every generator takes an explicit seed; values are returned as numpy
arrays of each leaf's own dtype (one array per leaf, in leaf order).

Record shapes follow the n-body particle of the paper's Fig. 2 / Fig. 3 and
the synthetic workloads used to measure the copy kernels:

* ``PARTICLE``  {pos{x,y,z}, vel{x,y,z}, mass}, all f32, 28 bytes;
* ``INT6``      {a,b,c,d: u32, e,f: i32}, 24 bytes (bit-packed integers);
* ``MIXED_F``   {x,y,z: f64, w: f32}, 32 bytes aligned / 28 packed;
* ``CFD``       {rho,u,v,w,e: f32, flag: i16, id: u16}, 24 bytes.
"""
from __future__ import annotations

import numpy as np

PARTICLE = [("pos.x", "f32"), ("pos.y", "f32"), ("pos.z", "f32"),
            ("vel.x", "f32"), ("vel.y", "f32"), ("vel.z", "f32"),
            ("mass", "f32")]
INT6 = [("a", "u32"), ("b", "u32"), ("c", "u32"), ("d", "u32"),
        ("e", "i32"), ("f", "i32")]
MIXED_F = [("x", "f64"), ("y", "f64"), ("z", "f64"), ("w", "f32")]
CFD = [("rho", "f32"), ("u", "f32"), ("v", "f32"), ("w", "f32"), ("e", "f32"),
       ("flag", "i16"), ("id", "u16")]

NP_DTYPE = {"u8": np.uint8, "u16": np.uint16, "u32": np.uint32, "u64": np.uint64,
            "i8": np.int8, "i16": np.int16, "i32": np.int32, "i64": np.int64,
            "f16": np.float16, "f32": np.float32, "f64": np.float64,
            "bf16": np.uint16}

BASE_SEED = 2302082510


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_fields(record, n: int, seed: int) -> list[np.ndarray]:
    """Floats U[-1, 1); integers uniform over their whole type range."""
    g = rng(seed)
    out = []
    for _, t in record:
        dt = NP_DTYPE[t]
        if t in ("f16", "f32", "f64"):
            out.append(g.uniform(-1.0, 1.0, n).astype(dt))
        elif t == "bf16":
            out.append(g.integers(0, 1 << 16, n, dtype=np.uint16))
        else:
            info = np.iinfo(dt)
            out.append(g.integers(int(info.min), int(info.max), n, dtype=dt,
                                  endpoint=True))
    return out


def particles(n: int, seed: int) -> list[np.ndarray]:
    """Particle record: pos and vel U[-1, 1), mass U[0, 1)."""
    g = rng(seed)
    cols = [g.uniform(-1.0, 1.0, n).astype(np.float32) for _ in range(6)]
    cols.append(g.uniform(0.0, 1.0, n).astype(np.float32))
    return cols


def int6(n: int, bits: int, seed: int) -> list[np.ndarray]:
    """INT6 record: unsigned leaves U[0, 2^b), signed U[-2^(b-1), 2^(b-1))."""
    g = rng(seed)
    out = []
    for _, t in INT6:
        if t == "u32":
            out.append(g.integers(0, 1 << bits, n, dtype=np.uint64).astype(np.uint32))
        else:
            lo, hi = -(1 << (bits - 1)), (1 << (bits - 1))
            out.append(g.integers(lo, hi, n, dtype=np.int64).astype(np.int32))
    return out


def mixed_f(n: int, seed: int, scale: float = 1e3) -> list[np.ndarray]:
    """MIXED_F record: x, y, z ~ N(0, scale) in f64; w = f32 of N(0, scale)."""
    g = rng(seed)
    cols = [g.normal(0.0, scale, n) for _ in range(3)]
    cols.append(g.normal(0.0, scale, n).astype(np.float32))
    return cols


def cfd(n: int, seed: int) -> list[np.ndarray]:
    """CFD record: floats U[-1, 1), flag U[-2^15, 2^15), id U[0, 2^16)."""
    g = rng(seed)
    cols = [g.uniform(-1.0, 1.0, n).astype(np.float32) for _ in range(5)]
    cols.append(g.integers(-(1 << 15), 1 << 15, n, dtype=np.int32).astype(np.int16))
    cols.append(g.integers(0, 1 << 16, n, dtype=np.int32).astype(np.uint16))
    return cols


def special_f64(n: int, seed: int) -> np.ndarray:
    """f64 values dense in the cases conversions get wrong: +-0, subnormals,
    +-INF, quiet and signalling NaN with payloads, the largest finite value,
    and random bit patterns over the whole exponent range."""
    g = rng(seed)
    fixed = np.array([0.0, -0.0, np.inf, -np.inf, 5e-324, -5e-324,
                      2.2250738585072014e-308, 1.7976931348623157e308,
                      -1.7976931348623157e308, 1.0, -1.0, 0.5, 65504.0, 65520.0,
                      3.4028234663852886e38, 3.4028235677973366e38,
                      1.401298464324817e-45, 7.006492321624085e-46],
                     dtype=np.float64)
    nan_bits = np.array([0x7FF8000000000000, 0xFFF8000000000001, 0x7FF0000000000001,
                         0x7FF4000000000000, 0x7FFFFFFFFFFFFFFF, 0xFFF0000020000000],
                        dtype=np.uint64)
    rand_bits = g.integers(0, 2**63, n, dtype=np.uint64) * np.uint64(2) + \
        g.integers(0, 2, n, dtype=np.uint64)
    out = np.concatenate([fixed.view(np.uint64), nan_bits, rand_bits])
    return out.view(np.float64)


def f32_range_f64(n: int, seed: int) -> np.ndarray:
    """f64 values whose exponents lie in and around the f32 range, with the
    29 mantissa bits below an f32 mantissa set to exactly half an f32 ulp
    (a tie), one unit either side of it, zero, or random: the cases where
    rounding f64 -> f32 to nearest even can go wrong."""
    g = rng(seed)
    sign = g.integers(0, 2, n, dtype=np.uint64) << np.uint64(63)
    # f64 exponents 1023-130 .. 1023+130 (f32 subnormals .. beyond f32 max)
    exp = g.integers(1023 - 130, 1023 + 131, n, dtype=np.uint64) << np.uint64(52)
    top = g.integers(0, 1 << 23, n, dtype=np.uint64) << np.uint64(29)
    half = np.uint64(1 << 28)
    low_choices = np.stack([np.full(n, half, np.uint64), np.full(n, half - np.uint64(1), np.uint64),
                            np.full(n, half + np.uint64(1), np.uint64), np.zeros(n, np.uint64),
                            g.integers(0, 1 << 29, n, dtype=np.uint64)])
    low = low_choices[g.integers(0, 5, n), np.arange(n)]
    top_all = np.full(n, np.uint64(((1 << 23) - 1) << 29), np.uint64)
    # a quarter of the values carry an all-ones f32 mantissa (rounding carries into the exponent)
    top = np.where(g.integers(0, 4, n) == 0, top_all, top)
    bits = sign | exp | top | low
    return bits.view(np.float64)


def special_f32(n: int, seed: int) -> np.ndarray:
    """f32 counterpart of ``special_f64``."""
    g = rng(seed)
    fixed = np.array([0.0, -0.0, np.inf, -np.inf, 1e-45, -1e-45, 1.1754944e-38,
                      3.4028235e38, -3.4028235e38, 1.0, -1.0, 65504.0, 65520.0,
                      65519.996, 6.1035156e-05, 5.9604645e-08, 2.9802322e-08],
                     dtype=np.float32)
    nan_bits = np.array([0x7FC00000, 0xFFC00001, 0x7F800001, 0x7FA00000, 0x7FFFFFFF],
                        dtype=np.uint32)
    rand_bits = g.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    out = np.concatenate([fixed.view(np.uint32), nan_bits, rand_bits])
    return out.view(np.float32)


# ---------------------------------------------------------------- device --
# Large inputs are drawn on the device with a seeded torch generator.  They
# are either one plain array per leaf (the values of each leaf, in record
# order) or raw random bytes for a whole blob.

def _torch_gen(seed: int, device):
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def device_random_bytes(size: int, seed: int, device="cuda"):
    """`size` uniformly random bytes (uint8 tensor) on `device`."""
    import torch
    g = _torch_gen(seed, device)
    return torch.randint(0, 256, (max(1, size),), dtype=torch.uint8, generator=g, device=device)


def device_fields(kind: str, n: int, seed: int, device="cuda", bits: int = 12):
    """Leaf arrays of n records on `device`, distributed like the host
    generators: kind is 'particle', 'int6' (with `bits`), 'mixed_f' or 'cfd'."""
    import torch
    g = _torch_gen(seed, device)

    def unif(lo, hi, dtype=torch.float32):
        return (torch.rand(n, generator=g, device=device, dtype=torch.float64) * (hi - lo) + lo).to(dtype)

    if kind == "particle":
        return [unif(-1.0, 1.0) for _ in range(6)] + [unif(0.0, 1.0)]
    if kind == "int6":
        out = []
        for _, t in INT6:
            if t == "u32":
                v = torch.randint(0, 1 << bits, (n,), generator=g, device=device, dtype=torch.int64)
            else:
                v = torch.randint(-(1 << (bits - 1)), 1 << (bits - 1), (n,), generator=g,
                                  device=device, dtype=torch.int64)
            out.append(v.to(torch.int32))
        return out
    if kind == "mixed_f":
        cols = [torch.randn(n, generator=g, device=device, dtype=torch.float64) * 1e3 for _ in range(3)]
        cols.append((torch.randn(n, generator=g, device=device, dtype=torch.float64) * 1e3).float())
        return cols
    if kind == "cfd":
        cols = [unif(-1.0, 1.0) for _ in range(5)]
        cols.append(torch.randint(-(1 << 15), 1 << 15, (n,), generator=g, device=device,
                                  dtype=torch.int32).to(torch.int16))
        cols.append(torch.randint(0, 1 << 16, (n,), generator=g, device=device,
                                  dtype=torch.int32).to(torch.int16))
        return cols
    raise ValueError(kind)
