// fconv.cuh -- floating-point format conversion on the device.
//
// BitpackFloatSoA and ChangeType (Sec. 3 of the paper) store floats with other
// exponent/mantissa widths.  The rule implemented (the paper only asks that
// floating-point semantics be kept as well as possible, NaN and INF included,
// and that overflow on packing give INF): round to nearest, ties to even;
// gradual underflow; an exponent that rounds up to all ones is INF; NaN keeps
// its sign and the top bits of its payload and has its top mantissa bit set.
//
// Formats are (E exponent bits, M mantissa bits), IEEE layout sign|exp|man,
// bias 2^(E-1)-1.  For the standard pairs of a non-NaN input, f64 <-> f32
// takes the integer routines below and f32 <-> f16 / bf16 the hardware
// conversions (cvt.rn), which round the same way.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace llgb {

__device__ __forceinline__ uint64_t low_bits64(int w)
{
    return w >= 64 ? ~0ull : ((1ull << w) - 1ull);
}

// General conversion with integer operations only.
static __device__ __noinline__ uint64_t fconv_general(uint64_t x, int se, int sm, int de, int dm)
{
    const uint32_t s_all = (1u << se) - 1u;
    const uint32_t d_all = (1u << de) - 1u;
    const uint64_t sign = (x >> (se + sm)) & 1ull;
    const uint32_t ex = (uint32_t)(x >> sm) & s_all;
    const uint64_t man = x & low_bits64(sm);
    const uint64_t out_sign = sign << (de + dm);
    const uint64_t out_inf = (uint64_t)d_all << dm;

    if (ex == s_all) {
        if (man == 0) return out_sign | out_inf;
        const uint64_t pay = dm >= sm ? (man << (dm - sm)) : (man >> (sm - dm));
        return out_sign | out_inf | pay | (1ull << (dm - 1));
    }
    if (ex == 0 && man == 0) return out_sign;

    const int s_bias = (1 << (se - 1)) - 1;
    const int d_bias = (1 << (de - 1)) - 1;
    uint64_t sig;
    int lsb_exp;  // value = sig * 2^lsb_exp
    if (ex) {
        sig = man | (1ull << sm);
        lsb_exp = (int)ex - s_bias - sm;
    } else {
        sig = man;
        lsb_exp = 1 - s_bias - sm;
    }
    const int top = 63 - __clzll((long long)sig);
    const int e_val = lsb_exp + top;
    const int e_min = 1 - d_bias;
    const bool normal = e_val >= e_min;
    const int quantum = (normal ? e_val : e_min) - dm;
    const int shift = quantum - lsb_exp;

    uint64_t r;
    if (shift <= 0) {
        r = sig << (-shift);
    } else if (shift >= 64) {
        r = 0;
    } else {
        const uint64_t kept = sig >> shift;
        const uint64_t rest = sig & ((1ull << shift) - 1ull);
        const uint64_t half = 1ull << (shift - 1);
        r = kept + ((rest > half || (rest == half && (kept & 1ull))) ? 1ull : 0ull);
    }
    // r carries the implicit bit for normal results; a rounding carry moves
    // into the exponent by itself.
    const uint64_t code = normal ? (((uint64_t)(e_val + d_bias - 1) << dm) + r) : r;
    if ((code >> dm) >= d_all) return out_sign | out_inf;
    return out_sign | code;
}

// f64 -> f32 with integer operations (the FP64 pipe of this GPU is narrow).
// Results in the normal f32 range are rounded here: the top 23 mantissa bits
// are kept, the 29 below decide the rounding, and a carry out of the
// mantissa moves into the exponent (rebiased from 1023 to 127; a carry into
// the all-ones exponent gives INF).  Zero, NaN, INF and subnormal results go
// through fconv_general.
__device__ __forceinline__ uint32_t f64_to_f32_bits(uint64_t x)
{
    const uint32_t hi = (uint32_t)(x >> 32), lo = (uint32_t)x;
    const uint32_t s = hi & 0x80000000u;
    const uint32_t e = (hi >> 20) & 0x7FFu;
    if (e - 897u < 254u) {  // f32 exponent 1 .. 254 before rounding
        // Drop the low 29 bits rounding to nearest, ties to even: adding
        // 2^28 - 1 plus the lowest kept bit carries into bit 29 exactly when
        // the dropped part exceeds half, or equals it with an odd kept part.
        // A carry out of the mantissa moves into the exponent.
        const uint64_t a = (((uint64_t)(hi & 0x7FFFFFFFu) << 32) | lo) + 0x0FFFFFFFull + ((lo >> 29) & 1u);
        return s | ((uint32_t)(a >> 29) - (896u << 23));
    }
    if (e > 1150u && e != 0x7FFu) return s | 0x7F800000u;   // beyond the f32 range: INF
    if ((hi & 0x7FFFFFFFu) == 0u && lo == 0u) return s;      // signed zero
    return (uint32_t)fconv_general(x, 11, 52, 8, 23);
}

// f32 -> f64 (exact) with integer operations: a normal input only rebiases
// its exponent and moves its mantissa up by 29 bits.
__device__ __forceinline__ uint64_t f32_to_f64_bits(uint32_t u)
{
    const uint32_t s = u & 0x80000000u, a = u & 0x7FFFFFFFu;
    if (a - 0x00800000u < 0x7F000000u)  // exponent 1 .. 254
        return ((uint64_t)(s | ((a >> 3) + (896u << 20))) << 32) | (uint64_t)(u << 29);
    if (a == 0u) return (uint64_t)s << 32;
    return fconv_general(u, 8, 23, 11, 52);  // subnormal, INF, NaN
}

// Conversion between two fixed formats, set up once per loop.  A value whose
// result is a normal number takes a few integer operations: the exponent is
// rebiased by adding a constant to the magnitude bits, and a narrowing drops
// k = sm - dm mantissa bits rounding to nearest, ties to even (add 2^(k-1) - 1
// plus the lowest kept bit; a carry moves into the exponent, up to INF).
// Zeros and finite values beyond the target's range are handled here too;
// NaN, INF, subnormal inputs and subnormal results go to fconv_general.
struct FmtConv {
    int se, sm, de, dm;
    int k;              // sm - dm: bits dropped (> 0) or appended (< 0)
    uint64_t absmask;   // magnitude bits of the source
    uint64_t in_inf;    // source INF code: magnitudes at or above are INF / NaN
    uint64_t lo, span;  // magnitudes in [lo, lo + span) give normal results
    uint64_t ovf;       // finite magnitudes at or above overflow to INF (~0: none)
    uint64_t half;      // narrowing: 2^(k-1) - 1
    uint64_t rebias;    // added to the shifted magnitude: (d_bias - s_bias) << dm, mod 2^64
    uint64_t inf_out;   // target INF code
};

__host__ __device__ inline FmtConv fmt_conv(int se, int sm, int de, int dm)
{
    FmtConv c;
    c.se = se;
    c.sm = sm;
    c.de = de;
    c.dm = dm;
    c.k = sm - dm;
    c.absmask = (se + sm >= 64) ? ~0ull : ((1ull << (se + sm)) - 1ull);
    c.in_inf = ((1ull << se) - 1ull) << sm;
    const int64_t s_bias = (1ll << (se - 1)) - 1, d_bias = (1ll << (de - 1)) - 1;
    // source exponents e whose result exponent e - s_bias + d_bias is 1 .. 2^de - 2
    const int64_t e_lo = s_bias - d_bias + 1, e_hi = (1ll << de) - 2 + s_bias - d_bias;
    const int64_t a = e_lo > 1 ? e_lo : 1, b = e_hi < (1ll << se) - 2 ? e_hi : (1ll << se) - 2;
    if (b >= a) {
        c.lo = (uint64_t)a << sm;
        c.span = ((uint64_t)(b + 1) << sm) - c.lo;
    } else {
        c.lo = 0;
        c.span = 0;
    }
    c.ovf = e_hi + 1 <= (1ll << se) - 2 ? ((uint64_t)(e_hi + 1) << sm) : ~0ull;
    c.half = c.k > 0 ? (1ull << (c.k - 1)) - 1ull : 0ull;
    c.rebias = (uint64_t)((d_bias - s_bias) * (int64_t)(1ll << dm));
    c.inf_out = ((1ull << de) - 1ull) << dm;
    return c;
}

__device__ __forceinline__ uint64_t fmt_convert(uint64_t x, const FmtConv& c)
{
    const uint64_t a = x & c.absmask;
    const uint64_t sign = (x >> (c.se + c.sm) & 1ull) << (c.de + c.dm);
    if (a - c.lo < c.span) {
        const uint64_t r = c.k > 0 ? ((a + c.half + ((a >> c.k) & 1ull)) >> c.k) : (a << -c.k);
        return sign | (r + c.rebias);
    }
    if (a == 0) return sign;
    if (a >= c.ovf && a < c.in_inf) return sign | c.inf_out;
    return fconv_general(x, c.se, c.sm, c.de, c.dm);
}

__device__ __forceinline__ bool is_nan_bits(uint64_t x, int e, int m)
{
    const uint64_t all = (1ull << e) - 1ull;
    return ((x >> m) & all) == all && (x & low_bits64(m)) != 0;
}

// Conversion with hardware fast paths for non-NaN standard pairs.
__device__ __forceinline__ uint64_t fconv(uint64_t x, int se, int sm, int de, int dm)
{
    if (!is_nan_bits(x, se, sm)) {
        if (se == 11 && sm == 52) {
            if (de == 8 && dm == 23) return f64_to_f32_bits(x);
            if (de == 11 && dm == 52) return x;
        } else if (se == 8 && sm == 23) {
            const float f = __uint_as_float((uint32_t)x);
            if (de == 11 && dm == 52) return f32_to_f64_bits((uint32_t)x);
            if (de == 5 && dm == 10) return (uint64_t)__half_as_ushort(__float2half_rn(f));
            if (de == 8 && dm == 7) return (uint64_t)__bfloat16_as_ushort(__float2bfloat16_rn(f));
            if (de == 8 && dm == 23) return x;
        } else if (se == 5 && sm == 10) {
            if (de == 8 && dm == 23) {
                const float f = __half2float(__ushort_as_half((unsigned short)x));
                return (uint64_t)__float_as_uint(f);
            }
        } else if (se == 8 && sm == 7) {
            if (de == 8 && dm == 23) return x << 16;
        }
    }
    return fconv_general(x, se, sm, de, dm);
}

}  // namespace llgb
