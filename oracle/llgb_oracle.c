/*
 * llgb_oracle.c -- plain, slow CPU oracle for mapping-driven record layouts.
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the CPU
 * baseline of the benchmark, never by the product path.  Shares no code with
 * the CUDA library.
 *
 * Every function is written for a reader checking it against the paper
 * (arXiv 2302.08251) by eye: one record, one field, one bit at a time, no
 * blocking and no reordering.  Where the paper leaves a detail open, the
 * reading taken is stated beside the code.
 */
#include "llgb_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define MAX_LEAVES 1024

/* ---------------------------------------------------------------- types -- */

int orc_type_size(int32_t t)
{
    switch (t) {
    case ORC_U8: case ORC_I8: return 1;
    case ORC_U16: case ORC_I16: case ORC_F16: case ORC_BF16: return 2;
    case ORC_U32: case ORC_I32: case ORC_F32: return 4;
    case ORC_U64: case ORC_I64: case ORC_F64: return 8;
    default: return 0;
    }
}

static int is_signed_int(int32_t t)
{
    return t == ORC_I8 || t == ORC_I16 || t == ORC_I32 || t == ORC_I64;
}

static int is_int(int32_t t)
{
    return t >= ORC_U8 && t <= ORC_I64;
}

/* IEEE-style (exponent bits, mantissa bits) of a floating-point leaf type. */
static int float_format(int32_t t, int* e, int* m)
{
    switch (t) {
    case ORC_F16: *e = 5; *m = 10; return 1;
    case ORC_BF16: *e = 8; *m = 7; return 1;
    case ORC_F32: *e = 8; *m = 23; return 1;
    case ORC_F64: *e = 11; *m = 52; return 1;
    default: return 0;
    }
}

static uint64_t low_mask(int w)
{
    return w >= 64 ? ~(uint64_t)0 : (((uint64_t)1 << w) - 1);
}

static uint64_t align_up(uint64_t x, uint64_t a)
{
    return (x + a - 1) / a * a;
}

/* ------------------------------------------------- wrapper record types -- */

/* Leaf types of the record that a wrapper mapping hands to its inner mapping.
 * Bytesplit (Sec. 3): every leaf becomes size-of-leaf u8 leaves, in leaf
 * order, byte j of a leaf being its j-th byte in little-endian order.
 * ChangeType (Sec. 3): a leaf whose type is some from[k] becomes to[k].
 * Returns the number of inner leaves, or -1. */
static int inner_types(const int32_t* types, int32_t nf, const orc_mapping* m,
                       int32_t* out)
{
    int count = 0;
    if (m->kind == ORC_BYTESPLIT) {
        for (int f = 0; f < nf; ++f) {
            int s = orc_type_size(types[f]);
            for (int j = 0; j < s; ++j) {
                if (count >= MAX_LEAVES) return -1;
                out[count++] = ORC_U8;
            }
        }
        return count;
    }
    if (m->kind == ORC_CHANGETYPE) {
        for (int f = 0; f < nf; ++f) {
            int32_t t = types[f];
            for (int k = 0; k < m->n_ct; ++k)
                if (m->ct_from[k] == t) { t = m->ct_to[k]; break; }
            out[count++] = t;
        }
        return count;
    }
    return -1;
}

/* Split (with Null, Sec. 3): the leaves whose bit is set in split_mask form,
 * in leaf order, the record of `inner`; the others that of `inner2`.  The
 * blobs of `inner` come first, then those of `inner2`. */
static void split_types(const int32_t* types, int32_t nf, const orc_mapping* m, int32_t* t0, int* n0,
                        int32_t* t1, int* n1)
{
    *n0 = *n1 = 0;
    for (int f = 0; f < nf; ++f) {
        if ((m->split_mask >> f) & 1u) t0[(*n0)++] = types[f];
        else t1[(*n1)++] = types[f];
    }
}

/* Part (0: inner, 1: inner2) of leaf f and its index in that part's record. */
static int split_index(const orc_mapping* m, int32_t f, int* part)
{
    const int sel = (int)((m->split_mask >> f) & 1u);
    int idx = 0;
    for (int g = 0; g < f; ++g)
        if ((int)((m->split_mask >> g) & 1u) == sel) ++idx;
    *part = sel ? 0 : 1;
    return idx;
}

/* Index of the first inner leaf that Bytesplit makes from leaf f. */
static int bytesplit_first(const int32_t* types, int32_t f)
{
    int first = 0;
    for (int g = 0; g < f; ++g) first += orc_type_size(types[g]);
    return first;
}

static int leaf_bits(const orc_mapping* m, int32_t f)
{
    return m->field_bits ? m->field_bits[f] : m->bits;
}

static void leaf_float(const orc_mapping* m, int32_t f, int* e, int* man)
{
    *e = m->field_exp ? m->field_exp[f] : m->exp_bits;
    *man = m->field_man ? m->field_man[f] : m->man_bits;
}

/* Width in bits of leaf f's code in a bit-packed mapping. */
static int code_width(const orc_mapping* m, int32_t f)
{
    if (m->kind == ORC_BITPACK_INT) return leaf_bits(m, f);
    int e = 0, man = 0;
    leaf_float(m, f, &e, &man);
    return 1 + e + man;
}

/* Where the code of leaf f of record i lies in a bit-packed mapping; returns
 * the blob, *bit its first bit.  bit_lanes == 0 (Sec. 3, SoA): blob f holds
 * leaf f's codes back to back.  bit_lanes == L: one blob of blocks of L
 * records; with R the bits of one record's codes, block i / L starts at bit
 * (i / L) L R and holds the L codes of leaf 0, then the L codes of leaf 1,
 * and so on; record i is lane i % L of its block. */
static int32_t bits_locate(int32_t nf, const orc_mapping* m, uint64_t i, int32_t f, uint64_t* bit)
{
    const uint64_t w = (uint64_t)code_width(m, f);
    if (m->bit_lanes == 0) {
        *bit = i * w;
        return f;
    }
    uint64_t R = 0, prefix = 0;
    for (int32_t g = 0; g < nf; ++g) {
        if (g == f) prefix = R;
        R += (uint64_t)code_width(m, g);
    }
    const uint64_t L = m->bit_lanes;
    *bit = (i / L) * L * R + L * prefix + (i % L) * w;
    return 0;
}

/* --------------------------------------------------------------- checks -- */

int orc_check(const int32_t* types, int32_t nf, const orc_mapping* m)
{
    if (!m || nf < 1 || nf > MAX_LEAVES) return 1;
    for (int f = 0; f < nf; ++f)
        if (orc_type_size(types[f]) == 0) return 2;
    switch (m->kind) {
    case ORC_AOS: case ORC_SOA_MB:
        return 0;
    case ORC_SOA_SB:
        if (m->subarray_align & (m->subarray_align - 1)) return 3;
        return 0;
    case ORC_AOSOA:
        return m->lanes >= 1 ? 0 : 3;
    case ORC_BITPACK_INT:
        /* Sec. 3: a bit count for integral leaves only. */
        for (int f = 0; f < nf; ++f) {
            int b = leaf_bits(m, f);
            if (!is_int(types[f])) return 4;
            if (b < 1 || b > 8 * orc_type_size(types[f])) return 5;
        }
        return 0;
    case ORC_BITPACK_FLOAT:
        /* Sec. 3: exponent and mantissa bits for floating-point leaves.
         * M >= 1 keeps NaN apart from INF; E >= 2 leaves a finite range. */
        for (int f = 0; f < nf; ++f) {
            int e = 0, man = 0, te = 0, tm = 0;
            leaf_float(m, f, &e, &man);
            if (!float_format(types[f], &te, &tm)) return 4;
            if (e < 2 || e > 11 || man < 1 || man > 52 || 1 + e + man > 64) return 5;
        }
        return 0;
    case ORC_BYTESPLIT: case ORC_CHANGETYPE: {
        int32_t it[MAX_LEAVES];
        if (!m->inner) return 6;
        if (m->kind == ORC_CHANGETYPE) {
            if (m->n_ct < 0 || m->n_ct > ORC_MAX_CT) return 7;
            for (int k = 0; k < m->n_ct; ++k) {
                int e, man;
                if (!float_format(m->ct_from[k], &e, &man)) return 7;
                if (!float_format(m->ct_to[k], &e, &man)) return 7;
            }
        }
        int n = inner_types(types, nf, m, it);
        if (n < 0) return 8;
        return orc_check(it, n, m->inner);
    }
    case ORC_NULL:
        return 0;
    case ORC_SPLIT: {
        int32_t t0[MAX_LEAVES], t1[MAX_LEAVES];
        int n0, n1, r;
        if (!m->inner || !m->inner2) return 6;
        if (nf < 64 && (m->split_mask >> nf) != 0) return 10;  /* selects no leaf beyond the record */
        split_types(types, nf, m, t0, &n0, t1, &n1);
        if (n0 == 0 || n1 == 0) return 10;                      /* both parts hold leaves */
        r = orc_check(t0, n0, m->inner);
        return r ? r : orc_check(t1, n1, m->inner2);
    }
    default:
        return 9;
    }
}

/* ------------------------------------------------------ affine mappings -- */

/* Byte offset of leaf f inside one record.  Aligned: C struct rules, each
 * leaf aligned to its own size.  Packed: leaves back to back. */
static uint64_t record_offset(const int32_t* types, int32_t f, int packed)
{
    uint64_t off = 0;
    for (int g = 0; g <= f; ++g) {
        uint64_t s = orc_type_size(types[g]);
        if (!packed) off = align_up(off, s);
        if (g == f) return off;
        off += s;
    }
    return off;
}

/* Bytes per record; aligned records are padded to the largest alignment. */
static uint64_t record_size(const int32_t* types, int32_t nf, int packed)
{
    uint64_t off = 0, max_align = 1;
    for (int g = 0; g < nf; ++g) {
        uint64_t s = orc_type_size(types[g]);
        if (!packed) off = align_up(off, s);
        off += s;
        if (s > max_align) max_align = s;
    }
    return packed ? off : align_up(off, max_align);
}

/* Start of leaf f's sub-array in the single SoA blob: the sub-arrays follow
 * each other in leaf order, each starting at a multiple of its alignment. */
static uint64_t soa_sb_base(const int32_t* types, int32_t f, uint64_t n,
                            uint64_t subarray_align)
{
    uint64_t base = 0;
    for (int g = 0; g <= f; ++g) {
        uint64_t s = orc_type_size(types[g]);
        uint64_t a = subarray_align ? subarray_align : s;
        base = align_up(base, a);
        if (g == f) return base;
        base += n * s;
    }
    return base;
}

/* Blob and byte offset of leaf f of record i in an affine mapping. */
static int affine_locate(const int32_t* types, int32_t nf, const orc_mapping* m,
                         uint64_t n, uint64_t i, int32_t f, uint64_t* off)
{
    uint64_t s = orc_type_size(types[f]);
    switch (m->kind) {
    case ORC_AOS:
        *off = i * record_size(types, nf, m->aos_packed)
             + record_offset(types, f, m->aos_packed);
        return 0;
    case ORC_SOA_MB:
        *off = i * s;
        return f;
    case ORC_SOA_SB:
        *off = soa_sb_base(types, f, n, m->subarray_align) + i * s;
        return 0;
    case ORC_AOSOA: {
        uint64_t lanes = m->lanes;
        uint64_t block = i / lanes, lane = i % lanes;
        *off = block * lanes * record_size(types, nf, 1)
             + lanes * record_offset(types, f, 1) + lane * s;
        return 0;
    }
    default:
        return -1;
    }
}

/* ---------------------------------------------------------- bit streams -- */

/* Bit k of a stream is bit (k mod 8) of byte floor(k / 8): LSB first.  This
 * equals LSB-first packing into little-endian words of any width. */
static uint64_t stream_get(const uint8_t* blob, uint64_t start, int w)
{
    uint64_t v = 0;
    for (int t = 0; t < w; ++t) {
        uint64_t k = start + (uint64_t)t;
        uint64_t bit = (blob[k >> 3] >> (k & 7)) & 1u;
        v |= bit << t;
    }
    return v;
}

static void stream_put(uint8_t* blob, uint64_t start, int w, uint64_t v)
{
    for (int t = 0; t < w; ++t) {
        uint64_t k = start + (uint64_t)t;
        uint8_t mask = (uint8_t)(1u << (k & 7));
        if ((v >> t) & 1u) blob[k >> 3] |= mask;
        else blob[k >> 3] &= (uint8_t)~mask;
    }
}

static uint64_t read_le(const uint8_t* p, int s)
{
    uint64_t v = 0;
    for (int j = 0; j < s; ++j) v |= (uint64_t)p[j] << (8 * j);
    return v;
}

static void write_le(uint8_t* p, int s, uint64_t v)
{
    for (int j = 0; j < s; ++j) p[j] = (uint8_t)(v >> (8 * j));
}

/* ---------------------------------------------------------- blob sizes -- */

int32_t orc_blob_count(const int32_t* types, int32_t nf, const orc_mapping* m)
{
    switch (m->kind) {
    case ORC_AOS: case ORC_SOA_SB: case ORC_AOSOA:
        return 1;
    case ORC_SOA_MB:
        return nf;
    case ORC_BITPACK_INT: case ORC_BITPACK_FLOAT:
        return m->bit_lanes ? 1 : nf;
    case ORC_BYTESPLIT: case ORC_CHANGETYPE: {
        int32_t it[MAX_LEAVES];
        int ni = inner_types(types, nf, m, it);
        return ni < 0 ? 0 : orc_blob_count(it, ni, m->inner);
    }
    case ORC_NULL:
        return 0;
    case ORC_SPLIT: {
        int32_t t0[MAX_LEAVES], t1[MAX_LEAVES];
        int n0, n1;
        split_types(types, nf, m, t0, &n0, t1, &n1);
        return orc_blob_count(t0, n0, m->inner) + orc_blob_count(t1, n1, m->inner2);
    }
    default:
        return 0;
    }
}

uint64_t orc_blob_size(const int32_t* types, int32_t nf, const orc_mapping* m,
                       uint64_t n, int32_t k)
{
    switch (m->kind) {
    case ORC_AOS:
        return n * record_size(types, nf, m->aos_packed);
    case ORC_SOA_MB:
        return n * (uint64_t)orc_type_size(types[k]);
    case ORC_SOA_SB:
        return soa_sb_base(types, nf - 1, n, m->subarray_align)
             + n * (uint64_t)orc_type_size(types[nf - 1]);
    case ORC_AOSOA: {
        uint64_t blocks = (n + m->lanes - 1) / m->lanes;
        return blocks * m->lanes * record_size(types, nf, 1);
    }
    case ORC_BITPACK_INT: case ORC_BITPACK_FLOAT: {
        /* whole 32-bit words; bits after the last value are zero */
        if (m->bit_lanes) {
            uint64_t R = 0;
            for (int32_t g = 0; g < nf; ++g) R += (uint64_t)code_width(m, g);
            const uint64_t blocks = (n + m->bit_lanes - 1) / m->bit_lanes;
            return 4 * ((blocks * m->bit_lanes * R + 31) / 32);
        }
        return 4 * ((n * (uint64_t)code_width(m, k) + 31) / 32);
    }
    case ORC_BYTESPLIT: case ORC_CHANGETYPE: {
        int32_t it[MAX_LEAVES];
        int ni = inner_types(types, nf, m, it);
        return orc_blob_size(it, ni, m->inner, n, k);
    }
    case ORC_SPLIT: {
        int32_t t0[MAX_LEAVES], t1[MAX_LEAVES];
        int n0, n1;
        split_types(types, nf, m, t0, &n0, t1, &n1);
        const int32_t b0 = orc_blob_count(t0, n0, m->inner);
        return k < b0 ? orc_blob_size(t0, n0, m->inner, n, k) : orc_blob_size(t1, n1, m->inner2, n, k - b0);
    }
    default:
        return 0;
    }
}

/* ---------------------------------------------------- float conversion -- */

static int msb_index(uint64_t x)
{
    int p = -1;
    while (x) { ++p; x >>= 1; }
    return p;
}

/* Round-to-nearest, ties-to-even conversion between binary formats with a
 * sign bit, `e` exponent bits (bias 2^(e-1)-1, all-ones exponent for INF and
 * NaN) and `m` stored mantissa bits.  Sec. 3 asks that floating-point
 * semantics be kept as well as possible, NaN and INF included, and that values
 * overflowing the packed format become INF; the rounding mode is not stated,
 * RNE (the IEEE default) is taken.  Steps:
 *   1 decode sign, exponent field and mantissa;
 *   2 all-ones exponent: INF stays INF; NaN keeps its sign and the top bits
 *     of its payload, with the top mantissa bit set (quiet);
 *   3 zero stays (signed) zero;
 *   4 otherwise the exact value is sig * 2^x;
 *   5 its unbiased exponent ev follows from the top bit of sig;
 *   6 the quantum q of the result is ev - M for normal results and
 *     emin - M below the normal range (gradual underflow);
 *   7 sig is scaled to that quantum, rounding to nearest, ties to even;
 *   8 the code is (biased exponent, fraction), a rounding carry running into
 *     the exponent;
 *   9 an exponent that reaches all ones means overflow: INF. */
uint64_t orc_convert(uint64_t x, int32_t src_e, int32_t src_m,
                     int32_t dst_e, int32_t dst_m)
{
    /* step 1 */
    uint64_t sign = (x >> (src_e + src_m)) & 1u;
    uint64_t e = (x >> src_m) & low_mask(src_e);
    uint64_t man = x & low_mask(src_m);
    uint64_t out_sign = sign << (dst_e + dst_m);
    uint64_t out_inf = low_mask(dst_e) << dst_m;

    /* step 2 */
    if (e == low_mask(src_e)) {
        if (man == 0) return out_sign | out_inf;
        uint64_t payload = dst_m >= src_m ? man << (dst_m - src_m)
                                          : man >> (src_m - dst_m);
        payload |= (uint64_t)1 << (dst_m - 1);
        return out_sign | out_inf | payload;
    }
    /* step 3 */
    if (e == 0 && man == 0) return out_sign;

    /* step 4 */
    int64_t src_bias = ((int64_t)1 << (src_e - 1)) - 1;
    uint64_t sig;
    int64_t xe;
    if (e != 0) {
        sig = ((uint64_t)1 << src_m) | man;
        xe = (int64_t)e - src_bias - src_m;
    } else {
        sig = man;
        xe = 1 - src_bias - src_m;
    }

    /* step 5 */
    int64_t ev = xe + msb_index(sig);
    int64_t dst_bias = ((int64_t)1 << (dst_e - 1)) - 1;
    int64_t emin = 1 - dst_bias;

    /* step 6 */
    int64_t q = ev >= emin ? ev - dst_m : emin - dst_m;

    /* step 7: scaled = sig * 2^(xe - q) */
    int64_t shift = q - xe;
    uint64_t r;
    if (shift <= 0) {
        r = sig << (-shift);
    } else if (shift >= 64) {
        r = 0; /* sig < 2^63 <= half a quantum */
    } else {
        uint64_t rem = sig & low_mask((int)shift);
        uint64_t half = (uint64_t)1 << (shift - 1);
        r = sig >> shift;
        if (rem > half || (rem == half && (r & 1u))) r += 1;
    }

    /* step 8: r holds the implicit bit for normal results, so adding it to
     * (biased - 1) << M lands on (biased << M) + fraction, and a rounding
     * carry to 2^(M+1) moves on to the next exponent by itself. */
    uint64_t code;
    if (ev >= emin) {
        uint64_t biased = (uint64_t)(ev + dst_bias);
        code = ((biased - 1) << dst_m) + r;
    } else {
        code = r; /* subnormal; a carry to 2^M is the smallest normal */
    }

    /* step 9 */
    if ((code >> dst_m) >= low_mask(dst_e)) return out_sign | out_inf;
    return out_sign | code;
}

/* ---------------------------------------------------------- load/store -- */

uint64_t orc_load(const int32_t* types, int32_t nf, const orc_mapping* m, uint64_t n,
                  uint8_t* const* blobs, uint64_t i, int32_t f)
{
    int32_t t = types[f];
    int s = orc_type_size(t);
    switch (m->kind) {
    case ORC_AOS: case ORC_SOA_SB: case ORC_SOA_MB: case ORC_AOSOA: {
        uint64_t off;
        int b = affine_locate(types, nf, m, n, i, f, &off);
        return read_le(blobs[b] + off, s);
    }
    case ORC_BITPACK_INT: {
        /* Sec. 3: unpacked when loaded.  Signed leaves are sign-extended from
         * bit b-1 (reading of the paper, which gives no sign rule). */
        int w = leaf_bits(m, f);
        uint64_t bit;
        int32_t b = bits_locate(nf, m, i, f, &bit);
        uint64_t code = stream_get(blobs[b], bit, w);
        if (is_signed_int(t) && ((code >> (w - 1)) & 1u)) code |= ~low_mask(w);
        return code & low_mask(8 * s);
    }
    case ORC_BITPACK_FLOAT: {
        int e = 0, man = 0, te = 0, tm = 0;
        leaf_float(m, f, &e, &man);
        float_format(t, &te, &tm);
        int w = 1 + e + man;
        uint64_t bit;
        int32_t b = bits_locate(nf, m, i, f, &bit);
        uint64_t code = stream_get(blobs[b], bit, w);
        return orc_convert(code, e, man, te, tm);
    }
    case ORC_BYTESPLIT: {
        int32_t it[MAX_LEAVES];
        int ni = inner_types(types, nf, m, it);
        int first = bytesplit_first(types, f);
        uint64_t v = 0;
        for (int j = 0; j < s; ++j) {
            uint64_t byte = orc_load(it, ni, m->inner, n, blobs, i, first + j);
            v |= (byte & 0xffu) << (8 * j);
        }
        return v;
    }
    case ORC_CHANGETYPE: {
        int32_t it[MAX_LEAVES];
        int ni = inner_types(types, nf, m, it);
        uint64_t u = orc_load(it, ni, m->inner, n, blobs, i, f);
        if (it[f] == t) return u;
        int ue = 0, um = 0, te = 0, tm = 0;
        float_format(it[f], &ue, &um);
        float_format(t, &te, &tm);
        return orc_convert(u, ue, um, te, tm);
    }
    case ORC_NULL:
        return 0;  /* Sec. 3: a default-constructed value */
    case ORC_SPLIT: {
        int32_t t0[MAX_LEAVES], t1[MAX_LEAVES];
        int n0, n1, part;
        split_types(types, nf, m, t0, &n0, t1, &n1);
        const int idx = split_index(m, f, &part);
        if (part == 0) return orc_load(t0, n0, m->inner, n, blobs, i, idx);
        return orc_load(t1, n1, m->inner2, n, blobs + orc_blob_count(t0, n0, m->inner), i, idx);
    }
    default:
        return 0;
    }
}

void orc_store(const int32_t* types, int32_t nf, const orc_mapping* m, uint64_t n,
               uint8_t* const* blobs, uint64_t i, int32_t f, uint64_t v)
{
    int32_t t = types[f];
    int s = orc_type_size(t);
    switch (m->kind) {
    case ORC_AOS: case ORC_SOA_SB: case ORC_SOA_MB: case ORC_AOSOA: {
        uint64_t off;
        int b = affine_locate(types, nf, m, n, i, f, &off);
        write_le(blobs[b] + off, s, v);
        return;
    }
    case ORC_BITPACK_INT: {
        /* Sec. 3: packed when stored: the low b bits of the two's-complement
         * value, i.e. v mod 2^b (wrap-around, no saturation). */
        int w = leaf_bits(m, f);
        uint64_t bit;
        int32_t b = bits_locate(nf, m, i, f, &bit);
        stream_put(blobs[b], bit, w, v & low_mask(w));
        return;
    }
    case ORC_BITPACK_FLOAT: {
        int e = 0, man = 0, te = 0, tm = 0;
        leaf_float(m, f, &e, &man);
        float_format(t, &te, &tm);
        int w = 1 + e + man;
        uint64_t bit;
        int32_t b = bits_locate(nf, m, i, f, &bit);
        stream_put(blobs[b], bit, w, orc_convert(v, te, tm, e, man));
        return;
    }
    case ORC_BYTESPLIT: {
        int32_t it[MAX_LEAVES];
        int ni = inner_types(types, nf, m, it);
        int first = bytesplit_first(types, f);
        for (int j = 0; j < s; ++j)
            orc_store(it, ni, m->inner, n, blobs, i, first + j, (v >> (8 * j)) & 0xffu);
        return;
    }
    case ORC_CHANGETYPE: {
        int32_t it[MAX_LEAVES];
        int ni = inner_types(types, nf, m, it);
        uint64_t u = v;
        if (it[f] != t) {
            int ue = 0, um = 0, te = 0, tm = 0;
            float_format(it[f], &ue, &um);
            float_format(t, &te, &tm);
            u = orc_convert(v, te, tm, ue, um);
        }
        orc_store(it, ni, m->inner, n, blobs, i, f, u);
        return;
    }
    case ORC_NULL:
        return;  /* Sec. 3: writes are discarded */
    case ORC_SPLIT: {
        int32_t t0[MAX_LEAVES], t1[MAX_LEAVES];
        int n0, n1, part;
        split_types(types, nf, m, t0, &n0, t1, &n1);
        const int idx = split_index(m, f, &part);
        if (part == 0) orc_store(t0, n0, m->inner, n, blobs, i, idx, v);
        else orc_store(t1, n1, m->inner2, n, blobs + orc_blob_count(t0, n0, m->inner), i, idx, v);
        return;
    }
    default:
        return;
    }
}

void orc_load_field(const int32_t* types, int32_t nf, const orc_mapping* m, uint64_t n,
                    uint8_t* const* blobs, int32_t f, uint64_t i0, uint64_t i1,
                    uint64_t* out)
{
    for (uint64_t i = i0; i < i1; ++i)
        out[i - i0] = orc_load(types, nf, m, n, blobs, i, f);
}

void orc_store_field(const int32_t* types, int32_t nf, const orc_mapping* m, uint64_t n,
                     uint8_t* const* blobs, int32_t f, uint64_t i0, uint64_t i1,
                     const uint64_t* in)
{
    for (uint64_t i = i0; i < i1; ++i)
        orc_store(types, nf, m, n, blobs, i, f, in[i - i0]);
}

void orc_convert_n(const uint64_t* in, uint64_t* out, uint64_t count,
                   int32_t src_e, int32_t src_m, int32_t dst_e, int32_t dst_m)
{
    for (uint64_t k = 0; k < count; ++k)
        out[k] = orc_convert(in[k], src_e, src_m, dst_e, dst_m);
}

/* ----------------------------------------------------------------- copy -- */

void orc_copy_range(const int32_t* types, int32_t nf, uint64_t n,
                    const orc_mapping* src_m, uint8_t* const* src_blobs,
                    const orc_mapping* dst_m, uint8_t* const* dst_blobs,
                    uint64_t i0, uint64_t i1)
{
    for (uint64_t i = i0; i < i1; ++i)
        for (int32_t f = 0; f < nf; ++f)
            orc_store(types, nf, dst_m, n, dst_blobs, i, f,
                      orc_load(types, nf, src_m, n, src_blobs, i, f));
}

/* Layout-aware copy (Sec. 1): the logical value of every leaf of every record
 * moves from the source mapping to the destination mapping.  Bytes of the
 * destination that belong to no leaf (struct padding, AoSoA lanes past n,
 * bits after the last packed value) end up zero. */
void orc_copy(const int32_t* types, int32_t nf, uint64_t n,
              const orc_mapping* src_m, uint8_t* const* src_blobs,
              const orc_mapping* dst_m, uint8_t* const* dst_blobs)
{
    int32_t nb = orc_blob_count(types, nf, dst_m);
    for (int32_t k = 0; k < nb; ++k)
        memset(dst_blobs[k], 0, (size_t)orc_blob_size(types, nf, dst_m, n, k));
    orc_copy_range(types, nf, n, src_m, src_blobs, dst_m, dst_blobs, 0, n);
}

/* --------------------------------------------------------------- n-body -- */

static double f32_bits_to_double(uint64_t bits)
{
    uint32_t u = (uint32_t)bits;
    float x;
    memcpy(&x, &u, sizeof x);
    return (double)x;
}

/* All-pairs n-body update and move (Sec. 5, Fig. 2; the interaction is the
 * softened Newtonian one with G = 1):
 *   a_i = sum_j m_j (p_j - p_i) / (|p_j - p_i|^2 + eps^2)^(3/2)
 *   v_i' = v_i + dt a_i;   p_i' = p_i + dt v_i'.
 * j runs over every particle, i included (its term is zero). */
void orc_nbody_step(const orc_mapping* m, uint64_t n, uint8_t* const* blobs,
                    double eps, double dt, uint64_t i0, uint64_t i1,
                    double* pos_out, double* vel_out)
{
    static const int32_t types[7] = {ORC_F32, ORC_F32, ORC_F32, ORC_F32,
                                     ORC_F32, ORC_F32, ORC_F32};
    double* pos = (double*)malloc(sizeof(double) * 3 * (n ? n : 1));
    double* mass = (double*)malloc(sizeof(double) * (n ? n : 1));
    for (uint64_t j = 0; j < n; ++j) {
        for (int k = 0; k < 3; ++k)
            pos[3 * j + k] = f32_bits_to_double(orc_load(types, 7, m, n, blobs, j, k));
        mass[j] = f32_bits_to_double(orc_load(types, 7, m, n, blobs, j, 6));
    }
    for (uint64_t i = i0; i < i1; ++i) {
        double a[3] = {0.0, 0.0, 0.0};
        for (uint64_t j = 0; j < n; ++j) {
            double d[3];
            for (int k = 0; k < 3; ++k) d[k] = pos[3 * j + k] - pos[3 * i + k];
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + eps * eps;
            double inv_r3 = 1.0 / (r2 * sqrt(r2));
            for (int k = 0; k < 3; ++k) a[k] += mass[j] * inv_r3 * d[k];
        }
        for (int k = 0; k < 3; ++k) {
            double v = f32_bits_to_double(orc_load(types, 7, m, n, blobs, i, 3 + k));
            double v_new = v + dt * a[k];
            vel_out[3 * (i - i0) + k] = v_new;
            pos_out[3 * (i - i0) + k] = pos[3 * i + k] + dt * v_new;
        }
    }
    free(pos);
    free(mass);
}

void orc_nbody_move(const orc_mapping* m, uint64_t n, uint8_t* const* blobs,
                    double dt, uint64_t i0, uint64_t i1, double* pos_out)
{
    static const int32_t types[7] = {ORC_F32, ORC_F32, ORC_F32, ORC_F32,
                                     ORC_F32, ORC_F32, ORC_F32};
    for (uint64_t i = i0; i < i1; ++i)
        for (int k = 0; k < 3; ++k) {
            const double p = f32_bits_to_double(orc_load(types, 7, m, n, blobs, i, k));
            const double v = f32_bits_to_double(orc_load(types, 7, m, n, blobs, i, 3 + k));
            pos_out[3 * (i - i0) + k] = p + dt * v;
        }
}

/* ------------------------------------------- access instrumentation -- */

void orc_nbody_access_counts(uint64_t n, uint64_t block, uint64_t* counts)
{
    const uint64_t blocks = n == 0 ? 0 : (n + block - 1) / block;
    for (int k = 0; k < 14; ++k) counts[k] = 0;
    /* reads: own positions (update), every record's position and mass once
     * per block (update), positions again (move) */
    for (int f = 0; f < 3; ++f) counts[f] = n + blocks * n + n;
    /* velocities: read in the update and in the move */
    for (int f = 3; f < 6; ++f) counts[f] = 2 * n;
    counts[6] = blocks * n;
    /* writes: velocities (update), positions (move) */
    for (int f = 0; f < 6; ++f) counts[7 + f] = n;
}

void orc_nbody_heatmap(const orc_mapping* m, uint64_t n, uint64_t block, uint64_t g, uint64_t* heat)
{
    static const int32_t types[7] = {ORC_F32, ORC_F32, ORC_F32, ORC_F32,
                                     ORC_F32, ORC_F32, ORC_F32};
    uint64_t counts[14], start[8] = {0};
    orc_nbody_access_counts(n, block, counts);
    const int32_t nb = orc_blob_count(types, 7, m);
    for (int32_t b = 0; b < nb; ++b) start[b + 1] = start[b] + (orc_blob_size(types, 7, m, n, b) + g - 1) / g;
    for (uint64_t k = 0; k < start[nb]; ++k) heat[k] = 0;
    for (uint64_t i = 0; i < n; ++i) {
        for (int32_t f = 0; f < 7; ++f) {
            uint64_t off = 0;
            const int b = affine_locate(types, 7, m, n, i, f, &off);
            if (b < 0) return;
            const uint64_t acc = counts[f] / n + counts[7 + f] / n; /* per element */
            for (uint64_t k = off / g; k <= (off + 3) / g; ++k) heat[start[b] + k] += acc;
        }
    }
}

