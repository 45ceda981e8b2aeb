/*
 * llgb_oracle.h -- plain, slow CPU oracle for mapping-driven record layouts.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this code; only the test suite, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no source with the CUDA library.
 *
 * What it computes (arXiv 2302.08251, "Updates on the Low-Level Abstraction of
 * Memory Access"):
 *   - a record dimension of leaf fields, flattened depth-first (Sec. 1, Fig. 1);
 *   - a linear array of n records (extents are linearised row-major before
 *     they reach the oracle, Sec. 2);
 *   - the mappings AoS, SoA single/multi blob, AoSoA<L> (Sec. 5, Fig. 3 text),
 *     BitpackIntSoA and BitpackFloatSoA (Sec. 3), also organised as AoSoA
 *     (the generalisation Sec. 3 announces), ChangeType (Sec. 3) and
 *     Bytesplit (Sec. 3);
 *   - the layout-aware copy (Sec. 1): every field of every record is loaded
 *     through the source mapping and stored through the destination mapping;
 *     every destination byte that no field owns is zero;
 *   - one all-pairs n-body step (Sec. 5, Fig. 2) in double precision, reading
 *     the particle records through a mapping, and its move phase alone.
 *
 * Values cross the API as uint64_t holding the little-endian bit pattern of
 * the field's own type, zero-extended to 64 bits.
 */
#ifndef LLGB_ORACLE_H
#define LLGB_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Leaf types. */
enum {
    ORC_U8 = 0, ORC_U16, ORC_U32, ORC_U64,
    ORC_I8, ORC_I16, ORC_I32, ORC_I64,
    ORC_F16, ORC_BF16, ORC_F32, ORC_F64,
    ORC_NTYPES
};

/* Mapping kinds. */
enum {
    ORC_AOS = 0,          /* array of structs; aligned (C struct rules) or packed */
    ORC_SOA_SB,           /* struct of arrays, one blob                            */
    ORC_SOA_MB,           /* struct of arrays, one blob per leaf                   */
    ORC_AOSOA,            /* arrays of structs of arrays, L lanes per block        */
    ORC_BITPACK_INT,      /* b-bit integers, one bit stream per leaf               */
    ORC_BITPACK_FLOAT,    /* (1+E+M)-bit floats, one bit stream per leaf           */
    ORC_BYTESPLIT,        /* each leaf split into bytes, forwarded to `inner`      */
    ORC_CHANGETYPE,       /* leaves of type from[k] stored as to[k] via `inner`    */
    ORC_NULL,             /* no storage: loads give 0, stores are discarded        */
    ORC_SPLIT             /* leaves in split_mask via `inner`, the rest via `inner2` */
};

#define ORC_MAX_CT 4

typedef struct orc_mapping {
    int32_t kind;
    int32_t aos_packed;          /* AoS: 0 = aligned, 1 = packed                   */
    uint64_t subarray_align;     /* SoA single blob: 0 = each leaf's own alignment */
    uint64_t lanes;              /* AoSoA: lanes per block (>= 1)                  */
    int32_t bits;                /* BitpackInt: bits per value, all leaves         */
    int32_t exp_bits;            /* BitpackFloat: exponent bits, all leaves        */
    int32_t man_bits;            /* BitpackFloat: mantissa bits, all leaves        */
    int32_t n_ct;                /* ChangeType: number of (from, to) pairs         */
    int32_t ct_from[ORC_MAX_CT];
    int32_t ct_to[ORC_MAX_CT];
    const int32_t* field_bits;   /* optional per-leaf override of `bits`           */
    const int32_t* field_exp;    /* optional per-leaf override of `exp_bits`       */
    const int32_t* field_man;    /* optional per-leaf override of `man_bits`       */
    const struct orc_mapping* inner; /* Bytesplit / ChangeType inner mapping; Split:
                                        mapping of the selected leaves            */
    uint64_t split_mask;         /* Split: bit f set = leaf f is selected          */
    const struct orc_mapping* inner2; /* Split: mapping of the other leaves        */
    uint64_t bit_lanes;          /* Bitpack*: 0 = one stream per leaf (SoA);
                                    L >= 1 = one blob of blocks of L records,
                                    each leaf's L codes in turn (AoSoA)        */
} orc_mapping;

/* Size in bytes of a leaf type; 0 for an unknown type. */
int orc_type_size(int32_t type);

/* Returns 0 when the mapping can hold the record, else a nonzero code. */
int orc_check(const int32_t* types, int32_t nf, const orc_mapping* m);

/* Number of blobs and the byte size of blob k for n records. */
int32_t orc_blob_count(const int32_t* types, int32_t nf, const orc_mapping* m);
uint64_t orc_blob_size(const int32_t* types, int32_t nf, const orc_mapping* m,
                       uint64_t n, int32_t k);

/* Load / store leaf f of record i through the mapping. */
uint64_t orc_load(const int32_t* types, int32_t nf, const orc_mapping* m, uint64_t n,
                  uint8_t* const* blobs, uint64_t i, int32_t f);
void orc_store(const int32_t* types, int32_t nf, const orc_mapping* m, uint64_t n,
               uint8_t* const* blobs, uint64_t i, int32_t f, uint64_t v);

/* Array forms of load / store / convert, for tests that touch many values:
 * out[k] = orc_load(..., i0 + k, f) for k < i1 - i0, and so on. */
void orc_load_field(const int32_t* types, int32_t nf, const orc_mapping* m, uint64_t n,
                    uint8_t* const* blobs, int32_t f, uint64_t i0, uint64_t i1,
                    uint64_t* out);
void orc_store_field(const int32_t* types, int32_t nf, const orc_mapping* m, uint64_t n,
                     uint8_t* const* blobs, int32_t f, uint64_t i0, uint64_t i1,
                     const uint64_t* in);
void orc_convert_n(const uint64_t* in, uint64_t* out, uint64_t count,
                   int32_t src_e, int32_t src_m, int32_t dst_e, int32_t dst_m);

/* Layout-aware copy of records [0, n): destination blobs are zeroed, then
 * every leaf of every record is loaded from src and stored into dst. */
void orc_copy(const int32_t* types, int32_t nf, uint64_t n,
              const orc_mapping* src_m, uint8_t* const* src_blobs,
              const orc_mapping* dst_m, uint8_t* const* dst_blobs);

/* Same as orc_copy restricted to records [i0, i1) and without zeroing; used to
 * time a bounded sample of a large copy. */
void orc_copy_range(const int32_t* types, int32_t nf, uint64_t n,
                    const orc_mapping* src_m, uint8_t* const* src_blobs,
                    const orc_mapping* dst_m, uint8_t* const* dst_blobs,
                    uint64_t i0, uint64_t i1);

/* Round-to-nearest-even conversion between IEEE-style binary formats given by
 * (exponent bits, mantissa bits), integer arithmetic only. */
uint64_t orc_convert(uint64_t bits, int32_t src_e, int32_t src_m,
                     int32_t dst_e, int32_t dst_m);

/* One all-pairs n-body step in double precision on the particle record
 * {pos.x, pos.y, pos.z, vel.x, vel.y, vel.z, mass} (all f32) held in a view
 * with mapping m.  Velocities of records [i0, i1) are updated with the
 * softened gravity sum over all n particles, then positions move with the new
 * velocities.  Results are written as doubles (3 per record, record-major)
 * for records [i0, i1) to pos_out and vel_out; the view is not modified. */
void orc_nbody_step(const orc_mapping* m, uint64_t n, uint8_t* const* blobs,
                    double eps, double dt, uint64_t i0, uint64_t i1,
                    double* pos_out, double* vel_out);

/* The move phase alone (Sec. 5): p_i + dt v_i in double precision for the
 * records [i0, i1), from the f32 pos and vel leaves the view holds; written
 * as doubles (3 per record, record-major) to pos_out.  The view is not
 * modified. */
void orc_nbody_move(const orc_mapping* m, uint64_t n, uint8_t* const* blobs,
                    double dt, uint64_t i0, uint64_t i1, double* pos_out);

/* Access instrumentation (Sec. 4, "Memory access instrumentation"):
 * FieldAccessCount counts the accesses per record field (reads and writes
 * apart: 2 counters per field), Heatmap the accesses touching each granule
 * of g bytes of every blob.  What is counted is the access schedule of the
 * tiled n-body step the CUDA library runs on the particle record, with
 * blocks of `block` particles (B = ceil(n / block) blocks) -- one step:
 *   update: each block reads pos.x/y/z of its own particles once, pos.x/y/z
 *           and mass of every record once, and reads and writes vel.x/y/z
 *           of its own particles once;
 *   move:   every particle's pos and vel are read once and pos written once.
 * orc_nbody_access_counts writes the 14 field counters of one step (reads of
 * leaves 0..6, then writes of leaves 0..6). */
void orc_nbody_access_counts(uint64_t n, uint64_t block, uint64_t* counts);

/* Heatmap of one such step at granularity g: for every record i and leaf f,
 * the accesses of that element in the step (reads + writes) are added to the
 * counter of every granule its 4 bytes touch.  Counters of blob b follow
 * those of blobs 0 .. b-1 (ceil(blob size / g) each).  `heat` is zeroed
 * first. */
void orc_nbody_heatmap(const orc_mapping* m, uint64_t n, uint64_t block, uint64_t g, uint64_t* heat);

#ifdef __cplusplus
}
#endif

#endif
