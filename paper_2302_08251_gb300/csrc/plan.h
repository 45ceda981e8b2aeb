// plan.h -- host-side mapping address compiler.
//
// Turns a record descriptor, extents and a mapping descriptor into a view
// plan (stored leaves, per-leaf recipes, blob sizes), and a pair of view plans
// into the tile kernel's JobDesc.
#pragma once

#include <stdint.h>

#include <string>
#include <vector>

#include "job.h"
#include "llgb.h"

struct llgb_record {
    std::vector<std::string> paths;
    std::vector<int32_t> types;
};

namespace llgb {

// BASE_SPLIT: a Split (or Null) view made of parts, each an ordinary plan
// (or no storage at all).
enum BaseKind { BASE_AOS, BASE_SOA_SB, BASE_SOA_MB, BASE_AOSOA, BASE_BITS_INT, BASE_BITS_FLOAT, BASE_SPLIT };
enum WrapKind { WRAP_NONE, WRAP_CHANGETYPE, WRAP_BYTESPLIT };

// How a logical leaf reaches its stored leaves.
struct Recipe {
    int op;     // LoadOp numbering (L_DIRECT, L_CT, L_BITS_INT, L_BITS_FLOAT, L_SPLIT)
    int first;  // first stored leaf
    int count;  // stored leaves used
};

struct StoredLeaf {
    int32_t type;   // stored type (u8 for byte-split leaves)
    int size;       // bytes (affine)
    int bits;       // bits per value (bit streams)
    int e, m;       // stored float format (bit-packed floats)
};

struct ViewPlan {
    std::vector<int32_t> types;  // logical leaf types
    llgb_extents ext{};
    uint64_t n = 0;
    int wrap = WRAP_NONE;
    int base = BASE_AOS;
    int aos_packed = 0;
    uint64_t subarray_align = 0;
    uint64_t lanes = 1;
    // Bit-packed bases: 0 = SoA (one stream per leaf); L = AoSoA, one blob of
    // blocks of L records, bit_block_bytes each, leaf g's L codes at byte
    // leaf_offset[g] of its block.
    uint64_t bit_lanes = 0;
    uint64_t bit_block_bytes = 0;
    std::vector<StoredLeaf> stored;
    std::vector<Recipe> recipes;       // one per logical leaf
    std::vector<uint64_t> leaf_offset; // AoS / AoSoA: offset inside the record
    std::vector<uint64_t> sb_base;     // SoA single blob: sub-array starts
    uint64_t record_bytes = 0;         // AoS: S (aligned or packed); AoSoA: packed
    std::vector<uint64_t> blob_sizes;
    std::vector<uint64_t> seg_end;     // per stored leaf: end of its run region
    std::vector<int> leaf_blob;        // per stored leaf: blob index
    std::string sig;                   // mapping signature (record, wrapper, layout), no sizes
    // BASE_SPLIT: the parts, each over the sub-record of part_fields[k] (in
    // leaf order); a null part stores nothing.  Part k's stored leaves and
    // blobs start at part_leaf0[k] / part_blob0[k] of this plan's.
    std::vector<ViewPlan> parts;
    std::vector<std::vector<int>> part_fields;
    std::vector<bool> part_null;
    std::vector<int> part_leaf0, part_blob0;
};

int type_size(int32_t t);
bool type_is_float(int32_t t, int* e, int* m);
bool type_is_int(int32_t t);
bool type_is_signed(int32_t t);

// Returns LLGB_OK or an error code, with a message in *why.
llgb_status plan_view(const llgb_record& rec, const llgb_extents& ext, const llgb_mapping_desc& map,
                      ViewPlan* out, std::string* why);

// Tile quantum (records) of a pair: tiles must be multiples of it.
uint32_t tile_quantum(const ViewPlan& src, const ViewPlan& dst);

// Image bytes per record on each side and code staging bytes per record.
void bytes_per_record(const ViewPlan& src, const ViewPlan& dst, double* src_bpr, double* dst_bpr,
                      uint32_t* code_bpr);

// Build the JobDesc for a pair with `tile` records per tile.
llgb_status plan_job(const ViewPlan& src, const std::vector<void*>& src_ptrs, const ViewPlan& dst,
                     const std::vector<void*>& dst_ptrs, uint32_t tile, JobDesc* job, std::string* why);

}  // namespace llgb
