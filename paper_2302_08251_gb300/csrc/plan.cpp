// plan.cpp -- mapping address compiler (host).
//
// View plans follow the mappings of arXiv 2302.08251:
//   AoS / SoA multi-blob / AoSoA (Sec. 5, Fig. 3 text), SoA single blob,
//   BitpackIntSoA and BitpackFloatSoA (Sec. 3), ChangeType and Bytesplit
//   (Sec. 3) over an AoS/SoA/AoSoA inner mapping,
// with the index-type rule of Sec. 2: a view whose record count or largest
// byte offset does not fit the chosen index type is rejected.
//
// Every plain layout is one affine form per leaf,
//     offset(i, f) = base_f + (i / L) * B + (i % L) * s_f,
// and every bit-packed leaf is the stream position i * w.  A tile of T
// records (T a multiple of 128 and of every lane count) therefore covers one
// contiguous run per blob region, and inside a tile image the same affine
// form holds with 32-bit tile-local offsets.
#include "plan.h"
#include "stream_specs.h"

#include <string.h>

#include <algorithm>
#include <functional>

namespace llgb {

int type_size(int32_t t)
{
    switch (t) {
    case LLGB_U8: case LLGB_I8: return 1;
    case LLGB_U16: case LLGB_I16: case LLGB_F16: case LLGB_BF16: return 2;
    case LLGB_U32: case LLGB_I32: case LLGB_F32: return 4;
    case LLGB_U64: case LLGB_I64: case LLGB_F64: return 8;
    default: return 0;
    }
}

bool type_is_float(int32_t t, int* e, int* m)
{
    int ee = 0, mm = 0;
    switch (t) {
    case LLGB_F16: ee = 5; mm = 10; break;
    case LLGB_BF16: ee = 8; mm = 7; break;
    case LLGB_F32: ee = 8; mm = 23; break;
    case LLGB_F64: ee = 11; mm = 52; break;
    default: return false;
    }
    if (e) *e = ee;
    if (m) *m = mm;
    return true;
}

bool type_is_int(int32_t t) { return t >= LLGB_U8 && t <= LLGB_I64; }
bool type_is_signed(int32_t t) { return t >= LLGB_I8 && t <= LLGB_I64; }

static uint64_t align_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

static bool mul_ok(uint64_t a, uint64_t b, uint64_t* out) { return !__builtin_mul_overflow(a, b, out); }

static uint64_t index_max(int itype)
{
    switch (itype) {
    case LLGB_IDX_I16: return 32767ull;
    case LLGB_IDX_U16: return 65535ull;
    case LLGB_IDX_I32: return 2147483647ull;
    case LLGB_IDX_U32: return 4294967295ull;
    case LLGB_IDX_I64: return 9223372036854775807ull;
    default: return ~0ull;
    }
}

static bool is_affine_kind(int k)
{
    return k == LLGB_MAP_AOS || k == LLGB_MAP_SOA_SB || k == LLGB_MAP_SOA_MB || k == LLGB_MAP_AOSOA;
}

static bool is_bits_base(int b) { return b == BASE_BITS_INT || b == BASE_BITS_FLOAT; }

// Split and Null (Sec. 3).  Null stores nothing: its leaves load as zero and
// their stores are dropped.  Split plans the sub-record of the leaves in
// split_mask (leaf order) with `inner` and that of the others with `inner2`,
// each as an ordinary view (recursively), and lays their stored leaves and
// blobs side by side, inner's first.
static llgb_status plan_split(const llgb_record& rec, const llgb_extents& ext, const llgb_mapping_desc& map,
                              ViewPlan& v, ViewPlan* out, std::string* why)
{
    const int nf = (int)rec.types.size();
    v.base = BASE_SPLIT;
    std::vector<std::vector<int>> fields;
    std::vector<const llgb_mapping_desc*> maps;
    if (map.kind == LLGB_MAP_NULL) {
        fields.emplace_back();
        for (int f = 0; f < nf; ++f) fields.back().push_back(f);
        maps.push_back(nullptr);
    } else {
        if (!map.inner || !map.inner2) {
            *why = "Split needs `inner` and `inner2`";
            return LLGB_ERR_INVALID_ARG;
        }
        if (nf < 64 && (map.split_mask >> nf) != 0) {
            *why = "Split selects a leaf beyond the record";
            return LLGB_ERR_INVALID_ARG;
        }
        std::vector<int> sel, rest;
        for (int f = 0; f < nf; ++f) ((map.split_mask >> f) & 1u ? sel : rest).push_back(f);
        if (sel.empty() || rest.empty()) {
            *why = "Split needs leaves on both sides";
            return LLGB_ERR_INVALID_ARG;
        }
        fields = {sel, rest};
        maps = {map.inner, map.inner2};
    }
    v.recipes.assign(nf, Recipe{L_NULL, 0, 0});
    std::string sig = "split" + std::to_string(map.kind == LLGB_MAP_NULL ? 0ull : map.split_mask) + "{";
    for (size_t k = 0; k < fields.size(); ++k) {
        ViewPlan part;
        const bool null = maps[k] == nullptr || maps[k]->kind == LLGB_MAP_NULL;
        v.part_leaf0.push_back((int)v.stored.size());
        v.part_blob0.push_back((int)v.blob_sizes.size());
        if (!null) {
            llgb_record sub;
            for (int f : fields[k]) {
                sub.paths.push_back(rec.paths[f]);
                sub.types.push_back(rec.types[f]);
            }
            const llgb_status st = plan_view(sub, ext, *maps[k], &part, why);
            if (st != LLGB_OK) return st;
            const int leaf0 = v.part_leaf0.back(), blob0 = v.part_blob0.back();
            for (size_t j = 0; j < fields[k].size(); ++j) {
                Recipe r = part.recipes[j];
                if (r.op != L_NULL) r.first += leaf0;
                v.recipes[fields[k][j]] = r;
            }
            for (size_t g = 0; g < part.stored.size(); ++g) {
                v.stored.push_back(part.stored[g]);
                v.seg_end.push_back(part.seg_end[g]);
                v.leaf_blob.push_back(part.leaf_blob[g] + blob0);
                v.leaf_offset.push_back(part.leaf_offset[g]);
                v.sb_base.push_back(part.sb_base[g]);
            }
            for (uint64_t b : part.blob_sizes) v.blob_sizes.push_back(b);
            sig += part.sig;
        }
        sig += "|";
        v.parts.push_back(std::move(part));
        v.part_fields.push_back(fields[k]);
        v.part_null.push_back(null);
    }
    if ((int)v.stored.size() > kMaxLeaves) {
        *why = "more than 32 stored leaves";
        return LLGB_ERR_UNSUPPORTED;
    }
    if ((int)v.blob_sizes.size() > kMaxBlobs) {
        *why = "more than 32 blobs";
        return LLGB_ERR_UNSUPPORTED;
    }
    v.sig = sig + "}";
    *out = std::move(v);
    return LLGB_OK;
}

llgb_status plan_view(const llgb_record& rec, const llgb_extents& ext, const llgb_mapping_desc& map,
                      ViewPlan* out, std::string* why)
{
    ViewPlan v;
    v.types = rec.types;
    v.ext = ext;
    const int nf = (int)rec.types.size();

    // --- extents (Sec. 2) ---
    if (ext.rank < 1 || ext.rank > 4 || ext.reserved != 0) {
        *why = "extents: rank must be 1..4 and reserved 0";
        return LLGB_ERR_INVALID_ARG;
    }
    if (ext.index_type < LLGB_IDX_I16 || ext.index_type > LLGB_IDX_U64) {
        *why = "extents: unknown index type";
        return LLGB_ERR_INVALID_ARG;
    }
    const uint64_t imax = index_max(ext.index_type);
    uint64_t n = 1;
    for (int d = 0; d < ext.rank; ++d) {
        if (ext.ext[d] > imax) {
            *why = "extent " + std::to_string(d) + " does not fit the index type";
            return LLGB_ERR_INDEX_OVERFLOW;
        }
        if (!mul_ok(n, ext.ext[d], &n)) {
            *why = "record count overflows 64 bits";
            return LLGB_ERR_INDEX_OVERFLOW;
        }
    }
    if (n > 0 && n - 1 > imax) {
        *why = "record count " + std::to_string(n) + " does not fit the index type";
        return LLGB_ERR_INDEX_OVERFLOW;
    }
    v.n = n;
    if (map.kind == LLGB_MAP_SPLIT || map.kind == LLGB_MAP_NULL) return plan_split(rec, ext, map, v, out, why);

    // --- wrappers (Sec. 3: ChangeType, Bytesplit) ---
    const llgb_mapping_desc* base = &map;
    std::vector<int32_t> stored_types;
    if (map.kind == LLGB_MAP_BYTESPLIT || map.kind == LLGB_MAP_CHANGETYPE) {
        if (!map.inner) {
            *why = "wrapper mapping without an inner mapping";
            return LLGB_ERR_INVALID_ARG;
        }
        base = map.inner;
        if (!is_affine_kind(base->kind)) {
            *why = "the inner mapping of Bytesplit/ChangeType must be AoS, SoA or AoSoA";
            return LLGB_ERR_UNSUPPORTED;
        }
        if (map.kind == LLGB_MAP_BYTESPLIT) {
            v.wrap = WRAP_BYTESPLIT;
            for (int f = 0; f < nf; ++f) {
                const int s = type_size(rec.types[f]);
                v.recipes.push_back({L_SPLIT, (int)stored_types.size(), s});
                for (int j = 0; j < s; ++j) stored_types.push_back(LLGB_U8);
            }
        } else {
            v.wrap = WRAP_CHANGETYPE;
            if (map.n_ct < 0 || map.n_ct > LLGB_MAX_CT) {
                *why = "ChangeType: n_ct must be 0..4";
                return LLGB_ERR_INVALID_ARG;
            }
            for (int k = 0; k < map.n_ct; ++k) {
                if (!type_is_float(map.ct_from[k], nullptr, nullptr) ||
                    !type_is_float(map.ct_to[k], nullptr, nullptr)) {
                    *why = "ChangeType: only floating-point type pairs are supported";
                    return LLGB_ERR_INVALID_ARG;
                }
            }
            for (int f = 0; f < nf; ++f) {
                int32_t t = rec.types[f];
                for (int k = 0; k < map.n_ct; ++k)
                    if (map.ct_from[k] == t) {
                        t = map.ct_to[k];
                        break;
                    }
                v.recipes.push_back({t == rec.types[f] ? (int)L_DIRECT : (int)L_CT, f, 1});
                stored_types.push_back(t);
            }
        }
    } else if (is_affine_kind(map.kind)) {
        for (int f = 0; f < nf; ++f) {
            v.recipes.push_back({L_DIRECT, f, 1});
            stored_types.push_back(rec.types[f]);
        }
    } else if (map.kind == LLGB_MAP_BITPACK_INT || map.kind == LLGB_MAP_BITPACK_FLOAT) {
        stored_types = rec.types;
    } else {
        *why = "unknown mapping kind";
        return LLGB_ERR_INVALID_ARG;
    }

    // --- stored leaves ---
    const int ns = (int)stored_types.size();
    if (ns > kMaxLeaves) {
        *why = "more than 32 stored leaves";
        return LLGB_ERR_UNSUPPORTED;
    }
    v.stored.resize(ns);
    for (int g = 0; g < ns; ++g) {
        v.stored[g].type = stored_types[g];
        v.stored[g].size = type_size(stored_types[g]);
        v.stored[g].bits = 8 * v.stored[g].size;
    }

    switch (base->kind) {
    case LLGB_MAP_AOS: v.base = BASE_AOS; break;
    case LLGB_MAP_SOA_SB: v.base = BASE_SOA_SB; break;
    case LLGB_MAP_SOA_MB: v.base = BASE_SOA_MB; break;
    case LLGB_MAP_AOSOA: v.base = BASE_AOSOA; break;
    case LLGB_MAP_BITPACK_INT: v.base = BASE_BITS_INT; break;
    default: v.base = BASE_BITS_FLOAT; break;
    }
    v.aos_packed = base->aos_packed ? 1 : 0;
    v.subarray_align = base->subarray_align;
    v.lanes = v.base == BASE_AOSOA ? base->lanes : 1;
    v.bit_lanes = is_bits_base(v.base) ? base->bit_lanes : 0;
    if (v.bit_lanes && (v.bit_lanes < 32 || v.bit_lanes > 1024 || (v.bit_lanes & (v.bit_lanes - 1)))) {
        *why = "bit-packed AoSoA: bit_lanes must be a power of two from 32 to 1024";
        return LLGB_ERR_UNSUPPORTED;
    }

    if (v.base == BASE_BITS_INT) {
        // Sec. 3 BitpackIntSoA: a bit count for integral leaves.
        for (int f = 0; f < nf; ++f) {
            const int b = base->field_bits ? base->field_bits[f] : base->bits;
            if (!type_is_int(rec.types[f])) {
                *why = "BitpackInt: leaf " + rec.paths[f] + " is not integral";
                return LLGB_ERR_INVALID_ARG;
            }
            if (b < 1 || b > 8 * type_size(rec.types[f])) {
                *why = "BitpackInt: bit count out of range for leaf " + rec.paths[f];
                return LLGB_ERR_INVALID_ARG;
            }
            v.stored[f].bits = b;
            v.recipes.push_back({L_BITS_INT, f, 1});
        }
    } else if (v.base == BASE_BITS_FLOAT) {
        // Sec. 3 BitpackFloatSoA: exponent and mantissa bits per leaf.
        for (int f = 0; f < nf; ++f) {
            const int e = base->field_exp ? base->field_exp[f] : base->exp_bits;
            const int m = base->field_man ? base->field_man[f] : base->man_bits;
            if (!type_is_float(rec.types[f], nullptr, nullptr)) {
                *why = "BitpackFloat: leaf " + rec.paths[f] + " is not floating point";
                return LLGB_ERR_INVALID_ARG;
            }
            if (e < 2 || e > 11 || m < 1 || m > 52 || 1 + e + m > 64) {
                *why = "BitpackFloat: need 2<=E<=11, 1<=M<=52, 1+E+M<=64";
                return LLGB_ERR_INVALID_ARG;
            }
            v.stored[f].e = e;
            v.stored[f].m = m;
            v.stored[f].bits = 1 + e + m;
            v.recipes.push_back({L_BITS_FLOAT, f, 1});
        }
    }
    if (v.base == BASE_SOA_SB && (v.subarray_align & (v.subarray_align - 1))) {
        *why = "SoA single blob: subarray_align must be 0 or a power of two";
        return LLGB_ERR_INVALID_ARG;
    }
    if (v.base == BASE_AOSOA && v.lanes < 1) {
        *why = "AoSoA: lanes must be >= 1";
        return LLGB_ERR_INVALID_ARG;
    }

    // --- layout and blob sizes ---
    v.leaf_offset.assign(ns, 0);
    v.sb_base.assign(ns, 0);
    v.seg_end.assign(ns, 0);
    v.leaf_blob.assign(ns, 0);
    bool ok = true;
    switch (v.base) {
    case BASE_AOS:
    case BASE_AOSOA: {
        const bool packed = v.base == BASE_AOSOA || v.aos_packed;
        uint64_t off = 0, max_align = 1;
        for (int g = 0; g < ns; ++g) {
            const uint64_t s = v.stored[g].size;
            if (!packed) off = align_up(off, s);
            v.leaf_offset[g] = off;
            off += s;
            max_align = std::max<uint64_t>(max_align, s);
        }
        v.record_bytes = packed ? off : align_up(off, max_align);
        uint64_t size = 0;
        if (v.base == BASE_AOS) {
            ok = mul_ok(n, v.record_bytes, &size);
        } else {
            const uint64_t blocks = n / v.lanes + (n % v.lanes ? 1 : 0);
            uint64_t recs = 0;
            ok = mul_ok(blocks, v.lanes, &recs) && mul_ok(recs, v.record_bytes, &size);
        }
        v.blob_sizes.push_back(size);
        for (int g = 0; g < ns; ++g) v.seg_end[g] = size;
        break;
    }
    case BASE_SOA_MB:
        for (int g = 0; g < ns; ++g) {
            uint64_t size = 0;
            ok = ok && mul_ok(n, (uint64_t)v.stored[g].size, &size);
            v.blob_sizes.push_back(size);
            v.seg_end[g] = size;
            v.leaf_blob[g] = g;
        }
        break;
    case BASE_SOA_SB: {
        uint64_t at = 0;
        for (int g = 0; g < ns; ++g) {
            const uint64_t s = v.stored[g].size;
            at = align_up(at, v.subarray_align ? v.subarray_align : s);
            v.sb_base[g] = at;
            uint64_t bytes = 0;
            ok = ok && mul_ok(n, s, &bytes) && !__builtin_add_overflow(at, bytes, &at);
            v.seg_end[g] = at;
        }
        v.blob_sizes.push_back(at);
        break;
    }
    default:  // bit streams: whole 32-bit words per leaf
        if (v.bit_lanes) {  // AoSoA organisation: runs of L codes, word-aligned
            uint64_t R = 0;
            for (int g = 0; g < ns; ++g) {
                v.leaf_offset[g] = v.bit_lanes * R / 8;
                R += v.stored[g].bits;
            }
            v.bit_block_bytes = v.bit_lanes * R / 8;
            const uint64_t blocks = n / v.bit_lanes + (n % v.bit_lanes ? 1 : 0);
            uint64_t size = 0;
            ok = mul_ok(blocks, v.bit_block_bytes, &size);
            v.blob_sizes.push_back(size);
            for (int g = 0; g < ns; ++g) v.seg_end[g] = size;
            break;
        }
        for (int g = 0; g < ns; ++g) {
            uint64_t bits = 0;
            ok = ok && mul_ok(n, (uint64_t)v.stored[g].bits, &bits);
            const uint64_t size = 4 * (bits / 32 + (bits % 32 ? 1 : 0));
            v.blob_sizes.push_back(size);
            v.seg_end[g] = size;
            v.leaf_blob[g] = g;
        }
        break;
    }
    if (!ok) {
        *why = "blob size overflows 64 bits";
        return LLGB_ERR_INDEX_OVERFLOW;
    }
    if ((int)v.blob_sizes.size() > kMaxBlobs) {
        *why = "more than 32 blobs";
        return LLGB_ERR_UNSUPPORTED;
    }
    for (uint64_t s : v.blob_sizes)
        if (s > 0 && s - 1 > imax) {
            *why = "largest byte offset " + std::to_string(s - 1) + " does not fit the index type";
            return LLGB_ERR_INDEX_OVERFLOW;
        }
    // Signature of the layout, for caches keyed by mapping pair.
    std::string sig = "w" + std::to_string(v.wrap) + "b" + std::to_string(v.base) + "p" + std::to_string(v.aos_packed) +
                      "a" + std::to_string(v.subarray_align) + "l" + std::to_string(v.lanes) + "o" +
                      std::to_string(v.bit_lanes) + ":";
    for (int f = 0; f < nf; ++f) sig += std::to_string(v.types[f]) + ",";
    sig += ":";
    for (const StoredLeaf& l : v.stored)
        sig += std::to_string(l.type) + "/" + std::to_string(l.bits) + "/" + std::to_string(l.e) + "/" +
               std::to_string(l.m) + ",";
    v.sig = sig;
    *out = std::move(v);
    return LLGB_OK;
}

static uint64_t gcd64(uint64_t a, uint64_t b)
{
    while (b) {
        const uint64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

static uint64_t lane_quantum(const ViewPlan& v, uint64_t q)
{
    if (v.base == BASE_AOSOA) q = q / gcd64(q, v.lanes) * v.lanes;
    if (v.bit_lanes) q = q / gcd64(q, v.bit_lanes) * v.bit_lanes;
    for (const ViewPlan& p : v.parts) q = lane_quantum(p, q);
    return q;
}

uint32_t tile_quantum(const ViewPlan& src, const ViewPlan& dst)
{
    const uint64_t q = lane_quantum(dst, lane_quantum(src, 128));
    return q > (1u << 20) ? 0u : (uint32_t)q;
}

static double image_bpr(const ViewPlan& v)
{
    switch (v.base) {
    case BASE_AOS:
    case BASE_AOSOA: return (double)v.record_bytes;
    case BASE_SPLIT: {
        double s = 0;
        for (size_t k = 0; k < v.parts.size(); ++k)
            if (!v.part_null[k]) s += image_bpr(v.parts[k]);
        return s;
    }
    default: {
        double s = 0;
        for (const StoredLeaf& l : v.stored) s += is_bits_base(v.base) ? l.bits / 8.0 : l.size;
        return s;
    }
    }
}

void bytes_per_record(const ViewPlan& src, const ViewPlan& dst, double* src_bpr, double* dst_bpr,
                      uint32_t* code_bpr)
{
    *src_bpr = image_bpr(src);
    *dst_bpr = image_bpr(dst);
    uint32_t c = 0;
    if (is_bits_base(dst.base))
        for (const StoredLeaf& l : dst.stored) c += l.bits > 32 ? 8 : 4;
    *code_bpr = c;
}

// Append the runs and leaf addressing of plan v (its blobs and stored leaves
// numbered from blob0 / leaf0 in the side) for tiles of `tile` records.
static llgb_status plan_side_part(const ViewPlan& v, int blob0, int leaf0, uint32_t tile, uint32_t ntiles,
                                  SideDesc* S, uint64_t& img, bool& bulk_ok, std::string* why)
{
    if (v.base == BASE_SPLIT) {
        for (size_t k = 0; k < v.parts.size(); ++k) {
            if (v.part_null[k]) continue;
            const llgb_status st = plan_side_part(v.parts[k], blob0 + v.part_blob0[k], leaf0 + v.part_leaf0[k], tile,
                                                  ntiles, S, img, bulk_ok, why);
            if (st != LLGB_OK) return st;
        }
        return LLGB_OK;
    }
    const int segs0 = S->nsegs;
    auto add_seg = [&](uint32_t blob, uint64_t gbase, uint64_t tile_bytes, uint64_t end) -> int64_t {
        if (S->nsegs >= kMaxSegs || tile_bytes > 0xFFFFFFFFull) return -1;
        SegDesc& d = S->segs[S->nsegs++];
        d.blob = blob0 + blob;
        d.gbase = gbase;
        d.tile_bytes = (uint32_t)tile_bytes;
        d.sbase = (uint32_t)img;
        // The last tile's run ends exactly where the region ends.
        const uint64_t last_start = gbase + (uint64_t)(ntiles - 1) * tile_bytes;
        if (end < last_start || end - last_start > tile_bytes || end > v.blob_sizes[blob]) return -1;
        d.tail_bytes = (uint32_t)(end - last_start);
        // Full tiles never run past the region.
        const uint64_t nfull = v.n / tile;
        if (gbase + nfull * tile_bytes > end) return -1;
        if ((gbase & 15u) || (tile_bytes & 15u)) bulk_ok = false;
        img += align_up(tile_bytes, 16) + kImageSlack;
        return d.sbase;
    };
    const int ns = (int)v.stored.size();
    S->nleaves = (uint16_t)std::max<int>(S->nleaves, leaf0 + ns);
    LeafDesc* leaves = S->leaves + leaf0;
    for (int g = 0; g < ns; ++g) {
        LeafDesc& L = leaves[g];
        L.size = (uint16_t)v.stored[g].size;
        L.lanes = 1;
        L.lshift = 0;
        L.kind = LEAF_AFFINE;
    }
    switch (v.base) {
    case BASE_AOS: {
        const int64_t sb = add_seg(0, 0, (uint64_t)tile * v.record_bytes, v.seg_end[0]);
        if (sb < 0) break;
        for (int g = 0; g < ns; ++g) {
            leaves[g].sbase = (uint32_t)(sb + v.leaf_offset[g]);
            leaves[g].bstride = (uint32_t)v.record_bytes;
        }
        break;
    }
    case BASE_AOSOA: {
        const int64_t sb = add_seg(0, 0, (uint64_t)tile * v.record_bytes, v.seg_end[0]);
        if (sb < 0) break;
        const uint32_t L = (uint32_t)v.lanes;
        uint8_t shift = 0xFF;
        for (uint8_t p = 0; p < 32; ++p)
            if ((1u << p) == L) shift = p;
        for (int g = 0; g < ns; ++g) {
            leaves[g].sbase = (uint32_t)(sb + L * v.leaf_offset[g]);
            leaves[g].bstride = (uint32_t)(L * v.record_bytes);
            leaves[g].lanes = L;
            leaves[g].lshift = shift;
        }
        break;
    }
    case BASE_SOA_MB:
    case BASE_SOA_SB:
        for (int g = 0; g < ns; ++g) {
            const uint64_t s = v.stored[g].size;
            const int64_t sb = add_seg(v.leaf_blob[g], v.sb_base[g], (uint64_t)tile * s, v.seg_end[g]);
            if (sb < 0) break;
            leaves[g].sbase = (uint32_t)sb;
            leaves[g].bstride = (uint32_t)s;
        }
        break;
    default:
        // a bit leaf's code of tile record r starts at bit
        //   8 (sbase + (r >> lshift) bstride) + (r & (lanes - 1)) bits;
        // a SoA stream is one run (lanes 0: mask all ones, lshift 31).
        if (v.bit_lanes) {
            const int64_t sb = add_seg(0, 0, (uint64_t)tile / v.bit_lanes * v.bit_block_bytes, v.seg_end[0]);
            if (sb < 0) break;
            uint8_t shift = 0;
            while ((1ull << shift) < v.bit_lanes) ++shift;
            for (int g = 0; g < ns; ++g) {
                leaves[g].sbase = (uint32_t)(sb + v.leaf_offset[g]);
                leaves[g].bstride = (uint32_t)v.bit_block_bytes;
                leaves[g].lanes = (uint32_t)v.bit_lanes;
                leaves[g].lshift = shift;
                leaves[g].kind = LEAF_BITS;
                leaves[g].bits = (uint8_t)v.stored[g].bits;
            }
            break;
        }
        for (int g = 0; g < ns; ++g) {
            const uint64_t w = v.stored[g].bits;
            const int64_t sb = add_seg(v.leaf_blob[g], 0, (uint64_t)tile * w / 8, v.seg_end[g]);
            if (sb < 0) break;
            leaves[g].sbase = (uint32_t)sb;
            leaves[g].bstride = 0;
            leaves[g].lanes = 0;
            leaves[g].lshift = 31;
            leaves[g].kind = LEAF_BITS;
            leaves[g].bits = (uint8_t)w;
        }
        break;
    }
    const int expect_segs = (v.base == BASE_AOS || v.base == BASE_AOSOA || v.bit_lanes) ? 1 : ns;
    if (S->nsegs - segs0 != expect_segs) {
        *why = "internal: a tile run does not fit its blob region";
        return LLGB_ERR_INVALID_ARG;
    }
    for (int g = 0; g < ns; ++g) {
        LeafDesc& L = leaves[g];
        uint32_t p = 8;
        while (p > 1 && ((L.sbase % p) || (L.bstride % p) || (L.lanes > 1 && (L.size % p)))) p /= 2;
        L.align = (uint8_t)p;
    }
    return LLGB_OK;
}

// Fill one side's runs and leaf addressing for tiles of `tile` records.
static llgb_status plan_side(const ViewPlan& v, const std::vector<void*>& ptrs, uint32_t tile, uint32_t ntiles,
                             SideDesc* S, std::string* why)
{
    memset(S, 0, sizeof *S);
    for (size_t k = 0; k < ptrs.size(); ++k) S->blobs[k] = static_cast<uint8_t*>(ptrs[k]);
    uint64_t img = 0;
    bool bulk_ok = true;
    const llgb_status st = plan_side_part(v, 0, 0, tile, ntiles, S, img, bulk_ok, why);
    if (st != LLGB_OK) return st;
    if (img > 0xFFFFFFFFull) {
        *why = "tile image too large";
        return LLGB_ERR_INVALID_ARG;
    }
    S->img_bytes = (uint32_t)img;
    S->bulk_ok = bulk_ok ? 1 : 0;
    return LLGB_OK;
}



static bool fmt_is(int e, int m, int fe, int fm) { return e == fe && m == fm; }

// The specialised loop a VALUE item can run in (FastKind), or FK_GENERIC.
static int fast_kind(const ItemDesc& it, const LeafDesc& A, const LeafDesc& B)
{
    const bool a_aff = A.kind == LEAF_AFFINE, b_aff = B.kind == LEAF_AFFINE;
    const bool a_al = A.kind == LEAF_BITS && (A.bits == 8 || A.bits == 16 || A.bits == 32 || A.bits == 64);
    const bool b_al = B.kind == LEAF_BITS && (B.bits == 8 || B.bits == 16 || B.bits == 32 || B.bits == 64);
    const int size = it.size;
    // integers: plain 4-byte leaf <-> bit stream of at most 32 bits
    if (it.lop == L_DIRECT && it.sop == S_BITS_INT && a_aff && size == 4 && A.align >= 4 && it.d_bits <= 32)
        return FK_PACK_INT32;
    if (it.lop == L_BITS_INT && it.sop == S_DIRECT && b_aff && size == 4 && B.align >= 4 && A.bits <= 32)
        return FK_UNPACK_INT32;
    // floats into / out of bit streams
    if (it.lop == L_DIRECT && it.sop == S_BITS_FLOAT && a_aff && A.align >= size && (size == 4 || size == 8)) {
        if (b_al && it.d_bits == 32 && size == 8 && fmt_is(it.d_e, it.d_m, 8, 23)) return FK_PACK_D_F32;
        if (b_al && it.d_bits == 32) return size == 8 ? FK_PACK_AL32_FROM8 : FK_PACK_AL32_FROM4;
        if (b_al && it.d_bits == 64) return size == 8 ? FK_PACK_AL64_FROM8 : FK_PACK_AL64_FROM4;
        if (b_al && it.d_bits == 16) return size == 8 ? FK_PACK_AL16_FROM8 : FK_PACK_AL16_FROM4;
        if (b_al && it.d_bits == 8) return size == 8 ? FK_PACK_AL8_FROM8 : FK_PACK_AL8_FROM4;
        return size == 8 ? FK_PACK_BITS_FROM8 : FK_PACK_BITS_FROM4;
    }
    if (it.lop == L_BITS_FLOAT && it.sop == S_DIRECT && b_aff && B.align >= size && (size == 4 || size == 8)) {
        if (a_al && A.bits == 32 && size == 8 && fmt_is(it.s_e, it.s_m, 8, 23)) return FK_UNPACK_F32_D;
        if (a_al && A.bits == 32) return size == 8 ? FK_UNPACK_AL32_TO8 : FK_UNPACK_AL32_TO4;
        if (a_al && A.bits == 64) return size == 8 ? FK_UNPACK_AL64_TO8 : FK_UNPACK_AL64_TO4;
        if (a_al && A.bits == 16) return size == 8 ? FK_UNPACK_AL16_TO8 : FK_UNPACK_AL16_TO4;
        if (a_al && A.bits == 8) return size == 8 ? FK_UNPACK_AL8_TO8 : FK_UNPACK_AL8_TO4;
        return size == 8 ? FK_UNPACK_BITS_TO8 : FK_UNPACK_BITS_TO4;
    }
    // ChangeType f64 <-> f32
    if (it.lop == L_DIRECT && it.sop == S_CT && a_aff && b_aff && size == 8 && it.d_size == 4 && A.align >= 8 &&
        B.align >= 4 && fmt_is(it.d_e, it.d_m, 8, 23))
        return FK_CT_D_F32;
    if (it.lop == L_CT && it.sop == S_DIRECT && a_aff && b_aff && size == 8 && it.s_size == 4 && A.align >= 4 &&
        B.align >= 8 && fmt_is(it.s_e, it.s_m, 8, 23))
        return FK_CT_F32_D;
    return FK_GENERIC;
}

// The specialised loops give each lane V consecutive records of every 32 V:
// V = 4, 2 or 1 for streams of <= 16, <= 32 or more bits (a lane's codes
// then fill 32..64 bits), and 16 bytes over the widest affine element
// otherwise.  An affine leaf must keep a lane's V records at a constant
// stride: one lane, or a power-of-two lane count that V divides and that
// divides 32 V.
static bool affine_for(const LeafDesc& L, int V)
{
    if (L.kind != LEAF_AFFINE) return true;
    if (L.lanes == 1) return true;
    return L.lshift != 0xFF && L.lanes % (uint32_t)V == 0 && L.lanes <= 32u * (uint32_t)V;
}

// Id of the compile-time stream format (stream_specs.h) of a VALUE item that
// packs a 4- or 8-byte affine leaf into a bit stream, or unpacks one, or 0:
// the leaf's type and the stream's width (and float format) must match an
// entry, and the affine leaf must allow the entry's records per lane.  The
// stream may be organised as SoA or as AoSoA (runs of L >= 32 codes, which
// the kernel-mode-1 loops address).
static int stream_spec_id(const ItemDesc& it, const LeafDesc& A, const LeafDesc& B)
{
    const bool pack = it.lop == L_DIRECT && (it.sop == S_BITS_INT || it.sop == S_BITS_FLOAT);
    const bool unpack = (it.lop == L_BITS_INT || it.lop == L_BITS_FLOAT) && it.sop == S_DIRECT;
    if (!pack && !unpack) return 0;
    const LeafDesc& P = pack ? A : B;  // the affine leaf
    const LeafDesc& S = pack ? B : A;  // the bit stream
    if (P.kind != LEAF_AFFINE || S.kind != LEAF_BITS) return 0;
    const int is_float = (pack ? it.sop == S_BITS_FLOAT : it.lop == L_BITS_FLOAT) ? 1 : 0;
    const int size = it.size;
    for (const StreamSpecInfo& sp : kStreamSpecs) {
        if (sp.is_float != is_float || sp.leaf_bytes != size || sp.bits != (int)S.bits) continue;
        if (sp.aosoa_only && S.lanes == 0) continue;
        if (is_float) {
            if (it.l_e != (size == 8 ? 11 : 8) || it.l_m != (size == 8 ? 52 : 23)) continue;
            if ((pack ? it.d_e : it.s_e) != sp.exp || (pack ? it.d_m : it.s_m) != sp.man) continue;
        }
        if ((int)P.align < size || !affine_for(P, stream_vpl(size, sp.bits))) return 0;
        return sp.id;
    }
    return 0;
}

static void set_fast_kind(ItemDesc& it, const LeafDesc& A, const LeafDesc& B)
{
    it.spec = (uint8_t)stream_spec_id(it, A, B);
    const int k = fast_kind(it, A, B);
    int V = 0;
    switch (k) {
    case FK_GENERIC: break;
    case FK_PACK_INT32:
    case FK_PACK_BITS_FROM8:
    case FK_PACK_BITS_FROM4: V = it.d_bits <= 16 ? 4 : (it.d_bits <= 32 ? 2 : 1); break;
    case FK_UNPACK_INT32:
    case FK_UNPACK_BITS_TO8:
    case FK_UNPACK_BITS_TO4: V = A.bits <= 16 ? 4 : (A.bits <= 32 ? 2 : 1); break;
    default: {
        const int widest = std::max(A.kind == LEAF_AFFINE ? (int)A.size : 0, B.kind == LEAF_AFFINE ? (int)B.size : 0);
        V = 16 / widest;
    }
    }
    // an AoSoA-organised bit leaf: a super-group of 32 V records must lie in
    // one run of its L codes
    auto runs_ok = [&](const LeafDesc& L) { return L.kind != LEAF_BITS || L.lanes == 0 || L.lanes >= 32u * V; };
    if (k != FK_GENERIC && affine_for(A, V) && affine_for(B, V) && runs_ok(A) && runs_ok(B)) {
        it.fast = (uint8_t)k;
        it.vpl = (uint8_t)V;
        it.runs = ((A.kind == LEAF_BITS && A.lanes) || (B.kind == LEAF_BITS && B.lanes)) ? 1 : 0;
    } else {
        it.fast = FK_GENERIC;
        it.vpl = 0;
    }
}

llgb_status plan_job(const ViewPlan& src, const std::vector<void*>& src_ptrs, const ViewPlan& dst,
                     const std::vector<void*>& dst_ptrs, uint32_t tile, JobDesc* job, std::string* why)
{
    memset(job, 0, sizeof *job);
    const uint32_t q = tile_quantum(src, dst);
    if (q == 0 || tile == 0 || tile % q) {
        *why = "tile size must be a positive multiple of " + std::to_string(q);
        return LLGB_ERR_INVALID_ARG;
    }
    const uint64_t n = src.n;
    const uint64_t ntiles64 = n == 0 ? 0 : (n - 1) / tile + 1;
    if (ntiles64 > 0xFFFFFFFFull) {
        *why = "too many tiles";
        return LLGB_ERR_INVALID_ARG;
    }
    job->n = n;
    job->tile = tile;
    job->ntiles = (uint32_t)ntiles64;
    job->nfull = (uint32_t)(n / tile);
    if (n == 0) return LLGB_OK;
    llgb_status st = plan_side(src, src_ptrs, tile, job->ntiles, &job->src, why);
    if (st != LLGB_OK) return st;
    st = plan_side(dst, dst_ptrs, tile, job->ntiles, &job->dst, why);
    if (st != LLGB_OK) return st;

    // Gaps between SoA single-blob sub-arrays belong to no leaf: zero them
    // (in every SoA single-blob part of a Split destination).
    std::function<bool(const ViewPlan&, int)> add_gaps = [&](const ViewPlan& v, int blob0) -> bool {
        if (v.base == BASE_SPLIT) {
            for (size_t k = 0; k < v.parts.size(); ++k)
                if (!v.part_null[k] && !add_gaps(v.parts[k], blob0 + v.part_blob0[k])) return false;
            return true;
        }
        if (v.base != BASE_SOA_SB) return true;
        for (size_t g = 1; g < v.stored.size(); ++g) {
            const uint64_t from = v.seg_end[g - 1], to = v.sb_base[g];
            if (to <= from) continue;
            if (job->nzeros >= kMaxZeros || to - from > 0xFFFFFFFFull) return false;
            ZeroRun& z = job->zeros[job->nzeros++];
            z.offset = from;
            z.bytes = (uint32_t)(to - from);
            z.blob = (uint32_t)blob0;
        }
        return true;
    };
    if (!add_gaps(dst, 0)) {
        *why = "too many or too large sub-array gaps";
        return LLGB_ERR_UNSUPPORTED;
    }

    // Bit-stream destination leaves (whether a generic item ORs into one is
    // known once the items exist, below).
    int8_t pack_of[kMaxLeaves];
    for (int g = 0; g < kMaxLeaves; ++g) pack_of[g] = -1;
    for (int g = 0; g < (int)dst.stored.size(); ++g) {
        if (job->dst.leaves[g].kind != LEAF_BITS) continue;
        if (job->npacks >= kMaxPacks) {
            *why = "more than 16 bit-packed leaves";
            return LLGB_ERR_UNSUPPORTED;
        }
        pack_of[g] = (int8_t)job->npacks;
        PackDesc& P = job->packs[job->npacks++];
        P.bits = (uint8_t)dst.stored[g].bits;
        P.dst_sbase = job->dst.leaves[g].sbase;
        P.aligned = (P.bits == 8 || P.bits == 16 || P.bits == 32 || P.bits == 64) ? 1 : 0;
        const LeafDesc& D = job->dst.leaves[g];
        P.leaf = (uint8_t)g;
        if (D.lanes) {  // AoSoA organisation: tile / L runs of L codes
            P.bytes = D.lanes * P.bits / 8;
            P.runs = (uint16_t)(tile / D.lanes);
        } else {
            P.bytes = (uint32_t)((uint64_t)tile * P.bits / 8);
            P.runs = 1;
        }
    }
    job->code_bytes = 0;

    // Items: one per leaf, or one per byte where a side splits bytes.
    const int nf = (int)src.types.size();
    auto too_many = [&]() -> llgb_status {
        *why = "more than 64 work items per tile";
        return LLGB_ERR_UNSUPPORTED;
    };
    auto add = [&](const ItemDesc& it) -> bool {
        if (job->nitems >= kMaxItems) return false;
        job->items[job->nitems++] = it;
        return true;
    };
    for (int f = 0; f < nf; ++f) {
        const Recipe a = src.recipes[f], b = dst.recipes[f];
        const int32_t t = src.types[f];
        if (b.op == L_NULL) continue;  // the destination stores nothing (Null)
        // A Null source loads 0, whose bytes are all zero: a destination that
        // stores bytes (plain or byte planes) then holds exactly the zero fill
        // of bytes no item owns, so the leaf needs no item -- and a job of
        // otherwise byte moves keeps its gather programs.
        if (a.op == L_NULL && (b.op == L_DIRECT || b.op == L_SPLIT)) continue;
        const int size = type_size(t);
        const bool a_bytes = a.op == L_DIRECT || a.op == L_SPLIT;
        const bool b_bytes = b.op == L_DIRECT || b.op == L_SPLIT;
        if (a_bytes && b_bytes && a.op != b.op && (size == 2 || size == 4 || size == 8)) {
            // A leaf to its byte planes or back (Bytesplit, Sec. 3): one item
            // transposes the bytes of 4 records per lane when every leaf
            // involved keeps a lane's 4 records at a constant stride.
            const bool split = b.op == L_SPLIT;
            const LeafDesc& whole = split ? job->src.leaves[a.first] : job->dst.leaves[b.first];
            const int planes0 = split ? b.first : a.first;
            bool ok = affine_for(whole, 4) && whole.kind == LEAF_AFFINE && whole.align >= size;
            for (int j = 0; j < size && ok; ++j) {
                const LeafDesc& P = split ? job->dst.leaves[planes0 + j] : job->src.leaves[planes0 + j];
                ok = P.kind == LEAF_AFFINE && affine_for(P, 4);
            }
            if (ok) {
                ItemDesc it{};
                it.op = ITEM_VALUE;
                it.size = (uint8_t)size;
                it.lop = (uint8_t)a.op;
                it.sop = (uint8_t)b.op;
                it.src_leaf = (uint8_t)a.first;
                it.dst_leaf = (uint8_t)b.first;
                const int k = size == 2 ? 0 : (size == 4 ? 1 : 2);
                it.fast = (uint8_t)((split ? FK_SPLIT2 : FK_JOIN2) + k);
                it.vpl = 4;
                if (!add(it)) return too_many();
                continue;
            }
        }
        if (a_bytes && b_bytes) {
            if (a.op == L_DIRECT && b.op == L_DIRECT) {
                ItemDesc it{};
                it.op = ITEM_MOVE;
                it.size = (uint8_t)size;
                it.src_leaf = (uint8_t)a.first;
                it.dst_leaf = (uint8_t)b.first;
                it.gran = (uint8_t)std::min<int>(
                    size, std::min<int>(job->src.leaves[a.first].align, job->dst.leaves[b.first].align));
                // whole aligned elements: the specialised loops (V = 4, 2 for 8 bytes)
                const int V = size == 8 ? 2 : 4;
                if (it.gran == size && (size == 1 || size == 2 || size == 4 || size == 8) &&
                    job->src.leaves[a.first].kind == LEAF_AFFINE && job->dst.leaves[b.first].kind == LEAF_AFFINE &&
                    affine_for(job->src.leaves[a.first], V) && affine_for(job->dst.leaves[b.first], V)) {
                    it.fast = (uint8_t)(FK_MOVE1 + (size == 1 ? 0 : size == 2 ? 1 : size == 4 ? 2 : 3));
                    it.vpl = (uint8_t)V;
                }
                if (!add(it)) return too_many();
            } else {
                for (int j = 0; j < size; ++j) {
                    ItemDesc it{};
                    it.op = ITEM_MOVE;
                    it.size = 1;
                    it.gran = 1;
                    it.src_leaf = (uint8_t)(a.op == L_SPLIT ? a.first + j : a.first);
                    it.src_byte = (uint8_t)(a.op == L_SPLIT ? 0 : j);
                    it.dst_leaf = (uint8_t)(b.op == L_SPLIT ? b.first + j : b.first);
                    it.dst_byte = (uint8_t)(b.op == L_SPLIT ? 0 : j);
                    if (!add(it)) return too_many();
                }
            }
            continue;
        }
        {
            ItemDesc it{};
            it.op = ITEM_VALUE;
            it.size = (uint8_t)size;
            it.lop = (uint8_t)a.op;
            it.sop = (uint8_t)b.op;  // StoreOp numbering matches LoadOp
            it.src_leaf = (uint8_t)a.first;
            it.dst_leaf = (uint8_t)b.first;
            it.is_signed = type_is_signed(t) ? 1 : 0;
            int le = 0, lm = 0;
            type_is_float(t, &le, &lm);
            it.l_e = (uint8_t)le;
            it.l_m = (uint8_t)lm;
            if (a.op == L_CT) {
                int e = 0, m = 0;
                type_is_float(src.stored[a.first].type, &e, &m);
                it.s_e = (uint8_t)e;
                it.s_m = (uint8_t)m;
                it.s_size = (uint8_t)src.stored[a.first].size;
            } else if (a.op == L_BITS_FLOAT) {
                it.s_e = (uint8_t)src.stored[a.first].e;
                it.s_m = (uint8_t)src.stored[a.first].m;
            }
            if (a.op == L_BITS_INT || a.op == L_BITS_FLOAT) it.s_bits = (uint8_t)src.stored[a.first].bits;
            if (b.op == L_CT) {
                int e = 0, m = 0;
                type_is_float(dst.stored[b.first].type, &e, &m);
                it.d_e = (uint8_t)e;
                it.d_m = (uint8_t)m;
                it.d_size = (uint8_t)dst.stored[b.first].size;
            } else if (b.op == L_BITS_FLOAT) {
                it.d_e = (uint8_t)dst.stored[b.first].e;
                it.d_m = (uint8_t)dst.stored[b.first].m;
            }
            if (b.op == L_BITS_INT || b.op == L_BITS_FLOAT) it.d_bits = (uint8_t)dst.stored[b.first].bits;
            set_fast_kind(it, job->src.leaves[a.first], job->dst.leaves[b.first]);
            if (!add(it)) return too_many();
        }
    }
    // Relative cost of a quad of each item, by which the consumer warps share
    // a tile.  Loops whose work grows with the element's bytes (Bytesplit's
    // byte planes, whole-element moves, f64 <-> f32 element conversions) cost
    // one unit per 4 bytes; the
    // converting loops cost about the same per record whatever the leaf's
    // size (their code stream dominates), one unit; record-by-record loops
    // (generic items, byte moves outside the specialised loops) more.
    for (int k = 0; k < job->nitems; ++k) {
        ItemDesc& it = job->items[k];
        int w = 1;
        if (it.op == ITEM_VALUE && it.fast == FK_GENERIC && !it.spec) {
            w = 6;
        } else if (it.op == ITEM_MOVE && it.fast == FK_GENERIC) {
            w = std::max(2, (int)it.size / std::max(1, (int)it.gran));
        } else if ((it.fast >= FK_SPLIT2 && it.fast <= FK_JOIN8) || (it.fast >= FK_MOVE1 && it.fast <= FK_MOVE8) ||
                   it.fast == FK_CT_D_F32 || it.fast == FK_CT_F32_D) {
            w = std::max(1, (int)it.size / 4);
        }
        it.weight = (uint8_t)std::min(8, w);
    }
    // Items on AoSoA-organised bit leaves choose the kernel mode: the generic
    // loop needs mode 1; the compile-time stream loops of such leaves are in
    // mode 3 (a job that needs both runs in mode 1, where the stream items take
    // the loops with run-time widths).
    job->seg = 0;
    for (int k = 0; k < job->nitems; ++k) {
        const ItemDesc& it = job->items[k];
        if (it.op != ITEM_VALUE) continue;
        const LeafDesc& A = job->src.leaves[it.src_leaf];
        const LeafDesc& B = job->dst.leaves[it.dst_leaf];
        if (!((A.kind == LEAF_BITS && A.lanes) || (B.kind == LEAF_BITS && B.lanes))) continue;
        if (it.spec) {
            if (job->seg == 0) job->seg = 3;
        } else if (it.fast == FK_GENERIC) {
            job->seg = 1;
        }
    }
    for (int k = 0; k < job->nitems; ++k) {
        const ItemDesc& it = job->items[k];
        if (it.op != ITEM_VALUE || (it.sop != S_BITS_INT && it.sop != S_BITS_FLOAT)) continue;
        PackDesc& P = job->packs[pack_of[it.dst_leaf]];
        // a compile-time stream item stores whole words, except in kernel mode 1,
        // where it runs the generic loop
        const bool generic = it.fast == FK_GENERIC && !(it.spec && job->seg != 1);
        P.ored = (generic && !P.aligned) ? 1 : 0;
        job->ored |= P.ored;
    }
    // Jobs made only of byte moves run full tiles through gather programs:
    // 2 source words per destination word when every move is at least
    // 2-byte grained and aligned, else up to 4.
    bool all_moves = job->npacks == 0;
    int min_gran = 8;
    for (int k = 0; k < job->nitems; ++k) {
        if (job->items[k].op != ITEM_MOVE) all_moves = false;
        min_gran = std::min<int>(min_gran, job->items[k].gran);
    }
    job->gather = all_moves ? (min_gran >= 2 ? 2 : 4) : 0;
    // Byte-plane destinations (equal runs, e.g. Bytesplit over SoA): neighbouring
    // consumer threads take words of different runs, which spreads the 4-word
    // gathers over the shared-memory banks.
    if (job->gather == 4 && job->dst.nsegs >= 4) {
        bool equal = true;
        for (int q = 1; q < job->dst.nsegs; ++q) equal &= job->dst.segs[q].tile_bytes == job->dst.segs[0].tile_bytes;
        job->interleave = equal ? 1 : 0;
    }
    return LLGB_OK;
}

}  // namespace llgb
