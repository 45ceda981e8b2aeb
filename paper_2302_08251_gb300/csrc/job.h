// job.h -- descriptor of one layout-aware copy, as the tile kernel sees it.
//
// The host planner (plan.cpp) compiles a (source view, destination view) pair
// into a JobDesc.  The kernel (copy.cu) moves the records tile by tile: the
// tile's bytes of each source run are staged into a shared-memory "image",
// every leaf of every record is moved (or converted) into the destination
// image, and the destination image's runs are written back.  Inside an image
// all addressing is 32-bit and tile-local, so no per-element arithmetic ever
// uses the 64-bit record index (Sec. 2 of the paper: 64-bit integer arithmetic
// is expensive on GPUs).
#pragma once

#include <stdint.h>

namespace llgb {

constexpr int kMaxBlobs = 32;   // blobs per side
constexpr int kMaxSegs = 32;    // contiguous runs per tile per side
constexpr int kMaxLeaves = 32;  // stored leaves per side
constexpr int kMaxItems = 64;   // per-tile work items
constexpr int kMaxPacks = 16;   // bit-stream destination leaves
constexpr int kImageSlack = 16; // bytes after every run in an image
constexpr int kMaxZeros = 32;   // destination byte ranges owned by no leaf
constexpr int kStageZeroBytes = 16;  // zero block at the end of every source stage
// Kernel modes: 0 value loops; 1 value loops with the generic loop of
// AoSoA-organised bit leaves; 2 / 4 gather programs of 2 / 4 source words;
// 3 value loops with the compile-time stream loops of AoSoA-organised bit
// leaves.
constexpr bool gather_mode(int mode) { return mode == 2 || mode == 4; }
// Warps of a CTA that issue its TMA copies: value kernels have a load warp
// and a store warp; gather kernels one warp for both.
constexpr unsigned producer_warps(int mode) { return gather_mode(mode) ? 1u : 2u; }

// One contiguous run of a tile in a blob.  For tile t it covers
// [gbase + t * tile_bytes, + tile_bytes) (the last tile: tail_bytes) and
// lands at image offset sbase.
struct SegDesc {
    uint64_t gbase;
    uint32_t tile_bytes;
    uint32_t tail_bytes;
    uint32_t sbase;
    uint32_t blob;
};

enum LeafKind : uint8_t { LEAF_AFFINE = 0, LEAF_BITS = 1 };

// Where record r's element of a stored leaf lives inside a tile image.
//   affine: sbase + (r / lanes) * bstride + (r % lanes) * size  (bytes)
//   bits:   bit r * bits of the LSB-first stream starting at sbase
struct LeafDesc {
    uint32_t sbase;
    uint32_t bstride;
    uint32_t lanes;
    uint16_t size;
    uint8_t kind;
    uint8_t lshift;  // log2(lanes), or 0xFF when lanes is not a power of two
    uint8_t bits;
    uint8_t align;   // power of two dividing every element address (1..8)
    uint8_t pad[2];
};

enum ItemOp : uint8_t { ITEM_MOVE = 0, ITEM_VALUE = 1 };
// L_NULL: the leaf has no storage (Null mapping): it loads as 0.
enum LoadOp : uint8_t { L_DIRECT = 0, L_CT = 1, L_BITS_INT = 2, L_BITS_FLOAT = 3, L_SPLIT = 4, L_NULL = 5 };
enum StoreOp : uint8_t { S_DIRECT = 0, S_CT = 1, S_BITS_INT = 2, S_BITS_FLOAT = 3, S_SPLIT = 4 };

// A unit of per-record work inside a tile.
//  MOVE:  copy `size` bytes from (src_leaf, byte src_byte of its element) to
//         (dst_leaf, byte dst_byte), in pieces of `gran` bytes.
//  VALUE: load the leaf's logical value (lop), store it (sop).
struct ItemDesc {
    uint8_t op;
    uint8_t size;        // MOVE: bytes; VALUE: logical value bytes
    uint8_t gran;        // MOVE: piece size (1, 2, 4, 8)
    uint8_t src_leaf;    // first source leaf (SPLIT: first of `size` byte leaves)
    uint8_t dst_leaf;
    uint8_t src_byte;
    uint8_t dst_byte;
    uint8_t lop;
    uint8_t sop;
    uint8_t is_signed;   // logical type is a signed integer
    uint8_t l_e, l_m;    // logical float format (0, 0 for integers)
    uint8_t s_e, s_m;    // source stored format (L_CT, L_BITS_FLOAT)
    uint8_t d_e, d_m;    // destination stored format (S_CT, S_BITS_FLOAT)
    uint8_t s_size;      // source stored bytes (L_CT)
    uint8_t d_size;      // destination stored bytes (S_CT)
    uint8_t s_bits;      // source bits (L_BITS_*)
    uint8_t d_bits;      // destination bits (S_BITS_*)
    uint8_t fast;        // FastKind of the specialised loop, FK_GENERIC if none
    uint8_t vpl;         // specialised loop: consecutive records per lane (1, 2, 4)
    uint8_t runs;        // specialised loop: a bit leaf of the item is AoSoA-organised
    uint8_t spec;        // id of the item's compile-time stream format (stream_specs.h), 0 if none
    uint8_t weight;      // relative cost of a quad (128 records) of the item, 1..8: warps share tiles by it
};

// Specialised VALUE loops (element sizes and conversion fixed at compile time).
enum FastKind : uint8_t {
    FK_GENERIC = 0,
    FK_PACK_INT32,        // 4-byte integer leaf -> stream of <= 32 bits
    FK_UNPACK_INT32,      // stream of <= 32 bits -> 4-byte integer leaf
    FK_PACK_D_F32,        // f64 leaf -> (8,23) stream, hardware conversion
    FK_PACK_AL32_FROM8,   // float leaf -> 32-bit stream (any format)
    FK_PACK_AL32_FROM4,
    FK_PACK_AL64_FROM8,   // -> 64-bit stream
    FK_PACK_AL64_FROM4,
    FK_PACK_AL16_FROM8,   // -> 16-bit stream
    FK_PACK_AL16_FROM4,
    FK_PACK_BITS_FROM8,   // -> stream of any other width
    FK_PACK_BITS_FROM4,
    FK_UNPACK_F32_D,      // (8,23) stream -> f64 leaf, hardware conversion
    FK_UNPACK_AL32_TO8,
    FK_UNPACK_AL32_TO4,
    FK_UNPACK_AL64_TO8,
    FK_UNPACK_AL64_TO4,
    FK_UNPACK_AL16_TO8,
    FK_UNPACK_AL16_TO4,
    FK_UNPACK_BITS_TO8,
    FK_UNPACK_BITS_TO4,
    FK_CT_D_F32,          // ChangeType store f64 -> f32
    FK_CT_F32_D,          // ChangeType load f32 -> f64
    FK_PACK_AL8_FROM8,    // -> 8-bit stream
    FK_PACK_AL8_FROM4,
    FK_UNPACK_AL8_TO8,
    FK_UNPACK_AL8_TO4,
    FK_SPLIT2,            // 2 / 4 / 8-byte leaf -> its byte planes (Bytesplit store)
    FK_SPLIT4,
    FK_SPLIT8,
    FK_JOIN2,             // byte planes -> 2 / 4 / 8-byte leaf (Bytesplit load)
    FK_JOIN4,
    FK_JOIN8,
    FK_MOVE1,             // whole 1 / 2 / 4 / 8-byte element between affine leaves
    FK_MOVE2,             // (MOVE items of jobs that also convert values)
    FK_MOVE4,
    FK_MOVE8
};

// A bit-stream destination leaf.  Specialised loops store whole words of the
// stream; a generic item ORs its codes into it (unless the width is 8, 16,
// 32 or 64 bits), and then the consumers zero the stream before every tile
// (`ored`): `runs` runs of `bytes` bytes from `dst_sbase`, the destination
// leaf's bstride apart (one run for a SoA stream; one per block for AoSoA).
struct PackDesc {
    uint32_t dst_sbase;  // destination image offset of the stream
    uint32_t bytes;      // bytes per run (a multiple of 4)
    uint8_t bits;
    uint8_t aligned;
    uint8_t ored;
    uint8_t leaf;        // destination leaf
    uint16_t runs;
    uint8_t pad[2];
};

struct SideDesc {
    uint8_t* blobs[kMaxBlobs];
    SegDesc segs[kMaxSegs];
    LeafDesc leaves[kMaxLeaves];
    uint32_t img_bytes;  // image size, multiple of 16
    uint16_t nsegs;
    uint16_t nleaves;
    uint8_t bulk_ok;     // full-tile runs are 16-byte aligned multiples of 16
    uint8_t pad[7];
};

// A destination byte range that no tile run covers and no leaf owns (the
// alignment gaps between SoA single-blob sub-arrays); written as zero by the
// CTA that handles the job's first tile.
struct ZeroRun {
    uint64_t offset;
    uint32_t bytes;
    uint32_t blob;
};

struct JobDesc {
    SideDesc src;
    SideDesc dst;
    ItemDesc items[kMaxItems];
    PackDesc packs[kMaxPacks];
    ZeroRun zeros[kMaxZeros];
    uint64_t n;          // records
    uint32_t tile;       // records per tile
    uint32_t ntiles;     // tiles covering n
    uint32_t nfull;      // tiles holding `tile` records
    uint32_t code_bytes; // code staging bytes
    uint16_t nitems;
    uint16_t npacks;
    uint16_t nzeros;
    uint8_t gather;      // full tiles use gather programs: 0 no, 2 or 4 source words
    uint8_t interleave;  // 4-word gathers: deal destination words round-robin over the runs
    uint8_t ored;        // some PackDesc has `ored` set: zero those streams before every tile
    uint8_t seg;         // kernel mode for AoSoA-organised bit leaves: 1 (generic loop), 3 (compile-time loops), else 0
    uint8_t pad[6];
    uint64_t program;    // device address of the job's gather program (gather_program_kernel), or 0: every CTA builds it
};

// Launch-wide parameters of the copy kernel.
struct CopyArgs {
    JobDesc job;                 // used when table == nullptr
    const JobDesc* table;        // batch: njobs descriptors in device memory
    const uint32_t* tile_start;  // batch: first global tile of each job (njobs+1)
    uint32_t njobs;
    uint32_t total_tiles;
    uint32_t src_stage_bytes;    // per stage: max image over jobs + kStageZeroBytes
    uint32_t dst_stage_bytes;
    uint32_t code_bytes;
    uint16_t src_stages;
    uint16_t dst_stages;
    uint32_t chunk;              // 0: CTA b takes tiles b, b + grid, ...; else tiles [b*chunk, (b+1)*chunk)
    const uint32_t* cta_tiles;   // if set (grid + 1 entries): CTA b takes tiles [cta_tiles[b], cta_tiles[b+1])
};

}  // namespace llgb
