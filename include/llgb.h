/*
 * llgb.h -- C ABI of the GB300 library for mapping-driven record layouts.
 *
 * The operations follow the problem statement of arXiv 2302.08251 ("Updates on
 * the Low-Level Abstraction of Memory Access"):
 *   - a record dimension of nested fields, flattened depth-first into leaves
 *     (Sec. 1, Fig. 1 concepts);
 *   - array extents, each static or dynamic, with a chosen index type used for
 *     index and offset arithmetic (Sec. 2);
 *   - an exchangeable mapping with its parameters (Sec. 1; new mappings Sec. 3;
 *     AoS / SoA multi-blob / AoSoA named in Sec. 5);
 *   - a view = mapping + blobs (Sec. 1, Sec. 2);
 *   - the layout-aware copy between views (Sec. 1), of which packing into and
 *     unpacking from the bit-packed mappings are special cases (Sec. 3);
 *   - a consumer that reads and writes records through a view: one all-pairs
 *     n-body step (Sec. 5, Fig. 2).
 *
 * Conventions for every call:
 *   - Device pointers are plain CUDA device addresses; host pointers are plain
 *     process addresses.  No PyTorch or CUDA types appear in the signatures:
 *     a stream is passed as `void*` holding a cudaStream_t (NULL = legacy
 *     default stream).
 *   - The library never allocates or frees blob memory.  The caller owns every
 *     blob and keeps it alive until the work queued on it has finished.
 *   - Calls return an llgb_status.  Host-side validation errors are returned
 *     before anything is queued.  Work is queued asynchronously on the given
 *     stream; errors raised by kernels (a wait that ran out of time) are
 *     recorded in a device status word read back by llgb_device_status().
 *   - llgb_last_error() returns a thread-local, human-readable message for the
 *     last failing call on the calling thread.
 *   - No C++ exception crosses this boundary.
 */
#ifndef LLGB_H
#define LLGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------- status -- */

typedef int32_t llgb_status;

enum {
    LLGB_OK = 0,
    LLGB_ERR_INVALID_ARG = 1,    /* null pointer, bad enum, bad parameter           */
    LLGB_ERR_INDEX_OVERFLOW = 2, /* n or an offset does not fit the index type      */
    LLGB_ERR_MISMATCH = 3,       /* views differ in record or record count          */
    LLGB_ERR_UNSUPPORTED = 4,    /* valid request that this library does not run    */
    LLGB_ERR_CUDA = 5,           /* a CUDA runtime call failed                      */
    LLGB_ERR_TIMEOUT = 6,        /* a bounded device wait gave up                   */
    LLGB_ERR_OOM = 7,            /* host or device allocation failed                */
    LLGB_ERR_UNBOUND = 8         /* view used before llgb_view_bind                 */
};

/* Message for the last failing call on this thread ("" if none). */
const char* llgb_last_error(void);

/* Library version string. */
const char* llgb_version(void);

/* ---------------------------------------------------------- leaf types -- */

enum {
    LLGB_U8 = 0, LLGB_U16, LLGB_U32, LLGB_U64,
    LLGB_I8, LLGB_I16, LLGB_I32, LLGB_I64,
    LLGB_F16, LLGB_BF16, LLGB_F32, LLGB_F64
};

/* -------------------------------------------------------------- record -- */

/* One leaf of the record dimension.  `path` names the leaf by its tags from
 * the root, dot separated ("pos.x"); leaves are given in depth-first order
 * (Sec. 1: records are addressed by tags; nested records flatten to leaves). */
typedef struct llgb_field_desc {
    const char* path;
    int32_t type; /* LLGB_U8 .. LLGB_F64 */
} llgb_field_desc;

typedef struct llgb_record llgb_record;

/* Create a record dimension from `n` leaves (1 <= n <= 64).  Paths are copied.
 * Errors: INVALID_ARG for n out of range, a null/empty/duplicate path or an
 * unknown type.  *out is owned by the caller; release with
 * llgb_record_destroy. */
llgb_status llgb_record_create(const llgb_field_desc* leaves, int32_t n,
                               llgb_record** out);
void llgb_record_destroy(llgb_record* rec);

/* Number of leaves. */
int32_t llgb_record_leaf_count(const llgb_record* rec);

/* Bytes of one record: packed = sum of leaf sizes; aligned = C struct rules
 * (each leaf aligned to its size, the record padded to the largest). */
llgb_status llgb_record_size(const llgb_record* rec, int32_t packed, uint64_t* out);

/* ------------------------------------------------------------- extents -- */

/* Index types (Sec. 2: the type used for all index and offset arithmetic). */
enum {
    LLGB_IDX_I16 = 0, LLGB_IDX_U16, LLGB_IDX_I32, LLGB_IDX_U32,
    LLGB_IDX_I64, LLGB_IDX_U64
};

/* Array extents (Sec. 2).  rank 1..4; ext[d] holds every extent, static or
 * not; bit d of static_mask marks extent d as known at compile time, in which
 * case kernels specialised for that value are used where they exist.  Records
 * are linearised row-major (last index fastest).  n = product of extents. */
typedef struct llgb_extents {
    int32_t rank;
    int32_t index_type;   /* LLGB_IDX_* */
    uint32_t static_mask;
    uint32_t reserved;    /* must be 0 */
    uint64_t ext[4];
} llgb_extents;

/* ------------------------------------------------------------- mapping -- */

enum {
    LLGB_MAP_AOS = 0,          /* array of structs                             */
    LLGB_MAP_SOA_SB,           /* struct of arrays, single blob                */
    LLGB_MAP_SOA_MB,           /* struct of arrays, one blob per leaf          */
    LLGB_MAP_AOSOA,            /* arrays of structs of arrays, `lanes` lanes    */
    LLGB_MAP_BITPACK_INT,      /* BitpackIntSoA: b-bit integers (Sec. 3)       */
    LLGB_MAP_BITPACK_FLOAT,    /* BitpackFloatSoA: (1+E+M)-bit floats (Sec. 3)  */
    LLGB_MAP_BYTESPLIT,        /* Bytesplit over `inner` (Sec. 3)              */
    LLGB_MAP_CHANGETYPE,       /* ChangeType over `inner` (Sec. 3)             */
    LLGB_MAP_NULL,             /* no storage (Sec. 3)                          */
    LLGB_MAP_SPLIT             /* leaves in split_mask via `inner`, the others
                                  via `inner2` (Sec. 3, with Null)              */
};

#define LLGB_MAX_CT 4

/* Mapping descriptor.  Fields not used by `kind` are ignored.
 *  AOS:           aos_packed = 0 aligned (C struct rules, default) / 1 packed.
 *  SOA_SB:        sub-arrays in leaf order in one blob, each starting at a
 *                 multiple of subarray_align (0 = the leaf's own size).
 *  SOA_MB:        blob k holds leaf k as a plain array.
 *  AOSOA:         blocks of `lanes` records; inside a block leaf k's lanes are
 *                 contiguous, leaves packed in order; the last block is whole
 *                 and its unused lanes are zero.
 *  BITPACK_INT:   integral leaves only; leaf k stored with field_bits[k] (or
 *                 `bits`) bits: the low b bits of the two's complement on
 *                 store, zero/sign extension on load; one LSB-first stream of
 *                 little-endian 32-bit words per leaf.
 *  BITPACK_FLOAT: floating-point leaves only; leaf k stored as sign, E =
 *                 field_exp[k] (or exp_bits) exponent bits, M = field_man[k]
 *                 (or man_bits) mantissa bits, IEEE-style, round to nearest
 *                 even, overflow to INF, NaN kept quiet; one stream per leaf.
 *                 2 <= E <= 11, 1 <= M <= 52, 1+E+M <= 64.
 *                 BITPACK_INT and BITPACK_FLOAT are organised by bit_lanes:
 *                 0 = SoA (the streams above, one blob per leaf); L = AoSoA:
 *                 one blob of blocks of L records, each block holding leaf
 *                 0's L codes, then leaf 1's, and so on (the generalisation
 *                 of the SoA organisation that Sec. 3 announces), the last
 *                 block whole with zero codes in its unused lanes.  L is a
 *                 power of two from 32 to 1024, so that every run of a
 *                 block's codes starts on a 32-bit word.
 *  BYTESPLIT:     each leaf becomes size-of-leaf u8 leaves (its little-endian
 *                 bytes) forwarded to `inner`.
 *  CHANGETYPE:    leaves of type ct_from[k] are stored as ct_to[k] (floating
 *                 point types) through `inner`; round to nearest even on store,
 *                 exact or RNE conversion back on load.
 *  NULL:          no blobs: loads give a zero value, stores are discarded.
 *  SPLIT:         the leaves whose bit is set in split_mask form (in leaf
 *                 order) the record of `inner`, the other leaves that of
 *                 `inner2`; the view's blobs are inner's, then inner2's.  Both
 *                 sides hold at least one leaf; any kind may be nested,
 *                 including SPLIT and NULL.
 * The `inner` of BYTESPLIT and CHANGETYPE must be an AOS, SOA_* or AOSOA
 * mapping. */
typedef struct llgb_mapping_desc {
    int32_t kind;
    int32_t aos_packed;
    uint64_t subarray_align;
    uint64_t lanes;
    int32_t bits;
    int32_t exp_bits;
    int32_t man_bits;
    int32_t n_ct;
    int32_t ct_from[LLGB_MAX_CT];
    int32_t ct_to[LLGB_MAX_CT];
    const int32_t* field_bits;
    const int32_t* field_exp;
    const int32_t* field_man;
    const struct llgb_mapping_desc* inner;
    uint64_t split_mask;                     /* SPLIT: bit f = leaf f to `inner` */
    const struct llgb_mapping_desc* inner2;  /* SPLIT: mapping of the others     */
    uint64_t bit_lanes;                      /* BITPACK_*: 0 SoA, else AoSoA lanes */
} llgb_mapping_desc;

/* ---------------------------------------------------------------- view -- */

typedef struct llgb_view llgb_view;

/* Plan a view of `rec` with extents `ext` and mapping `map` (both copied).
 * Computes the blob count and sizes; binds no memory.
 * Errors: INVALID_ARG (bad descriptor), INDEX_OVERFLOW (n or the largest
 * byte offset does not fit the index type), UNSUPPORTED (a nesting of
 * wrappers or a leaf count the GPU planner does not handle).
 * The view keeps a reference to nothing the caller passed. */
llgb_status llgb_view_create(const llgb_record* rec, const llgb_extents* ext,
                             const llgb_mapping_desc* map, llgb_view** out);
void llgb_view_destroy(llgb_view* view);

int32_t llgb_view_blob_count(const llgb_view* view);
uint64_t llgb_view_blob_size(const llgb_view* view, int32_t k);
uint64_t llgb_view_record_count(const llgb_view* view);

/* Bind `n` device blobs (n = llgb_view_blob_count, each at least
 * llgb_view_blob_size bytes, each 16-byte aligned).  The view borrows the
 * pointers; the caller keeps ownership.  Errors: INVALID_ARG (count, null or
 * misaligned pointer). */
llgb_status llgb_view_bind(llgb_view* view, void* const* dev_ptrs, int32_t n);

/* ---------------------------------------------------------------- copy -- */

/* Layout-aware copy (Sec. 1): for every record i < n and leaf f, the logical
 * value of (i, f) is loaded through src's mapping and stored through dst's;
 * every byte of every dst blob that no (i, f) owns is written with zero.
 * Both views must have the same record (leaf types) and the same n; index
 * types may differ.  src and dst blobs must not overlap.  Queued on `stream`.
 * A copy that runs gather programs (byte permutations, such as every pair of
 * plain mappings) takes them from a cache of the library: the first copy of
 * a tile layout on a device and CUDA context (outside stream capture; a
 * device reset starts the cache anew) allocates its program,
 * at most ~150 KB, with cudaMalloc, builds it with a small kernel on a
 * stream of the library's own and waits for that kernel; later copies of
 * the same layout, on any stream, only read it.  The cache holds at most
 * 64 MB per process and is never freed; past that, and during capture, every
 * CTA of the copy builds its program itself (slower for copies of a few
 * hundred MB or less, same bytes).
 * Errors: MISMATCH, UNBOUND, UNSUPPORTED, CUDA. */
llgb_status llgb_copy(const llgb_view* src, llgb_view* dst, void* stream);

/* Pack: copy from a plain (AoS/SoA/AoSoA) view into a BITPACK_* view.
 * Unpack: the reverse.  Same semantics as llgb_copy; the kinds are checked
 * (Sec. 3: values are packed on store and unpacked on load). */
llgb_status llgb_pack(const llgb_view* plain, llgb_view* packed, void* stream);
llgb_status llgb_unpack(const llgb_view* packed, llgb_view* plain, void* stream);

/* Which tile engine a copy runs.  Both move the same bytes.
 *   AUTO:   the library's choice -- gather programs for jobs made only of
 *           byte moves with more than two tiles per CTA, else value loops;
 *   VALUE:  the value loops (per-item loops over each warp's share);
 *   GATHER: per-thread gather programs where the job allows (only byte
 *           moves, within the CTA's program capacity), else value loops. */
typedef enum llgb_engine { LLGB_ENGINE_AUTO = 0, LLGB_ENGINE_VALUE = 1, LLGB_ENGINE_GATHER = 2 } llgb_engine;

/* How tiles move between global and shared memory: the TMA engine (bulk
 * copies issued by one producer warp per direction) or plain coalesced loads
 * and stores by the consumer threads.  Both move the same bytes; which one is
 * faster depends on the pair (many small runs per tile favour plain stores).
 * The last tile of a view, and runs that are not 16-byte aligned, always take
 * plain accesses. */
typedef enum llgb_staging {
    LLGB_STAGING_TMA = 0,         /* TMA loads and stores (default)            */
    LLGB_STAGING_PLAIN_STORE = 1, /* TMA loads, plain stores                   */
    LLGB_STAGING_PLAIN_LOAD = 2,  /* plain loads, TMA stores                   */
    LLGB_STAGING_PLAIN = 3        /* plain loads and stores                    */
} llgb_staging;

/* Launch shape of the copy kernel.  All zero = the library's choice. */
typedef struct llgb_launch_config {
    int32_t tile_records;   /* records per tile; multiple of 128 and of lanes */
    int32_t src_stages;     /* source tiles in flight per CTA (1..8)           */
    int32_t dst_stages;     /* destination tiles in flight per CTA (1..4)      */
    int32_t threads;        /* threads per CTA: 128, 256 or 512                */
    int32_t ctas_per_sm;    /* resident CTAs per SM (1..8)                      */
    int32_t engine;         /* llgb_engine                                     */
    int32_t staging;        /* llgb_staging                                    */
    int32_t reserved;       /* must be 0                                       */
} llgb_launch_config;

/* The launch shape llgb_copy uses for this pair (after autotuning, if any). */
llgb_status llgb_copy_config(const llgb_view* src, const llgb_view* dst,
                             llgb_launch_config* out);

/* What llgb_copy (with cfg, or the library's shape when cfg is NULL or all
 * zero) and a batch entry would run for this pair, planned on the host only:
 * no memory need be bound, nothing is launched.
 *   kernel_mode, batch_kernel_mode: 0 value loops; 1 value loops with
 *     AoSoA-organised bit leaves in the generic loop; 3 value loops with
 *     AoSoA-organised bit leaves in the compile-time stream loops; 2 / 4
 *     gather programs of 2 / 4 source words (a single copy, and the same pair
 *     in a batch or an arena copy);
 *   tile_records, tiles: the tiling; items: work items per tile, of which
 *     generic_items convert values record by record (the others run loops
 *     specialised at compile time, or move bytes), and stream_items pack or
 *     unpack a SoA bit stream whose width and float format are compile-time
 *     constants of one of the library's specialised loops (integer widths 1,
 *     3, 7, 12, 17, 31 of 4-byte leaves; f64 and f32 leaves in the (E, M)
 *     formats E in {5, 8, 11}, M in {2, 10, 23, 52}), in kernel mode 0 for
 *     SoA streams and mode 3 for streams organised as AoSoA.
 * All zero for n = 0.  Errors: INVALID_ARG, MISMATCH, UNSUPPORTED. */
typedef struct llgb_plan_info {
    int32_t kernel_mode;
    int32_t batch_kernel_mode;
    int32_t tile_records;
    int32_t items;
    int32_t generic_items;
    int32_t stream_items;
    uint64_t tiles;
} llgb_plan_info;

llgb_status llgb_copy_plan(const llgb_view* src, const llgb_view* dst, const llgb_launch_config* cfg,
                           llgb_plan_info* out);

/* llgb_copy with an explicit launch shape.  Errors as llgb_copy, plus
 * INVALID_ARG for a shape that does not fit the pair. */
llgb_status llgb_copy_with(const llgb_view* src, llgb_view* dst,
                           const llgb_launch_config* cfg, void* stream);

/* --------------------------------------------------------------- batch -- */

/* Many layout-aware copies (Sec. 1) in one or a few launches: a batch plans
 * every (src[k], dst[k]) pair once, groups the jobs by kernel mode and builds
 * a device descriptor table per group (allocated with cudaMalloc on the
 * current device, released by llgb_batch_destroy).  Each launch moves every
 * pair exactly as llgb_copy would, same bytes.  Views keep their bound blobs
 * for the life of the batch (rebinding a view requires a new batch).  Pairs
 * with n = 0 are skipped.  Gather jobs take their programs from the cache
 * that llgb_copy describes (creation may allocate and wait for the build
 * kernel once per new tile layout).  A batch arena uses the programs the
 * cache already holds (a lookup: it allocates and waits for nothing) and has
 * its CTAs build the others; the allocation-free batch does not use the
 * cache.
 * Errors: as llgb_copy, plus OOM. */
typedef struct llgb_batch llgb_batch;

llgb_status llgb_batch_create(int32_t n, const llgb_view* const* src, llgb_view* const* dst,
                              llgb_batch** out);

/* Queue every copy of the batch on `stream`.  use_graph != 0: the launches
 * are captured once into a CUDA graph (on a private stream) and the graph is
 * replayed on `stream`. */
llgb_status llgb_batch_launch(llgb_batch* b, void* stream, int32_t use_graph);

/* Kernel launches per llgb_batch_launch, total tiles and algorithmic bytes
 * (every source and destination blob byte).  Any pointer may be NULL. */
llgb_status llgb_batch_info(const llgb_batch* b, int32_t* launches, uint64_t* tiles, uint64_t* bytes);

/* Waits for the batch's last queued launch, then frees it. */
void llgb_batch_destroy(llgb_batch* b);

/* Batch arena: batched copies for a loop that submits new pairs all the
 * time (a request loop).  llgb_batch_create allocates and fills device tables
 * (cudaMalloc, a blocking cudaMemcpy) and llgb_batch_destroy frees them
 * (cudaFree): calls that can synchronise the whole device.  An arena
 * allocates, once, descriptor tables for `slots` copies of at most
 * `max_pairs` pairs each, in device memory and in pinned host memory, on the
 * current device.  llgb_batch_arena_copy then moves src[k] -> dst[k] for
 * k < n exactly as llgb_copy does (same bytes), queued on `stream`: it plans
 * the pairs, writes their tables into the next slot's pinned staging and
 * queues one cudaMemcpyAsync of them and the copy kernels (one per kernel
 * mode) on `stream`.  Nothing synchronises the device; the host waits only
 * when the slot it takes is still in use by a copy `slots` calls back.
 * Calls may use different streams; the views' blobs must stay alive until
 * the work queued on them has finished.  An arena is used from any thread
 * (calls are serialised) on the device it was made on.
 * Errors: create -- INVALID_ARG (max_pairs 1..65536, slots 1..64), OOM, CUDA;
 * copy -- as llgb_copy, plus INVALID_ARG (n > max_pairs, another device). */
typedef struct llgb_batch_arena llgb_batch_arena;

llgb_status llgb_batch_arena_create(int32_t max_pairs, int32_t slots, llgb_batch_arena** out);
llgb_status llgb_batch_arena_copy(llgb_batch_arena* a, int32_t n, const llgb_view* const* src,
                                  llgb_view* const* dst, void* stream);
/* Waits for the arena's queued copies, then frees it. */
void llgb_batch_arena_destroy(llgb_batch_arena* a);

/* Batched copy that allocates no device memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate device
 * memory while they run -- cudaMalloc/cudaFree may synchronise the whole
 * device (too slow for latency-critical loops), a host framework's caching
 * allocator may already own all free HBM (a fresh cudaMalloc then fails), or
 * the deployment fixes its device memory at start-up.
 *
 * It moves src[k] -> dst[k] for k < n exactly as llgb_copy does (same bytes),
 * queued on `stream`, with no cudaMalloc, cudaFree or other allocating call.
 * The descriptor tables live in one static device array of this library
 * (about 370 KB, holding at most 64 view pairs), which every GPU that loads
 * the library keeps until the process exits.  They reach that array as the
 * parameters of small upload kernels queued on `stream` ahead of the copy
 * kernels, so no host memory is read after the call returns.
 *   - n <= 64; larger n returns LLGB_ERR_INVALID_ARG (split the work).
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture on the device.  The address is kept per
 *     device and CUDA context: after a device reset (a new context) the next
 *     call looks it up again, and is then again a first call.
 *   - Every call on a device shares the array and overwrites all of it that
 *     the call uses (no state survives between calls).  Calls queued on one
 *     stream run one after the other.  Calls that overlap on the GPU -- on
 *     different streams, or from different host threads -- race on the
 *     array; order them (one stream, or events).
 * Errors: as llgb_copy. */
llgb_status llgb_batch_copy_noalloc(int32_t n, const llgb_view* const* src, llgb_view* const* dst,
                                    void* stream);

/* Autotuner: time candidate launch shapes of llgb_copy(src, dst) on `stream`
 * (each candidate runs the copy 4 times; dst is written) -- first the
 * default shape at other stage counts, and tile records, stages, threads and
 * CTAs per SM with TMA staging, then the staging
 * schemes (llgb_staging) of the fastest shape.  The default shape and the
 * four fastest are timed twice more (best of three); a shape or staging
 * scheme replaces the default only when it is at least 2% faster, so that
 * run-to-run noise does not pick a shape.  The result is kept for this
 * mapping pair and power-of-two record count, and used in later llgb_copy,
 * llgb_batch_create, llgb_batch_arena_copy and llgb_batch_copy_noalloc calls
 * of this process.  A batch entry whose record count has no tuned shape takes
 * the pair's shape tuned for the largest count (in a batch, other entries
 * keep the SMs busy, so a small view needs no small tile).  *best (may be
 * NULL) receives it.  Synchronizes the stream. */
llgb_status llgb_autotune(const llgb_view* src, llgb_view* dst, void* stream, llgb_launch_config* best);

/* Forget every tuned launch shape. */
llgb_status llgb_autotune_clear(void);

/* Persist the tuned launch shapes: save writes every shape of this process
 * to the JSON file `path` ({"llgb_autotune": 1, "entries": {key: [tile_records,
 * src_stages, dst_stages, threads, ctas_per_sm, engine, staging]}}, keyed by
 * mapping pair and power-of-two record count); load adds a file's shapes to
 * those of this process (an entry of the file replaces one with its key), so
 * that a later process skips the tuning.  A shape that no longer fits a pair
 * makes its copies fail with INVALID_ARG: files belong to one build of the
 * library.  Errors: INVALID_ARG (null path, unreadable or malformed file,
 * a value out of range), OOM. */
llgb_status llgb_autotune_save(const char* path);
llgb_status llgb_autotune_load(const char* path);

/* -------------------------------------------------------------- n-body -- */

/* One all-pairs n-body step (Sec. 5, Fig. 2) on a view whose record is the
 * particle {pos.x, pos.y, pos.z, vel.x, vel.y, vel.z, mass} (7 f32 leaves, in
 * this order) under an AOS, SOA_SB, SOA_MB or AOSOA mapping (any lane
 * count).  Update: for
 * every i, v_i += dt * sum_j m_j (p_j - p_i) / (|p_j - p_i|^2 + eps^2)^(3/2),
 * j over all particles; then move: p_i += dt * v_i.  FP32 arithmetic; the
 * result bits do not depend on the mapping.  Queued on `stream` (two
 * kernels).  Errors: INVALID_ARG (not the particle record), UNBOUND,
 * UNSUPPORTED (a bit-packed, Bytesplit, ChangeType or Split view, or
 * n >= 2^31), CUDA. */
llgb_status llgb_nbody_step(llgb_view* particles, float eps, float dt, void* stream);

/* The two phases of llgb_nbody_step apart, each with a chosen traversal of
 * the records (Sec. 5: the single loop over the flat index that a mapping-
 * agnostic consumer writes, against loops nested the way the mapping lays
 * records out, which the paper leaves open for AoSoA):
 *   LLGB_TRAVERSE_INDEX: one thread per record index i; every access maps i
 *       through the mapping (for AoSoA with L lanes, i / L and i % L).
 *   LLGB_TRAVERSE_BLOCKS: the walk follows the layout.  Move: for AoSoA, one
 *       AoSoA block after another, the block's 3 L pos floats updated as one
 *       contiguous run from the 3 L vel floats after them (16-byte accesses
 *       when L is a multiple of 4); for SoA, 4 consecutive records of each
 *       leaf per thread (16-byte accesses when the leaf arrays are 16-byte
 *       aligned); an AoS record is its own block.  Update: addresses advance
 *       as a (block, lane) cursor, one division per thread instead of one per
 *       access.
 * Both traversals give the same result bits, and llgb_nbody_update followed
 * by llgb_nbody_move gives the bits of llgb_nbody_step.  AoSoA views may have
 * any lane count.  Errors: as llgb_nbody_step, plus INVALID_ARG (unknown
 * traversal). */
typedef enum llgb_traversal { LLGB_TRAVERSE_INDEX = 0, LLGB_TRAVERSE_BLOCKS = 1 } llgb_traversal;

/* Update only: v_i += dt * sum_j m_j (p_j - p_i) / (|p_j - p_i|^2 + eps^2)^(3/2). */
llgb_status llgb_nbody_update(llgb_view* particles, float eps, float dt, int32_t traversal, void* stream);

/* Move only: p_i += dt * v_i (one fused multiply-add per leaf). */
llgb_status llgb_nbody_move(llgb_view* particles, float dt, int32_t traversal, void* stream);

/* FP32 throughput probe, the roofline of the n-body update (an FP32 ALU-bound
 * loop).  The paper has no counterpart: it measures the peak the n-body's
 * TFLOP/s are divided by.  Queues one kernel on `stream` whose threads fill
 * every warp slot of every SM and each run 16 independent fused
 * multiply-add chains for `iters` rounds; *fmas (host) receives the number of
 * FMAs it performs (2 FLOP each).  Time it with events on `stream`.  `sink`:
 * one device float the kernel may write.  Errors: INVALID_ARG, CUDA. */
llgb_status llgb_fma_probe(uint32_t iters, float* sink, uint64_t* fmas, void* stream);

/* --------------------------------------------- access instrumentation -- */

/* FieldAccessCount and Heatmap (Sec. 4, "Memory access instrumentation") of
 * the n-body consumer: llgb_nbody_step, with every access it makes through
 * the view counted as a side effect.  The result bits are those of
 * llgb_nbody_step.
 *   field_counts: NULL, or 14 device uint64 counters, 8-byte aligned,
 *       incremented (not zeroed): reads of leaves 0..6, then writes of
 *       leaves 0..6 (FieldAccessCount: two counters per record field).
 *   count_mode: how field_counts are incremented --
 *       LLGB_COUNT_ATOMIC: one global atomic increment per access (the
 *           paper's scheme);
 *       LLGB_COUNT_BLOCK: per-CTA shared-memory counters added to the global
 *           ones once per CTA (the same counts).
 *   heat, granularity: NULL, or llgb_heatmap_counters(particles, g) device
 *       uint64 counters, 8-byte aligned, incremented: counter k of blob b
 *       (after the counters of blobs 0 .. b-1) counts the accesses touching
 *       bytes [k g, (k+1) g) of blob b; an access of a 4-byte leaf touches
 *       every granule its bytes overlap.  g: a power of two (1 = bytes,
 *       64 = cache lines).  One global atomic increment per touched granule.
 * Accesses of one step: the update reads each particle's pos once, the pos
 * and mass of every particle once per 64-particle block of the update
 * (B = ceil(n / 64) blocks), and reads and writes each vel once; the move
 * reads each pos and vel once and writes each pos once.
 * Errors: as llgb_nbody_step, plus INVALID_ARG (count mode, granularity,
 * alignment). */
typedef enum llgb_count_mode { LLGB_COUNT_ATOMIC = 1, LLGB_COUNT_BLOCK = 2 } llgb_count_mode;

llgb_status llgb_nbody_step_instrumented(llgb_view* particles, float eps, float dt, uint64_t* field_counts,
                                         int32_t count_mode, uint64_t* heat, uint64_t granularity, void* stream);

/* Number of Heatmap counters of `view` at `granularity` bytes (a power of
 * two): the sum over its blobs of ceil(blob bytes / granularity). */
llgb_status llgb_heatmap_counters(const llgb_view* view, uint64_t granularity, uint64_t* counters);

/* -------------------------------------------------------------- status -- */

/* Read the device status word that kernels set when a bounded wait gives up
 * (LLGB_ERR_TIMEOUT); 0 when none did.  Synchronizes the current device.
 * reset != 0 clears the word. */
llgb_status llgb_device_status(int32_t* code, int32_t reset);

/* Self-test of the failure detection of the copy kernels.  Every wait of a
 * copy kernel on one of its pipeline barriers is bounded (2 s); when one runs
 * out, the kernel stops its CTA's work, records LLGB_ERR_TIMEOUT in the device
 * status word and returns, so that the CUDA context stays usable.  This call
 * queues one small kernel on `stream` that takes that same bounded wait on a
 * barrier no thread ever arrives on, with the limit `limit_ns` (1 us .. 10 s)
 * instead of 2 s: it gives up after limit_ns, records LLGB_ERR_TIMEOUT and
 * returns.  `waited_ns` (a device uint64, 8-byte aligned, or NULL) receives the
 * time the wait took.  Read the status with llgb_device_status.
 * Errors: INVALID_ARG (limit out of range, misaligned pointer), CUDA. */
llgb_status llgb_wait_selftest(uint64_t limit_ns, uint64_t* waited_ns, void* stream);

#ifdef __cplusplus
}
#endif

#endif
