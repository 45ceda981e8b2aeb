// capi.cpp -- the C ABI declared in include/llgb.h.
//
// Host-side validation, planning and launch.  No exception leaves this file:
// every entry point catches and turns failures into an llgb_status with a
// thread-local message.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <map>
#include <mutex>
#include <new>
#include <set>
#include <string>
#include <vector>

#include "job.h"
#include "kernels.h"
#include "llgb.h"
#include "plan.h"

// A planned copy into a view, kept so that repeated llgb_copy calls of the
// same pair skip the host planning: valid while the source view, both views'
// bound blobs, the current device and the tuned launch shapes are unchanged.
struct CopyPlanCache {
    bool valid = false;
    uint64_t src_id = 0, src_bind = 0, dst_bind = 0, tune_gen = 0;
    int device = -1;
    int mode = 0, grid = 0, threads = 0;
    size_t smem = 0;
    llgb::CopyArgs args;
};

struct llgb_view {
    llgb::ViewPlan plan;
    std::vector<void*> ptrs;
    bool bound = false;
    uint64_t id = 0;         // unique over the process, never reused
    uint64_t bind_gen = 0;   // counts llgb_view_bind calls
    std::mutex cache_mu;
    CopyPlanCache cache;     // the last copy planned into this view
};

using namespace llgb;

namespace {

std::atomic<uint64_t> g_view_ids{1};
std::atomic<uint64_t> g_tune_gen{1};  // bumped whenever a tuned launch shape changes

thread_local std::string t_error;

llgb_status fail(llgb_status s, const std::string& msg)
{
    t_error = msg;
    return s;
}

llgb_status cuda_fail(cudaError_t e, const char* what)
{
    return fail(LLGB_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

struct DeviceInfo {
    int sms = 0;
    int max_smem = 0;       // dynamic shared memory one CTA may opt into
    int smem_per_sm = 0;    // shared memory of an SM
    int reserved_smem = 0;  // shared memory the system reserves per CTA
};

DeviceInfo device_info()
{
    static std::mutex mu;
    static std::vector<DeviceInfo> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return {};
    std::lock_guard<std::mutex> lock(mu);
    if ((int)cache.size() <= dev) cache.resize(dev + 1);
    if (cache[dev].sms == 0) {
        cudaDeviceGetAttribute(&cache[dev].sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&cache[dev].max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaDeviceGetAttribute(&cache[dev].smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        cudaDeviceGetAttribute(&cache[dev].reserved_smem, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    }
    return cache[dev];
}

// `ctas` CTAs of `smem` dynamic shared memory each are resident on one SM
// together (without a device: the limits of this GPU family).
bool smem_fits(size_t smem, int ctas)
{
    const DeviceInfo dev = device_info();
    const size_t per_cta = dev.max_smem > 0 ? (size_t)dev.max_smem : 232448;
    const size_t per_sm = dev.smem_per_sm > 0 ? (size_t)dev.smem_per_sm : 233472;
    const size_t reserved = dev.max_smem > 0 ? (size_t)dev.reserved_smem : 1024;
    return smem <= per_cta && (size_t)ctas * (smem + reserved) <= per_sm;
}

bool same_record(const ViewPlan& a, const ViewPlan& b) { return a.types == b.types; }

// Shared memory a launch shape needs for a pair (JobDesc planned at `tile`).
size_t smem_needed(const JobDesc& J, const llgb_launch_config& c)
{
    return copy_shared_header_bytes() + (size_t)c.src_stages * (J.src.img_bytes + kStageZeroBytes) +
           (size_t)c.dst_stages * J.dst.img_bytes + J.code_bytes;
}

bool valid_threads(int t) { return t == 128 || t == 256 || t == 512; }

// Plain consumer loads and / or stores instead of TMA bulk copies
// (llgb_staging): the kernel then moves every tile of that side the way it
// moves unaligned runs.
void apply_staging(JobDesc* job, int staging)
{
    if (staging & LLGB_STAGING_PLAIN_STORE) job->dst.bulk_ok = 0;
    if (staging & LLGB_STAGING_PLAIN_LOAD) job->src.bulk_ok = 0;
}

// Gather programs built once on the GPU and shared by every CTA of every
// copy whose job has the same tile-local layout (the program depends on the
// leaves' image addressing, the items, the tile and the CTA's consumer
// count -- not on record counts or blob addresses).  Kept for the process:
// at most kProgramCacheBytes of device memory; past that, and during stream
// capture, jobs carry no program and every CTA builds its own.
constexpr size_t kProgramCacheBytes = 64u << 20;

struct ProgramEntry {
    JobDesc key;
    int device = -1, mode = 0;
    uint64_t context = 0;  // a device reset makes a new context, and the old buffers invalid
    uint32_t consumers = 0;
    uint32_t* dev = nullptr;
};

// Identity of the CUDA context current on this thread (0 if it cannot be
// read), through the driver entry points the runtime hands out.
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

uint64_t context_identity()
{
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

std::mutex prog_mu;
std::multimap<uint64_t, ProgramEntry> prog_cache;
size_t prog_bytes = 0;
std::map<std::pair<int, uint64_t>, cudaStream_t> prog_streams;  // per device and context: the stream programs are built on

static_assert(sizeof(JobDesc) % 8 == 0, "program keys are hashed in 8-byte words");

JobDesc program_key(const JobDesc& J)
{
    JobDesc k = J;
    k.n = 0;
    k.ntiles = k.nfull = 0;
    k.program = 0;
    for (SideDesc* S : {&k.src, &k.dst}) {
        memset(S->blobs, 0, sizeof S->blobs);
        S->bulk_ok = 0;
        for (SegDesc& g : S->segs) {
            g.gbase = 0;
            g.tail_bytes = 0;
        }
    }
    k.nzeros = 0;
    memset(k.zeros, 0, sizeof k.zeros);
    return k;
}

// FNV-1a over 8-byte words (n a multiple of 8; JobDesc is).
uint64_t hash_words(const void* p, size_t n)
{
    uint64_t h = 1469598103934665603ull;
    for (size_t i = 0; i + 8 <= n; i += 8) {
        uint64_t w;
        memcpy(&w, static_cast<const unsigned char*>(p) + i, 8);
        h = (h ^ w) * 1099511628211ull;
    }
    return h;
}

// Device address of J's gather program for `mode` CTAs of `threads`
// threads, built (once per layout, device and consumer count) on a stream of
// the library's own and waited for, so that copies on any stream may use it;
// 0 when none can be had (the caller's stream is capturing, the cache is
// full, or a CUDA call failed).  build false: a lookup only, which allocates
// and waits for nothing (0 if the layout has no program yet).
uint64_t gather_program(const JobDesc& J, int mode, int threads, cudaStream_t caller, bool build = true)
{
    if (!gather_mode(mode) || J.gather == 0) return 0;
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return 0;
    const uint64_t context = context_identity();
    if (context == 0) return 0;  // no way to tell a reset device's buffers from live ones
    const uint32_t consumers = (uint32_t)threads - 32u * producer_warps(mode);
    static thread_local JobDesc key;
    key = program_key(J);
    const uint64_t h = hash_words(&key, sizeof key) ^ ((uint64_t)device << 56) ^ ((uint64_t)mode << 48) ^ consumers;
    std::lock_guard<std::mutex> lock(prog_mu);
    auto range = prog_cache.equal_range(h);
    for (auto it = range.first; it != range.second; ++it) {
        const ProgramEntry& e = it->second;
        if (e.device == device && e.context == context && e.mode == mode && e.consumers == consumers &&
            memcmp(&e.key, &key, sizeof key) == 0)
            return (uint64_t)(uintptr_t)e.dev;
    }
    const size_t bytes = gather_program_words(mode, consumers) * 4u;
    if (!build || prog_bytes + bytes > kProgramCacheBytes) return 0;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(caller, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return 0;
    }
    cudaStream_t& ps = prog_streams[{device, context}];
    if (!ps && cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking) != cudaSuccess) {
        ps = nullptr;
        cudaGetLastError();
        return 0;
    }
    uint32_t* dev = nullptr;
    if (cudaMalloc(&dev, bytes) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (launch_gather_program(J, mode, consumers, dev, ps) != cudaSuccess || cudaStreamSynchronize(ps) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(dev);
        return 0;
    }
    ProgramEntry e;
    e.key = key;
    e.device = device;
    e.context = context;
    e.mode = mode;
    e.consumers = consumers;
    e.dev = dev;
    prog_cache.emplace(h, e);
    prog_bytes += bytes;
    return (uint64_t)(uintptr_t)dev;
}

// Kernel mode of a planned job under a launch shape: its gather form when the
// gather programs cover the destination image with the consumer threads,
// else the general kernel (0).
int job_mode(const JobDesc& J, int threads)
{
    if (J.seg) return J.seg;
    int mode = J.gather;
    if (mode == 0) return 0;
    // words the gather programs cover: every run (interleaved), or the whole
    // image up to its last slack (linear)
    uint64_t words = (J.dst.img_bytes - kImageSlack) / 4u;
    if (J.interleave) {
        words = 0;
        for (int q = 0; q < J.dst.nsegs; ++q) words += ((J.dst.segs[q].tile_bytes + 15u) & ~15u) / 4u;
    }
    // the producer warps of every CTA issue TMA copies; the rest run the programs
    if (words > (uint64_t)gather_words_per_thread(mode) * (uint64_t)(threads - 32 * (int)producer_warps(mode))) mode = 0;
    return mode;
}

// Launch shapes chosen by llgb_autotune, keyed by mapping pair and the
// record count's power of two.
std::mutex tune_mu;
std::map<std::string, llgb_launch_config> tune_cache;

std::string tune_key(const llgb_view* src, const llgb_view* dst)
{
    int bucket = 0;
    while (bucket < 63 && (1ull << (bucket + 1)) <= src->plan.n) ++bucket;
    return src->plan.sig + "|" + dst->plan.sig + "|" + std::to_string(bucket);
}

// any_bucket: a batch entry, whose batch keeps the SMs busy, takes the pair's
// shape tuned for its largest record count when its own count has none.
bool tuned_config(const llgb_view* src, const llgb_view* dst, llgb_launch_config* out, bool any_bucket = false)
{
    std::lock_guard<std::mutex> lock(tune_mu);
    auto it = tune_cache.find(tune_key(src, dst));
    if (it != tune_cache.end()) {
        *out = it->second;
        return true;
    }
    if (!any_bucket) return false;
    const std::string prefix = src->plan.sig + "|" + dst->plan.sig + "|";
    int best_bucket = -1;
    for (const auto& kv : tune_cache) {
        if (kv.first.compare(0, prefix.size(), prefix) != 0) continue;
        const int bucket = atoi(kv.first.c_str() + prefix.size());
        if (bucket > best_bucket) {
            best_bucket = bucket;
            *out = kv.second;
        }
    }
    return best_bucket >= 0;
}

// A job whose every item packs an integer leaf into a bit stream in a
// specialised loop: little consumer work per byte read.
static bool int_pack_job(const JobDesc& J)
{
    if (J.nitems == 0) return false;
    for (int i = 0; i < J.nitems; ++i) {
        const ItemDesc& it = J.items[i];
        if (it.op != ITEM_VALUE || it.lop != L_DIRECT || it.sop != S_BITS_INT) return false;
        if (it.fast == FK_GENERIC && it.spec == 0) return false;
    }
    return true;
}

// Default launch shape (from launch-shape sweeps on GB300).
//  * Gather jobs (byte permutations) run two 256-thread CTAs per SM on
//    tiles of up to ~16 KB, shrunk until the CTA's gather programs cover
//    them (a thread's program holds a fixed number of destination words):
//    the largest such tile keeps the most bytes in flight (2^26-record
//    particle SoA -> AoS: 384-record tiles 0.84, 512-record tiles 0.97 of
//    measured HBM) -- or, with four or more destination runs per tile, one
//    512-thread CTA on ~30 KB tiles.
//  * Other jobs run one 512-thread CTA per SM with two source and two
//    destination stages of the largest tile that fits (at most 4096
//    records): per-tile costs are then spread over the most records.
//    Integer-stream packs, whose consumers have little to do per byte
//    read, run two 256-thread CTAs per SM instead: each has its own load
//    pipeline, and together they keep more bytes in flight (b = 1 pack
//    0.80 -> 0.91, b = 12 0.94 -> 0.98 of measured HBM); float packs and
//    unpacks measured faster with one 512-thread CTA.
// Small views keep at least two tiles per CTA.
// for_batch: the pair is one entry of a batch, whose other entries keep the
// SMs busy, so a small view keeps its full-size tile.
llgb_status default_config(const llgb_view* src, const llgb_view* dst, llgb_launch_config* out, bool for_batch = false)
{
    const DeviceInfo dev = device_info();
    const int sms = dev.sms > 0 ? dev.sms : 152;
    const uint32_t q = tile_quantum(src->plan, dst->plan);
    if (q == 0) return fail(LLGB_ERR_UNSUPPORTED, "AoSoA lane counts give no usable tile size");
    std::vector<void*> none_s(src->plan.blob_sizes.size(), nullptr), none_d(dst->plan.blob_sizes.size(), nullptr);
    static thread_local JobDesc probe;
    std::string why;
    if (plan_job(src->plan, none_s, dst->plan, none_d, q, &probe, &why) != LLGB_OK)
        return fail(LLGB_ERR_UNSUPPORTED, why);
    const bool gather = probe.gather != 0;
    llgb_launch_config c{};
    double sb = 0, db = 0;
    uint32_t cb = 0;
    bytes_per_record(src->plan, dst->plan, &sb, &db, &cb);
    uint64_t tile;
    if (gather && probe.dst.nsegs >= 4) {
        // many destination runs (SoA-like destinations): one 512-thread CTA
        // per SM, whose programs cover ~30 KB tiles, issues a quarter as many
        // bulk stores per byte as two 256-thread CTAs on 12 KB tiles
        c.threads = 512;
        c.ctas_per_sm = 1;
        c.src_stages = 4;
        c.dst_stages = 2;
        tile = (uint64_t)(30720.0 / std::max(std::max(sb, db), 1.0)) / q * q;
    } else if (gather) {
        c.threads = 256;
        c.ctas_per_sm = 2;
        c.src_stages = 4;
        c.dst_stages = 3;
        tile = (uint64_t)(16384.0 / std::max(std::max(sb, db), 1.0)) / q * q;
    } else {
        const bool light = int_pack_job(probe);
        c.threads = light ? 256 : 512;
        c.ctas_per_sm = light ? 2 : 1;
        c.src_stages = 2;
        c.dst_stages = 2;
        const double budget = 227.0 * 1024 / c.ctas_per_sm - (double)copy_shared_header_bytes() - 64.0;
        tile = (uint64_t)(budget / (2.0 * (std::max(sb, 1.0) + std::max(db, 1.0)))) / q * q;
        tile = std::min<uint64_t>(tile, 4096 / q * q);
        // integer-stream packs: a multiple of 256 records, so that every
        // stream run of a tile is whole 32-byte sectors (measured: b = 1
        // pack 0.88 at 2176 records, 0.94 at 2048; b = 31 0.93 at 1152,
        // 0.96 at 1024; b = 17 the other way, 0.96 at 1408, 0.94 at 1280)
        const uint64_t q256 = std::max<uint64_t>(q, 256u / q * q);
        if (light && q256 % q == 0 && tile >= 2 * q256) tile = tile / q256 * q256;
    }
    if (tile < q) tile = q;
    if (!for_batch) {
        const uint64_t n = src->plan.n;
        const uint64_t want = (n + 2ull * sms * c.ctas_per_sm - 1) / (2ull * sms * c.ctas_per_sm);
        const uint64_t small = std::max<uint64_t>(q, (want + q - 1) / q * q);
        tile = std::min(tile, small);
    }
    for (;;) {
        if (plan_job(src->plan, none_s, dst->plan, none_d, (uint32_t)tile, &probe, &why) != LLGB_OK)
            return fail(LLGB_ERR_UNSUPPORTED, why);
        // a gather job keeps its tile within what the CTA's programs cover
        if (gather && tile > q && job_mode(probe, c.threads) == 0) {
            tile -= q;
            continue;
        }
        if (smem_fits(smem_needed(probe, c), c.ctas_per_sm)) break;
        if (c.src_stages > 2) {
            --c.src_stages;
            continue;
        }
        if (c.dst_stages > 2) {
            --c.dst_stages;
            continue;
        }
        if (tile <= q) {
            if (c.ctas_per_sm > 1) {
                c.ctas_per_sm = 1;
                continue;
            }
            return fail(LLGB_ERR_UNSUPPORTED, "record too large for a shared-memory tile");
        }
        tile -= q;
    }
    c.tile_records = (int32_t)tile;
    *out = c;
    return LLGB_OK;
}

// A job of a batch, planned at its launch shape's tile -- capped so that its
// source and destination images each stay within a quarter of a CTA's
// shared memory: a batch kernel sizes every stage for the largest image of
// its group, and two source plus two destination stages of any mix of such
// jobs then fit.  Jobs of at most kFewTiles tiles run the value loops: every
// CTA that meets a gather job builds its program, which short jobs do not
// repay.
constexpr uint32_t kFewTiles = 4;
// In a batch a gather job shares its CTAs' time with other jobs, and every
// CTA that meets it builds its programs again: jobs of at most this many
// tiles move their bytes in the value loops instead, and a gather group runs
// at most one CTA per kGatherTilesPerCta of its tiles.
constexpr uint32_t kFewGatherTiles = 16;
constexpr uint64_t kGatherTilesPerCta = 8;

// fit_gather: a job made of byte moves keeps its gather programs by running
// in CTAs of its own launch shape's thread count (*threads_out), its tile
// shrunk until those CTAs' programs cover it; otherwise (fit_gather false)
// its mode is judged for `threads`-thread CTAs as planned.
llgb_status plan_batch_job(const llgb_view* src, const llgb_view* dst, JobDesc* job, int* mode, int threads,
                           bool fit_gather = false, int* threads_out = nullptr)
{
    llgb_launch_config c{};
    if (!tuned_config(src, dst, &c, fit_gather)) {
        const llgb_status st = default_config(src, dst, &c, fit_gather);
        if (st != LLGB_OK) return st;
    }
    const DeviceInfo dev = device_info();
    const size_t per_cta = dev.max_smem > 0 ? (size_t)dev.max_smem : 232448;
    const size_t side_cap = (per_cta - copy_shared_header_bytes()) / 4 - kStageZeroBytes;
    const uint32_t q = tile_quantum(src->plan, dst->plan);
    uint32_t tile = (uint32_t)c.tile_records;
    std::string why;
    for (;;) {
        const llgb_status st = plan_job(src->plan, src->ptrs, dst->plan, dst->ptrs, tile, job, &why);
        if (st != LLGB_OK) return fail(st, why);
        if ((job->src.img_bytes <= side_cap && job->dst.img_bytes <= side_cap) || tile <= q) break;
        tile -= q;
    }
    if (fit_gather && job->gather && job->ntiles > kFewTiles) {
        threads = c.threads;
        while (job_mode(*job, threads) == 0 && tile > q) {
            tile -= q;
            const llgb_status st = plan_job(src->plan, src->ptrs, dst->plan, dst->ptrs, tile, job, &why);
            if (st != LLGB_OK) return fail(st, why);
        }
    }
    apply_staging(job, c.staging);
    // few-tile jobs take the value loops; run-addressed bit jobs need mode 1 for them
    const uint32_t few = fit_gather && job->gather ? kFewGatherTiles : kFewTiles;
    *mode = job->ntiles <= few ? job->seg : job_mode(*job, threads);
    if (threads_out) *threads_out = gather_mode(*mode) ? threads : 0;
    return LLGB_OK;
}

llgb_status check_pair(const llgb_view* src, const llgb_view* dst)
{
    if (!src || !dst) return fail(LLGB_ERR_INVALID_ARG, "null view");
    if (!same_record(src->plan, dst->plan)) return fail(LLGB_ERR_MISMATCH, "views have different records");
    if (src->plan.n != dst->plan.n) return fail(LLGB_ERR_MISMATCH, "views have different record counts");
    if (!src->bound || !dst->bound) return fail(LLGB_ERR_UNBOUND, "view used before llgb_view_bind");
    return LLGB_OK;
}

// Kernel mode of a single copy's job under launch shape c on `grid` CTAs.
int copy_mode(const JobDesc& J, const llgb_launch_config& c, int grid)
{
    int mode = c.engine == LLGB_ENGINE_VALUE ? J.seg : job_mode(J, c.threads);
    // a gather program is built once per job by every CTA: with at most two
    // tiles per CTA that costs more than it saves, and the value loops
    // (whole-element moves) need no program
    if (c.engine == LLGB_ENGINE_AUTO && gather_mode(mode) && J.ntiles <= 2u * (uint32_t)grid) mode = 0;
    return mode;
}

llgb_status run_copy(const llgb_view* src, llgb_view* dst, const llgb_launch_config* cfg_in, void* stream)
{
    llgb_status st = check_pair(src, dst);
    if (st != LLGB_OK) return st;
    if (src->plan.n == 0) return LLGB_OK;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool library_shape = !(cfg_in && cfg_in->tile_records != 0);
    int device = 0;
    cudaGetDevice(&device);
    const uint64_t tune_gen = g_tune_gen.load();
    std::lock_guard<std::mutex> lock(dst->cache_mu);
    CopyPlanCache& C = dst->cache;
    if (library_shape && C.valid && C.src_id == src->id && C.src_bind == src->bind_gen &&
        C.dst_bind == dst->bind_gen && C.device == device && C.tune_gen == tune_gen) {
        const cudaError_t e = launch_copy(C.args, C.mode, C.grid, C.threads, C.smem, s);
        if (e != cudaSuccess) return cuda_fail(e, "copy kernel launch");
        return LLGB_OK;
    }
    llgb_launch_config c{};
    if (!library_shape) {
        c = *cfg_in;
    } else if (!tuned_config(src, dst, &c)) {
        st = default_config(src, dst, &c);
        if (st != LLGB_OK) return st;
    }
    if (!valid_threads(c.threads) || c.src_stages < 1 || c.src_stages > 8 || c.dst_stages < 1 ||
        c.dst_stages > 4 || c.ctas_per_sm < 1 || c.ctas_per_sm > 8)
        return fail(LLGB_ERR_INVALID_ARG, "launch config out of range");
    static thread_local CopyArgs args;
    memset(&args, 0, sizeof args);
    std::string why;
    st = plan_job(src->plan, src->ptrs, dst->plan, dst->ptrs, (uint32_t)c.tile_records, &args.job, &why);
    if (st != LLGB_OK) return fail(st, why);
    apply_staging(&args.job, c.staging);
    const DeviceInfo dev = device_info();
    const size_t smem = smem_needed(args.job, c);
    if (!smem_fits(smem, c.ctas_per_sm))
        return fail(LLGB_ERR_INVALID_ARG, "launch config needs more shared memory than an SM has");
    args.table = nullptr;
    args.tile_start = nullptr;
    args.njobs = 1;
    args.total_tiles = args.job.ntiles;
    args.src_stage_bytes = args.job.src.img_bytes + kStageZeroBytes;
    args.dst_stage_bytes = args.job.dst.img_bytes;
    args.code_bytes = args.job.code_bytes;
    args.src_stages = (uint16_t)c.src_stages;
    args.dst_stages = (uint16_t)c.dst_stages;
    const int sms = dev.sms > 0 ? dev.sms : 152;
    const int grid = (int)std::min<uint64_t>(args.total_tiles, (uint64_t)sms * c.ctas_per_sm);
    const int mode = copy_mode(args.job, c, grid);
    if (c.threads / 32 <= (int)producer_warps(mode))
        return fail(LLGB_ERR_INVALID_ARG, "launch config leaves no consumer warp");
    if (gather_mode(mode)) args.job.program = gather_program(args.job, mode, c.threads, s);
    cudaError_t e = launch_copy(args, mode, grid, c.threads, smem, s);
    if (e != cudaSuccess) return cuda_fail(e, "copy kernel launch");
    if (library_shape) {
        C.args = args;
        C.mode = mode;
        C.grid = grid;
        C.threads = c.threads;
        C.smem = smem;
        C.src_id = src->id;
        C.src_bind = src->bind_gen;
        C.dst_bind = dst->bind_gen;
        C.device = device;
        C.tune_gen = tune_gen;
        C.valid = true;
    } else {
        C.valid = false;
    }
    return LLGB_OK;
}

bool is_bitpacked(const llgb_view* v)
{
    return v && (v->plan.base == BASE_BITS_INT || v->plan.base == BASE_BITS_FLOAT);
}

}  // namespace

// Helpers for the allocation-free batched entry point (noalloc.cu).
namespace llgb {

llgb_status internal_fail(llgb_status status, const char* message) { return fail(status, message); }

llgb_status internal_plan_pair(const llgb_view* src, const llgb_view* dst, JobDesc* job, int* mode, int threads)
{
    llgb_status st = check_pair(src, dst);
    if (st != LLGB_OK) return st;
    return plan_batch_job(src, dst, job, mode, threads);
}

bool internal_empty(const llgb_view* v) { return v->plan.n == 0; }

void internal_device_limits(int* sms, size_t* smem_cap)
{
    const DeviceInfo dev = device_info();
    *sms = dev.sms > 0 ? dev.sms : 152;
    *smem_cap = dev.max_smem > 0 ? (size_t)dev.max_smem : 232448;
}

bool internal_smem_fits(size_t smem, int ctas) { return smem_fits(smem, ctas); }

}  // namespace llgb

namespace {

// A group of a batch: the jobs of one kernel mode, run by one launch of the
// copy kernel over a descriptor table (args.table / args.tile_start are set
// once the tables have a device address).
struct BatchGroup {
    int mode = 0;
    int threads = 256;
    int grid = 0;
    size_t smem = 0;
    std::vector<JobDesc> jobs;
    std::vector<uint32_t> starts;     // first tile of each job, then the total
    std::vector<uint32_t> cta_tiles;  // first tile of each CTA, then the total
    CopyArgs args;
};

// Tiles of a group split over its CTAs by bytes rather than by count: a tile
// weighs its job's source and destination image bytes plus a fixed cost, and
// CTA b takes the tiles whose weight falls into the b-th equal part.  Jobs of
// one group differ several-fold in bytes per tile.
constexpr double kTileFixedBytes = 8192.0;

void balance_ctas(BatchGroup& g)
{
    const size_t nj = g.jobs.size();
    std::vector<double> w(nj);
    double total = 0.0;
    for (size_t j = 0; j < nj; ++j) {
        w[j] = (double)g.jobs[j].src.img_bytes + (double)g.jobs[j].dst.img_bytes + kTileFixedBytes;
        total += w[j] * (double)g.jobs[j].ntiles;
    }
    const uint32_t grid = (uint32_t)g.grid;
    g.cta_tiles.assign(grid + 1u, 0u);
    size_t j = 0;
    double before = 0.0;  // weight of the tiles of jobs 0 .. j-1
    for (uint32_t b = 1; b < grid; ++b) {
        const double target = total * (double)b / (double)grid;
        while (j + 1 < nj && before + w[j] * (double)g.jobs[j].ntiles <= target) {
            before += w[j] * (double)g.jobs[j].ntiles;
            ++j;
        }
        double into = std::ceil((target - before) / w[j]);
        if (into < 0.0) into = 0.0;
        uint32_t t = g.starts[j] + (uint32_t)std::min<double>(into, (double)g.jobs[j].ntiles);
        g.cta_tiles[b] = std::max(t, g.cta_tiles[b - 1]);
    }
    g.cta_tiles[grid] = g.starts[nj];
}

// Plan every (src[k], dst[k]) pair once and group the jobs by kernel mode
// and, for gather jobs, the CTA size their programs were sized for.  Each
// group gets its launch shape: stages sized for the largest images of the
// group; value groups run two 256-thread CTAs per SM where they fit, else one
// of 512; 256-thread gather groups two CTAs, 512-thread ones one.
// Gather jobs' programs: kProgramsBuild takes them from the program cache,
// building missing ones (which may allocate and wait for a small build
// kernel); kProgramsLookup takes only those the cache already holds; the
// CTAs build the rest, and every program with kProgramsNone.
enum { kProgramsNone = 0, kProgramsLookup = 1, kProgramsBuild = 2 };
llgb_status plan_groups(int32_t n, const llgb_view* const* src, llgb_view* const* dst, std::vector<BatchGroup>* out,
                        uint64_t* bytes, uint64_t* tiles, int programs = kProgramsNone, cudaStream_t stream = nullptr)
{
    const DeviceInfo dev = device_info();
    const int sms = dev.sms > 0 ? dev.sms : 152;
    std::vector<BatchGroup> groups;
    *bytes = 0;
    *tiles = 0;
    for (int32_t k = 0; k < n; ++k) {
        llgb_status st = check_pair(src[k], dst[k]);
        if (st != LLGB_OK) return fail(st, "batch entry " + std::to_string(k) + ": " + t_error);
        if (src[k]->plan.n == 0) continue;
        JobDesc J;
        int mode = 0, threads = 0;
        st = plan_batch_job(src[k], dst[k], &J, &mode, 256, true, &threads);
        if (st != LLGB_OK) return fail(st, "batch entry " + std::to_string(k) + ": " + t_error);
        BatchGroup* g = nullptr;
        for (BatchGroup& x : groups)
            if (x.mode == mode && (!gather_mode(mode) || x.threads == threads)) g = &x;
        if (!g) {
            groups.emplace_back();
            g = &groups.back();
            g->mode = mode;
            g->threads = gather_mode(mode) ? threads : 0;
        }
        if (programs != kProgramsNone && gather_mode(mode))
            J.program = gather_program(J, mode, threads, stream, programs == kProgramsBuild);
        g->jobs.push_back(J);
        for (uint64_t s : src[k]->plan.blob_sizes) *bytes += s;
        for (uint64_t s : dst[k]->plan.blob_sizes) *bytes += s;
        *tiles += J.ntiles;
    }
    out->clear();
    for (BatchGroup& g : groups) {
        // tile numbers are per group, starting at 0
        uint64_t total = 0;
        uint32_t src_bytes = 0, dst_bytes = 0;
        g.starts.clear();
        for (size_t q = 0; q < g.jobs.size(); ++q) {
            g.starts.push_back((uint32_t)total);
            total += g.jobs[q].ntiles;
            src_bytes = std::max(src_bytes, g.jobs[q].src.img_bytes);
            dst_bytes = std::max(dst_bytes, g.jobs[q].dst.img_bytes);
        }
        if (total > 0xFFFFFFFFull) return fail(LLGB_ERR_UNSUPPORTED, "batch has too many tiles");
        g.starts.push_back((uint32_t)total);
        const bool gather = gather_mode(g.mode);
        const bool wide_gather = gather && g.threads == 512;
        int ctas = wide_gather ? 1 : 2;
        uint16_t ns = gather ? 4 : 2, nd = gather ? (wide_gather ? 2 : 3) : 2;
        auto need = [&]() {
            return copy_shared_header_bytes() + (size_t)ns * (src_bytes + kStageZeroBytes) + (size_t)nd * dst_bytes;
        };
        while (!smem_fits(need(), ctas) && (ns > 2 || nd > 2 || ctas > 1)) {
            if (ns > 2) --ns;
            else if (nd > 2) --nd;
            else ctas = 1;
        }
        if (!smem_fits(need(), 1)) return fail(LLGB_ERR_UNSUPPORTED, "batch tiles do not fit shared memory");
        if (!gather || g.threads == 0) g.threads = ctas == 1 ? 512 : 256;  // one CTA per SM: a full-size one
        // a 256-thread gather group that fell to one CTA per SM keeps its 256 threads (its programs' size)
        g.smem = need();
        g.grid = (int)std::min<uint64_t>(total, (uint64_t)sms * ctas);
        if (gather) g.grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(g.grid, total / kGatherTilesPerCta));
        memset(&g.args, 0, sizeof g.args);
        g.args.njobs = (uint32_t)g.jobs.size();
        g.args.total_tiles = (uint32_t)total;
        g.args.src_stage_bytes = src_bytes + kStageZeroBytes;
        g.args.dst_stage_bytes = dst_bytes;
        g.args.code_bytes = 0;
        g.args.src_stages = ns;
        g.args.dst_stages = nd;
        g.args.chunk = (uint32_t)((total + g.grid - 1) / g.grid);
        balance_ctas(g);
        out->push_back(std::move(g));
    }
    return LLGB_OK;
}

llgb_status enqueue_groups(const std::vector<BatchGroup>& groups, cudaStream_t stream)
{
    for (const BatchGroup& g : groups) {
        const cudaError_t e = launch_copy(g.args, g.mode, g.grid, g.threads, g.smem, stream);
        if (e != cudaSuccess) return cuda_fail(e, "batch kernel launch");
    }
    return LLGB_OK;
}

}  // namespace

// A batch: every job planned once, grouped by kernel mode; each group is one
// launch of the copy kernel over a device descriptor table of its own.
struct llgb_batch {
    std::vector<BatchGroup> groups;
    std::vector<void*> device_tables;  // per group: its jobs, then its tile starts
    uint64_t bytes = 0;
    uint64_t tiles = 0;
    int device = 0;
    cudaStream_t capture = nullptr;
    std::vector<cudaStream_t> branches;  // one per group after the first, while capturing
    std::vector<cudaEvent_t> joins;      // fork / join events of the capture
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;

    ~llgb_batch()
    {
        if (done) {
            cudaEventSynchronize(done);
            cudaEventDestroy(done);
        }
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        for (cudaEvent_t e : joins) cudaEventDestroy(e);
        for (cudaStream_t st : branches) cudaStreamDestroy(st);
        if (capture) cudaStreamDestroy(capture);
        for (void* p : device_tables)
            if (p) cudaFree(p);
    }
};

// A batch arena: descriptor tables for `slots` batched copies of up to
// max_pairs pairs each, in device memory and in pinned host staging, both
// allocated once at creation.  A copy takes the next slot (waiting, on the
// host, only until that slot's previous copy has finished on the device),
// writes its tables into the slot's staging, and queues one asynchronous
// table copy and its kernels on the caller's stream.
struct llgb_batch_arena {
    int32_t max_pairs = 0;
    int32_t nslots = 0;
    size_t slot_bytes = 0;
    uint8_t* d_mem = nullptr;
    uint8_t* h_mem = nullptr;
    std::vector<cudaEvent_t> done;  // per slot: its last copy's kernels are done
    int next = 0;
    int device = 0;
    std::mutex mu;
    std::vector<BatchGroup> groups;  // scratch of the current call

    ~llgb_batch_arena()
    {
        for (cudaEvent_t e : done) {
            cudaEventSynchronize(e);
            cudaEventDestroy(e);
        }
        if (d_mem) cudaFree(d_mem);
        if (h_mem) cudaFreeHost(h_mem);
    }
};

namespace {

// Groups of at most 5 kernel modes, gather modes in two CTA sizes: a slot
// holds max_pairs jobs, then the tile starts of every group (max_pairs + 7
// entries).
constexpr int kArenaGroups = 7;

// ... and the CTA ranges of every group (at most 2 CTAs per SM, plus one).
size_t arena_slot_bytes(int32_t max_pairs, int sms)
{
    const size_t starts = ((size_t)max_pairs + kArenaGroups) * sizeof(uint32_t);
    const size_t ctas = (size_t)kArenaGroups * (2 * (size_t)sms + 1) * sizeof(uint32_t);
    return ((size_t)max_pairs * sizeof(JobDesc) + starts + ctas + 255) / 256 * 256;
}

llgb_status batch_build(int32_t n, const llgb_view* const* src, llgb_view* const* dst, llgb_batch* b)
{
    cudaGetDevice(&b->device);
    llgb_status st = plan_groups(n, src, dst, &b->groups, &b->bytes, &b->tiles, kProgramsBuild);
    if (st != LLGB_OK) return st;
    for (BatchGroup& g : b->groups) {
        const size_t table_bytes = g.jobs.size() * sizeof(JobDesc);
        const size_t starts_bytes = g.starts.size() * sizeof(uint32_t);
        const size_t cta_bytes = g.cta_tiles.size() * sizeof(uint32_t);
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, table_bytes + starts_bytes + cta_bytes);
        if (e == cudaSuccess) b->device_tables.push_back(p);
        uint8_t* d = static_cast<uint8_t*>(p);
        if (e == cudaSuccess) e = cudaMemcpy(d, g.jobs.data(), table_bytes, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(d + table_bytes, g.starts.data(), starts_bytes, cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(d + table_bytes + starts_bytes, g.cta_tiles.data(), cta_bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess)
            return e == cudaErrorMemoryAllocation ? fail(LLGB_ERR_OOM, "batch descriptor table")
                                                  : cuda_fail(e, "batch descriptor table");
        g.args.table = reinterpret_cast<const JobDesc*>(d);
        g.args.tile_start = reinterpret_cast<const uint32_t*>(d + table_bytes);
        g.args.cta_tiles = reinterpret_cast<const uint32_t*>(d + table_bytes + starts_bytes);
    }
    return LLGB_OK;
}

llgb_status batch_enqueue(llgb_batch* b, cudaStream_t stream) { return enqueue_groups(b->groups, stream); }

}  // namespace

extern "C" {

const char* llgb_last_error(void) { return t_error.c_str(); }

const char* llgb_version(void) { return "llgb 0.1 (sm_103a)"; }

llgb_status llgb_record_create(const llgb_field_desc* leaves, int32_t n, llgb_record** out)
{
    try {
        if (!leaves || !out) return fail(LLGB_ERR_INVALID_ARG, "null argument");
        if (n < 1 || n > 64) return fail(LLGB_ERR_INVALID_ARG, "leaf count must be 1..64");
        auto* r = new llgb_record;
        std::set<std::string> seen;
        for (int k = 0; k < n; ++k) {
            if (!leaves[k].path || !leaves[k].path[0] || type_size(leaves[k].type) == 0 ||
                !seen.insert(leaves[k].path).second) {
                delete r;
                return fail(LLGB_ERR_INVALID_ARG, "leaf " + std::to_string(k) + ": bad path or type");
            }
            r->paths.emplace_back(leaves[k].path);
            r->types.push_back(leaves[k].type);
        }
        *out = r;
        return LLGB_OK;
    } catch (const std::bad_alloc&) {
        return fail(LLGB_ERR_OOM, "out of host memory");
    } catch (...) {
        return fail(LLGB_ERR_INVALID_ARG, "unexpected error");
    }
}

void llgb_record_destroy(llgb_record* rec) { delete rec; }

int32_t llgb_record_leaf_count(const llgb_record* rec) { return rec ? (int32_t)rec->types.size() : 0; }

llgb_status llgb_record_size(const llgb_record* rec, int32_t packed, uint64_t* out)
{
    if (!rec || !out) return fail(LLGB_ERR_INVALID_ARG, "null argument");
    uint64_t off = 0, max_align = 1;
    for (int32_t t : rec->types) {
        const uint64_t s = type_size(t);
        if (!packed) off = (off + s - 1) / s * s;
        off += s;
        max_align = std::max(max_align, s);
    }
    *out = packed ? off : (off + max_align - 1) / max_align * max_align;
    return LLGB_OK;
}

llgb_status llgb_view_create(const llgb_record* rec, const llgb_extents* ext, const llgb_mapping_desc* map,
                             llgb_view** out)
{
    try {
        if (!rec || !ext || !map || !out) return fail(LLGB_ERR_INVALID_ARG, "null argument");
        auto* v = new llgb_view;
        std::string why;
        const llgb_status st = plan_view(*rec, *ext, *map, &v->plan, &why);
        if (st != LLGB_OK) {
            delete v;
            return fail(st, why);
        }
        v->ptrs.assign(v->plan.blob_sizes.size(), nullptr);
        v->id = g_view_ids.fetch_add(1);
        *out = v;
        return LLGB_OK;
    } catch (const std::bad_alloc&) {
        return fail(LLGB_ERR_OOM, "out of host memory");
    } catch (...) {
        return fail(LLGB_ERR_INVALID_ARG, "unexpected error");
    }
}

void llgb_view_destroy(llgb_view* view) { delete view; }

int32_t llgb_view_blob_count(const llgb_view* view) { return view ? (int32_t)view->plan.blob_sizes.size() : 0; }

uint64_t llgb_view_blob_size(const llgb_view* view, int32_t k)
{
    if (!view || k < 0 || k >= (int32_t)view->plan.blob_sizes.size()) return 0;
    return view->plan.blob_sizes[k];
}

uint64_t llgb_view_record_count(const llgb_view* view) { return view ? view->plan.n : 0; }

llgb_status llgb_view_bind(llgb_view* view, void* const* dev_ptrs, int32_t n)
{
    if (!view) return fail(LLGB_ERR_INVALID_ARG, "null view");
    if (n != (int32_t)view->plan.blob_sizes.size()) return fail(LLGB_ERR_INVALID_ARG, "wrong blob count");
    if (n > 0 && !dev_ptrs) return fail(LLGB_ERR_INVALID_ARG, "null pointer array");
    for (int k = 0; k < n; ++k) {
        const uintptr_t p = reinterpret_cast<uintptr_t>(dev_ptrs[k]);
        if (view->plan.blob_sizes[k] > 0 && (p == 0 || (p & 15u)))
            return fail(LLGB_ERR_INVALID_ARG, "blob " + std::to_string(k) + " is null or not 16-byte aligned");
    }
    for (int k = 0; k < n; ++k) view->ptrs[k] = dev_ptrs[k];
    view->bound = true;
    ++view->bind_gen;
    return LLGB_OK;
}

llgb_status llgb_copy(const llgb_view* src, llgb_view* dst, void* stream)
{
    try {
        return run_copy(src, dst, nullptr, stream);
    } catch (...) {
        return fail(LLGB_ERR_INVALID_ARG, "unexpected error");
    }
}

llgb_status llgb_copy_with(const llgb_view* src, llgb_view* dst, const llgb_launch_config* cfg, void* stream)
{
    try {
        if (!cfg) return fail(LLGB_ERR_INVALID_ARG, "null launch config");
        if (cfg->reserved) return fail(LLGB_ERR_INVALID_ARG, "reserved field must be 0");
        if (cfg->engine < LLGB_ENGINE_AUTO || cfg->engine > LLGB_ENGINE_GATHER)
            return fail(LLGB_ERR_INVALID_ARG, "unknown engine");
        if (cfg->staging < LLGB_STAGING_TMA || cfg->staging > LLGB_STAGING_PLAIN)
            return fail(LLGB_ERR_INVALID_ARG, "unknown staging");
        if (cfg->tile_records <= 0) return fail(LLGB_ERR_INVALID_ARG, "tile_records must be positive");
        return run_copy(src, dst, cfg, stream);
    } catch (...) {
        return fail(LLGB_ERR_INVALID_ARG, "unexpected error");
    }
}

llgb_status llgb_copy_config(const llgb_view* src, const llgb_view* dst, llgb_launch_config* out)
{
    if (!src || !dst || !out) return fail(LLGB_ERR_INVALID_ARG, "null argument");
    if (!same_record(src->plan, dst->plan) || src->plan.n != dst->plan.n)
        return fail(LLGB_ERR_MISMATCH, "views differ in record or count");
    if (tuned_config(src, dst, out)) return LLGB_OK;
    return default_config(src, dst, out);
}

llgb_status llgb_copy_plan(const llgb_view* src, const llgb_view* dst, const llgb_launch_config* cfg,
                           llgb_plan_info* out)
{
    try {
        if (!src || !dst || !out) return fail(LLGB_ERR_INVALID_ARG, "null argument");
        if (!same_record(src->plan, dst->plan) || src->plan.n != dst->plan.n)
            return fail(LLGB_ERR_MISMATCH, "views differ in record or count");
        *out = llgb_plan_info{};
        if (src->plan.n == 0) return LLGB_OK;
        llgb_launch_config c{};
        if (cfg && cfg->tile_records != 0) {
            c = *cfg;
        } else if (!tuned_config(src, dst, &c)) {
            const llgb_status st = default_config(src, dst, &c);
            if (st != LLGB_OK) return st;
        }
        static thread_local JobDesc J;
        std::string why;
        llgb_status st = plan_job(src->plan, src->ptrs, dst->plan, dst->ptrs, (uint32_t)c.tile_records, &J, &why);
        if (st != LLGB_OK) return fail(st, why);
        const DeviceInfo dev = device_info();
        const int sms = dev.sms > 0 ? dev.sms : 152;
        const int grid = (int)std::min<uint64_t>(J.ntiles, (uint64_t)sms * c.ctas_per_sm);
        out->kernel_mode = copy_mode(J, c, grid);
        out->tile_records = (int32_t)J.tile;
        out->tiles = J.ntiles;
        out->items = J.nitems;
        for (int k = 0; k < J.nitems; ++k) {
            if (J.items[k].op == ITEM_VALUE && J.items[k].fast == FK_GENERIC && !J.items[k].spec) ++out->generic_items;
            if (J.items[k].spec) ++out->stream_items;
        }
        int bmode = 0, bthreads = 0;
        st = plan_batch_job(src, dst, &J, &bmode, 256, true, &bthreads);
        if (st != LLGB_OK) return st;
        out->batch_kernel_mode = bmode;
        return LLGB_OK;
    } catch (...) {
        return fail(LLGB_ERR_INVALID_ARG, "unexpected error");
    }
}

llgb_status llgb_pack(const llgb_view* plain, llgb_view* packed, void* stream)
{
    if (is_bitpacked(plain) || !is_bitpacked(packed))
        return fail(LLGB_ERR_INVALID_ARG, "pack needs a plain source and a bit-packed destination");
    return llgb_copy(plain, packed, stream);
}

llgb_status llgb_unpack(const llgb_view* packed, llgb_view* plain, void* stream)
{
    if (!is_bitpacked(packed) || is_bitpacked(plain))
        return fail(LLGB_ERR_INVALID_ARG, "unpack needs a bit-packed source and a plain destination");
    return llgb_copy(packed, plain, stream);
}

}  // extern "C"

namespace {

// The particle view the n-body kernels read, plus for each leaf its blob and
// the byte offset of its base in that blob (for heatmap counters).  *layout:
// 0 AoS, 1 SoA, 2 AoSoA.
llgb_status particle_view(llgb_view* particles, ParticleView* v, int* kind, int* blob, uint64_t* boff,
                          int* layout = nullptr)
{
    if (!particles) return fail(LLGB_ERR_INVALID_ARG, "null view");
    const ViewPlan& p = particles->plan;
    if (p.types != std::vector<int32_t>(7, LLGB_F32))
        return fail(LLGB_ERR_INVALID_ARG, "n-body needs the 7-leaf f32 particle record");
    if (p.wrap != WRAP_NONE || p.base == BASE_BITS_INT || p.base == BASE_BITS_FLOAT || p.base == BASE_SPLIT)
        return fail(LLGB_ERR_UNSUPPORTED, "n-body reads AoS, SoA or AoSoA views");
    if (!particles->bound) return fail(LLGB_ERR_UNBOUND, "view used before llgb_view_bind");
    if (p.n > 0x7FFFFFFFull) return fail(LLGB_ERR_UNSUPPORTED, "n-body needs n < 2^31");
    *v = ParticleView{};
    v->n = (uint32_t)p.n;
    *kind = PV_GENERIC;
    int lay = 2;
    for (int f = 0; f < 7; ++f) blob[f] = 0;
    switch (p.base) {
    case BASE_AOS:  // 28-byte record, aligned and packed alike
        for (int f = 0; f < 7; ++f) boff[f] = 4u * f;
        v->bstride = 28;
        v->lanes = 1;
        *kind = PV_AOS;
        lay = 0;
        break;
    case BASE_SOA_MB:
        for (int f = 0; f < 7; ++f) {
            blob[f] = f;
            boff[f] = 0;
        }
        v->bstride = 4;
        v->lanes = 0xFFFFFFFFu;
        *kind = PV_SOA;
        lay = 1;
        break;
    case BASE_SOA_SB:
        for (int f = 0; f < 7; ++f) boff[f] = p.sb_base[f];
        v->bstride = 4;
        v->lanes = 0xFFFFFFFFu;
        *kind = PV_SOA;
        lay = 1;
        break;
    default: {  // AoSoA
        const uint64_t L = p.lanes;
        if (28 * L > 0xFFFFFFFFull) return fail(LLGB_ERR_UNSUPPORTED, "AoSoA block too large for the n-body");
        for (int f = 0; f < 7; ++f) boff[f] = L * 4 * f;
        v->bstride = (uint32_t)(28 * L);
        v->lanes = (uint32_t)L;
        if (L & (L - 1)) {
            *kind = PV_DIV;
        } else {
            v->lmask = (uint32_t)(L - 1);
            while ((1ull << v->lshift) < L) ++v->lshift;
            *kind = L == 32 ? PV_AOSOA32 : PV_GENERIC;
        }
        break;
    }
    }
    // (block, lane) cursor steps of 32 records
    if (lay == 1) {
        v->step_lanes = 32;
        v->step_off = 128;
        v->wrap_off = 0;
    } else {
        const uint64_t L = v->lanes;
        v->step_lanes = (uint32_t)(32 % L);
        v->step_off = (32 / L) * v->bstride + (32 % L) * 4;
        v->wrap_off = v->bstride - 4 * L;
    }
    for (int f = 0; f < 7; ++f) v->base[f] = static_cast<uint8_t*>(particles->ptrs[blob[f]]) + boff[f];
    if (layout) *layout = lay;
    return LLGB_OK;
}

// Heatmap counters of a view at granularity g: ceil(blob bytes / g) per blob;
// start[b] = counters of the blobs before b.
uint64_t heat_layout(const llgb_view* v, uint64_t g, std::vector<uint64_t>* start)
{
    start->assign(1, 0);
    for (uint64_t s : v->plan.blob_sizes) start->push_back(start->back() + (s + g - 1) / g);
    return start->back();
}

}  // namespace

extern "C" {

llgb_status llgb_nbody_step(llgb_view* particles, float eps, float dt, void* stream)
{
    ParticleView v;
    int kind = 0, layout = 0, blob[7];
    uint64_t boff[7];
    const llgb_status st = particle_view(particles, &v, &kind, blob, boff, &layout);
    if (st != LLGB_OK) return st;
    const cudaError_t e = launch_nbody(v, kind, layout, eps, dt, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "n-body launch");
    return LLGB_OK;
}

llgb_status llgb_nbody_update(llgb_view* particles, float eps, float dt, int32_t traversal, void* stream)
{
    if (traversal != LLGB_TRAVERSE_INDEX && traversal != LLGB_TRAVERSE_BLOCKS)
        return fail(LLGB_ERR_INVALID_ARG, "unknown traversal");
    ParticleView v;
    int kind = 0, blob[7];
    uint64_t boff[7];
    const llgb_status st = particle_view(particles, &v, &kind, blob, boff);
    if (st != LLGB_OK) return st;
    const cudaError_t e = launch_nbody_update(v, kind, traversal, eps, dt, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "n-body update launch");
    return LLGB_OK;
}

llgb_status llgb_nbody_move(llgb_view* particles, float dt, int32_t traversal, void* stream)
{
    if (traversal != LLGB_TRAVERSE_INDEX && traversal != LLGB_TRAVERSE_BLOCKS)
        return fail(LLGB_ERR_INVALID_ARG, "unknown traversal");
    ParticleView v;
    int kind = 0, layout = 0, blob[7];
    uint64_t boff[7];
    const llgb_status st = particle_view(particles, &v, &kind, blob, boff, &layout);
    if (st != LLGB_OK) return st;
    const cudaError_t e = launch_nbody_move(v, kind, layout, traversal, dt, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "n-body move launch");
    return LLGB_OK;
}

llgb_status llgb_heatmap_counters(const llgb_view* view, uint64_t granularity, uint64_t* counters)
{
    if (!view || !counters) return fail(LLGB_ERR_INVALID_ARG, "null argument");
    if (granularity == 0 || (granularity & (granularity - 1)))
        return fail(LLGB_ERR_INVALID_ARG, "granularity must be a power of two");
    std::vector<uint64_t> start;
    *counters = heat_layout(view, granularity, &start);
    return LLGB_OK;
}

llgb_status llgb_nbody_step_instrumented(llgb_view* particles, float eps, float dt, uint64_t* field_counts,
                                         int32_t count_mode, uint64_t* heat, uint64_t granularity, void* stream)
{
    ParticleView v;
    int kind = 0, blob[7];
    uint64_t boff[7];
    llgb_status st = particle_view(particles, &v, &kind, blob, boff);
    if (st != LLGB_OK) return st;
    if (field_counts && count_mode != LLGB_COUNT_ATOMIC && count_mode != LLGB_COUNT_BLOCK)
        return fail(LLGB_ERR_INVALID_ARG, "unknown count mode");
    if ((reinterpret_cast<uintptr_t>(field_counts) | reinterpret_cast<uintptr_t>(heat)) & 7u)
        return fail(LLGB_ERR_INVALID_ARG, "counters must be 8-byte aligned");
    NbodyInstr in{};
    in.counts = reinterpret_cast<unsigned long long*>(field_counts);
    in.count_mode = count_mode;
    if (heat) {
        if (granularity == 0 || (granularity & (granularity - 1)))
            return fail(LLGB_ERR_INVALID_ARG, "granularity must be a power of two");
        std::vector<uint64_t> start;
        heat_layout(particles, granularity, &start);
        in.heat = reinterpret_cast<unsigned long long*>(heat);
        while ((1ull << in.gshift) < granularity) ++in.gshift;
        for (int f = 0; f < 7; ++f) {
            in.boff[f] = boff[f];
            in.hstart[f] = start[blob[f]];
        }
    }
    const cudaError_t e = launch_nbody_instrumented(v, kind == PV_DIV, in, eps, dt, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "n-body launch");
    return LLGB_OK;
}

llgb_status llgb_batch_create(int32_t n, const llgb_view* const* src, llgb_view* const* dst, llgb_batch** out)
{
    try {
        if (!out || n < 0 || (n > 0 && (!src || !dst))) return fail(LLGB_ERR_INVALID_ARG, "bad batch arguments");
        auto* b = new llgb_batch;
        const llgb_status st = batch_build(n, src, dst, b);
        if (st != LLGB_OK) {
            delete b;
            return st;
        }
        *out = b;
        return LLGB_OK;
    } catch (const std::bad_alloc&) {
        return fail(LLGB_ERR_OOM, "out of host memory");
    } catch (...) {
        return fail(LLGB_ERR_INVALID_ARG, "unexpected error");
    }
}

llgb_status llgb_batch_launch(llgb_batch* b, void* stream, int32_t use_graph)
{
    if (!b) return fail(LLGB_ERR_INVALID_ARG, "null batch");
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (!b->done && (e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming)) != cudaSuccess)
        return cuda_fail(e, "batch event");
    if (!use_graph) {
        const llgb_status st = batch_enqueue(b, s);
        if (st != LLGB_OK) return st;
    } else {
        if (!b->exec) {
            for (const BatchGroup& g : b->groups)
                if ((e = prepare_copy(g.mode, g.smem)) != cudaSuccess) return cuda_fail(e, "kernel attributes");
            if ((e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking)) != cudaSuccess)
                return cuda_fail(e, "capture stream");
            // the groups touch disjoint views: each becomes its own branch of
            // the graph (forked from and joined back into the capture stream),
            // so one group's last CTAs overlap the next group's first
            const size_t ng = b->groups.size();
            for (size_t k = 1; k < ng; ++k) {
                cudaStream_t br = nullptr;
                cudaEvent_t fork = nullptr, join = nullptr;
                if ((e = cudaStreamCreateWithFlags(&br, cudaStreamNonBlocking)) == cudaSuccess) b->branches.push_back(br);
                if (e == cudaSuccess && (e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming)) == cudaSuccess)
                    b->joins.push_back(fork);
                if (e == cudaSuccess && (e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming)) == cudaSuccess)
                    b->joins.push_back(join);
                if (e != cudaSuccess) return cuda_fail(e, "graph branches");
            }
            if ((e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
                return cuda_fail(e, "begin capture");
            llgb_status st = LLGB_OK;
            for (size_t k = 1; k < ng && st == LLGB_OK && e == cudaSuccess; ++k) {
                e = cudaEventRecord(b->joins[2 * (k - 1)], b->capture);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(b->branches[k - 1], b->joins[2 * (k - 1)], 0);
                if (e == cudaSuccess) {
                    const BatchGroup& g = b->groups[k];
                    e = launch_copy(g.args, g.mode, g.grid, g.threads, g.smem, b->branches[k - 1]);
                }
                if (e == cudaSuccess) e = cudaEventRecord(b->joins[2 * (k - 1) + 1], b->branches[k - 1]);
            }
            if (e == cudaSuccess && ng > 0) {
                const BatchGroup& g = b->groups[0];
                e = launch_copy(g.args, g.mode, g.grid, g.threads, g.smem, b->capture);
            }
            for (size_t k = 1; k < ng && e == cudaSuccess; ++k)
                e = cudaStreamWaitEvent(b->capture, b->joins[2 * (k - 1) + 1], 0);
            if (e != cudaSuccess) st = cuda_fail(e, "batch capture");
            e = cudaStreamEndCapture(b->capture, &b->graph);
            if (st != LLGB_OK) return st;
            if (e != cudaSuccess) return cuda_fail(e, "end capture");
            if ((e = cudaGraphInstantiate(&b->exec, b->graph, 0)) != cudaSuccess) return cuda_fail(e, "graph instantiate");
        }
        if ((e = cudaGraphLaunch(b->exec, s)) != cudaSuccess) return cuda_fail(e, "graph launch");
    }
    if ((e = cudaEventRecord(b->done, s)) != cudaSuccess) return cuda_fail(e, "batch event record");
    return LLGB_OK;
}

llgb_status llgb_batch_info(const llgb_batch* b, int32_t* launches, uint64_t* tiles, uint64_t* bytes)
{
    if (!b) return fail(LLGB_ERR_INVALID_ARG, "null batch");
    if (launches) *launches = (int32_t)b->groups.size();
    if (tiles) *tiles = b->tiles;
    if (bytes) *bytes = b->bytes;
    return LLGB_OK;
}

void llgb_batch_destroy(llgb_batch* b) { delete b; }

llgb_status llgb_batch_arena_create(int32_t max_pairs, int32_t slots, llgb_batch_arena** out)
{
    try {
        if (!out || max_pairs < 1 || max_pairs > 65536 || slots < 1 || slots > 64)
            return fail(LLGB_ERR_INVALID_ARG, "arena needs 1..65536 pairs and 1..64 slots");
        auto* a = new llgb_batch_arena;
        a->max_pairs = max_pairs;
        a->nslots = slots;
        const DeviceInfo dev = device_info();
        a->slot_bytes = arena_slot_bytes(max_pairs, dev.sms > 0 ? dev.sms : 152);
        cudaGetDevice(&a->device);
        cudaError_t e = cudaMalloc(&a->d_mem, a->slot_bytes * (size_t)slots);
        if (e == cudaSuccess) e = cudaMallocHost(&a->h_mem, a->slot_bytes * (size_t)slots);
        for (int k = 0; e == cudaSuccess && k < slots; ++k) {
            cudaEvent_t ev = nullptr;
            e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e == cudaSuccess) a->done.push_back(ev);
        }
        if (e != cudaSuccess) {
            delete a;
            return e == cudaErrorMemoryAllocation ? fail(LLGB_ERR_OOM, "arena tables") : cuda_fail(e, "arena tables");
        }
        *out = a;
        return LLGB_OK;
    } catch (const std::bad_alloc&) {
        return fail(LLGB_ERR_OOM, "out of host memory");
    } catch (...) {
        return fail(LLGB_ERR_INVALID_ARG, "unexpected error");
    }
}

llgb_status llgb_batch_arena_copy(llgb_batch_arena* a, int32_t n, const llgb_view* const* src,
                                  llgb_view* const* dst, void* stream)
{
    try {
        if (!a || n < 0 || (n > 0 && (!src || !dst))) return fail(LLGB_ERR_INVALID_ARG, "bad arena arguments");
        if (n > a->max_pairs) return fail(LLGB_ERR_INVALID_ARG, "more pairs than the arena was made for");
        int device = 0;
        cudaGetDevice(&device);
        if (device != a->device) return fail(LLGB_ERR_INVALID_ARG, "arena used on another device than it was made on");
        std::lock_guard<std::mutex> lock(a->mu);
        uint64_t bytes = 0, tiles = 0;
        llgb_status st = plan_groups(n, src, dst, &a->groups, &bytes, &tiles, kProgramsLookup);
        if (st != LLGB_OK || a->groups.empty()) return st;
        const int slot = a->next;
        a->next = (a->next + 1) % a->nslots;
        // the slot's previous copy must have read its tables
        cudaError_t e = cudaEventSynchronize(a->done[slot]);
        if (e != cudaSuccess) return cuda_fail(e, "arena slot wait");
        uint8_t* h = a->h_mem + (size_t)slot * a->slot_bytes;
        uint8_t* d = a->d_mem + (size_t)slot * a->slot_bytes;
        size_t at = 0;
        for (BatchGroup& g : a->groups) {
            memcpy(h + at, g.jobs.data(), g.jobs.size() * sizeof(JobDesc));
            g.args.table = reinterpret_cast<const JobDesc*>(d + at);
            at += g.jobs.size() * sizeof(JobDesc);
        }
        for (BatchGroup& g : a->groups) {
            memcpy(h + at, g.starts.data(), g.starts.size() * sizeof(uint32_t));
            g.args.tile_start = reinterpret_cast<const uint32_t*>(d + at);
            at += g.starts.size() * sizeof(uint32_t);
        }
        for (BatchGroup& g : a->groups) {
            if (at + g.cta_tiles.size() * sizeof(uint32_t) > a->slot_bytes)
                return fail(LLGB_ERR_UNSUPPORTED, "arena slot too small for the CTA ranges");
            memcpy(h + at, g.cta_tiles.data(), g.cta_tiles.size() * sizeof(uint32_t));
            g.args.cta_tiles = reinterpret_cast<const uint32_t*>(d + at);
            at += g.cta_tiles.size() * sizeof(uint32_t);
        }
        const cudaStream_t s = static_cast<cudaStream_t>(stream);
        if ((e = cudaMemcpyAsync(d, h, at, cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return cuda_fail(e, "arena table copy");
        st = enqueue_groups(a->groups, s);
        if ((e = cudaEventRecord(a->done[slot], s)) != cudaSuccess) return cuda_fail(e, "arena event record");
        return st;
    } catch (const std::bad_alloc&) {
        return fail(LLGB_ERR_OOM, "out of host memory");
    } catch (...) {
        return fail(LLGB_ERR_INVALID_ARG, "unexpected error");
    }
}

void llgb_batch_arena_destroy(llgb_batch_arena* a) { delete a; }

llgb_status llgb_autotune(const llgb_view* src, llgb_view* dst, void* stream, llgb_launch_config* best)
{
    try {
        llgb_status st = check_pair(src, dst);
        if (st != LLGB_OK) return st;
        llgb_launch_config base{};
        st = default_config(src, dst, &base);
        if (st != LLGB_OK) return st;
        if (src->plan.n == 0) {
            if (best) *best = base;
            return LLGB_OK;
        }
        const cudaStream_t s = static_cast<cudaStream_t>(stream);
        const uint32_t q = tile_quantum(src->plan, dst->plan);
        double sb = 0, db = 0;
        uint32_t cb = 0;
        bytes_per_record(src->plan, dst->plan, &sb, &db, &cb);
        const double per_rec = std::max(std::max(sb, db), 1.0);
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        cudaError_t e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
        if (e != cudaSuccess) {
            if (e0) cudaEventDestroy(e0);
            return cuda_fail(e, "autotune events");
        }
        // time one shape: a warm-up copy (which also rejects shapes that do
        // not fit the pair), then three timed copies
        auto time_shape = [&](const llgb_launch_config& c) -> float {
            if (run_copy(src, dst, &c, stream) != LLGB_OK) return -1.0f;
            cudaEventRecord(e0, s);
            bool ok = true;
            for (int r = 0; r < 3 && ok; ++r) ok = run_copy(src, dst, &c, stream) == LLGB_OK;
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess || !ok) return -1.0f;
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            return ms;
        };
        // 1. tile size, threads and CTAs per SM, pipeline depths (TMA staging)
        std::vector<llgb_launch_config> cands{base};
        // the default shape with other pipeline depths (which of 3 and 4
        // source stages is faster differs from pair to pair)
        for (int ns : {2, 3, 4, 5})
            for (int nd : {2, 3, 4}) {
                llgb_launch_config c = base;
                if (ns == base.src_stages && nd == base.dst_stages) continue;
                c.src_stages = ns;
                c.dst_stages = nd;
                cands.push_back(c);
            }
        for (double target : {6144.0, 12288.0, 24576.0, 49152.0, 73728.0})
            for (int threads : {256, 512})
                for (int ns : {2, 3, 4})
                    for (int nd : {2, 3}) {
                        llgb_launch_config c{};
                        c.tile_records = (int32_t)std::max<uint64_t>(q, (uint64_t)(target / per_rec) / q * q);
                        c.threads = threads;
                        c.ctas_per_sm = threads == 256 ? 2 : 1;
                        c.src_stages = ns;
                        c.dst_stages = nd;
                        cands.push_back(c);
                    }
        // Timings on a shared memory system vary by a few percent from run to
        // run: the four fastest shapes and the default are timed twice more
        // and keep their best time, and a shape replaces the default only when
        // that is at least kMargin faster.
        constexpr float kMargin = 0.02f;
        std::vector<std::pair<float, size_t>> timed;
        for (size_t i = 0; i < cands.size(); ++i) {
            const float ms = time_shape(cands[i]);
            if (ms >= 0.0f) timed.push_back({ms, i});
        }
        std::sort(timed.begin(), timed.end());
        std::vector<size_t> finalists{0};
        for (size_t i = 0; i < timed.size() && finalists.size() < 5; ++i)
            if (timed[i].second != 0) finalists.push_back(timed[i].second);
        auto best_of = [&](const llgb_launch_config& c, float first) {
            float ms = first;
            for (int r = 0; r < 2; ++r) {
                const float t = time_shape(c);
                if (t >= 0.0f && (ms < 0.0f || t < ms)) ms = t;
            }
            return ms;
        };
        auto first_time = [&](size_t i) {
            for (const auto& t : timed)
                if (t.second == i) return t.first;
            return -1.0f;
        };
        const float base_ms = best_of(base, first_time(0));
        float best_ms = base_ms >= 0.0f ? base_ms : 1e30f;
        llgb_launch_config winner = base;
        for (size_t k = 1; k < finalists.size(); ++k) {
            const float ms = best_of(cands[finalists[k]], first_time(finalists[k]));
            if (ms >= 0.0f && ms < best_ms) {
                best_ms = ms;
                winner = cands[finalists[k]];
            }
        }
        if (base_ms >= 0.0f && best_ms > (1.0f - kMargin) * base_ms) {
            winner = base;
            best_ms = base_ms;
        }
        // 2. the staging scheme of the winning shape, under the same margin
        const llgb_launch_config shape = winner;
        const float shape_ms = best_ms;
        for (int staging : {LLGB_STAGING_PLAIN_STORE, LLGB_STAGING_PLAIN_LOAD, LLGB_STAGING_PLAIN}) {
            llgb_launch_config c = shape;
            c.staging = staging;
            const float ms = best_of(c, time_shape(c));
            if (ms >= 0.0f && ms < best_ms && ms <= (1.0f - kMargin) * shape_ms) {
                best_ms = ms;
                winner = c;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        t_error.clear();
        {
            std::lock_guard<std::mutex> lock(tune_mu);
            tune_cache[tune_key(src, dst)] = winner;
        }
        g_tune_gen.fetch_add(1);
        if (best) *best = winner;
        return LLGB_OK;
    } catch (...) {
        return fail(LLGB_ERR_INVALID_ARG, "unexpected error");
    }
}

// The tuned shapes as JSON: {"llgb_autotune": 1, "entries": {"<pair key>":
// [tile_records, src_stages, dst_stages, threads, ctas_per_sm, engine,
// staging], ...}}.  Keys are the mapping pair and record-count bucket that
// llgb_autotune files a shape under (letters, digits and , : / { } |).
llgb_status llgb_autotune_save(const char* path)
{
    try {
        if (!path) return fail(LLGB_ERR_INVALID_ARG, "null path");
        std::string out = "{\"llgb_autotune\": 1, \"entries\": {";
        {
            std::lock_guard<std::mutex> lock(tune_mu);
            bool first = true;
            for (const auto& kv : tune_cache) {
                const llgb_launch_config& c = kv.second;
                out += first ? "\n  \"" : ",\n  \"";
                first = false;
                out += kv.first + "\": [" + std::to_string(c.tile_records) + ", " + std::to_string(c.src_stages) +
                       ", " + std::to_string(c.dst_stages) + ", " + std::to_string(c.threads) + ", " +
                       std::to_string(c.ctas_per_sm) + ", " + std::to_string(c.engine) + ", " +
                       std::to_string(c.staging) + "]";
            }
        }
        out += "\n}}\n";
        FILE* f = fopen(path, "wb");
        if (!f) return fail(LLGB_ERR_INVALID_ARG, std::string("cannot write ") + path);
        const bool ok = fwrite(out.data(), 1, out.size(), f) == out.size();
        if (fclose(f) != 0 || !ok) return fail(LLGB_ERR_INVALID_ARG, std::string("cannot write ") + path);
        return LLGB_OK;
    } catch (...) {
        return fail(LLGB_ERR_OOM, "out of host memory");
    }
}

llgb_status llgb_autotune_load(const char* path)
{
    try {
        if (!path) return fail(LLGB_ERR_INVALID_ARG, "null path");
        FILE* f = fopen(path, "rb");
        if (!f) return fail(LLGB_ERR_INVALID_ARG, std::string("cannot read ") + path);
        std::string text;
        char buf[4096];
        size_t got;
        while ((got = fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, got);
        fclose(f);
        if (text.find("\"llgb_autotune\": 1") == std::string::npos)
            return fail(LLGB_ERR_INVALID_ARG, "not an llgb autotune file");
        size_t at = text.find("\"entries\"");
        if (at == std::string::npos) return fail(LLGB_ERR_INVALID_ARG, "autotune file has no entries");
        at = text.find('{', at);
        std::map<std::string, llgb_launch_config> parsed;
        while (at != std::string::npos) {
            const size_t k0 = text.find('"', at + 1);
            if (k0 == std::string::npos) break;
            const size_t k1 = text.find('"', k0 + 1);
            const size_t l0 = text.find('[', k1);
            const size_t l1 = text.find(']', l0);
            if (k1 == std::string::npos || l0 == std::string::npos || l1 == std::string::npos)
                return fail(LLGB_ERR_INVALID_ARG, "malformed autotune entry");
            int v[7];
            if (sscanf(text.c_str() + l0, "[%d , %d , %d , %d , %d , %d , %d ]", &v[0], &v[1], &v[2], &v[3], &v[4],
                       &v[5], &v[6]) != 7)
                return fail(LLGB_ERR_INVALID_ARG, "malformed autotune entry");
            llgb_launch_config c{};
            c.tile_records = v[0];
            c.src_stages = v[1];
            c.dst_stages = v[2];
            c.threads = v[3];
            c.ctas_per_sm = v[4];
            c.engine = v[5];
            c.staging = v[6];
            if (c.tile_records <= 0 || !valid_threads(c.threads) || c.src_stages < 1 || c.src_stages > 8 ||
                c.dst_stages < 1 || c.dst_stages > 4 || c.ctas_per_sm < 1 || c.ctas_per_sm > 8 ||
                c.engine < LLGB_ENGINE_AUTO || c.engine > LLGB_ENGINE_GATHER || c.staging < LLGB_STAGING_TMA ||
                c.staging > LLGB_STAGING_PLAIN)
                return fail(LLGB_ERR_INVALID_ARG, "autotune entry out of range");
            parsed[text.substr(k0 + 1, k1 - k0 - 1)] = c;
            at = text.find(',', l1);
            if (at != std::string::npos && text.find('"', at) == std::string::npos) break;
        }
        {
            std::lock_guard<std::mutex> lock(tune_mu);
            for (const auto& kv : parsed) tune_cache[kv.first] = kv.second;
        }
        g_tune_gen.fetch_add(1);
        return LLGB_OK;
    } catch (...) {
        return fail(LLGB_ERR_OOM, "out of host memory");
    }
}

llgb_status llgb_autotune_clear(void)
{
    std::lock_guard<std::mutex> lock(tune_mu);
    tune_cache.clear();
    g_tune_gen.fetch_add(1);
    return LLGB_OK;
}

llgb_status llgb_fma_probe(uint32_t iters, float* sink, uint64_t* fmas, void* stream)
{
    if (!sink || !fmas || iters == 0) return fail(LLGB_ERR_INVALID_ARG, "null argument or zero rounds");
    const cudaError_t e = launch_fma_probe(iters, sink, fmas, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "FMA probe launch");
    return LLGB_OK;
}

llgb_status llgb_wait_selftest(uint64_t limit_ns, uint64_t* waited_ns, void* stream)
{
    if (limit_ns < 1000ull || limit_ns > 10000000000ull)
        return fail(LLGB_ERR_INVALID_ARG, "limit_ns must be 1 us .. 10 s");
    if (reinterpret_cast<uintptr_t>(waited_ns) & 7u) return fail(LLGB_ERR_INVALID_ARG, "waited_ns must be 8-byte aligned");
    const cudaError_t e = launch_wait_selftest(limit_ns, reinterpret_cast<unsigned long long*>(waited_ns),
                                               static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "wait self-test launch");
    return LLGB_OK;
}

llgb_status llgb_device_status(int32_t* code, int32_t reset)
{
    if (!code) return fail(LLGB_ERR_INVALID_ARG, "null argument");
    unsigned v = 0;
    const cudaError_t e = read_device_status(&v, reset != 0);
    if (e != cudaSuccess) return cuda_fail(e, "device status");
    *code = (int32_t)v;
    return LLGB_OK;
}

}  // extern "C"
