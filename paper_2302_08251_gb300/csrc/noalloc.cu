// noalloc.cu -- batched copy that allocates no device memory.
//
// llgb_batch_create keeps its descriptor tables in memory it obtains with
// cudaMalloc.  Some callers cannot allocate device memory while they run:
// cudaMalloc and cudaFree may synchronise the whole device, which stalls
// latency-critical loops; a host framework's caching allocator may already
// own all free HBM, so a fresh cudaMalloc fails; and some deployments fix
// their device memory at start-up and forbid allocation afterwards.
// llgb_batch_copy_noalloc serves them: the same copy kernel reads its
// descriptor table from a fixed array in this library's static device
// memory, which every GPU that loads the library holds until the process
// exits.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "job.h"
#include "kernels.h"
#include "llgb.h"

namespace llgb {
llgb_status internal_fail(llgb_status status, const char* message);
llgb_status internal_plan_pair(const llgb_view* src, const llgb_view* dst, JobDesc* job, int* mode, int threads);
bool internal_empty(const llgb_view* v);
void internal_device_limits(int* sms, size_t* smem_cap);
bool internal_smem_fits(size_t smem, int ctas);
size_t copy_shared_header_bytes();
}  // namespace llgb

using namespace llgb;

namespace {

constexpr int kNoallocPairs = 64;      // most pairs one call accepts
constexpr int kModes = 5;              // kernel modes: general, 2-word and 4-word gathers, AoSoA bits (generic, compile-time)
constexpr int kMaxDevices = 64;
constexpr size_t kTableBytes = (size_t)kNoallocPairs * sizeof(JobDesc);
constexpr int kStartsPerMode = (kNoallocPairs + 1 + 3) / 4 * 4;  // tile starts of one mode, padded to 16 bytes
constexpr size_t kStartsBytes = (size_t)kModes * kStartsPerMode * sizeof(uint32_t);
constexpr size_t kScratchBytes = (kTableBytes + kStartsBytes + 255) / 256 * 256;
static_assert(kTableBytes % 16 == 0 && sizeof(JobDesc) % 8 == 0, "tables are moved in 16-byte words");
static_assert(kStartsBytes % 16 == 0, "tile starts are moved in 16-byte words");

// The descriptor tables and tile starts of the current call (about 370 KB).
// Shared by every call on a device; see llgb_batch_copy_noalloc.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// One piece of a call's descriptors, carried to the device as kernel
// parameters: `words` 16-byte words for the scratch array from word `at` on.
// Parameters are copied when the kernel is queued, so the host memory they
// came from is free again as soon as the launch returns.
constexpr uint32_t kUploadWords = 1984;  // 31,744 bytes: within the 32 KB parameter limit
struct UploadArgs {
    uint32_t at;
    uint32_t words;
    uint32_t pad[2];
    uint4 data[kUploadWords];
};

__global__ void noalloc_upload(const __grid_constant__ UploadArgs a)
{
    uint4* dst = reinterpret_cast<uint4*>(g_noalloc_scratch) + a.at;
    for (uint32_t k = threadIdx.x; k < a.words; k += blockDim.x) dst[k] = a.data[k];
}

// Identity of the CUDA context current on this thread (0 if none can be
// read): a device reset or a context re-creation gives a new identity, and
// with it a new copy of the scratch array at a new address.
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

uint64_t current_context_id()
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

struct ScratchEntry {
    void* ptr = nullptr;     // device address of g_noalloc_scratch
    uint64_t context = 0;    // the context it belongs to
};
std::mutex setup_mu;
ScratchEntry device_scratch[kMaxDevices];

// Device address of the scratch array in the current device's context.  In
// host code the array's name only stands in for the symbol, so the address
// is asked for once per device and context, with that device current.
llgb_status scratch_address(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return internal_fail(LLGB_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return internal_fail(LLGB_ERR_UNSUPPORTED, "device ordinal out of range");
    const uint64_t ctx = current_context_id();
    std::lock_guard<std::mutex> lock(setup_mu);
    ScratchEntry& s = device_scratch[dev];
    if (!s.ptr || ctx == 0 || s.context != ctx) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return internal_fail(LLGB_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed");
        s.ptr = p;
        s.context = current_context_id();  // the lookup made the device's context current if it was not
    }
    *out = s.ptr;
    return LLGB_OK;
}

// A call's descriptors as they go to the scratch array: the tables of all
// groups back to back, then the tile starts of all groups.
struct Staging {
    JobDesc jobs[kNoallocPairs];
    uint32_t starts[kModes][kStartsPerMode];
};
static_assert(offsetof(Staging, starts) == kTableBytes, "staging mirrors the scratch array");
thread_local Staging staging;
thread_local UploadArgs upload;

// Queue uploads of staging bytes [from, to) (multiples of 16) to the same
// offsets of the scratch array.
cudaError_t upload_range(size_t from, size_t to, cudaStream_t s)
{
    const uint4* words = reinterpret_cast<const uint4*>(&staging);
    for (size_t w = from / 16; w < to / 16; w += kUploadWords) {
        const size_t k = to / 16 - w < kUploadWords ? to / 16 - w : kUploadWords;
        upload.at = (uint32_t)w;
        upload.words = (uint32_t)k;
        memcpy(upload.data, words + w, k * 16);
        noalloc_upload<<<1, 256, 0, s>>>(upload);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

extern "C" llgb_status llgb_batch_copy_noalloc(int32_t n, const llgb_view* const* src, llgb_view* const* dst,
                                               void* stream)
{
    if (n < 0 || (n > 0 && (!src || !dst))) return internal_fail(LLGB_ERR_INVALID_ARG, "bad batch arguments");
    if (n > kNoallocPairs)
        return internal_fail(LLGB_ERR_INVALID_ARG, "llgb_batch_copy_noalloc takes at most 64 view pairs per call");
    void* scratch = nullptr;
    llgb_status st = scratch_address(&scratch);
    if (st != LLGB_OK) return st;

    // Plan every pair and order the jobs by kernel mode.
    int mode_of[kNoallocPairs];
    int order[kNoallocPairs];
    int count[kModes] = {0, 0, 0, 0, 0};
    static thread_local JobDesc planned[kNoallocPairs];
    int njobs = 0;
    for (int32_t k = 0; k < n; ++k) {
        if (!src[k] || !dst[k]) return internal_fail(LLGB_ERR_INVALID_ARG, "null view");
        if (internal_empty(src[k])) {
            JobDesc probe;
            int m = 0;
            st = internal_plan_pair(src[k], dst[k], &probe, &m, 256);  // still validates the pair
            if (st != LLGB_OK) return st;
            continue;
        }
        int m = 0;
        st = internal_plan_pair(src[k], dst[k], &planned[njobs], &m, 256);
        if (st != LLGB_OK) return st;
        mode_of[njobs] = m == 0 ? 0 : (m == 2 ? 1 : (m == 4 ? 2 : (m == 1 ? 3 : 4)));
        ++count[mode_of[njobs]];
        ++njobs;
    }
    if (njobs == 0) return LLGB_OK;
    int at[kModes] = {0, count[0], count[0] + count[1], count[0] + count[1] + count[2],
                      count[0] + count[1] + count[2] + count[3]};
    for (int q = 0; q < njobs; ++q) order[at[mode_of[q]]++] = q;
    for (int q = 0; q < njobs; ++q) staging.jobs[q] = planned[order[q]];

    int sms = 152;
    size_t smem_cap = 232448;
    internal_device_limits(&sms, &smem_cap);
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    struct Launch {
        CopyArgs args;
        int grid;
        int threads;
        size_t smem;
    };
    static thread_local Launch launch[kModes];
    int first = 0;
    for (int g = 0; g < kModes; ++g) {
        launch[g].grid = 0;
        if (count[g] == 0) continue;
        uint64_t total = 0;
        uint32_t src_bytes = 0, dst_bytes = 0;
        for (int q = 0; q < count[g]; ++q) {
            const JobDesc& J = staging.jobs[first + q];
            staging.starts[g][q] = (uint32_t)total;
            total += J.ntiles;
            src_bytes = src_bytes > J.src.img_bytes ? src_bytes : J.src.img_bytes;
            dst_bytes = dst_bytes > J.dst.img_bytes ? dst_bytes : J.dst.img_bytes;
        }
        if (total > 0xFFFFFFFFull) return internal_fail(LLGB_ERR_UNSUPPORTED, "batch has too many tiles");
        staging.starts[g][count[g]] = (uint32_t)total;
        int ctas = 2;
        const bool gather = g == 1 || g == 2;
        uint16_t ns = gather ? 4 : 2, nd = gather ? 3 : 2;
        auto need = [&]() {
            return copy_shared_header_bytes() + (size_t)ns * (src_bytes + kStageZeroBytes) + (size_t)nd * dst_bytes;
        };
        while (!internal_smem_fits(need(), ctas) && (ns > 2 || nd > 2 || ctas > 1)) {
            if (ns > 2) --ns;
            else if (nd > 2) --nd;
            else ctas = 1;
        }
        if (!internal_smem_fits(need(), 1)) return internal_fail(LLGB_ERR_UNSUPPORTED, "batch tiles do not fit shared memory");
        launch[g].threads = ctas == 1 ? 512 : 256;
        CopyArgs& a = launch[g].args;
        memset(&a, 0, sizeof a);
        a.table = reinterpret_cast<const JobDesc*>(scratch) + first;
        a.tile_start = reinterpret_cast<const uint32_t*>(static_cast<unsigned char*>(scratch) + kTableBytes) +
                       (size_t)g * kStartsPerMode;
        a.njobs = (uint32_t)count[g];
        a.total_tiles = (uint32_t)total;
        a.src_stage_bytes = src_bytes + kStageZeroBytes;
        a.dst_stage_bytes = dst_bytes;
        a.src_stages = ns;
        a.dst_stages = nd;
        launch[g].grid = (int)(total < (uint64_t)sms * ctas ? total : (uint64_t)sms * ctas);
        a.chunk = (uint32_t)((total + launch[g].grid - 1) / launch[g].grid);
        launch[g].smem = need();
        first += count[g];
    }

    // The descriptors go into the static array by kernel parameters, then
    // the copy kernels run, all in stream order.
    cudaError_t e = upload_range(0, (size_t)njobs * sizeof(JobDesc), s);
    if (e == cudaSuccess) e = upload_range(kTableBytes, kTableBytes + sizeof staging.starts, s);
    if (e != cudaSuccess) return internal_fail(LLGB_ERR_CUDA, cudaGetErrorString(e));
    for (int g = 0; g < kModes; ++g) {
        if (launch[g].grid == 0) continue;
        const int mode = g == 0 ? 0 : (g == 1 ? 2 : (g == 2 ? 4 : (g == 3 ? 1 : 3)));
        e = launch_copy(launch[g].args, mode, launch[g].grid, launch[g].threads, launch[g].smem, s);
        if (e != cudaSuccess) return internal_fail(LLGB_ERR_CUDA, cudaGetErrorString(e));
    }
    return LLGB_OK;
}
