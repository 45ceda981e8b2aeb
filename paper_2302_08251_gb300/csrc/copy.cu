// copy.cu -- the layout-aware copy kernel (Sec. 1 of the paper: layout-aware
// copies between views with different mappings; Sec. 3: pack on store,
// unpack on load, ChangeType, Bytesplit).
//
// One persistent kernel serves every mapping pair and, through a descriptor
// table, many views per launch.  Each CTA walks its share of tiles:
//
//   1. the source runs of the tile are brought into a shared-memory image,
//      with 1-D TMA bulk copies (cp.async.bulk + mbarrier) for full tiles,
//      `src_stages` tiles ahead of the one being converted;
//   2. every item (a leaf moved byte for byte, or a value loaded, converted
//      and stored) runs over the tile's records, one record per thread, from
//      the source image into the destination image; bit-stream destinations
//      first stage their codes, then one thread per 32-bit output word gathers
//      the codes that overlap it;
//   3. the destination runs go back to global memory with bulk stores
//      (cp.async.bulk ... bulk_group), `dst_stages` tiles in flight.
//
// The last tile of a view, and views whose runs are not 16-byte aligned, use
// plain coalesced loads and stores instead of TMA.  Every wait on an mbarrier
// is bounded; on expiry the kernel records LLGB_ERR_TIMEOUT in the device
// status word and returns.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fconv.cuh"
#include "job.h"
#include "kernels.h"
#include "llgb.h"

namespace llgb {

__device__ unsigned int g_device_status;

// ------------------------------------------------------------------ PTX --

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_barrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ uint64_t global_timer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of `bar` to complete, for at most ~2 s.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    for (uint32_t spin = 0; spin < (1u << 30); ++spin) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((spin & 63u) == 0 && global_timer_ns() - t0 > 2000000000ull) break;
    }
    return false;
}

__device__ __forceinline__ void bulk_load(void* sdst, const void* gsrc, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(sdst)),
        "l"(gsrc), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void bulk_store(void* gdst, const void* ssrc, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst),
                 "r"(smem_addr(ssrc)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

__device__ __forceinline__ void bulk_wait_read(int allowed)
{
    switch (allowed) {
    case 0: asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); break;
    case 1: asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); break;
    case 2: asm volatile("cp.async.bulk.wait_group.read 2;" ::: "memory"); break;
    default: asm volatile("cp.async.bulk.wait_group.read 3;" ::: "memory"); break;
    }
}

__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ------------------------------------------------------- image access --

__device__ __forceinline__ uint32_t elem_off(const LeafDesc& L, uint32_t r)
{
    if (L.lanes == 1) return L.sbase + r * L.bstride;
    if (L.lshift != 0xFF)
        return L.sbase + (r >> L.lshift) * L.bstride + (r & (L.lanes - 1u)) * L.size;
    return L.sbase + (r / L.lanes) * L.bstride + (r % L.lanes) * L.size;
}

__device__ __forceinline__ uint64_t ld_elem(const uint8_t* p, int size, int align)
{
    if (align >= size) {
        switch (size) {
        case 1: return *p;
        case 2: return *reinterpret_cast<const uint16_t*>(p);
        case 4: return *reinterpret_cast<const uint32_t*>(p);
        default: return *reinterpret_cast<const uint64_t*>(p);
        }
    }
    uint64_t v = 0;
    for (int j = 0; j < size; ++j) v |= (uint64_t)p[j] << (8 * j);
    return v;
}

__device__ __forceinline__ void st_elem(uint8_t* p, int size, int align, uint64_t v)
{
    if (align >= size) {
        switch (size) {
        case 1: *p = (uint8_t)v; return;
        case 2: *reinterpret_cast<uint16_t*>(p) = (uint16_t)v; return;
        case 4: *reinterpret_cast<uint32_t*>(p) = (uint32_t)v; return;
        default: *reinterpret_cast<uint64_t*>(p) = v; return;
        }
    }
    for (int j = 0; j < size; ++j) p[j] = (uint8_t)(v >> (8 * j));
}

// w bits starting at bit `pos` of the LSB-first stream at `base` (4-aligned,
// readable for 8 bytes past the last value).
__device__ __forceinline__ uint64_t ld_bits(const uint8_t* base, uint32_t pos, int w)
{
    const uint32_t* words = reinterpret_cast<const uint32_t*>(base);
    const uint32_t q = pos >> 5, sh = pos & 31u;
    uint64_t v = ((uint64_t)words[q] | ((uint64_t)words[q + 1] << 32)) >> sh;
    if (sh + (uint32_t)w > 64u) v |= (uint64_t)words[q + 2] << (64u - sh);
    return v & low_bits64(w);
}

template <int G>
struct UInt;
template <>
struct UInt<1> { using T = uint8_t; };
template <>
struct UInt<2> { using T = uint16_t; };
template <>
struct UInt<4> { using T = uint32_t; };
template <>
struct UInt<8> { using T = uint64_t; };

template <int G>
__device__ __forceinline__ void move_loop(const LeafDesc A, const LeafDesc B, uint32_t sb, uint32_t db,
                                          uint32_t size, const uint8_t* simg, uint8_t* dimg,
                                          uint32_t tile, uint32_t nvalid)
{
    using W = typename UInt<G>::T;
    for (uint32_t r = threadIdx.x; r < tile; r += blockDim.x) {
        const uint32_t so = elem_off(A, r) + sb;
        const uint32_t dof = elem_off(B, r) + db;
        if (r < nvalid) {
            for (uint32_t p = 0; p < size; p += G)
                *reinterpret_cast<W*>(dimg + dof + p) = *reinterpret_cast<const W*>(simg + so + p);
        } else {
            for (uint32_t p = 0; p < size; p += G) *reinterpret_cast<W*>(dimg + dof + p) = W(0);
        }
    }
}

__device__ __forceinline__ uint64_t load_value(const ItemDesc& I, const SideDesc& S, const uint8_t* simg,
                                               uint32_t r)
{
    switch (I.lop) {
    case L_DIRECT: {
        const LeafDesc& L = S.leaves[I.src_leaf];
        return ld_elem(simg + elem_off(L, r), I.size, L.align);
    }
    case L_CT: {
        const LeafDesc& L = S.leaves[I.src_leaf];
        const uint64_t u = ld_elem(simg + elem_off(L, r), I.s_size, L.align);
        return fconv(u, I.s_e, I.s_m, I.l_e, I.l_m);
    }
    case L_BITS_INT: {
        const LeafDesc& L = S.leaves[I.src_leaf];
        uint64_t c = ld_bits(simg + L.sbase, r * L.bits, L.bits);
        if (I.is_signed && ((c >> (L.bits - 1)) & 1ull)) c |= ~low_bits64(L.bits);
        return c & low_bits64(8 * I.size);
    }
    case L_BITS_FLOAT: {
        const LeafDesc& L = S.leaves[I.src_leaf];
        const uint64_t c = ld_bits(simg + L.sbase, r * L.bits, L.bits);
        return fconv(c, I.s_e, I.s_m, I.l_e, I.l_m);
    }
    default: {  // L_SPLIT
        uint64_t v = 0;
        for (int j = 0; j < I.size; ++j) {
            const LeafDesc& L = S.leaves[I.src_leaf + j];
            v |= (uint64_t)simg[elem_off(L, r)] << (8 * j);
        }
        return v;
    }
    }
}

__device__ __forceinline__ void store_code(const PackDesc& P, uint8_t* codes, uint32_t r, uint64_t c)
{
    if (P.wide)
        reinterpret_cast<uint64_t*>(codes + P.code_off)[r] = c;
    else
        reinterpret_cast<uint32_t*>(codes + P.code_off)[r] = (uint32_t)c;
}

__device__ __forceinline__ void store_value(const ItemDesc& I, const JobDesc& J, uint8_t* dimg, uint8_t* codes,
                                            uint32_t r, uint64_t v)
{
    const SideDesc& D = J.dst;
    switch (I.sop) {
    case S_DIRECT: {
        const LeafDesc& L = D.leaves[I.dst_leaf];
        st_elem(dimg + elem_off(L, r), I.size, L.align, v);
        return;
    }
    case S_CT: {
        const LeafDesc& L = D.leaves[I.dst_leaf];
        st_elem(dimg + elem_off(L, r), I.d_size, L.align, fconv(v, I.l_e, I.l_m, I.d_e, I.d_m));
        return;
    }
    case S_BITS_INT:
        store_code(J.packs[I.slot], codes, r, v & low_bits64(I.d_bits));
        return;
    case S_BITS_FLOAT:
        store_code(J.packs[I.slot], codes, r, fconv(v, I.l_e, I.l_m, I.d_e, I.d_m));
        return;
    default: {  // S_SPLIT
        for (int j = 0; j < I.size; ++j) {
            const LeafDesc& L = D.leaves[I.dst_leaf + j];
            dimg[elem_off(L, r)] = (uint8_t)(v >> (8 * j));
        }
        return;
    }
    }
}

__device__ void run_items(const JobDesc& J, const uint8_t* simg, uint8_t* dimg, uint8_t* codes,
                          uint32_t nvalid)
{
    const uint32_t tile = J.tile;
    for (int it = 0; it < J.nitems; ++it) {
        const ItemDesc I = J.items[it];
        if (I.op == ITEM_MOVE) {
            const LeafDesc A = J.src.leaves[I.src_leaf];
            const LeafDesc B = J.dst.leaves[I.dst_leaf];
            switch (I.gran) {
            case 8: move_loop<8>(A, B, I.src_byte, I.dst_byte, I.size, simg, dimg, tile, nvalid); break;
            case 4: move_loop<4>(A, B, I.src_byte, I.dst_byte, I.size, simg, dimg, tile, nvalid); break;
            case 2: move_loop<2>(A, B, I.src_byte, I.dst_byte, I.size, simg, dimg, tile, nvalid); break;
            default: move_loop<1>(A, B, I.src_byte, I.dst_byte, I.size, simg, dimg, tile, nvalid); break;
            }
        } else {
            for (uint32_t r = threadIdx.x; r < tile; r += blockDim.x) {
                const uint64_t v = r < nvalid ? load_value(I, J.src, simg, r) : 0ull;
                store_value(I, J, dimg, codes, r, v);
            }
        }
    }
}

// One thread per 32-bit word of each bit-stream destination: OR together the
// staged codes that overlap the word.
__device__ void run_packs(const JobDesc& J, uint8_t* dimg, const uint8_t* codes)
{
    const uint32_t tile = J.tile;
    for (int k = 0; k < J.npacks; ++k) {
        const PackDesc P = J.packs[k];
        const uint32_t w = P.bits;
        const uint32_t nwords = tile * w / 32u;
        uint32_t* out = reinterpret_cast<uint32_t*>(dimg + P.dst_sbase);
        for (uint32_t q = threadIdx.x; q < nwords; q += blockDim.x) {
            const uint32_t bit0 = q * 32u;
            const uint32_t jlo = bit0 / w;
            uint32_t jhi = (bit0 + 31u) / w;
            if (jhi > tile - 1u) jhi = tile - 1u;
            uint32_t word = 0;
            for (uint32_t j = jlo; j <= jhi; ++j) {
                const uint64_t c = P.wide ? reinterpret_cast<const uint64_t*>(codes + P.code_off)[j]
                                          : (uint64_t) reinterpret_cast<const uint32_t*>(codes + P.code_off)[j];
                const int pos = (int)(j * w) - (int)bit0;
                word |= pos >= 0 ? (uint32_t)(c << pos) : (uint32_t)(c >> (-pos));
            }
            out[q] = word;
        }
    }
}

// Plain copy of `bytes` between global and shared memory by all threads.
__device__ void plain_copy(uint8_t* dst, const uint8_t* src, uint32_t bytes)
{
    const uintptr_t both = reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src);
    uint32_t done = 0;
    if ((both & 15u) == 0) {
        const uint32_t n16 = bytes / 16u;
        for (uint32_t k = threadIdx.x; k < n16; k += blockDim.x)
            reinterpret_cast<uint4*>(dst)[k] = reinterpret_cast<const uint4*>(src)[k];
        done = n16 * 16u;
    } else if ((both & 3u) == 0) {
        const uint32_t n4 = bytes / 4u;
        for (uint32_t k = threadIdx.x; k < n4; k += blockDim.x)
            reinterpret_cast<uint32_t*>(dst)[k] = reinterpret_cast<const uint32_t*>(src)[k];
        done = n4 * 4u;
    }
    for (uint32_t k = done + threadIdx.x; k < bytes; k += blockDim.x) dst[k] = src[k];
}

__device__ __forceinline__ uint32_t job_of(const CopyArgs& a, uint32_t g)
{
    if (a.table == nullptr) return 0;
    uint32_t lo = 0, hi = a.njobs;  // tile_start[lo] <= g < tile_start[hi]
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (a.tile_start[mid] <= g) lo = mid;
        else hi = mid;
    }
    return lo;
}

struct __align__(16) CopyShared {
    uint64_t full[8];
    int abort;
    int cur_job;
    int pad[2];
    JobDesc job;
};

__device__ __forceinline__ uint32_t align16(uint32_t x) { return (x + 15u) & ~15u; }

__global__ void __launch_bounds__(1024) copy_kernel(const __grid_constant__ CopyArgs a)
{
    extern __shared__ __align__(128) uint8_t smem[];
    CopyShared& H = *reinterpret_cast<CopyShared*>(smem);
    uint8_t* src_stage = smem + align16(sizeof(CopyShared));
    uint8_t* dst_stage = src_stage + a.src_stages * a.src_stage_bytes;
    uint8_t* codes = dst_stage + a.dst_stages * a.dst_stage_bytes;

    const uint32_t G = gridDim.x;
    const uint32_t first = blockIdx.x;
    if (first >= a.total_tiles) return;
    const uint32_t count = (a.total_tiles - first + G - 1u) / G;
    const uint32_t NS = a.src_stages, ND = a.dst_stages;

    if (threadIdx.x == 0) {
        for (uint32_t s = 0; s < NS; ++s) mbar_init(&H.full[s], 1);
        fence_barrier_init();
        H.abort = 0;
        H.cur_job = -1;
    }
    __syncthreads();

    // Producer side (thread 0): issue the TMA loads of this CTA's k-th tile.
    auto issue = [&](uint32_t k) {
        const uint32_t g = first + k * G;
        const uint32_t j = job_of(a, g);
        const JobDesc* J = a.table ? a.table + j : &a.job;
        const uint32_t t = g - (a.table ? a.tile_start[j] : 0u);
        if (t >= J->nfull || !J->src.bulk_ok) return;
        const uint32_t s = k % NS;
        uint8_t* img = src_stage + s * a.src_stage_bytes;
        uint32_t total = 0;
        for (int q = 0; q < J->src.nsegs; ++q) total += J->src.segs[q].tile_bytes;
        mbar_arrive_expect_tx(&H.full[s], total);
        for (int q = 0; q < J->src.nsegs; ++q) {
            const SegDesc& S = J->src.segs[q];
            bulk_load(img + S.sbase, J->src.blobs[S.blob] + S.gbase + (uint64_t)t * S.tile_bytes,
                      S.tile_bytes, &H.full[s]);
        }
    };

    if (threadIdx.x == 0)
        for (uint32_t k = 0; k < NS && k < count; ++k) issue(k);

    uint32_t phase = 0;
    uint32_t k = 0;
    for (; k < count; ++k) {
        const uint32_t g = first + k * G;
        const uint32_t j = job_of(a, g);
        if ((int)j != H.cur_job) {
            __syncthreads();
            if (threadIdx.x == 0) bulk_wait_read(0);
            __syncthreads();
            const JobDesc* src_desc = a.table ? a.table + j : &a.job;
            const uint2* from = reinterpret_cast<const uint2*>(src_desc);
            uint2* to = reinterpret_cast<uint2*>(&H.job);
            for (uint32_t w = threadIdx.x; w < sizeof(JobDesc) / 8u; w += blockDim.x) to[w] = from[w];
            uint4* z = reinterpret_cast<uint4*>(dst_stage);
            const uint32_t zwords = (ND * a.dst_stage_bytes + a.code_bytes) / 16u;
            for (uint32_t w = threadIdx.x; w < zwords; w += blockDim.x) z[w] = make_uint4(0, 0, 0, 0);
            __syncthreads();
            if (threadIdx.x == 0) H.cur_job = (int)j;
        }
        const JobDesc& J = H.job;
        const uint32_t t = g - (a.table ? a.tile_start[j] : 0u);
        const uint32_t nvalid = (t + 1u < J.ntiles) ? J.tile : (uint32_t)(J.n - (uint64_t)t * J.tile);
        const uint32_t s = k % NS, d = k % ND;
        uint8_t* simg = src_stage + s * a.src_stage_bytes;
        uint8_t* dimg = dst_stage + d * a.dst_stage_bytes;
        const bool bulk_in = t < J.nfull && J.src.bulk_ok;
        const bool bulk_out = t < J.nfull && J.dst.bulk_ok;

        if (bulk_in) {
            if (!mbar_wait_bounded(&H.full[s], (phase >> s) & 1u)) H.abort = 1;
            phase ^= 1u << s;
        } else {
            const bool last = (t + 1u == J.ntiles);
            for (int q = 0; q < J.src.nsegs; ++q) {
                const SegDesc& S = J.src.segs[q];
                plain_copy(simg + S.sbase, J.src.blobs[S.blob] + S.gbase + (uint64_t)t * S.tile_bytes,
                           last ? S.tail_bytes : S.tile_bytes);
            }
        }
        if (threadIdx.x == 0) bulk_wait_read((int)ND - 1);
        __syncthreads();
        if (H.abort) break;

        if (t == 0) {
            for (int q = 0; q < J.nzeros; ++q) {
                const ZeroRun& Z = J.zeros[q];
                uint8_t* p = J.dst.blobs[Z.blob] + Z.offset;
                for (uint32_t b = threadIdx.x; b < Z.bytes; b += blockDim.x) p[b] = 0;
            }
        }
        run_items(J, simg, dimg, codes, nvalid);
        if (J.npacks) {
            __syncthreads();
            run_packs(J, dimg, codes);
        }
        fence_proxy_async();
        __syncthreads();

        if (bulk_out) {
            if (threadIdx.x == 0) {
                for (int q = 0; q < J.dst.nsegs; ++q) {
                    const SegDesc& S = J.dst.segs[q];
                    bulk_store(J.dst.blobs[S.blob] + S.gbase + (uint64_t)t * S.tile_bytes, dimg + S.sbase,
                               S.tile_bytes);
                }
                bulk_commit();
            }
        } else {
            const bool last = (t + 1u == J.ntiles);
            for (int q = 0; q < J.dst.nsegs; ++q) {
                const SegDesc& S = J.dst.segs[q];
                plain_copy(J.dst.blobs[S.blob] + S.gbase + (uint64_t)t * S.tile_bytes, dimg + S.sbase,
                           last ? S.tail_bytes : S.tile_bytes);
            }
        }
        if (threadIdx.x == 0 && k + NS < count) issue(k + NS);
    }

    if (threadIdx.x == 0) {
        if (H.abort) {
            atomicOr(&g_device_status, (unsigned)LLGB_ERR_TIMEOUT);
            // let the loads already issued land before the CTA goes away
            for (uint32_t q = k + 1; q < k + NS && q < count; ++q) {
                const uint32_t s = q % NS;
                mbar_wait_bounded(&H.full[s], (phase >> s) & 1u);
            }
        }
        bulk_wait_all();
    }
}

// ------------------------------------------------------------ launcher --

size_t copy_shared_header_bytes() { return (sizeof(CopyShared) + 15u) & ~size_t(15); }

cudaError_t launch_copy(const CopyArgs& args, int grid, int threads, size_t smem_bytes, cudaStream_t stream)
{
    static thread_local int configured_dev = -1;
    static thread_local size_t configured_bytes = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev != configured_dev || smem_bytes > configured_bytes) {
        e = cudaFuncSetAttribute(copy_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
        if (e != cudaSuccess) return e;
        configured_dev = dev;
        configured_bytes = smem_bytes;
    }
    copy_kernel<<<grid, threads, smem_bytes, stream>>>(args);
    return cudaGetLastError();
}

cudaError_t read_device_status(unsigned* out, bool reset)
{
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return e;
    e = cudaMemcpyFromSymbol(out, g_device_status, sizeof(unsigned));
    if (e != cudaSuccess) return e;
    if (reset) {
        const unsigned zero = 0;
        e = cudaMemcpyToSymbol(g_device_status, &zero, sizeof(unsigned));
    }
    return e;
}

}  // namespace llgb
