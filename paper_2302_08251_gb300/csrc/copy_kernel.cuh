// copy_kernel.cuh -- the layout-aware copy kernel (Sec. 1 of the paper: layout-aware
// copies between views with different mappings; Sec. 3: pack on store,
// unpack on load, ChangeType, Bytesplit).
//
// One persistent kernel serves every mapping pair and, through a descriptor
// table, many views per launch.  Each CTA walks its share of tiles with one
// load warp, one store warp and several consumer warps, synchronised by
// mbarriers:
//
//   1. the load warp brings the source runs of a tile into a shared-memory
//      image with 1-D TMA bulk copies (cp.async.bulk + mbarrier transaction
//      counts), `src_stages` tiles ahead of the consumers;
//   2. the consumers convert the tile into a destination image: jobs made of
//      byte moves run per-thread gather programs (PRMT); other jobs run their
//      items (a leaf moved byte for byte, or a value loaded, converted and
//      stored), each warp over its fixed share of the tile, in loops
//      specialised for the common cases (V consecutive records per lane,
//      stream words assembled with warp shuffles, byte planes by 4 x 4
//      byte transposes);
//   3. the store warp writes the destination runs back with bulk stores
//      (cp.async.bulk ... bulk_group) as soon as the consumers release them,
//      and hands each destination stage back once its store has read it.
//
// Value kernels have a load warp and a store warp; gather kernels, whose
// consumers need every warp, one warp that does both.
//
// The last tile of a view, and views whose runs are not 16-byte aligned, use
// plain coalesced loads and stores instead of TMA.  Every wait on an mbarrier
// is bounded; on expiry the kernel records LLGB_ERR_TIMEOUT in the device
// status word and returns.
//
// Each kernel mode is compiled in a translation unit of its own
// (copy_mode0.cu, copy_mode1.cu, copy_mode3.cu, copy_gather.cu), so that the
// modes build in parallel; every unit holds its own device status word, and the host reads
// them all (copy.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "fconv.cuh"
#include "job.h"
#include "kernels.h"
#include "llgb.h"

namespace llgb {

// Status word of this translation unit's kernels (LLGB_ERR_TIMEOUT when a
// bounded wait gave up).
static __device__ unsigned int g_device_status;

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

// try_wait that may suspend the thread for up to `hint_ns` until the phase
// completes, instead of returning at once: waiting warps then leave the issue
// slots to the warps that have work.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, uint32_t parity, uint32_t hint_ns)
{
    uint32_t done;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return done != 0;
}

// Longest wait of a copy kernel on one mbarrier phase.
constexpr uint64_t kWaitLimitNs = 2000000000ull;

// Wait for phase `parity` of `bar` to complete, for at most limit_ns (and at
// most 2^30 suspended polls of up to 20 us each).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns = kWaitLimitNs)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    for (uint32_t spin = 0; spin < (1u << 30); ++spin) {
        if (mbar_try_wait_sleep(bar, parity, 20000u)) return true;
        if (global_timer_ns() - t0 > limit_ns) break;
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

// The head of a CTA's dynamic shared memory; the stage images follow it.
struct __align__(16) CopyShared {
    uint64_t full[8];    // source stage s holds its tile (TMA transaction count)
    uint64_t empty[8];   // consumers are done reading source stage s
    uint64_t dfull[4];   // consumers have written destination stage d
    uint64_t dempty[4];  // the store of destination stage d has read it
    int abort;
    uint32_t cons_base;  // first consumer thread: 32 x the producer warps
    int pad[2];
    JobDesc job;         // the consumers' copy of the current job
};

extern __shared__ __align__(128) uint8_t g_smem[];

// The first warps of a CTA issue the TMA loads and stores (producer_warps
// of the kernel mode); the other warps are consumers, and every per-tile
// loop below is strided over them only.
__device__ __forceinline__ uint32_t cons_base() { return reinterpret_cast<const CopyShared*>(g_smem)->cons_base; }
__device__ __forceinline__ uint32_t ctid() { return threadIdx.x - cons_base(); }
__device__ __forceinline__ uint32_t cnum() { return blockDim.x - cons_base(); }

__device__ __forceinline__ void consumer_sync()
{
    asm volatile("bar.sync 1, %0;" ::"r"(cnum()) : "memory");
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

// Leaf addressing held in registers for a whole loop.
struct LeafRegs {
    uint32_t sbase, bstride, lanes, size, lshift, align, bits;
};

__device__ __forceinline__ LeafRegs leaf_regs(const LeafDesc& L)
{
    return LeafRegs{L.sbase, L.bstride, L.lanes, L.size, L.lshift, L.align, L.bits};
}

__device__ __forceinline__ uint32_t eoff(const LeafRegs& L, uint32_t r)
{
    if (L.lanes == 1) return L.sbase + r * L.bstride;
    if (L.lshift != 0xFF) return L.sbase + (r >> L.lshift) * L.bstride + (r & (L.lanes - 1u)) * L.size;
    return L.sbase + (r / L.lanes) * L.bstride + (r % L.lanes) * L.size;
}

// The records a loop visits: r0, r0 + step, ... below r1.
struct Span {
    uint32_t r0, r1, step;
};

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
__device__ __forceinline__ void move_loop(const LeafRegs A, const LeafRegs B, uint32_t sb, uint32_t db,
                                          uint32_t size, const uint8_t* __restrict__ simg,
                                          uint8_t* __restrict__ dimg, Span sp, uint32_t nvalid)
{
    using W = typename UInt<G>::T;
    for (uint32_t r = sp.r0; r < sp.r1; r += sp.step) {
        const uint32_t so = eoff(A, r) + sb;
        const uint32_t dof = eoff(B, r) + db;
        const bool live = r < nvalid;
        for (uint32_t p = 0; p < size; p += G)
            *reinterpret_cast<W*>(dimg + dof + p) = live ? *reinterpret_cast<const W*>(simg + so + p) : W(0);
    }
}

__device__ __forceinline__ bool byte_aligned_width(uint32_t w) { return w == 8 || w == 16 || w == 32 || w == 64; }

__device__ __forceinline__ void red_or_shared(uint32_t* p, uint32_t v)
{
    asm volatile("red.shared.or.b32 [%0], %1;" ::"r"(smem_addr(p)), "r"(v) : "memory");
}

// OR the w-bit code c into the zeroed LSB-first stream at `base`, at bit pos.
__device__ __forceinline__ void or_bits(uint8_t* base, uint32_t pos, uint32_t w, uint64_t c)
{
    if (c == 0) return;
    uint32_t* words = reinterpret_cast<uint32_t*>(base) + (pos >> 5);
    const uint32_t sh = pos & 31u;
    const uint32_t lo = (uint32_t)c, hi = (uint32_t)(c >> 32);
    red_or_shared(words, lo << sh);
    if (sh + w > 32u) red_or_shared(words + 1, sh ? __funnelshift_l(lo, hi, sh) : hi);
    if (sh + w > 64u) red_or_shared(words + 2, hi >> (32u - sh));
}

// One VALUE item: load the logical value through LOP, store it through SOP.
// Two records per iteration keep two independent chains in flight.  SEG: a
// bit leaf of the item is organised as AoSoA (runs of `lanes` codes,
// `bstride` bytes apart); a separate instantiation, so that SoA streams keep
// their plain addressing (and its register budget).
template <int LOP, int SOP, bool SEG = false>
__device__ __noinline__ void value_loop(const ItemDesc& I, const JobDesc& J, const uint8_t* __restrict__ simg,
                                        uint8_t* __restrict__ dimg, Span sp, uint32_t nvalid)
{
    const LeafRegs A = leaf_regs(J.src.leaves[I.src_leaf]);
    const LeafRegs B = leaf_regs(J.dst.leaves[I.dst_leaf]);
    const int size = I.size;
    const uint64_t lmask = low_bits64(8 * size);
    const bool is_bits_src = LOP == L_BITS_INT || LOP == L_BITS_FLOAT;
    const bool a_aligned = is_bits_src && byte_aligned_width(A.bits);
    const uint32_t abytes = A.bits / 8u;
    const uint64_t smask = low_bits64(A.bits);
    const bool d_aligned = (SOP == S_BITS_INT || SOP == S_BITS_FLOAT) && byte_aligned_width(I.d_bits);
    const uint32_t dbytes = I.d_bits / 8u;
    const uint64_t dmask = low_bits64(I.d_bits);

    auto load = [&](uint32_t r) -> uint64_t {
        if (r >= nvalid) return 0ull;
        if (LOP == L_NULL) return 0ull;  // Null mapping: a zero value
        if (LOP == L_DIRECT) return ld_elem(simg + eoff(A, r), size, A.align);
        if (LOP == L_CT) return fconv(ld_elem(simg + eoff(A, r), I.s_size, A.align), I.s_e, I.s_m, I.l_e, I.l_m);
        if (is_bits_src) {
            // the run holding record r, and r's lane in it
            const uint8_t* run = SEG ? simg + A.sbase + (r >> A.lshift) * A.bstride : simg + A.sbase;
            const uint32_t rl = SEG ? r & (A.lanes - 1u) : r;
            uint64_t c;
            if (a_aligned) {
                c = ld_elem(run + rl * abytes, (int)abytes, SEG ? (int)min(abytes, A.align) : (int)abytes);
            } else if (A.bits <= 32) {
                const uint32_t* wd = reinterpret_cast<const uint32_t*>(run);
                const uint32_t pos = rl * A.bits;
                c = __funnelshift_r(wd[pos >> 5], wd[(pos >> 5) + 1], pos & 31u) & (uint32_t)smask;
            } else {
                c = ld_bits(run, rl * A.bits, A.bits);
            }
            if (LOP == L_BITS_INT) {
                if (I.is_signed && ((c >> (A.bits - 1)) & 1ull)) c |= ~smask;
                return c & lmask;
            }
            return fconv(c, I.s_e, I.s_m, I.l_e, I.l_m);
        }
        uint64_t v = 0;  // L_SPLIT
        for (int j = 0; j < size; ++j) {
            const LeafRegs S = leaf_regs(J.src.leaves[I.src_leaf + j]);
            v |= (uint64_t)simg[eoff(S, r)] << (8 * j);
        }
        return v;
    };
    auto store = [&](uint32_t r, uint64_t v) {
        if (SOP == S_DIRECT) {
            st_elem(dimg + eoff(B, r), size, B.align, v);
        } else if (SOP == S_CT) {
            st_elem(dimg + eoff(B, r), I.d_size, B.align, fconv(v, I.l_e, I.l_m, I.d_e, I.d_m));
        } else if (SOP == S_BITS_INT || SOP == S_BITS_FLOAT) {
            const uint64_t c = SOP == S_BITS_INT ? (v & dmask) : fconv(v, I.l_e, I.l_m, I.d_e, I.d_m);
            uint8_t* run = SEG ? dimg + B.sbase + (r >> B.lshift) * B.bstride : dimg + B.sbase;
            const uint32_t rl = SEG ? r & (B.lanes - 1u) : r;
            if (d_aligned)
                st_elem(run + rl * dbytes, (int)dbytes, SEG ? (int)min(dbytes, B.align) : (int)dbytes, c);
            else
                or_bits(run, rl * I.d_bits, I.d_bits, c);
        } else {  // S_SPLIT
            for (int j = 0; j < size; ++j) {
                const LeafRegs D = leaf_regs(J.dst.leaves[I.dst_leaf + j]);
                dimg[eoff(D, r)] = (uint8_t)(v >> (8 * j));
            }
        }
    };
    for (uint32_t r = sp.r0; r < sp.r1; r += 2u * sp.step) {
        const uint32_t r2 = r + sp.step;
        const uint64_t v1 = load(r);
        const uint64_t v2 = r2 < sp.r1 ? load(r2) : 0ull;
        store(r, v1);
        if (r2 < sp.r1) store(r2, v2);
    }
}

// SEGOK: the kernel mode that runs jobs with AoSoA-organised bit leaves (1);
// the other value mode (0) never calls their loops, which keeps its register
// budget (calls share the kernel's registers).
template <int LOP, bool SEGOK>
__device__ __forceinline__ void value_dispatch(const ItemDesc& I, const JobDesc& J, const uint8_t* simg,
                                               uint8_t* dimg, Span sp, uint32_t nvalid)
{
    constexpr bool bits_src = LOP == L_BITS_INT || LOP == L_BITS_FLOAT;
    const bool seg_src = bits_src && J.src.leaves[I.src_leaf].lanes != 0;
    const bool seg_dst = (I.sop == S_BITS_INT || I.sop == S_BITS_FLOAT) && J.dst.leaves[I.dst_leaf].lanes != 0;
    if constexpr (SEGOK) {
        if (seg_src || seg_dst) {  // AoSoA-organised bit leaves
            switch (I.sop) {
            case S_BITS_INT: value_loop<LOP, S_BITS_INT, true>(I, J, simg, dimg, sp, nvalid); return;
            case S_BITS_FLOAT: value_loop<LOP, S_BITS_FLOAT, true>(I, J, simg, dimg, sp, nvalid); return;
            default:
                if constexpr (bits_src) {
                    switch (I.sop) {
                    case S_DIRECT: value_loop<LOP, S_DIRECT, true>(I, J, simg, dimg, sp, nvalid); return;
                    case S_CT: value_loop<LOP, S_CT, true>(I, J, simg, dimg, sp, nvalid); return;
                    default: value_loop<LOP, S_SPLIT, true>(I, J, simg, dimg, sp, nvalid); return;
                    }
                }
                return;
            }
        }
    }
    switch (I.sop) {
    case S_DIRECT: value_loop<LOP, S_DIRECT>(I, J, simg, dimg, sp, nvalid); break;
    case S_CT: value_loop<LOP, S_CT>(I, J, simg, dimg, sp, nvalid); break;
    case S_BITS_INT: value_loop<LOP, S_BITS_INT>(I, J, simg, dimg, sp, nvalid); break;
    case S_BITS_FLOAT: value_loop<LOP, S_BITS_FLOAT>(I, J, simg, dimg, sp, nvalid); break;
    default: value_loop<LOP, S_SPLIT>(I, J, simg, dimg, sp, nvalid); break;
    }
}

// ------------------------------------------------------ fast value loops --
//
// A VALUE item whose element sizes and conversion are among the common cases
// runs here.  Lane l of a warp takes V consecutive records (V = 1, 2 or 4,
// chosen by the planner per item) of each "super-group" of 32 V records, so
//  * an affine leaf's elements of a lane sit at a lane constant plus a step
//    per super-group, and are moved with vector loads / stores where they
//    are contiguous;
//  * a w-bit stream's super-group is exactly C = V w whole words (32 <= C <=
//    64 for w >= 8), and the lane's codes form one C-bit chunk at a lane-
//    constant bit offset: a lane reads its chunk with three word loads and
//    two funnel shifts, and assembles output word k from the (at most two,
//    for C >= 32) chunks that reach it, fetched with warp shuffles -- codes
//    are stored as whole words, never ORed into shared memory.

enum FastLoad { FL_AFF = 0, FL_AL = 1, FL_BITS = 2 };
enum FastStore { FS_AFF = 0, FS_AL = 1, FS_BITS = 2 };
// FC_SAME: one float format on both sides (only a NaN changes: it is quieted).
enum FastConv { FC_INT = 0, FC_D2F = 1, FC_F2D = 2, FC_RT = 3, FC_SAME = 4, FC_NONE = 5 };

template <int SZ>
__device__ __forceinline__ uint64_t ld_sz(const uint8_t* p)
{
    if (SZ == 1) return *p;
    if (SZ == 2) return *reinterpret_cast<const uint16_t*>(p);
    if (SZ == 4) return *reinterpret_cast<const uint32_t*>(p);
    return *reinterpret_cast<const uint64_t*>(p);
}

// Shared-memory accesses at 32-bit shared-window addresses.  The loops
// below are separate functions that see the stage images only through
// pointers, so they address them explicitly (no 64-bit generic addressing).
// Loads carry no memory clobber: within a loop the source image is only
// read and the destination image only written.
template <int SZ>
__device__ __forceinline__ uint64_t lds(uint32_t a)
{
    if constexpr (SZ == 1) {
        uint16_t v;
        asm("ld.shared.u8 %0, [%1];" : "=h"(v) : "r"(a));
        return v & 0xFFu;
    } else if constexpr (SZ == 2) {
        uint16_t v;
        asm("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(a));
        return v;
    } else if constexpr (SZ == 4) {
        uint32_t v;
        asm("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
        return v;
    } else {
        uint64_t v;
        asm("ld.shared.u64 %0, [%1];" : "=l"(v) : "r"(a));
        return v;
    }
}

template <int SZ>
__device__ __forceinline__ void sts(uint32_t a, uint64_t v)
{
    if constexpr (SZ == 1) asm volatile("st.shared.u8 [%0], %1;" ::"r"(a), "h"((uint16_t)(v & 0xFFu)));
    else if constexpr (SZ == 2) asm volatile("st.shared.u16 [%0], %1;" ::"r"(a), "h"((uint16_t)v));
    else if constexpr (SZ == 4) asm volatile("st.shared.u32 [%0], %1;" ::"r"(a), "r"((uint32_t)v));
    else asm volatile("st.shared.u64 [%0], %1;" ::"r"(a), "l"(v));
}

__device__ __forceinline__ uint2 lds_v2(uint32_t a)
{
    uint2 v;
    asm("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a));
    return v;
}

__device__ __forceinline__ uint4 lds_v4(uint32_t a)
{
    uint4 v;
    asm("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
    return v;
}

__device__ __forceinline__ void sts_v2(uint32_t a, uint32_t x, uint32_t y)
{
    asm volatile("st.shared.v2.u32 [%0], {%1, %2};" ::"r"(a), "r"(x), "r"(y));
}

__device__ __forceinline__ void sts_v4(uint32_t a, uint32_t x, uint32_t y, uint32_t z, uint32_t w)
{
    asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(x), "r"(y), "r"(z), "r"(w));
}

// One side's lane constants: element v of the lane's records in super-group
// g sits at off + g * step + v * vstride; `vec`: the V elements are
// contiguous and aligned for vector access.
struct LaneRun {
    uint32_t off, step, vstride;
    bool vec;
};

template <int V, int SZ>
__device__ __forceinline__ bool run_vec_ok(uint32_t off, uint32_t step, uint32_t vstride)
{
    constexpr uint32_t A = (V * SZ) >= 16 ? 16u : (uint32_t)(V * SZ);
    return V * SZ >= 4 && vstride == (uint32_t)SZ && off % A == 0u && step % A == 0u;
}

// Affine leaves with one lane, or a power-of-two lane count that V divides
// and that divides 32 V (the planner checks).
template <int V, int SZ>
__device__ __forceinline__ LaneRun affine_run(const LeafDesc& L, uint32_t lane)
{
    const uint32_t r = (uint32_t)V * lane;
    LaneRun R;
    R.step = ((32u * V) >> L.lshift) * L.bstride;
    R.off = L.sbase + (r >> L.lshift) * L.bstride + (r & (L.lanes - 1u)) * L.size;
    R.vstride = L.lanes == 1 ? L.bstride : L.size;
    R.vec = run_vec_ok<V, SZ>(R.off, R.step, R.vstride);
    return R;
}

// Where super-group g of a bit leaf starts, relative to super-group 0:
// (g >> ksh) * bstride + (g & kmask) * step.  A SoA stream is one run (ksh
// 31, kmask all ones: g * step); an AoSoA-organised leaf has 2^ksh
// super-groups per run of L codes (L >= 32 V), runs bstride bytes apart.
struct SgSteps {
    uint32_t step, bstride, ksh, kmask;
};

__device__ __forceinline__ SgSteps sg_steps(const LeafDesc& L, uint32_t step, int V)
{
    if (L.lanes == 0) return SgSteps{step, 0u, 31u, 0xFFFFFFFFu};
    const uint32_t ksh = L.lshift - 5u - (V == 4 ? 2u : (V == 2 ? 1u : 0u));
    return SgSteps{step, L.bstride, ksh, (1u << ksh) - 1u};
}

__device__ __forceinline__ uint32_t sg_off(const SgSteps& S, uint32_t g)
{
    return (g >> S.ksh) * S.bstride + (g & S.kmask) * S.step;
}

// Whole-byte streams: a dense array of SZ-byte codes (per run).
template <int V, int SZ>
__device__ __forceinline__ LaneRun stream_run(const LeafDesc& L, uint32_t lane)
{
    LaneRun R;
    R.step = 32u * V * SZ;
    R.off = L.sbase + (uint32_t)V * lane * SZ;
    R.vstride = SZ;
    R.vec = run_vec_ok<V, SZ>(R.off, R.step, R.vstride) && (L.bstride % 16u == 0u);
    return R;
}

// The V elements of a lane as 32-bit words (V * SZ >= 4 bytes, vector path).
template <int V, int SZ, typename T>
__device__ __forceinline__ void words_to_elems(const uint32_t* w, T (&x)[V])
{
#pragma unroll
    for (int v = 0; v < V; ++v) {
        if constexpr (SZ == 8) x[v] = (T)((uint64_t)w[2 * v] | ((uint64_t)w[2 * v + 1] << 32));
        else if constexpr (SZ == 4) x[v] = w[v];
        else if constexpr (SZ == 2) x[v] = (w[v / 2] >> (16 * (v % 2))) & 0xFFFFu;
        else x[v] = (w[v / 4] >> (8 * (v % 4))) & 0xFFu;
    }
}

template <int V, int SZ, typename T>
__device__ __forceinline__ void elems_to_words(const T (&x)[V], uint32_t* w)
{
#pragma unroll
    for (int q = 0; q < V * SZ / 4; ++q) w[q] = 0u;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        if constexpr (SZ == 8) {
            w[2 * v] = (uint32_t)x[v];
            w[2 * v + 1] = (uint32_t)((uint64_t)x[v] >> 32);
        } else if constexpr (SZ == 4) {
            w[v] = (uint32_t)x[v];
        } else if constexpr (SZ == 2) {
            w[v / 2] |= ((uint32_t)x[v] & 0xFFFFu) << (16 * (v % 2));
        } else {
            w[v / 4] |= ((uint32_t)x[v] & 0xFFu) << (8 * (v % 4));
        }
    }
}

template <int V, int SZ, typename T>
__device__ __forceinline__ void ld_run(uint32_t p, const LaneRun& R, T (&x)[V])
{
    constexpr int BYTES = V * SZ;
    if constexpr (BYTES >= 4) {
        if (R.vec) {
            uint32_t w[BYTES / 4];
            if constexpr (BYTES % 16 == 0) {
#pragma unroll
                for (int q = 0; q < BYTES / 16; ++q) {
                    const uint4 t = lds_v4(p + 16u * q);
                    w[4 * q] = t.x;
                    w[4 * q + 1] = t.y;
                    w[4 * q + 2] = t.z;
                    w[4 * q + 3] = t.w;
                }
            } else if constexpr (BYTES == 8) {
                const uint2 t = lds_v2(p);
                w[0] = t.x;
                w[1] = t.y;
            } else {
                w[0] = (uint32_t)lds<4>(p);
            }
            words_to_elems<V, SZ, T>(w, x);
            return;
        }
    }
    if constexpr (V == 4) {
        // Strided elements (an AoS-like leaf): the lanes of 8-lane quarter q
        // read element (v + q) & 3 at step v instead of element v.  With
        // every lane at the same element, lanes whose records lie a bank
        // cycle apart collide (8-way at a 24-byte record); spread over the
        // quarters, they collide 4x less often, at any stride.
        const uint32_t r = (threadIdx.x >> 3) & 3u;
        T y[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) y[v] = (T)lds<SZ>(p + ((v + r) & 3u) * R.vstride);
        // y[v] is element (v + r) & 3: rotate back by r
        T z[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) z[e] = (r & 1u) ? y[(e + 3) & 3] : y[e];
#pragma unroll
        for (int e = 0; e < 4; ++e) x[e] = (r & 2u) ? z[(e + 2) & 3] : z[e];
        return;
    }
#pragma unroll
    for (int v = 0; v < V; ++v) x[v] = (T)lds<SZ>(p + v * R.vstride);
}

template <int V, int SZ, typename T>
__device__ __forceinline__ void st_run(uint32_t p, const LaneRun& R, const T (&x)[V])
{
    constexpr int BYTES = V * SZ;
    if constexpr (BYTES >= 4) {
        if (R.vec) {
            uint32_t w[BYTES / 4];
            elems_to_words<V, SZ, T>(x, w);
            if constexpr (BYTES % 16 == 0) {
#pragma unroll
                for (int q = 0; q < BYTES / 16; ++q) sts_v4(p + 16u * q, w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
            } else if constexpr (BYTES == 8) {
                sts_v2(p, w[0], w[1]);
            } else {
                sts<4>(p, w[0]);
            }
            return;
        }
    }
    if constexpr (V == 4) {
        // strided elements, each 8-lane quarter starting at another element
        // as in ld_run
        const uint32_t r = (threadIdx.x >> 3) & 3u;
        T z[4], y[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) z[e] = (r & 1u) ? x[(e + 1) & 3] : x[e];
#pragma unroll
        for (int e = 0; e < 4; ++e) y[e] = (r & 2u) ? z[(e + 2) & 3] : z[e];
        // y[v] is element (v + r) & 3
#pragma unroll
        for (int v = 0; v < 4; ++v) sts<SZ>(p + ((v + r) & 3u) * R.vstride, (uint64_t)y[v]);
        return;
    }
#pragma unroll
    for (int v = 0; v < V; ++v) sts<SZ>(p + v * R.vstride, (uint64_t)x[v]);
}

// x << s and x >> s with PTX semantics: shift amounts of 32 or more (also
// "negative" ones, as unsigned) give 0.
__device__ __forceinline__ uint32_t shl_c(uint32_t x, uint32_t s)
{
    uint32_t r;
    asm("shl.b32 %0, %1, %2;" : "=r"(r) : "r"(x), "r"(s));
    return r;
}

// floor(a / b) for a < 2^15 and 0 < b <= 2^7: a float quotient is within one
// of the exact one, and one integer check each way makes it exact.
__device__ __forceinline__ uint32_t small_div(uint32_t a, uint32_t b)
{
    uint32_t q = (uint32_t)__fmul_rz((float)a, __frcp_rn((float)b));
    if (q * b > a) --q;
    if ((q + 1u) * b <= a) ++q;
    return q;
}

// Lane constants of a stream of C-bit chunks (C = V w bits per lane; a
// super-group is C words).  Reading: the lane's chunk starts `sh` bits into
// word `word` of the super-group.  Writing, round m (words k = lane + 32 m
// < C): the chunk of lane l0 reaches word k from chunk bit rsh on; the next
// chunks (nterm - 1 of them; at most one when C >= 32) start inside word k
// at bit j C - rsh (t1 for j = 1; 32 when there is none).
struct ChunkLane {
    uint32_t word, sh;
    uint32_t l0[2], rsh[2], t1[2], nterm[2], jmax[2];
};

__device__ __forceinline__ ChunkLane chunk_lane(uint32_t C, uint32_t lane, bool writing)
{
    ChunkLane K;
    const uint32_t bit = lane * C;
    K.word = bit >> 5;
    K.sh = bit & 31u;
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        K.l0[m] = 0u;
        K.rsh[m] = 0u;
        K.t1[m] = 32u;
        K.nterm[m] = 0u;
        K.jmax[m] = 0u;
        if (!writing) continue;
        const uint32_t k = lane + 32u * m;
        if (k < C) {
            const uint32_t b0 = 32u * k;
            K.l0[m] = small_div(b0, C);
            K.rsh[m] = b0 - K.l0[m] * C;
            K.nterm[m] = min(31u, small_div(b0 + 31u, C)) - K.l0[m] + 1u;
            if (K.nterm[m] >= 2u) K.t1[m] = C - K.rsh[m];
        }
        K.jmax[m] = __reduce_max_sync(0xFFFFFFFFu, K.nterm[m]);
    }
    return K;
}

// Word k = lane + 32 m of a super-group whose lanes hold chunks (lo, hi).
// MANY: chunks narrower than 32 bits, so more than two reach a word.
template <bool MANY>
__device__ __forceinline__ uint32_t chunk_word(uint32_t lo, uint32_t hi, uint32_t C, const ChunkLane& K, int m)
{
    const uint32_t l0 = K.l0[m];
    const uint32_t lo0 = __shfl_sync(0xFFFFFFFFu, lo, l0);
    const uint32_t hi0 = __shfl_sync(0xFFFFFFFFu, hi, l0);
    uint32_t word = (uint32_t)((((uint64_t)hi0 << 32) | lo0) >> K.rsh[m]);
    if constexpr (!MANY) {
        const uint32_t lo1 = __shfl_sync(0xFFFFFFFFu, lo, (l0 + 1u) & 31u);
        return word | shl_c(lo1, K.t1[m]);
    } else {
        for (uint32_t j = 1; j < K.jmax[m]; ++j) {
            const uint32_t v = __shfl_sync(0xFFFFFFFFu, lo, (l0 + j) & 31u);
            word |= j < K.nterm[m] ? shl_c(v, j * C - K.rsh[m]) : 0u;
        }
        return word;
    }
}

// The item fields a conversion needs, held in registers for a whole loop.
struct ConvRegs {
    uint32_t wa, wb;
    bool is_signed;
    int se, sm, de, dm;  // stored -> logical (on load) or logical -> stored
    uint64_t absmask, inf, quiet;  // FC_SAME: |x| above the INF code is a NaN
    FmtConv fc;                    // FC_RT
};

template <int CV, bool ON_LOAD, typename T>
__device__ __forceinline__ T fast_convert(T x, const ConvRegs& c)
{
    if (CV == FC_INT) {
        if (ON_LOAD) {
            if (c.is_signed) {
                const uint32_t up = 32u - c.wa;  // 0 for 32-bit codes
                return (T)(uint32_t)(((int32_t)((uint32_t)x << up)) >> up);
            }
            return (T)(uint32_t)x;
        }
        return x;  // the pack masks codes to their width
    }
    if (CV == FC_NONE) return x;
    if (CV == FC_D2F) return (T)f64_to_f32_bits((uint64_t)x);
    if (CV == FC_F2D) return (T)f32_to_f64_bits((uint32_t)x);
    if (CV == FC_SAME) return (x & (T)c.absmask) > (T)c.inf ? (x | (T)c.quiet) : x;
    return (T)fmt_convert((uint64_t)x, c.fc);
}

// LK / SK: how the source / destination element is reached; SZL / SZS:
// element bytes of affine leaves and whole-byte streams; CV: the conversion,
// applied on the load side (stream -> leaf) when CONV_ON_LOAD; V: records
// per lane; MANY: stream chunks narrower than 32 bits.  Super-groups
// [g0, g1) of the tile; records at or past nvalid read as zero (and so are
// written as zero).  Super-groups whose records are all valid run without
// any checks.
// RUNS: a stream side is AoSoA-organised (super-group offsets by sg_off); a
// separate instantiation, so that SoA streams keep one multiply per address.
template <int LK, int SK, int SZL, int SZS, int CV, bool CONV_ON_LOAD, int V, bool MANY, bool RUNS = false>
__device__ __noinline__ void fast_loop(const ItemDesc& I, const JobDesc& J, const uint8_t* simg, uint8_t* dimg,
                                       uint32_t g0, uint32_t g1, uint32_t nvalid)
{
    // element / code type: 32-bit where every value and code fits
    using T = typename std::conditional<(SZL <= 4 && SZS <= 4 && V > 1), uint32_t, uint64_t>::type;
    constexpr uint32_t B = 4u / V;  // super-groups in flight: 4 records per lane
    const uint32_t lane = threadIdx.x & 31u;
    const LeafDesc LA = J.src.leaves[I.src_leaf];
    const LeafDesc LB = J.dst.leaves[I.dst_leaf];
    ConvRegs cr;
    cr.wa = LA.bits;
    cr.wb = I.d_bits;
    cr.is_signed = I.is_signed != 0;
    cr.se = CONV_ON_LOAD ? I.s_e : I.l_e;
    cr.sm = CONV_ON_LOAD ? I.s_m : I.l_m;
    cr.de = CONV_ON_LOAD ? I.l_e : I.d_e;
    cr.dm = CONV_ON_LOAD ? I.l_m : I.d_m;
    if constexpr (CV == FC_SAME) {
        cr.absmask = low_bits64(cr.se + cr.sm);
        cr.inf = low_bits64(cr.se) << cr.sm;
        cr.quiet = 1ull << (cr.sm > 0 ? cr.sm - 1 : 0);
    } else {
        cr.absmask = cr.inf = cr.quiet = 0;
    }
    if constexpr (CV == FC_RT) cr.fc = fmt_conv(cr.se, cr.sm, cr.de, cr.dm);
    const uint32_t wa = cr.wa, wb = cr.wb;
    const uint32_t sa = smem_addr(simg), da = smem_addr(dimg);

    LaneRun RA{}, RB{};
    ChunkLane KA{}, KB{};
    SgSteps GA{}, GB{};
    uint32_t ca = 0u, cb = 0u, abase = 0u, bbase = 0u;
    if (LK == FL_AFF) {
        RA = affine_run<V, SZL>(LA, lane);
    } else if (LK == FL_AL) {
        RA = stream_run<V, SZL>(LA, lane);
        GA = sg_steps(LA, RA.step, V);
    } else {
        ca = (uint32_t)V * wa;
        KA = chunk_lane(ca, lane, false);
        abase = sa + LA.sbase + 4u * KA.word;
        GA = sg_steps(LA, 4u * ca, V);
    }
    if (SK == FS_AFF) {
        RB = affine_run<V, SZS>(LB, lane);
    } else if (SK == FS_AL) {
        RB = stream_run<V, SZS>(LB, lane);
        GB = sg_steps(LB, RB.step, V);
    } else {
        cb = (uint32_t)V * wb;
        KB = chunk_lane(cb, lane, true);
        bbase = da + LB.sbase + 4u * lane;
        GB = sg_steps(LB, 4u * cb, V);
    }
    const T amask = (T)low_bits64((int)wa), bmask = (T)low_bits64((int)wb);

    auto body = [&](uint32_t g, auto check_tag) {
        constexpr bool CHECK = decltype(check_tag)::value;
        T x[B][V];
#pragma unroll
        for (uint32_t b = 0; b < B; ++b) {
            const uint32_t gg = g + b;
            const uint32_t rec0 = 32u * V * gg + (uint32_t)V * lane;
            if (CHECK) {
#pragma unroll
                for (int v = 0; v < V; ++v) x[b][v] = 0u;
                if (gg >= g1 || rec0 >= nvalid) continue;
            }
            if (LK == FL_BITS) {
                const uint32_t p = abase + (RUNS ? sg_off(GA, gg) : gg * GA.step);
                const uint32_t w0 = (uint32_t)lds<4>(p), w1 = (uint32_t)lds<4>(p + 4u), w2 = (uint32_t)lds<4>(p + 8u);
                const uint64_t chunk = ((uint64_t)__funnelshift_r(w1, w2, KA.sh) << 32) | __funnelshift_r(w0, w1, KA.sh);
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const T c = (T)(chunk >> (v * wa)) & amask;
                    x[b][v] = (!CHECK || rec0 + v < nvalid) ? c : (T)0u;
                }
            } else {
                const uint32_t p = sa + RA.off + (RUNS && LK == FL_AL ? sg_off(GA, gg) : gg * RA.step);
                if (!CHECK || rec0 + V <= nvalid) {
                    ld_run<V, SZL, T>(p, RA, x[b]);
                } else {
#pragma unroll
                    for (int v = 0; v < V; ++v) x[b][v] = rec0 + v < nvalid ? (T)lds<SZL>(p + v * RA.vstride) : (T)0u;
                }
            }
        }
#pragma unroll
        for (uint32_t b = 0; b < B; ++b)
#pragma unroll
            for (int v = 0; v < V; ++v) x[b][v] = fast_convert<CV, CONV_ON_LOAD>(x[b][v], cr);
#pragma unroll
        for (uint32_t b = 0; b < B; ++b) {
            const uint32_t gg = g + b;
            if (CHECK && gg >= g1) break;
            if (SK == FS_BITS) {
                uint64_t chunk = 0;
#pragma unroll
                for (int v = 0; v < V; ++v) chunk |= (uint64_t)(x[b][v] & bmask) << (v * wb);
                const uint32_t lo = (uint32_t)chunk, hi = (uint32_t)(chunk >> 32);
                const uint32_t q = bbase + (RUNS ? sg_off(GB, gg) : gg * GB.step);
                const uint32_t w0 = chunk_word<MANY>(lo, hi, cb, KB, 0);
                if (lane < cb) sts<4>(q, w0);
                if (cb > 32u) {
                    const uint32_t w1 = chunk_word<MANY>(lo, hi, cb, KB, 1);
                    if (lane + 32u < cb) sts<4>(q + 128u, w1);
                }
            } else {
                st_run<V, SZS, T>(da + RB.off + (RUNS && SK == FS_AL ? sg_off(GB, gg) : gg * RB.step), RB, x[b]);
            }
        }
    };
    const uint32_t gfull = min(g1, max(g0, nvalid / (32u * V)));  // super-groups below hold valid records only
    uint32_t g = g0;
    for (; g + B <= gfull; g += B) body(g, std::false_type{});
    for (; g < g1; g += B) body(g, std::true_type{});
}

// ------------------------------------------------------- byte planes --
//
// Bytesplit (Sec. 3 of the paper) stores byte j of every value of a leaf in
// plane j.  Lane l takes 4 consecutive records of a super-group of 128: the
// 4 SZ-byte values are a 4 x SZ byte matrix, and plane j's word for those
// records is its column j.  SZ = 4 is one 4 x 4 byte transpose (8 PRMT),
// SZ = 8 two, SZ = 2 two PRMT per direction; the transpose is its own
// inverse, so splitting and joining share it.

__device__ __forceinline__ void transpose4x4(uint32_t& a, uint32_t& b, uint32_t& c, uint32_t& d)
{
    const uint32_t t0 = __byte_perm(a, b, 0x5140), t1 = __byte_perm(a, b, 0x7362);
    const uint32_t t2 = __byte_perm(c, d, 0x5140), t3 = __byte_perm(c, d, 0x7362);
    a = __byte_perm(t0, t2, 0x5410);
    b = __byte_perm(t0, t2, 0x7632);
    c = __byte_perm(t1, t3, 0x5410);
    d = __byte_perm(t1, t3, 0x7632);
}

// The 4 records' values as SZ words (row-major: word q holds bytes
// 4q .. 4q+3 of the 4 x SZ matrix read value by value) <-> plane words.
template <int SZ>
__device__ __forceinline__ void rows_to_planes(uint32_t (&w)[SZ])
{
    if constexpr (SZ == 2) {
        const uint32_t p0 = __byte_perm(w[0], w[1], 0x6420), p1 = __byte_perm(w[0], w[1], 0x7531);
        w[0] = p0;
        w[1] = p1;
    } else if constexpr (SZ == 4) {
        transpose4x4(w[0], w[1], w[2], w[3]);
    } else {
        // values are (lo, hi) word pairs: lo words give planes 0..3, hi words 4..7
        uint32_t a = w[0], b = w[2], c = w[4], d = w[6];
        uint32_t e = w[1], f = w[3], g = w[5], h = w[7];
        transpose4x4(a, b, c, d);
        transpose4x4(e, f, g, h);
        w[0] = a; w[1] = b; w[2] = c; w[3] = d;
        w[4] = e; w[5] = f; w[6] = g; w[7] = h;
    }
}

template <int SZ>
__device__ __forceinline__ void planes_to_rows(uint32_t (&w)[SZ])
{
    if constexpr (SZ == 2) {
        const uint32_t r0 = __byte_perm(w[0], w[1], 0x5140), r1 = __byte_perm(w[0], w[1], 0x7362);
        w[0] = r0;
        w[1] = r1;
    } else if constexpr (SZ == 4) {
        transpose4x4(w[0], w[1], w[2], w[3]);
    } else {
        uint32_t a = w[0], b = w[1], c = w[2], d = w[3];
        uint32_t e = w[4], f = w[5], g = w[6], h = w[7];
        transpose4x4(a, b, c, d);
        transpose4x4(e, f, g, h);
        w[0] = a; w[2] = b; w[4] = c; w[6] = d;
        w[1] = e; w[3] = f; w[5] = g; w[7] = h;
    }
}

// The quads [g0, g1) of a split or join whose planes are vector runs at one
// common step (SoA-like planes) and whose records are all valid: one plane
// address step per quad and no per-plane or per-record checks.  Returns the
// first quad it left to split_loop (g0 when the planes do not qualify).  A
// function of its own, so that the general loop's per-plane state does not
// add to the registers the kernel keeps across the call.
template <int SZ, bool JOIN>
__device__ __noinline__ uint32_t split_uni(const ItemDesc& I, const JobDesc& J, const uint8_t* simg, uint8_t* dimg,
                                           uint32_t g0, uint32_t g1, uint32_t nvalid)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t sa = smem_addr(simg), da = smem_addr(dimg);
    const LaneRun RW = affine_run<4, SZ>(JOIN ? J.dst.leaves[I.dst_leaf] : J.src.leaves[I.src_leaf], lane);
    bool uni = RW.vec;
    uint32_t pbase[SZ], pstep = 0;
#pragma unroll
    for (int j = 0; j < SZ; ++j) {
        const LaneRun RP = affine_run<4, 1>(JOIN ? J.src.leaves[I.src_leaf + j] : J.dst.leaves[I.dst_leaf + j], lane);
        if (j == 0) pstep = RP.step;
        uni = uni && RP.vec && RP.step == pstep;
        pbase[j] = (JOIN ? sa : da) + RP.off;
    }
    if (!uni) return g0;
    const uint32_t gfull = min(g1, max(g0, nvalid / 128u));
    uint32_t wa = (JOIN ? da : sa) + RW.off + g0 * RW.step, pa = g0 * pstep;
    for (uint32_t g = g0; g < gfull; ++g, wa += RW.step, pa += pstep) {
        uint32_t w[SZ];
        if (!JOIN) {
            uint64_t x[4];
            ld_run<4, SZ, uint64_t>(wa, RW, x);
            elems_to_words<4, SZ, uint64_t>(x, w);
            rows_to_planes<SZ>(w);
#pragma unroll
            for (int j = 0; j < SZ; ++j) sts<4>(pbase[j] + pa, w[j]);
        } else {
#pragma unroll
            for (int j = 0; j < SZ; ++j) w[j] = (uint32_t)lds<4>(pbase[j] + pa);
            planes_to_rows<SZ>(w);
            uint64_t x[4];
            words_to_elems<4, SZ, uint64_t>(w, x);
            st_run<4, SZ, uint64_t>(wa, RW, x);
        }
    }
    return gfull;
}

// JOIN false: leaf -> planes (store side split); true: planes -> leaf.
template <int SZ, bool JOIN>
__device__ __noinline__ void split_loop(const ItemDesc& I, const JobDesc& J, const uint8_t* simg, uint8_t* dimg,
                                        uint32_t g0, uint32_t g1, uint32_t nvalid)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t sa = smem_addr(simg), da = smem_addr(dimg);
    const LeafDesc& LW = JOIN ? J.dst.leaves[I.dst_leaf] : J.src.leaves[I.src_leaf];
    const LaneRun RW = affine_run<4, SZ>(LW, lane);
    const uint32_t wbase = (JOIN ? da : sa) + RW.off;
    LaneRun RP[SZ];
    uint32_t pbase[SZ];
#pragma unroll
    for (int j = 0; j < SZ; ++j) {
        RP[j] = affine_run<4, 1>(JOIN ? J.src.leaves[I.src_leaf + j] : J.dst.leaves[I.dst_leaf + j], lane);
        pbase[j] = (JOIN ? sa : da) + RP[j].off;
    }
    for (uint32_t g = g0; g < g1; ++g) {
        const uint32_t rec0 = 128u * g + 4u * lane;
        const uint32_t nv = rec0 >= nvalid ? 0u : min(4u, nvalid - rec0);  // valid records of the lane
        uint32_t w[SZ];
        if (!JOIN) {
            uint64_t x[4];
            if (nv == 4u) {
                ld_run<4, SZ, uint64_t>(wbase + g * RW.step, RW, x);
            } else {
#pragma unroll
                for (int v = 0; v < 4; ++v) x[v] = (uint32_t)v < nv ? lds<SZ>(wbase + g * RW.step + v * RW.vstride) : 0u;
            }
            elems_to_words<4, SZ, uint64_t>(x, w);
            rows_to_planes<SZ>(w);
#pragma unroll
            for (int j = 0; j < SZ; ++j) {
                const uint32_t a = pbase[j] + g * RP[j].step;
                if (RP[j].vec) {
                    sts<4>(a, w[j]);
                } else {
#pragma unroll
                    for (int v = 0; v < 4; ++v) sts<1>(a + v * RP[j].vstride, (w[j] >> (8 * v)) & 0xFFu);
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < SZ; ++j) {
                const uint32_t a = pbase[j] + g * RP[j].step;
                if (RP[j].vec) {
                    w[j] = (uint32_t)lds<4>(a);
                } else {
                    w[j] = 0u;
#pragma unroll
                    for (int v = 0; v < 4; ++v) w[j] |= (uint32_t)lds<1>(a + v * RP[j].vstride) << (8 * v);
                }
                // bytes of records at or past nvalid read as zero
                w[j] &= nv >= 4u ? 0xFFFFFFFFu : ((1u << (8u * nv)) - 1u);
            }
            planes_to_rows<SZ>(w);
            uint64_t x[4];
            words_to_elems<4, SZ, uint64_t>(w, x);
            st_run<4, SZ, uint64_t>(wbase + g * RW.step, RW, x);
        }
    }
}

// Runs a VALUE item over quads [q0, q1) (128 records each) in its
// specialised loop; false when it has none.
__device__ __forceinline__ bool run_fast(const ItemDesc& I, const JobDesc& J, const uint8_t* simg, uint8_t* dimg,
                                         uint32_t q0, uint32_t q1, uint32_t nvalid)
{
#define LLGB_FAST_V(LK, SK, SZL, SZS, CV, OL, V, MANY)                                                 \
    do {                                                                                                \
        if (I.runs)                                                                                     \
            fast_loop<LK, SK, SZL, SZS, CV, OL, V, MANY, true>(I, J, simg, dimg, q0 * (4u / V), q1 * (4u / V), \
                                                               nvalid);                                 \
        else                                                                                            \
            fast_loop<LK, SK, SZL, SZS, CV, OL, V, MANY>(I, J, simg, dimg, q0 * (4u / V), q1 * (4u / V), nvalid); \
    } while (0)
// streams: V from the width; chunks under 32 bits (widths below 8) take MANY
#define LLGB_FAST(K, LK, SK, SZL, SZS, CV, OL)                                             \
    case K:                                                                                \
        if (I.vpl == 4) {                                                                  \
            if (width < 8u) LLGB_FAST_V(LK, SK, SZL, SZS, CV, OL, 4, true);                \
            else LLGB_FAST_V(LK, SK, SZL, SZS, CV, OL, 4, false);                          \
        } else if (I.vpl == 2) LLGB_FAST_V(LK, SK, SZL, SZS, CV, OL, 2, false);            \
        else LLGB_FAST_V(LK, SK, SZL, SZS, CV, OL, 1, false);                              \
        return true;
#define LLGB_FAST1(K, LK, SK, SZL, SZS, CV, OL, V) \
    case K: LLGB_FAST_V(LK, SK, SZL, SZS, CV, OL, V, false); return true;
// stream and leaf of one float format: no rounding, only NaN quieting
#define LLGB_FAST_SAME(K, LK, SK, SZL, SZS, OL, V)                    \
    case K:                                                          \
        if (OL ? (I.s_e == I.l_e && I.s_m == I.l_m) : (I.l_e == I.d_e && I.l_m == I.d_m)) \
            LLGB_FAST_V(LK, SK, SZL, SZS, FC_SAME, OL, V, false);        \
        else LLGB_FAST_V(LK, SK, SZL, SZS, FC_RT, OL, V, false);        \
        return true;
    const uint32_t width = I.sop == S_BITS_INT || I.sop == S_BITS_FLOAT ? I.d_bits : I.s_bits;
    switch (I.fast) {
        LLGB_FAST(FK_PACK_INT32, FL_AFF, FS_BITS, 4, 4, FC_INT, false)
        LLGB_FAST(FK_UNPACK_INT32, FL_BITS, FS_AFF, 4, 4, FC_INT, true)
        LLGB_FAST(FK_PACK_BITS_FROM8, FL_AFF, FS_BITS, 8, 8, FC_RT, false)
        LLGB_FAST(FK_PACK_BITS_FROM4, FL_AFF, FS_BITS, 4, 4, FC_RT, false)
        LLGB_FAST(FK_UNPACK_BITS_TO8, FL_BITS, FS_AFF, 8, 8, FC_RT, true)
        LLGB_FAST(FK_UNPACK_BITS_TO4, FL_BITS, FS_AFF, 4, 4, FC_RT, true)
        LLGB_FAST1(FK_PACK_D_F32, FL_AFF, FS_AL, 8, 4, FC_D2F, false, 2)
        LLGB_FAST1(FK_PACK_AL32_FROM8, FL_AFF, FS_AL, 8, 4, FC_RT, false, 2)
        LLGB_FAST_SAME(FK_PACK_AL32_FROM4, FL_AFF, FS_AL, 4, 4, false, 4)
        LLGB_FAST_SAME(FK_PACK_AL64_FROM8, FL_AFF, FS_AL, 8, 8, false, 2)
        LLGB_FAST1(FK_PACK_AL64_FROM4, FL_AFF, FS_AL, 4, 8, FC_RT, false, 4)
        LLGB_FAST1(FK_PACK_AL16_FROM8, FL_AFF, FS_AL, 8, 2, FC_RT, false, 2)
        LLGB_FAST1(FK_PACK_AL16_FROM4, FL_AFF, FS_AL, 4, 2, FC_RT, false, 4)
        LLGB_FAST1(FK_PACK_AL8_FROM8, FL_AFF, FS_AL, 8, 1, FC_RT, false, 2)
        LLGB_FAST1(FK_PACK_AL8_FROM4, FL_AFF, FS_AL, 4, 1, FC_RT, false, 4)
        LLGB_FAST1(FK_UNPACK_F32_D, FL_AL, FS_AFF, 4, 8, FC_F2D, true, 2)
        LLGB_FAST1(FK_UNPACK_AL32_TO8, FL_AL, FS_AFF, 4, 8, FC_RT, true, 2)
        LLGB_FAST_SAME(FK_UNPACK_AL32_TO4, FL_AL, FS_AFF, 4, 4, true, 4)
        LLGB_FAST_SAME(FK_UNPACK_AL64_TO8, FL_AL, FS_AFF, 8, 8, true, 2)
        LLGB_FAST1(FK_UNPACK_AL64_TO4, FL_AL, FS_AFF, 8, 4, FC_RT, true, 4)
        LLGB_FAST1(FK_UNPACK_AL16_TO8, FL_AL, FS_AFF, 2, 8, FC_RT, true, 2)
        LLGB_FAST1(FK_UNPACK_AL16_TO4, FL_AL, FS_AFF, 2, 4, FC_RT, true, 4)
        LLGB_FAST1(FK_UNPACK_AL8_TO8, FL_AL, FS_AFF, 1, 8, FC_RT, true, 2)
        LLGB_FAST1(FK_UNPACK_AL8_TO4, FL_AL, FS_AFF, 1, 4, FC_RT, true, 4)
        LLGB_FAST1(FK_CT_D_F32, FL_AFF, FS_AFF, 8, 4, FC_D2F, false, 2)
        LLGB_FAST1(FK_CT_F32_D, FL_AFF, FS_AFF, 4, 8, FC_F2D, true, 2)
        LLGB_FAST1(FK_MOVE1, FL_AFF, FS_AFF, 1, 1, FC_NONE, false, 4)
        LLGB_FAST1(FK_MOVE2, FL_AFF, FS_AFF, 2, 2, FC_NONE, false, 4)
        LLGB_FAST1(FK_MOVE4, FL_AFF, FS_AFF, 4, 4, FC_NONE, false, 4)
        LLGB_FAST1(FK_MOVE8, FL_AFF, FS_AFF, 8, 8, FC_NONE, false, 2)
    case FK_SPLIT2: split_loop<2, false>(I, J, simg, dimg, split_uni<2, false>(I, J, simg, dimg, q0, q1, nvalid), q1, nvalid); return true;
    case FK_SPLIT4: split_loop<4, false>(I, J, simg, dimg, split_uni<4, false>(I, J, simg, dimg, q0, q1, nvalid), q1, nvalid); return true;
    case FK_SPLIT8: split_loop<8, false>(I, J, simg, dimg, split_uni<8, false>(I, J, simg, dimg, q0, q1, nvalid), q1, nvalid); return true;
    case FK_JOIN2: split_loop<2, true>(I, J, simg, dimg, split_uni<2, true>(I, J, simg, dimg, q0, q1, nvalid), q1, nvalid); return true;
    case FK_JOIN4: split_loop<4, true>(I, J, simg, dimg, split_uni<4, true>(I, J, simg, dimg, q0, q1, nvalid), q1, nvalid); return true;
    case FK_JOIN8: split_loop<8, true>(I, J, simg, dimg, split_uni<8, true>(I, J, simg, dimg, q0, q1, nvalid), q1, nvalid); return true;
    default: return false;
    }
#undef LLGB_FAST_SAME
#undef LLGB_FAST1
#undef LLGB_FAST
#undef LLGB_FAST_V
}

}  // namespace llgb

#include "stream_loops.cuh"

namespace llgb {

// Zero the bit streams that generic items OR their codes into.
static __device__ __noinline__ void zero_streams(const JobDesc& J, uint8_t* dimg)
{
    for (int k = 0; k < J.npacks; ++k) {
        const PackDesc& P = J.packs[k];
        if (!P.ored) continue;
        if (P.runs == 1) {
            uint4* z = reinterpret_cast<uint4*>(dimg + P.dst_sbase);
            for (uint32_t q = ctid(); q < (P.bytes + 15u) / 16u; q += cnum()) z[q] = make_uint4(0, 0, 0, 0);
            continue;
        }
        const uint32_t wpr = P.bytes / 4u;  // words per run
        const uint32_t stride = J.dst.leaves[P.leaf].bstride;
        for (uint32_t w = ctid(); w < P.runs * wpr; w += cnum()) {
            const uint32_t run = w / wpr;
            *reinterpret_cast<uint32_t*>(dimg + P.dst_sbase + run * stride + 4u * (w - run * wpr)) = 0u;
        }
    }
}

// Quads [q0, q1) (128 records each) of one item.
template <int MODE>
__device__ __forceinline__ void run_item_quads(const JobDesc& J, const ItemDesc& I, const uint8_t* simg,
                                               uint8_t* dimg, uint32_t q0, uint32_t q1, uint32_t nvalid)
{
    constexpr bool SEGOK = MODE == 1;  // the generic loop of AoSoA-organised bit leaves
    const Span sp{128u * q0 + (threadIdx.x & 31u), 128u * q1, 32u};
    // the loops of the compile-time stream formats: SoA streams in kernel
    // mode 0, any organisation in mode 3 (mode 1 runs them in its other loops)
    if constexpr (MODE != 1) {
        if (I.spec && run_spec<MODE == 3>(I, J, simg, dimg, q0, q1, nvalid)) return;
    }
    if (I.op == ITEM_MOVE && I.fast != FK_GENERIC && run_fast(I, J, simg, dimg, q0, q1, nvalid)) return;
    if (I.op == ITEM_MOVE) {
        const LeafRegs A = leaf_regs(J.src.leaves[I.src_leaf]);
        const LeafRegs B = leaf_regs(J.dst.leaves[I.dst_leaf]);
        switch (I.gran) {
        case 8: move_loop<8>(A, B, I.src_byte, I.dst_byte, I.size, simg, dimg, sp, nvalid); break;
        case 4: move_loop<4>(A, B, I.src_byte, I.dst_byte, I.size, simg, dimg, sp, nvalid); break;
        case 2: move_loop<2>(A, B, I.src_byte, I.dst_byte, I.size, simg, dimg, sp, nvalid); break;
        default: move_loop<1>(A, B, I.src_byte, I.dst_byte, I.size, simg, dimg, sp, nvalid); break;
        }
    } else if (!run_fast(I, J, simg, dimg, q0, q1, nvalid)) {
        switch (I.lop) {
        case L_DIRECT: value_dispatch<L_DIRECT, SEGOK>(I, J, simg, dimg, sp, nvalid); break;
        case L_CT: value_dispatch<L_CT, SEGOK>(I, J, simg, dimg, sp, nvalid); break;
        case L_BITS_INT: value_dispatch<L_BITS_INT, SEGOK>(I, J, simg, dimg, sp, nvalid); break;
        case L_BITS_FLOAT: value_dispatch<L_BITS_FLOAT, SEGOK>(I, J, simg, dimg, sp, nvalid); break;
        case L_NULL: value_dispatch<L_NULL, SEGOK>(I, J, simg, dimg, sp, nvalid); break;
        default: value_dispatch<L_SPLIT, SEGOK>(I, J, simg, dimg, sp, nvalid); break;
        }
    }
}

// The tile's work is nitems x (tile / 128) quads, laid out item by item; a
// quad of item i costs ItemDesc::weight units (an item of 8-byte elements
// about twice one of 4-byte elements).  The weighted quads are cut into
// cnum/32 equal contiguous shares; consumer warp w takes share w of every tile
// of a job: quads [quad, Q) of `item`, the whole items after it, and quads
// [0, end_quad) of end_item.
struct ItemShare {
    uint32_t item, quad, end_item, end_quad;
};

// The (item, quad) at which weighted position p falls: the first quad whose
// weighted start is at or past p.
__device__ __forceinline__ void weighted_quad(const JobDesc& J, uint32_t Q, uint32_t p, uint32_t& item, uint32_t& quad)
{
    uint32_t acc = 0;
    for (uint32_t i = 0; i < J.nitems; ++i) {
        const uint32_t w = J.items[i].weight;
        const uint32_t span = w * Q;
        if (p < acc + span) {
            const uint32_t q = (p - acc + w - 1u) / w;
            item = q < Q ? i : i + 1u;
            quad = q < Q ? q : 0u;
            return;
        }
        acc += span;
    }
    item = J.nitems;
    quad = 0u;
}

__device__ __forceinline__ ItemShare item_share(const JobDesc& J)
{
    const uint32_t w = ctid() >> 5, nw = cnum() >> 5;
    const uint32_t Q = J.tile >> 7;
    uint32_t total = 0;  // <= 64 items x 8 x 2^10 quads
    for (uint32_t i = 0; i < J.nitems; ++i) total += J.items[i].weight * Q;
    ItemShare S;
    weighted_quad(J, Q, total * w / nw, S.item, S.quad);
    weighted_quad(J, Q, total * (w + 1u) / nw, S.end_item, S.end_quad);
    return S;
}

template <int MODE>
__device__ void run_items(const JobDesc& J, const uint8_t* simg, uint8_t* dimg, uint32_t nvalid, ItemShare S)
{
    const uint32_t Q = J.tile >> 7;
    uint32_t it = S.item, q0 = S.quad;
    while (it < S.end_item || (it == S.end_item && q0 < S.end_quad)) {
        const uint32_t q1 = it == S.end_item ? S.end_quad : Q;
        if (q1 > q0) run_item_quads<MODE>(J, J.items[it], simg, dimg, q0, q1, nvalid);
        ++it;
        q0 = 0;
    }
}

// Byte moves only (the items of a gather job, for its last tile).
__device__ __forceinline__ void run_moves(const JobDesc& J, const uint8_t* simg, uint8_t* dimg, uint32_t nvalid)
{
    for (int it = 0; it < J.nitems; ++it) {
        const ItemDesc I = J.items[it];
        const LeafRegs A = leaf_regs(J.src.leaves[I.src_leaf]);
        const LeafRegs B = leaf_regs(J.dst.leaves[I.dst_leaf]);
        const Span sp{ctid(), J.tile, cnum()};
        switch (I.gran) {
        case 8: move_loop<8>(A, B, I.src_byte, I.dst_byte, I.size, simg, dimg, sp, nvalid); break;
        case 4: move_loop<4>(A, B, I.src_byte, I.dst_byte, I.size, simg, dimg, sp, nvalid); break;
        case 2: move_loop<2>(A, B, I.src_byte, I.dst_byte, I.size, simg, dimg, sp, nvalid); break;
        default: move_loop<1>(A, B, I.src_byte, I.dst_byte, I.size, simg, dimg, sp, nvalid); break;
        }
    }
}

// ------------------------------------------------------ gather programs --
//
// A job made only of byte moves permutes bytes: destination image byte o of
// every full tile comes from the same source image byte (or is zero).  Each
// thread derives, once per job, a program for each of its destination words
// w = ctid + k * cnum: up to four source words and the byte selectors
// that assemble the word with PRMT.  A full tile then costs a few loads, one
// or three PRMTs and one store per destination word.

// Destination words per thread: 16 for the 2-word form, 12 for the 4-word
// form (registers: 2 resp. 4 per word).
template <int FORM>
struct GatherMax {
    static constexpr int value = FORM == 2 ? 16 : (FORM == 4 ? 12 : 1);
};

// Source byte of destination image byte o, or -1 (padding, zero fill).
// *run receives how many of the following destination bytes (o + 1, ...)
// continue the same item's bytes of the same element, and so come from the
// following source bytes.
__device__ __forceinline__ int32_t gather_source(const JobDesc& J, uint32_t o, uint32_t* run)
{
    *run = 0;
    const SideDesc& D = J.dst;
    // d / bs, from the previous leaf's quotient when the strides agree: the
    // leaves of one AoS record or AoSoA block lie within one stride of each
    // other, so the quotient moves by at most one and needs no division
    uint32_t qs = 0, qb = 0;
    auto blocks = [&](uint32_t d, uint32_t bs) -> uint32_t {
        if (bs == qs) {
            const uint32_t t = qb * bs;
            if (d >= t && d - t < bs) return qb;
            if (d < t && t - d <= bs) return --qb;
            if (d >= t + bs && d - t - bs < bs) return ++qb;
        }
        qs = bs;
        qb = d / bs;
        return qb;
    };
    for (int g = 0; g < D.nleaves; ++g) {
        const LeafDesc& L = D.leaves[g];
        if (o < L.sbase) continue;
        const uint32_t d = o - L.sbase;
        uint32_t r, e;
        if (L.lanes == 1) {
            r = blocks(d, L.bstride);
            e = d - r * L.bstride;
            if (e >= L.size || r >= J.tile) continue;
        } else {
            const uint32_t blk = blocks(d, L.bstride);
            const uint32_t rem = d - blk * L.bstride;
            const uint32_t lane = (L.size & (L.size - 1u)) == 0u ? rem >> (__ffs(L.size) - 1) : rem / L.size;
            e = rem - lane * L.size;
            if (lane >= L.lanes) continue;
            r = blk * L.lanes + lane;
            if (r >= J.tile) continue;
        }
        for (int it = 0; it < J.nitems; ++it) {
            const ItemDesc& I = J.items[it];
            if (I.dst_leaf != g || e < I.dst_byte || e >= (uint32_t)I.dst_byte + I.size) continue;
            *run = (uint32_t)I.dst_byte + I.size - e - 1u;
            return (int32_t)(eoff(leaf_regs(J.src.leaves[I.src_leaf]), r) + I.src_byte + (e - I.dst_byte));
        }
        return -1;
    }
    return -1;
}

template <int FORM>
struct GatherProgram {
    static constexpr int K = GatherMax<FORM>::value;
    uint32_t idx01[K];                         // source word indices i0 | i1 << 16
    uint32_t sel01[K];                         // q0 | q1 << 16
    uint32_t idx23[FORM == 4 ? K : 1];         // i2 | i3 << 16
    uint32_t sel2[FORM == 4 ? K : 1];          // q2
    uint32_t dstw[FORM == 4 ? (K + 1) / 2 : 1]; // destination word of slot k (16 bits each; 0xFFFF: none)
};

// Destination word of consumer slot x: x itself, or -- interleaved -- word
// x / nsegs of run x % nsegs (all runs of equal size).  0xFFFFFFFF: none.
__device__ __forceinline__ uint32_t gather_slot_word(const JobDesc& J, uint32_t x, uint32_t nwords)
{
    if (!J.interleave) return x < nwords ? x : 0xFFFFFFFFu;
    const uint32_t nseg = J.dst.nsegs;
    const uint32_t seg = x % nseg, p = x / nseg;
    const uint32_t seg_words = ((J.dst.segs[seg].tile_bytes + 15u) & ~15u) / 4u;
    return p < seg_words ? J.dst.segs[seg].sbase / 4u + p : 0xFFFFFFFFu;
}

// The gather program entry of destination word w (0xFFFFFFFF: none): source
// word indices i0 | i1 << 16 (and i2 | i3 << 16 for the 4-word form) and
// the PRMT selectors that assemble the word from them.  Padding bytes read
// source word zero_word.
template <int FORM>
__device__ __forceinline__ void gather_slot(const JobDesc& J, uint32_t zero_word, uint32_t w, uint32_t& i01,
                                            uint32_t& s01, uint32_t& i23, uint32_t& q2)
{
    uint32_t word[4], byte[4];
    // one lookup per run of an item's contiguous bytes: a word of a 4-byte
    // field takes one, not four
    int32_t src = -1;
    uint32_t run = 0;
#pragma unroll 1
    for (int b = 0; b < 4; ++b) {
        if (src >= 0 && run > 0) {
            ++src;
            --run;
        } else {
            src = w != 0xFFFFFFFFu ? gather_source(J, 4u * w + b, &run) : -1;
        }
        word[b] = src < 0 ? zero_word : (uint32_t)src >> 2;
        byte[b] = src < 0 ? 0u : (uint32_t)src & 3u;
    }
    uint32_t u[4] = {word[0], word[0], word[0], word[0]};
    int nu = 1;
#pragma unroll
    for (int b = 1; b < 4; ++b) {
        bool seen = false;
        for (int x = 0; x < 4; ++x) seen |= (x < nu && u[x] == word[b]);
        if (!seen) {
            if (nu == 1) u[1] = word[b];
            else if (nu == 2) u[2] = word[b];
            else u[3] = word[b];
            ++nu;
        }
    }
    uint32_t q0 = 0, q1 = 0;
    q2 = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const uint32_t sh = 4u * b;
        if (word[b] == u[0]) {
            q0 |= byte[b] << sh;
            q2 |= (uint32_t)b << sh;
        } else if (word[b] == u[1]) {
            q0 |= (4u + byte[b]) << sh;
            q2 |= (uint32_t)b << sh;
        } else if (word[b] == u[2]) {
            q1 |= byte[b] << sh;
            q2 |= (4u + b) << sh;
        } else {
            q1 |= (4u + byte[b]) << sh;
            q2 |= (4u + b) << sh;
        }
    }
    if (FORM == 2 && nu > 2) atomicOr(&g_device_status, 0x100u);  // planner broke its promise
    i01 = u[0] | (u[1] << 16);
    s01 = q0 | (q1 << 16);
    i23 = u[2] | (u[3] << 16);
}

// Every consumer thread derives its own slots of the job's program (slot k
// of consumer c is destination word c + k * consumers, or, interleaved, the
// word that gather_slot_word deals it).
template <int FORM>
__device__ __forceinline__ void build_gather(const JobDesc& J, uint32_t zero_word, uint32_t nwords,
                                             GatherProgram<FORM>& G)
{
    // Rolled over k so that gather_slot is expanded once; each result is
    // steered into its register slot by an unrolled select.
#pragma unroll 1
    for (int k = 0; k < GatherProgram<FORM>::K; ++k) {
        const uint32_t w = FORM == 4 ? gather_slot_word(J, ctid() + k * cnum(), nwords)
                                     : (ctid() + k * cnum() < nwords ? ctid() + k * cnum() : 0xFFFFFFFFu);
        uint32_t i01, s01, i23, q2;
        gather_slot<FORM>(J, zero_word, w, i01, s01, i23, q2);
#pragma unroll
        for (int kk = 0; kk < GatherProgram<FORM>::K; ++kk) {
            if (kk == k) {
                G.idx01[kk] = i01;
                G.sel01[kk] = s01;
                if (FORM == 4) {
                    G.idx23[kk] = i23;
                    G.sel2[kk] = q2;
                    const uint32_t half = (w == 0xFFFFFFFFu ? 0xFFFFu : (w & 0xFFFFu)) << (16 * (kk & 1));
                    G.dstw[kk / 2] = (G.dstw[kk / 2] & ~(0xFFFFu << (16 * (kk & 1)))) | half;
                }
            }
        }
    }
}

// A job's gather program in global memory, built once by
// gather_program_kernel for CTAs of `cn` consumer threads: a header
// {kProgramMagic, cn, FORM, K}, then per slot k the words of GatherProgram
// (2 for the 2-word form: idx01, sel01; 5 for the 4-word form: idx01,
// sel01, idx23, sel2, destination word), word f of slot k of consumer c at
// (k F + f) cn + c, so that a CTA's consumers read them with coalesced
// loads.  Source indices name the padding word kZeroMarker, which a loading
// CTA replaces by its own zero word (a batch sizes stages for its largest
// job).
constexpr uint32_t kProgramMagic = 0x6C6C6770u;
constexpr uint32_t kProgramHeader = 4;
constexpr uint32_t kZeroMarker = 0xFFFFu;  // above every image word index (images < 256 KB)

template <int FORM>
__device__ __host__ constexpr uint32_t gather_program_fields() { return FORM == 2 ? 2u : 5u; }

template <int FORM>
__global__ void gather_program_kernel(const JobDesc job, uint32_t cn, uint32_t* __restrict__ out)
{
    constexpr uint32_t K = GatherMax<FORM>::value, F = gather_program_fields<FORM>();
    __shared__ JobDesc J;
    {
        const uint2* from = reinterpret_cast<const uint2*>(&job);
        uint2* to = reinterpret_cast<uint2*>(&J);
        for (uint32_t w = threadIdx.x; w < sizeof(JobDesc) / 8u; w += blockDim.x) to[w] = from[w];
    }
    __syncthreads();
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        out[0] = kProgramMagic;
        out[1] = cn;
        out[2] = (uint32_t)FORM;
        out[3] = K;
    }
    if (i >= K * cn) return;
    const uint32_t k = i / cn, c = i - k * cn, x = c + k * cn;
    const uint32_t nwords = (J.dst.img_bytes - kImageSlack) / 4u;
    const uint32_t w = FORM == 4 ? gather_slot_word(J, x, nwords) : (x < nwords ? x : 0xFFFFFFFFu);
    uint32_t i01, s01, i23, q2;
    gather_slot<FORM>(J, kZeroMarker, w, i01, s01, i23, q2);
    uint32_t* o = out + kProgramHeader;
    o[(k * F + 0u) * cn + c] = i01;
    o[(k * F + 1u) * cn + c] = s01;
    if constexpr (FORM == 4) {
        o[(k * F + 2u) * cn + c] = i23;
        o[(k * F + 3u) * cn + c] = q2;
        o[(k * F + 4u) * cn + c] = w == 0xFFFFFFFFu ? 0xFFFFu : (w & 0xFFFFu);
    }
}

// This consumer thread's slots from a built program; false (nothing loaded)
// when the program was built for another consumer count or form.
template <int FORM>
__device__ __forceinline__ bool load_gather(const uint32_t* prog, uint32_t zero_word, GatherProgram<FORM>& G)
{
    constexpr uint32_t K = GatherMax<FORM>::value, F = gather_program_fields<FORM>();
    const uint32_t cn = cnum(), c = ctid();
    if (prog[0] != kProgramMagic || prog[1] != cn || prog[2] != (uint32_t)FORM || prog[3] != K) return false;
    const uint32_t* o = prog + kProgramHeader;
    auto fix = [&](uint32_t v) {
        const uint32_t lo = v & 0xFFFFu, hi = v >> 16;
        return (lo == kZeroMarker ? zero_word : lo) | ((hi == kZeroMarker ? zero_word : hi) << 16);
    };
#pragma unroll
    for (uint32_t k = 0; k < K; ++k) {
        G.idx01[k] = fix(o[(k * F + 0u) * cn + c]);
        G.sel01[k] = o[(k * F + 1u) * cn + c];
        if constexpr (FORM == 4) {
            G.idx23[k] = fix(o[(k * F + 2u) * cn + c]);
            G.sel2[k] = o[(k * F + 3u) * cn + c];
            const uint32_t w = o[(k * F + 4u) * cn + c] & 0xFFFFu;
            G.dstw[k / 2] = (k & 1u) ? (G.dstw[k / 2] & 0xFFFFu) | (w << 16) : w;
        }
    }
    return true;
}

template <int FORM>
__device__ __forceinline__ void run_gather(const GatherProgram<FORM>& G, const uint8_t* simg, uint8_t* dimg,
                                           uint32_t nwords)
{
    const uint32_t* __restrict__ s = reinterpret_cast<const uint32_t*>(simg);
    uint32_t* __restrict__ d = reinterpret_cast<uint32_t*>(dimg);
    constexpr int K = GatherProgram<FORM>::K;
    // every source word first, then the stores: K loads in flight per thread
    uint32_t a[K], b[K], c[FORM == 4 ? K : 1], e[FORM == 4 ? K : 1];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        a[k] = s[G.idx01[k] & 0xFFFFu];
        b[k] = s[G.idx01[k] >> 16];
        if (FORM == 4) {
            c[k] = s[G.idx23[k] & 0xFFFFu];
            e[k] = s[G.idx23[k] >> 16];
        }
    }
    const uint32_t c0 = ctid(), cn = cnum();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const uint32_t w = FORM == 4 ? (G.dstw[k / 2] >> (16 * (k & 1))) & 0xFFFFu : c0 + k * cn;
        if (FORM == 4 ? w != 0xFFFFu : w < nwords) {
            if (FORM == 2) {
                d[w] = __byte_perm(a[k], b[k], G.sel01[k] & 0xFFFFu);
            } else {
                const uint32_t t0 = __byte_perm(a[k], b[k], G.sel01[k] & 0xFFFFu);
                const uint32_t t1 = __byte_perm(c[k], e[k], G.sel01[k] >> 16);
                d[w] = __byte_perm(t0, t1, G.sel2[k]);
            }
        }
    }
}

// Plain copy of `bytes` between global and shared memory by the consumers.
static __device__ void plain_copy(uint8_t* dst, const uint8_t* src, uint32_t bytes)
{
    const uint32_t c0 = ctid(), cn = cnum();
    const uintptr_t both = reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src);
    uint32_t done = 0;
    if ((both & 15u) == 0) {
        const uint32_t n16 = bytes / 16u;
        for (uint32_t k = c0; k < n16; k += cn)
            reinterpret_cast<uint4*>(dst)[k] = reinterpret_cast<const uint4*>(src)[k];
        done = n16 * 16u;
    } else if ((both & 3u) == 0) {
        const uint32_t n4 = bytes / 4u;
        for (uint32_t k = c0; k < n4; k += cn)
            reinterpret_cast<uint32_t*>(dst)[k] = reinterpret_cast<const uint32_t*>(src)[k];
        done = n4 * 4u;
    }
    for (uint32_t k = done + c0; k < bytes; k += cn) dst[k] = src[k];
}

// Global tile index of this CTA's k-th tile (see CopyArgs::chunk).
__device__ __forceinline__ uint32_t tile_index(const CopyArgs& a, uint32_t first, uint32_t k)
{
    return (a.chunk || a.cta_tiles) ? first + k : first + k * gridDim.x;
}

// The job of global tile g, for a role that walks its tiles in order: tiles
// [start, next) belong to `job`; a CTA's tiles are contiguous in batches, so
// a step past `next` is almost always into the next job (one load), and only
// the first tile (or a step back) searches the table.
struct JobCursor {
    uint32_t job = 0, start = 1, next = 0;  // empty until the first lookup
};

__device__ __forceinline__ uint32_t job_of(const CopyArgs& a, uint32_t g, JobCursor& c)
{
    if (a.table == nullptr) {
        c.start = 0;
        return 0;
    }
    if (g >= c.start && g < c.next) return c.job;
    if (c.start <= c.next && g >= c.next && c.job + 1u < a.njobs) {
        const uint32_t after = a.tile_start[c.job + 2u];
        if (g < after) {
            c.job += 1u;
            c.start = c.next;
            c.next = after;
            return c.job;
        }
    }
    uint32_t lo = 0, hi = a.njobs;  // tile_start[lo] <= g < tile_start[hi]
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (a.tile_start[mid] <= g) lo = mid;
        else hi = mid;
    }
    c.job = lo;
    c.start = a.tile_start[lo];
    c.next = a.tile_start[lo + 1u];
    return lo;
}

__device__ __forceinline__ uint32_t align16(uint32_t x) { return (x + 15u) & ~15u; }

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Run addressing of one side of a job, held in the producer warp's
// registers: lane q keeps run q (base address, bytes per tile, image offset).
struct LaneRuns {
    int job = -1;
    const uint8_t* gptr = nullptr;
    uint32_t bytes = 0, sbase = 0, total = 0, nfull = 0;
    int nsegs = 0;
    bool bulk = false;
};

__device__ __forceinline__ void lane_runs_load(LaneRuns& L, const SideDesc& S, const JobDesc* J, int j, uint32_t lane)
{
    L.job = j;
    L.nsegs = S.nsegs;
    L.nfull = J->nfull;
    L.bulk = S.bulk_ok;
    if ((int)lane < L.nsegs) {
        const SegDesc seg = S.segs[lane];
        L.gptr = S.blobs[seg.blob] + seg.gbase;
        L.bytes = seg.tile_bytes;
        L.sbase = seg.sbase;
    } else {
        L.gptr = nullptr;
        L.bytes = 0;
        L.sbase = 0;
    }
    L.total = __reduce_add_sync(0xFFFFFFFFu, L.bytes);
}

// After an abort the consumers may have left: wait (bounded) for the loads
// of the last src_stages issued tiles, which may still be landing in shared
// memory, before the CTA exits.
static __device__ void drain_loads(const CopyArgs& a, CopyShared& H, uint32_t first, uint32_t issued)
{
    const uint32_t NS = a.src_stages;
    JobCursor jc;
    for (uint32_t k = issued > NS ? issued - NS : 0u; k < issued; ++k) {
        const uint32_t g = tile_index(a, first, k);
        const uint32_t j = job_of(a, g, jc);
        const JobDesc* J = a.table ? a.table + j : &a.job;
        const uint32_t t = g - jc.start;
        if (t < J->nfull && J->src.bulk_ok) (void)mbar_wait_bounded(&H.full[k % NS], (k / NS) & 1u);
    }
}

// One warp for both directions (gather kernels, whose consumers are cheap
// per byte and need every warp): TMA loads `src_stages` tiles ahead, bulk
// stores as the consumers finish each destination stage.
static __device__ void producer(const CopyArgs& a, CopyShared& H, uint8_t* src_stage, uint8_t* dst_stage, uint32_t first,
                         uint32_t count)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t NS = a.src_stages, ND = a.dst_stages;
    volatile int* abort_flag = &H.abort;
    LaneRuns in, out;
    JobCursor in_c, out_c;
    uint32_t issued = 0;  // tiles whose loads have been issued: 0 .. issued-1

    auto issue_load = [&](uint32_t k) {
        const uint32_t g = tile_index(a, first, k);
        const uint32_t j = job_of(a, g, in_c);
        const uint32_t t = g - in_c.start;
        if ((int)j != in.job) {
            const JobDesc* J = a.table ? a.table + j : &a.job;
            lane_runs_load(in, J->src, J, (int)j, lane);
        }
        issued = k + 1u;
        if (!(t < in.nfull && in.bulk)) return;
        const uint32_t s = k % NS;
        if (lane == 0) mbar_arrive_expect_tx(&H.full[s], in.total);
        if ((int)lane < in.nsegs)
            bulk_load(src_stage + s * a.src_stage_bytes + in.sbase, in.gptr + (uint64_t)t * in.bytes, in.bytes,
                      &H.full[s]);
    };

    for (uint32_t k = 0; k < NS && k < count; ++k) issue_load(k);
    for (uint32_t k = 0; k < count; ++k) {
        const uint32_t d = k % ND;
        if (!mbar_wait_bounded(&H.dfull[d], (k / ND) & 1u)) {
            *abort_flag = 1;
            break;
        }
        const uint32_t g = tile_index(a, first, k);
        const uint32_t j = job_of(a, g, out_c);
        const uint32_t t = g - out_c.start;
        if ((int)j != out.job) {
            const JobDesc* J = a.table ? a.table + j : &a.job;
            lane_runs_load(out, J->dst, J, (int)j, lane);
        }
        if (t < out.nfull && out.bulk && (int)lane < out.nsegs)
            bulk_store(const_cast<uint8_t*>(out.gptr) + (uint64_t)t * out.bytes,
                       dst_stage + d * a.dst_stage_bytes + out.sbase, out.bytes);
        bulk_commit();  // one group per tile (empty for tiles the consumers stored)
        // The consumers released tile k's source stage before they arrived
        // on dfull: its next load goes out before any wait on the stores.
        if (k + NS < count) {
            if (!mbar_wait_bounded(&H.empty[k % NS], (k / NS) & 1u)) {
                *abort_flag = 1;
                break;
            }
            issue_load(k + NS);
        }
        // Release stage d for tile k+ND as soon as tile k's store has read it.
        bulk_wait_read(0);
        __syncwarp();
        if (lane == 0) mbar_arrive(&H.dempty[d]);
        if (*abort_flag) break;
    }
    bulk_wait_all();
    if (*abort_flag) drain_loads(a, H, first, issued);
}

// Load warp: brings tile k into source stage k % NS with TMA bulk loads as
// soon as the consumers have released the stage's previous tile.
static __device__ void load_producer(const CopyArgs& a, CopyShared& H, uint8_t* src_stage, uint32_t first, uint32_t count)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t NS = a.src_stages;
    volatile int* abort_flag = &H.abort;
    LaneRuns in;
    JobCursor in_c;
    uint32_t issued = 0;        // tiles whose loads have been issued: 0 .. issued-1
    uint32_t s = 0, round = 0;  // k % NS, (k / NS) & 1
    for (uint32_t k = 0; k < count; ++k) {
        if (k >= NS && !mbar_wait_bounded(&H.empty[s], round ^ 1u)) {
            *abort_flag = 1;
            break;
        }
        const uint32_t g = tile_index(a, first, k);
        const uint32_t j = job_of(a, g, in_c);
        const uint32_t t = g - in_c.start;
        if ((int)j != in.job) {
            const JobDesc* J = a.table ? a.table + j : &a.job;
            lane_runs_load(in, J->src, J, (int)j, lane);
        }
        issued = k + 1u;
        if (t < in.nfull && in.bulk) {
            if (lane == 0) mbar_arrive_expect_tx(&H.full[s], in.total);
            if ((int)lane < in.nsegs)
                bulk_load(src_stage + s * a.src_stage_bytes + in.sbase, in.gptr + (uint64_t)t * in.bytes, in.bytes,
                          &H.full[s]);
        }
        if (*abort_flag) break;
        if (++s == NS) {
            s = 0;
            round ^= 1u;
        }
    }
    if (*abort_flag) drain_loads(a, H, first, issued);
}

// Store warp: writes destination stage k % ND back with TMA bulk stores once
// the consumers have finished tile k, and releases the stage for tile k+ND
// as soon as the store has read it.  Loads and stores are issued by two
// warps so that neither waits behind the other's (serial) issue.
static __device__ void store_producer(const CopyArgs& a, CopyShared& H, uint8_t* dst_stage, uint32_t first, uint32_t count)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t ND = a.dst_stages;
    volatile int* abort_flag = &H.abort;
    LaneRuns out;
    JobCursor out_c;
    uint32_t d = 0, round = 0;  // k % ND, (k / ND) & 1
    for (uint32_t k = 0; k < count; ++k) {
        if (!mbar_wait_bounded(&H.dfull[d], round)) {
            *abort_flag = 1;
            break;
        }
        const uint32_t g = tile_index(a, first, k);
        const uint32_t j = job_of(a, g, out_c);
        const uint32_t t = g - out_c.start;
        if ((int)j != out.job) {
            const JobDesc* J = a.table ? a.table + j : &a.job;
            lane_runs_load(out, J->dst, J, (int)j, lane);
        }
        if (t < out.nfull && out.bulk && (int)lane < out.nsegs)
            bulk_store(const_cast<uint8_t*>(out.gptr) + (uint64_t)t * out.bytes,
                       dst_stage + d * a.dst_stage_bytes + out.sbase, out.bytes);
        bulk_commit();  // one group per tile (empty for tiles the consumers stored)
        bulk_wait_read(0);
        __syncwarp();
        if (lane == 0) mbar_arrive(&H.dempty[d]);
        if (*abort_flag) break;
        if (++d == ND) {
            d = 0;
            round ^= 1u;
        }
    }
    bulk_wait_all();
}

// Bounded wait that gives up at once after an abort (the phase may never
// complete then); a timeout records the abort for every role.
__device__ __forceinline__ void wait_or_abort(CopyShared& H, uint64_t* bar, uint32_t parity)
{
    volatile int* abort_flag = &H.abort;
    if (*abort_flag) return;
    if (!mbar_wait_bounded(bar, parity)) *abort_flag = 1;
}

// Consumer warps: convert each tile from its source stage into a destination
// stage, or load / store it themselves where TMA does not apply.
template <int MODE>
__device__ void consumer(const CopyArgs& a, CopyShared& H, uint8_t* src_stage, uint8_t* dst_stage, uint8_t* codes,
                         uint32_t first, uint32_t count)
{
    const uint32_t NS = a.src_stages, ND = a.dst_stages;
    const uint32_t zero_word = (a.src_stage_bytes - kStageZeroBytes) / 4u;
    const bool warp_leader = (threadIdx.x & 31u) == 0;
    GatherProgram<gather_mode(MODE) ? MODE : 2> gp;
    uint32_t gather_words = 0;
    uint32_t phase = 0;        // per source stage: parity of the next full phase
    uint32_t zeroed = 0;       // destination stages whose padding bytes are zero (current job)
    int cur_job = -1;
    uint32_t s = 0, d = 0;     // stages of tile k: k % NS, k % ND
    uint32_t dround = 0;       // parity of k / ND
    ItemShare share{0u, 0u, 0u, 0u};
    JobCursor jc;

    for (uint32_t k = 0; k < count; ++k) {
        const uint32_t g = tile_index(a, first, k);
        const uint32_t j = job_of(a, g, jc);
        if ((int)j != cur_job) {
            consumer_sync();
            const uint2* from = reinterpret_cast<const uint2*>(a.table ? a.table + j : &a.job);
            uint2* to = reinterpret_cast<uint2*>(&H.job);
            for (uint32_t w = ctid(); w < sizeof(JobDesc) / 8u; w += cnum()) to[w] = from[w];
            consumer_sync();
            cur_job = (int)j;
            zeroed = 0;
            if constexpr (!gather_mode(MODE)) {
                share = item_share(H.job);
            } else {
                gather_words = (H.job.dst.img_bytes - kImageSlack) / 4u;
                const uint32_t* prog = reinterpret_cast<const uint32_t*>(H.job.program);
                if (!(prog && load_gather<MODE>(prog, zero_word, gp))) build_gather<MODE>(H.job, zero_word, gather_words, gp);
            }
        }
        const JobDesc& J = H.job;
        const uint32_t t = g - jc.start;
        const uint32_t nvalid = (t + 1u < J.ntiles) ? J.tile : (uint32_t)(J.n - (uint64_t)t * J.tile);
        uint8_t* simg = src_stage + s * a.src_stage_bytes;
        uint8_t* dimg = dst_stage + d * a.dst_stage_bytes;
        const bool bulk_in = t < J.nfull && J.src.bulk_ok;
        const bool bulk_out = t < J.nfull && J.dst.bulk_ok;

        // Consumer warps run without a per-tile barrier: each waits on the
        // stage barriers itself, so warps may drift apart by up to
        // min(src_stages, dst_stages) tiles.  The barriers below are taken
        // at the same tiles by every warp, aborted or not (a wait that timed
        // out sets H.abort, and later waits return at once).
        bool sync_needed = false;
        if (bulk_in) {
            wait_or_abort(H, &H.full[s], (phase >> s) & 1u);
            phase ^= 1u << s;
        } else {
            consumer_sync();  // every warp is done with the stage's previous tile
            const bool last = (t + 1u == J.ntiles);
            for (int q = 0; q < J.src.nsegs; ++q) {
                const SegDesc& S = J.src.segs[q];
                plain_copy(simg + S.sbase, J.src.blobs[S.blob] + S.gbase + (uint64_t)t * S.tile_bytes,
                           last ? S.tail_bytes : S.tile_bytes);
            }
            sync_needed = true;
        }
        wait_or_abort(H, &H.dempty[d], dround ^ 1u);

        // Items write leaf bytes only: their stage must start with zero padding.
        // (A gather program writes every word, zeros included.)  The store
        // of the stage's previous tile has read it (dempty), and that tile's
        // writers all arrived before the store was issued.
        const bool items_here = !gather_mode(MODE) || t >= J.nfull;
        if (items_here && !(zeroed & (1u << d))) {
            uint4* z = reinterpret_cast<uint4*>(dimg);
            for (uint32_t w = ctid(); w < a.dst_stage_bytes / 16u; w += cnum()) z[w] = make_uint4(0, 0, 0, 0);
            zeroed |= 1u << d;
            sync_needed = true;
        }
        if (!gather_mode(MODE) && J.ored) {
            zero_streams(J, dimg);
            sync_needed = true;
        }
        if (sync_needed) consumer_sync();
        if (t == 0) {
            for (int q = 0; q < J.nzeros; ++q) {
                const ZeroRun& Z = J.zeros[q];
                uint8_t* p = J.dst.blobs[Z.blob] + Z.offset;
                for (uint32_t b = ctid(); b < Z.bytes; b += cnum()) p[b] = 0;
            }
        }
        if constexpr (gather_mode(MODE)) {
            if (t < J.nfull) {
                run_gather<MODE>(gp, simg, dimg, gather_words);
                zeroed |= 1u << d;
            } else {
                run_moves(J, simg, dimg, nvalid);
            }
        } else {
            run_items<MODE>(J, simg, dimg, nvalid, share);
        }
        fence_proxy_async();
        __syncwarp();
        if (warp_leader) mbar_arrive(&H.empty[s]);
        if (!bulk_out) {
            consumer_sync();
            const bool last = (t + 1u == J.ntiles);
            for (int q = 0; q < J.dst.nsegs; ++q) {
                const SegDesc& S = J.dst.segs[q];
                plain_copy(J.dst.blobs[S.blob] + S.gbase + (uint64_t)t * S.tile_bytes, dimg + S.sbase,
                           last ? S.tail_bytes : S.tile_bytes);
            }
            __syncwarp();
        }
        if (warp_leader) mbar_arrive(&H.dfull[d]);
        if (++s == NS) s = 0;
        if (++d == ND) {
            d = 0;
            dround ^= 1u;
        }
    }
}

// MODE 0: general items and packs (compile-time loops of SoA bit streams).
// MODE 1: the same, for jobs whose bit leaves organised as AoSoA need the
// generic loop.  MODE 3: the same, with the compile-time loops of bit leaves
// organised as AoSoA.  MODE 2 / 4: every job is made of byte moves; full tiles
// run gather programs of that form.
template <int MODE>
__global__ void __launch_bounds__(512, 1) copy_kernel(const __grid_constant__ CopyArgs a)
{
    CopyShared& H = *reinterpret_cast<CopyShared*>(g_smem);
    uint8_t* src_stage = g_smem + align16(sizeof(CopyShared));
    uint8_t* dst_stage = src_stage + a.src_stages * a.src_stage_bytes;
    uint8_t* codes = dst_stage + a.dst_stages * a.dst_stage_bytes;

    const uint32_t G = gridDim.x;
    uint32_t first, count;  // this CTA's tiles: first + k (contiguous) or first + k * grid
    if (a.cta_tiles) {
        first = a.cta_tiles[blockIdx.x];
        const uint32_t end = a.cta_tiles[blockIdx.x + 1];
        if (first >= end) return;
        count = end - first;
    } else if (a.chunk) {
        const uint64_t begin = (uint64_t)blockIdx.x * a.chunk;
        if (begin >= a.total_tiles) return;
        const uint64_t left = a.total_tiles - begin;
        first = (uint32_t)begin;
        count = left < a.chunk ? (uint32_t)left : a.chunk;
    } else {
        first = blockIdx.x;
        if (first >= a.total_tiles) return;
        count = (a.total_tiles - first + G - 1u) / G;
    }
    const uint32_t NS = a.src_stages, ND = a.dst_stages;
    constexpr uint32_t P = producer_warps(MODE);
    const uint32_t consumer_warps = blockDim.x / 32u - P;

    // The last 16 bytes of every source stage hold zeros: gather programs
    // read destination padding from there.
    const uint32_t zero_word = (a.src_stage_bytes - kStageZeroBytes) / 4u;
    if (threadIdx.x < NS * 4u)
        reinterpret_cast<uint32_t*>(src_stage + (threadIdx.x / 4u) * a.src_stage_bytes)[zero_word + threadIdx.x % 4u] = 0u;
    if (threadIdx.x == 0) {
        for (uint32_t s = 0; s < NS; ++s) {
            mbar_init(&H.full[s], 1);
            mbar_init(&H.empty[s], consumer_warps);
        }
        for (uint32_t d = 0; d < ND; ++d) {
            mbar_init(&H.dfull[d], consumer_warps);
            mbar_init(&H.dempty[d], 1);
        }
        fence_barrier_init();
        H.abort = 0;
        H.cons_base = 32u * P;
    }
    __syncthreads();

    if (P == 2 && threadIdx.x < 32u)
        load_producer(a, H, src_stage, first, count);
    else if (P == 2 && threadIdx.x < 64u)
        store_producer(a, H, dst_stage, first, count);
    else if (P == 1 && threadIdx.x < 32u)
        producer(a, H, src_stage, dst_stage, first, count);
    else
        consumer<MODE>(a, H, src_stage, dst_stage, codes, first, count);

    // Both roles return after bounded waits, so every thread gets here.
    __syncthreads();
    if (H.abort && threadIdx.x == 0) atomicOr(&g_device_status, (unsigned)LLGB_ERR_TIMEOUT);
}

// Host side of one translation unit: its kernels' shared-memory limit and
// launch, and its status word.
template <int MODE>
static cudaError_t prepare_mode(size_t smem_bytes)
{
    static thread_local int configured_dev = -1;
    static thread_local size_t configured_bytes = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev != configured_dev || smem_bytes > configured_bytes) {
        e = cudaFuncSetAttribute(copy_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
        if (e != cudaSuccess) return e;
        configured_dev = dev;
        configured_bytes = smem_bytes;
    }
    return cudaSuccess;
}

template <int MODE>
static cudaError_t launch_mode(const CopyArgs& args, int grid, int threads, size_t smem_bytes, cudaStream_t stream)
{
    cudaError_t e = prepare_mode<MODE>(smem_bytes);
    if (e != cudaSuccess) return e;
    copy_kernel<MODE><<<grid, threads, smem_bytes, stream>>>(args);
    return cudaGetLastError();
}

// OR this unit's status word into *out (after the caller synchronised the
// device); reset clears it.
static cudaError_t unit_status(unsigned* out, bool reset)
{
    unsigned v = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_device_status, sizeof(unsigned));
    if (e != cudaSuccess) return e;
    *out |= v;
    if (reset && v) {
        const unsigned zero = 0;
        e = cudaMemcpyToSymbol(g_device_status, &zero, sizeof(unsigned));
    }
    return e;
}

}  // namespace llgb
