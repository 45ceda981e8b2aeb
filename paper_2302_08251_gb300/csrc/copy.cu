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
                                          uint8_t* __restrict__ dimg, uint32_t tile, uint32_t nvalid)
{
    using W = typename UInt<G>::T;
    for (uint32_t r = threadIdx.x; r < tile; r += blockDim.x) {
        const uint32_t so = eoff(A, r) + sb;
        const uint32_t dof = eoff(B, r) + db;
        const bool live = r < nvalid;
        for (uint32_t p = 0; p < size; p += G)
            *reinterpret_cast<W*>(dimg + dof + p) = live ? *reinterpret_cast<const W*>(simg + so + p) : W(0);
    }
}

// One VALUE item: load the logical value through LOP, store it through SOP.
template <int LOP, int SOP>
__device__ __noinline__ void value_loop(const ItemDesc I, const JobDesc& J, const uint8_t* __restrict__ simg,
                                        uint8_t* __restrict__ dimg, uint8_t* __restrict__ codes,
                                        uint32_t tile, uint32_t nvalid)
{
    const LeafRegs A = leaf_regs(J.src.leaves[I.src_leaf]);
    const LeafRegs B = leaf_regs(J.dst.leaves[I.dst_leaf]);
    const int size = I.size;
    const uint64_t lmask = low_bits64(8 * size);
    uint32_t code_off = 0;
    bool wide = false;
    if (SOP == S_BITS_INT || SOP == S_BITS_FLOAT) {
        code_off = J.packs[I.slot].code_off;
        wide = J.packs[I.slot].wide;
    }
    const uint64_t dmask = low_bits64(I.d_bits);
    const uint64_t smask = low_bits64(A.bits);
    for (uint32_t r = threadIdx.x; r < tile; r += blockDim.x) {
        uint64_t v = 0;
        if (r < nvalid) {
            if (LOP == L_DIRECT) {
                v = ld_elem(simg + eoff(A, r), size, A.align);
            } else if (LOP == L_CT) {
                v = fconv(ld_elem(simg + eoff(A, r), I.s_size, A.align), I.s_e, I.s_m, I.l_e, I.l_m);
            } else if (LOP == L_BITS_INT) {
                uint64_t c = ld_bits(simg + A.sbase, r * A.bits, A.bits);
                if (I.is_signed && ((c >> (A.bits - 1)) & 1ull)) c |= ~smask;
                v = c & lmask;
            } else if (LOP == L_BITS_FLOAT) {
                v = fconv(ld_bits(simg + A.sbase, r * A.bits, A.bits), I.s_e, I.s_m, I.l_e, I.l_m);
            } else {  // L_SPLIT
                for (int j = 0; j < size; ++j) {
                    const LeafRegs S = leaf_regs(J.src.leaves[I.src_leaf + j]);
                    v |= (uint64_t)simg[eoff(S, r)] << (8 * j);
                }
            }
        }
        if (SOP == S_DIRECT) {
            st_elem(dimg + eoff(B, r), size, B.align, v);
        } else if (SOP == S_CT) {
            st_elem(dimg + eoff(B, r), I.d_size, B.align, fconv(v, I.l_e, I.l_m, I.d_e, I.d_m));
        } else if (SOP == S_BITS_INT || SOP == S_BITS_FLOAT) {
            const uint64_t c = SOP == S_BITS_INT ? (v & dmask) : fconv(v, I.l_e, I.l_m, I.d_e, I.d_m);
            if (wide)
                reinterpret_cast<uint64_t*>(codes + code_off)[r] = c;
            else
                reinterpret_cast<uint32_t*>(codes + code_off)[r] = (uint32_t)c;
        } else {  // S_SPLIT
            for (int j = 0; j < size; ++j) {
                const LeafRegs D = leaf_regs(J.dst.leaves[I.dst_leaf + j]);
                dimg[eoff(D, r)] = (uint8_t)(v >> (8 * j));
            }
        }
    }
}

template <int LOP>
__device__ __forceinline__ void value_dispatch(const ItemDesc& I, const JobDesc& J, const uint8_t* simg,
                                               uint8_t* dimg, uint8_t* codes, uint32_t tile, uint32_t nvalid)
{
    switch (I.sop) {
    case S_DIRECT: value_loop<LOP, S_DIRECT>(I, J, simg, dimg, codes, tile, nvalid); break;
    case S_CT: value_loop<LOP, S_CT>(I, J, simg, dimg, codes, tile, nvalid); break;
    case S_BITS_INT: value_loop<LOP, S_BITS_INT>(I, J, simg, dimg, codes, tile, nvalid); break;
    case S_BITS_FLOAT: value_loop<LOP, S_BITS_FLOAT>(I, J, simg, dimg, codes, tile, nvalid); break;
    default: value_loop<LOP, S_SPLIT>(I, J, simg, dimg, codes, tile, nvalid); break;
    }
}

__device__ void run_items(const JobDesc& J, const uint8_t* simg, uint8_t* dimg, uint8_t* codes,
                          uint32_t nvalid)
{
    const uint32_t tile = J.tile;
    for (int it = 0; it < J.nitems; ++it) {
        const ItemDesc I = J.items[it];
        if (I.op == ITEM_MOVE) {
            const LeafRegs A = leaf_regs(J.src.leaves[I.src_leaf]);
            const LeafRegs B = leaf_regs(J.dst.leaves[I.dst_leaf]);
            switch (I.gran) {
            case 8: move_loop<8>(A, B, I.src_byte, I.dst_byte, I.size, simg, dimg, tile, nvalid); break;
            case 4: move_loop<4>(A, B, I.src_byte, I.dst_byte, I.size, simg, dimg, tile, nvalid); break;
            case 2: move_loop<2>(A, B, I.src_byte, I.dst_byte, I.size, simg, dimg, tile, nvalid); break;
            default: move_loop<1>(A, B, I.src_byte, I.dst_byte, I.size, simg, dimg, tile, nvalid); break;
            }
        } else {
            switch (I.lop) {
            case L_DIRECT: value_dispatch<L_DIRECT>(I, J, simg, dimg, codes, tile, nvalid); break;
            case L_CT: value_dispatch<L_CT>(I, J, simg, dimg, codes, tile, nvalid); break;
            case L_BITS_INT: value_dispatch<L_BITS_INT>(I, J, simg, dimg, codes, tile, nvalid); break;
            case L_BITS_FLOAT: value_dispatch<L_BITS_FLOAT>(I, J, simg, dimg, codes, tile, nvalid); break;
            default: value_dispatch<L_SPLIT>(I, J, simg, dimg, codes, tile, nvalid); break;
            }
        }
    }
}

// Byte moves only (the items of a gather job, for its last tile).
__device__ __forceinline__ void run_moves(const JobDesc& J, const uint8_t* simg, uint8_t* dimg, uint32_t nvalid)
{
    for (int it = 0; it < J.nitems; ++it) {
        const ItemDesc I = J.items[it];
        const LeafRegs A = leaf_regs(J.src.leaves[I.src_leaf]);
        const LeafRegs B = leaf_regs(J.dst.leaves[I.dst_leaf]);
        switch (I.gran) {
        case 8: move_loop<8>(A, B, I.src_byte, I.dst_byte, I.size, simg, dimg, J.tile, nvalid); break;
        case 4: move_loop<4>(A, B, I.src_byte, I.dst_byte, I.size, simg, dimg, J.tile, nvalid); break;
        case 2: move_loop<2>(A, B, I.src_byte, I.dst_byte, I.size, simg, dimg, J.tile, nvalid); break;
        default: move_loop<1>(A, B, I.src_byte, I.dst_byte, I.size, simg, dimg, J.tile, nvalid); break;
        }
    }
}

// One thread per 32-bit word of a bit-stream destination: OR together the
// codes that overlap the word.
template <bool DIRECT, bool WIDE>
__device__ __noinline__ void pack_loop(const PackDesc P, const JobDesc& J, const uint8_t* __restrict__ simg,
                                       uint8_t* __restrict__ dimg, const uint8_t* __restrict__ codes,
                                       uint32_t tile, uint32_t nvalid)
{
    const uint32_t w = P.bits;
    const uint32_t nwords = tile * w / 32u;
    uint32_t* out = reinterpret_cast<uint32_t*>(dimg + P.dst_sbase);
    LeafRegs A{};
    if (DIRECT) A = leaf_regs(J.src.leaves[P.src_leaf]);
    const uint64_t mask = low_bits64(w);
    const int ssize = P.src_size;
    for (uint32_t q = threadIdx.x; q < nwords; q += blockDim.x) {
        const uint32_t bit0 = q * 32u;
        const uint32_t jlo = w == 1 ? bit0 : __umulhi(bit0, P.magic);
        uint32_t jhi = w == 1 ? bit0 + 31u : __umulhi(bit0 + 31u, P.magic);
        if (jhi > tile - 1u) jhi = tile - 1u;
        uint32_t word = 0;
        for (uint32_t j = jlo; j <= jhi; ++j) {
            uint64_t c;
            if (DIRECT)
                c = j < nvalid ? (ld_elem(simg + eoff(A, j), ssize, A.align) & mask) : 0ull;
            else if (WIDE)
                c = reinterpret_cast<const uint64_t*>(codes + P.code_off)[j];
            else
                c = reinterpret_cast<const uint32_t*>(codes + P.code_off)[j];
            const int pos = (int)(j * w) - (int)bit0;
            word |= pos >= 0 ? (uint32_t)(c << pos) : (uint32_t)(c >> (-pos));
        }
        out[q] = word;
    }
}

__device__ void run_packs(const JobDesc& J, const uint8_t* simg, uint8_t* dimg, const uint8_t* codes,
                          uint32_t nvalid)
{
    for (int k = 0; k < J.npacks; ++k) {
        const PackDesc P = J.packs[k];
        if (P.direct)
            pack_loop<true, false>(P, J, simg, dimg, codes, J.tile, nvalid);
        else if (P.wide)
            pack_loop<false, true>(P, J, simg, dimg, codes, J.tile, nvalid);
        else
            pack_loop<false, false>(P, J, simg, dimg, codes, J.tile, nvalid);
    }
}

// ------------------------------------------------------ gather programs --
//
// A job made only of byte moves permutes bytes: destination image byte o of
// every full tile comes from the same source image byte (or is zero).  Each
// thread derives, once per job, a program for each of its destination words
// w = tid + k * blockDim.x: up to four source words and the byte selectors
// that assemble the word with PRMT.  A full tile then costs a few loads, one
// or three PRMTs and one store per destination word.

// Destination words per thread: 16 for the 2-word form, 12 for the 4-word
// form (registers: 2 resp. 4 per word).
template <int FORM>
struct GatherMax {
    static constexpr int value = FORM == 2 ? 16 : (FORM == 4 ? 12 : 1);
};

// Source image byte feeding destination image byte o, or -1 (no leaf: zero).
__device__ __forceinline__ int32_t gather_source(const JobDesc& J, uint32_t o)
{
    const SideDesc& D = J.dst;
    for (int g = 0; g < D.nleaves; ++g) {
        const LeafDesc& L = D.leaves[g];
        if (o < L.sbase) continue;
        const uint32_t d = o - L.sbase;
        uint32_t r, e;
        if (L.lanes == 1) {
            r = d / L.bstride;
            e = d - r * L.bstride;
            if (e >= L.size || r >= J.tile) continue;
        } else {
            const uint32_t blk = d / L.bstride;
            const uint32_t rem = d - blk * L.bstride;
            const uint32_t lane = rem / L.size;
            e = rem - lane * L.size;
            if (lane >= L.lanes) continue;
            r = blk * L.lanes + lane;
            if (r >= J.tile) continue;
        }
        for (int it = 0; it < J.nitems; ++it) {
            const ItemDesc& I = J.items[it];
            if (I.dst_leaf != g || e < I.dst_byte || e >= (uint32_t)I.dst_byte + I.size) continue;
            return (int32_t)(eoff(leaf_regs(J.src.leaves[I.src_leaf]), r) + I.src_byte + (e - I.dst_byte));
        }
        return -1;
    }
    return -1;
}

template <int FORM>
struct GatherProgram {
    static constexpr int K = GatherMax<FORM>::value;
    uint32_t idx01[K];                 // source word indices i0 | i1 << 16
    uint32_t sel01[K];                 // q0 | q1 << 16
    uint32_t idx23[FORM == 4 ? K : 1]; // i2 | i3 << 16
    uint32_t sel2[FORM == 4 ? K : 1];  // q2
};

template <int FORM>
__device__ __forceinline__ void build_gather(const JobDesc& J, uint32_t zero_word, uint32_t nwords,
                                             GatherProgram<FORM>& G)
{
    // Rolled over k so that gather_source is expanded once; each result is
    // steered into its register slot by an unrolled select.
#pragma unroll 1
    for (int k = 0; k < GatherProgram<FORM>::K; ++k) {
        const uint32_t w = threadIdx.x + k * blockDim.x;
        uint32_t word[4], byte[4];
#pragma unroll 1
        for (int b = 0; b < 4; ++b) {
            const int32_t src = w < nwords ? gather_source(J, 4u * w + b) : -1;
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
        uint32_t q0 = 0, q1 = 0, q2 = 0;
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
        const uint32_t i01 = u[0] | (u[1] << 16), s01 = q0 | (q1 << 16);
        const uint32_t i23 = u[2] | (u[3] << 16);
#pragma unroll
        for (int kk = 0; kk < GatherProgram<FORM>::K; ++kk) {
            if (kk == k) {
                G.idx01[kk] = i01;
                G.sel01[kk] = s01;
                if (FORM == 4) {
                    G.idx23[kk] = i23;
                    G.sel2[kk] = q2;
                }
            }
        }
    }
}

template <int FORM>
__device__ __forceinline__ void run_gather(const GatherProgram<FORM>& G, const uint8_t* simg, uint8_t* dimg,
                                           uint32_t nwords)
{
    const uint32_t* __restrict__ s = reinterpret_cast<const uint32_t*>(simg);
    uint32_t* __restrict__ d = reinterpret_cast<uint32_t*>(dimg);
#pragma unroll
    for (int k = 0; k < GatherProgram<FORM>::K; ++k) {
        const uint32_t w = threadIdx.x + k * blockDim.x;
        if (w < nwords) {
            const uint32_t a = s[G.idx01[k] & 0xFFFFu], b = s[G.idx01[k] >> 16];
            if (FORM == 2) {
                d[w] = __byte_perm(a, b, G.sel01[k] & 0xFFFFu);
            } else {
                const uint32_t c = s[G.idx23[k] & 0xFFFFu], e = s[G.idx23[k] >> 16];
                const uint32_t t0 = __byte_perm(a, b, G.sel01[k] & 0xFFFFu);
                const uint32_t t1 = __byte_perm(c, e, G.sel01[k] >> 16);
                d[w] = __byte_perm(t0, t1, G.sel2[k]);
            }
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

// MODE 0: general items and packs.  MODE 2 / 4: every job is made of byte
// moves; full tiles run gather programs of that form.
template <int MODE>
__global__ void __launch_bounds__(512, 1) copy_kernel(const __grid_constant__ CopyArgs a)
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
    // The last 16 bytes of every source stage hold zeros: gather programs
    // read destination padding from there.
    const uint32_t zero_word = (a.src_stage_bytes - kStageZeroBytes) / 4u;
    if (threadIdx.x < NS * 4u)
        reinterpret_cast<uint32_t*>(src_stage + (threadIdx.x / 4u) * a.src_stage_bytes)[zero_word + threadIdx.x % 4u] = 0u;

    if (threadIdx.x == 0) {
        for (uint32_t s = 0; s < NS; ++s) mbar_init(&H.full[s], 1);
        fence_barrier_init();
        H.abort = 0;
        H.cur_job = -1;
    }
    __syncthreads();
    GatherProgram<MODE> gp;
    uint32_t gather_words = 0;

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
            if (MODE != 0) {
                gather_words = (H.job.dst.img_bytes - kImageSlack) / 4u;
                build_gather<MODE>(H.job, zero_word, gather_words, gp);
            }
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
        if (MODE != 0) {
            if (t < J.nfull)
                run_gather<MODE>(gp, simg, dimg, gather_words);
            else
                run_moves(J, simg, dimg, nvalid);
        } else {
            run_items(J, simg, dimg, codes, nvalid);
            if (J.npacks) {
                __syncthreads();
                run_packs(J, simg, dimg, codes, nvalid);
            }
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

int gather_words_per_thread(int mode) { return mode == 2 ? GatherMax<2>::value : (mode == 4 ? GatherMax<4>::value : 0); }

template <int MODE>
static cudaError_t launch_mode(const CopyArgs& args, int grid, int threads, size_t smem_bytes, cudaStream_t stream)
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
    copy_kernel<MODE><<<grid, threads, smem_bytes, stream>>>(args);
    return cudaGetLastError();
}

cudaError_t launch_copy(const CopyArgs& args, int mode, int grid, int threads, size_t smem_bytes,
                        cudaStream_t stream)
{
    switch (mode) {
    case 2: return launch_mode<2>(args, grid, threads, smem_bytes, stream);
    case 4: return launch_mode<4>(args, grid, threads, smem_bytes, stream);
    default: return launch_mode<0>(args, grid, threads, smem_bytes, stream);
    }
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
