// stream_loops.cuh -- pack and unpack loops of SoA bit streams whose format
// is known at compile time (the formats of stream_specs.h).  Included by
// copy_kernel.cuh after the shared-memory and lane helpers it uses.
//
// Pack (Sec. 3: values are packed when stored).  A warp takes super-groups of
// 32 V records; lane l holds records V l .. V l + V - 1 of each:
//   1. the lane loads its V leaf elements with one vector access and turns
//      them into w-bit codes (the low w bits of an integer; a float rounded
//      to (E, M), nearest even, by constant-shift integer arithmetic);
//   2. the codes form the lane's chunk of C = V w bits (code v at bit v w);
//   3. narrow chunks (C < 32) are merged over T = 2, 4 or 8 neighbouring
//      lanes (a shuffle per doubling), so that every merged chunk has
//      CC = T C bits with 32 <= CC <= 64;
//   4. output word k of the super-group takes bits [32 k, 32 k + 32) of the
//      merged chunks: at most two of them reach it, fetched with shuffles from
//      lanes j0 T and (j0 + 1) T (j0 = floor(32 k / CC)); lane k builds and
//      stores word k (two rounds when the super-group has more than 32 words).
// Unpack (values are unpacked when loaded): lane l reads its C-bit chunk at
// bit l C of the super-group (two or three words and funnel shifts), splits
// it into V codes, converts them and stores its V elements with one vector
// access.
// Records at or past the tile's valid count are taken as zero (and so written
// as zero).  Float values whose result is not a normal number of the target
// -- zeros included -- and NaN and INF inputs are redone by fconv_general;
// the warp votes on whether any lane has one, so the common case pays one
// vote.
#pragma once

#include "stream_specs.h"

namespace llgb {

// Rounding conversion of a normal number between binary formats (SE, SM) ->
// (DE, DM), by integer operations on the bit pattern: the magnitude bits
// (exponent and mantissa) are shifted by k = SM - DM with rounding to
// nearest, ties to even (add 2^(k-1) - 1 plus the lowest kept bit, then drop k
// bits: a carry moves into the exponent, and past the largest exponent it
// gives the INF code), and the exponent is rebiased by adding a constant --
// folded into the rounding constant as (DB - SB) 2^SM before the shift.
// `bad` is set for inputs this does not cover: source exponents whose target
// exponent is out of range (zero, subnormal or overflowing results,
// subnormal inputs, INF, NaN); the range test reads only the exponent field's
// word.
template <int SE, int SM, int DE, int DM>
__device__ __forceinline__ uint64_t conv_fast(uint64_t x, bool& bad)
{
    constexpr int SB = (1 << (SE - 1)) - 1, DB = (1 << (DE - 1)) - 1;
    constexpr int K = SM - DM;
    constexpr int E_LO = (SB - DB + 1) > 1 ? (SB - DB + 1) : 1;
    constexpr int E_HI = ((1 << DE) - 2 + SB - DB) < ((1 << SE) - 2) ? ((1 << DE) - 2 + SB - DB) : ((1 << SE) - 2);
    if constexpr (SE + SM == 63 && K >= 33 && 1 + DE + DM <= 32 && DE <= 12) {
        // f64 narrowed to at most 19 mantissa bits: exponent and kept bits lie
        // in the high word, and the low word only tells, as a sticky bit with
        // the lowest kept bit, whether the dropped bits reach past a tie --
        // the 64-bit sum's carry out of the low word -- so the rounding runs
        // on the high word alone
        const uint32_t hi = (uint32_t)(x >> 32), lo = (uint32_t)x;
        const uint32_t ah = hi & 0x7FFFFFFFu;
        bad = ah - ((uint32_t)E_LO << (SM - 32)) >= ((uint32_t)(E_HI - E_LO + 1) << (SM - 32));
        constexpr uint32_t C32 = (uint32_t)(((1ll << (K - 33)) - 1ll) + (int64_t)(DB - SB) * (1ll << (SM - 32)));
        const uint32_t carry = (uint32_t)(lo != 0u) | ((ah >> (K - 32)) & 1u);
        const uint32_t r = (ah + C32 + carry) >> (K - 32);
        return (uint64_t)(((hi >> 31) << (DE + DM)) | r);
    } else if constexpr (SE + SM == 31 && K > 0 && DE + SM <= 31) {
        // f32 narrowed to a format whose rebiased exponent still fits the word
        const uint32_t x32 = (uint32_t)x, a32 = x32 & 0x7FFFFFFFu;
        bad = (a32 >> SM) - (uint32_t)E_LO > (uint32_t)(E_HI - E_LO);
        constexpr uint32_t C32 = (uint32_t)(((1ll << (K - 1)) - 1ll) + (int64_t)(DB - SB) * (1ll << SM));
        const uint32_t r = (a32 + C32 + ((a32 >> K) & 1u)) >> K;
        return (uint64_t)(((x32 >> 31) << (DE + DM)) | r);
    }
    constexpr uint64_t AMASK = (SE + SM >= 64) ? ~0ull : ((1ull << (SE + SM)) - 1ull);
    const uint64_t a = x & AMASK;
    if constexpr (SM >= 32) {  // the exponent field lies in the high word
        const uint32_t ah = (uint32_t)(a >> 32);
        bad = ah - ((uint32_t)E_LO << (SM - 32)) >= ((uint32_t)(E_HI - E_LO + 1) << (SM - 32));
    } else {
        const uint32_t e = (uint32_t)(a >> SM);
        bad = e - (uint32_t)E_LO > (uint32_t)(E_HI - E_LO);
    }
    uint64_t r;
    if constexpr (K > 0) {
        constexpr uint64_t C = ((1ull << (K - 1)) - 1ull) + (uint64_t)((int64_t)(DB - SB) * (int64_t)(1ll << SM));
        r = (a + C + ((a >> K) & 1ull)) >> K;
    } else {
        r = (a << (-K)) + (uint64_t)((int64_t)(DB - SB) * (int64_t)(1ll << DM));
    }
    return (((x >> (SE + SM)) & 1ull) << (DE + DM)) | r;
}

// One entry of stream_specs.h: leaf type, code format and loop shape.
template <int FL, int SZ_, int E_, int M_, int W_>
struct StreamSpec {
    static constexpr bool FLOAT = FL != 0;
    static constexpr int SZ = SZ_;                  // leaf bytes
    static constexpr int E = E_, M = M_, W = W_;    // code format
    static constexpr int LE = SZ == 8 ? 11 : 8;     // leaf float format
    static constexpr int LM = SZ == 8 ? 52 : 23;
    static constexpr int V = stream_vpl(SZ, W);     // records per lane per super-group
    static constexpr int C = V * W;                 // chunk bits per lane = words per super-group
    static constexpr int T = C >= 32 ? 1 : (2 * C >= 32 ? 2 : (4 * C >= 32 ? 4 : 8));
    static constexpr int CC = T * C;                // merged chunk bits (32 .. 64)
    static constexpr int ROUNDS = (C + 31) / 32;    // output words per lane per super-group
    static constexpr int B = 4 / V;                 // super-groups per iteration (4 records per lane)
    // pack: integer codes of 4-record lanes take two super-groups per
    // iteration (two independent shuffle chains; measured faster), floats one
    static constexpr int BP = (V == 4 && !FLOAT) ? 2 : B;
    using Elem = typename std::conditional<SZ == 8, uint64_t, uint32_t>::type;
    using Code = typename std::conditional<(W > 32), uint64_t, uint32_t>::type;
    static constexpr uint64_t CODE_MASK = W >= 64 ? ~0ull : ((1ull << W) - 1ull);
    static_assert(CC >= 32 && CC <= 64, "merged chunks hold 32 to 64 bits");
};

// Words a lane reads for its chunk in unpack: its chunk starts at bit
// (l C) mod 32 of its first word.
template <int C>
constexpr int chunk_read_words()
{
    int most = 0;
    for (int l = 0; l < 32; ++l) {
        const int need = ((l * C) % 32 + C + 31) / 32;
        most = need > most ? need : most;
    }
    return most;
}

// Super-group addressing of a bit stream in the RUNS loops, which also take
// streams organised as AoSoA: blocks of L records, each leaf's L codes one
// run of L W bits (a whole number of words), runs `bstride` bytes apart.
// Word k of super-group g's codes (read as one stream of 32 V W bits) lies at
//   (g >> ksh) * bs + (g & kmask) * step + word_off(k)
// past the leaf's first run:
//   SoA (one run):   ksh 31, kmask all ones, step 4 C, word_off(k) = 4 k;
//   L >= 32 V:       L / (32 V) super-groups per run: ksh = log2 of that,
//                    bs = bstride, step = 4 C, word_off(k) = 4 k;
//   L <  32 V:       R = 32 V / L runs per super-group: ksh 0, kmask 0,
//                    bs = R bstride, step 0, word_off(k) = (k / wpr) bstride
//                    + 4 (k mod wpr), wpr = L W / 32 words per run.
struct SgAddr {
    uint32_t ksh, kmask, bs, step;
    uint32_t lshift, wpr, bstride;  // L < 32 V: run words and stride
    bool split;                     // L < 32 V
};

__device__ __forceinline__ SgAddr sg_addr(const LeafDesc& L, uint32_t V, uint32_t W)
{
    SgAddr A{31u, 0xFFFFFFFFu, 0u, 4u * V * W, 0u, 0u, 0u, false};
    if (L.lanes == 0) return A;
    const uint32_t vsh = V == 4 ? 2u : (V == 2 ? 1u : 0u);
    if (L.lshift >= 5u + vsh) {
        A.ksh = L.lshift - 5u - vsh;
        A.kmask = (1u << A.ksh) - 1u;
        A.bs = L.bstride;
        return A;
    }
    A.split = true;
    A.ksh = 0u;
    A.kmask = 0u;
    A.step = 0u;
    A.bs = (32u * V >> L.lshift) * L.bstride;
    A.lshift = L.lshift;
    A.wpr = (L.lanes * W) >> 5;
    A.bstride = L.bstride;
    return A;
}

__device__ __forceinline__ uint32_t sg_base(const SgAddr& A, uint32_t g) { return (g >> A.ksh) * A.bs + (g & A.kmask) * A.step; }

__device__ __forceinline__ uint32_t sg_word_off(const SgAddr& A, uint32_t k)
{
    if (!A.split) return 4u * k;
    const uint32_t run = k / A.wpr;
    return run * A.bstride + 4u * (k - run * A.wpr);
}

template <class S, bool RUNS>
__device__ __noinline__ void stream_pack(const ItemDesc& I, const JobDesc& J, const uint8_t* simg, uint8_t* dimg,
                                         uint32_t g0, uint32_t g1, uint32_t nvalid)
{
    constexpr int V = S::V, W = S::W, C = S::C, T = S::T, CC = S::CC, ROUNDS = S::ROUNDS, B = S::BP;
    constexpr bool WIDE = CC > 32;              // merged chunks have a high word
    constexpr bool NEXT = (CC % 32) != 0;       // a word can reach into the next merged chunk
    using Elem = typename S::Elem;
    using Code = typename S::Code;
    using Chunk = typename std::conditional<WIDE, uint64_t, uint32_t>::type;
    const uint32_t lane = threadIdx.x & 31u;
    const LaneRun RA = affine_run<V, S::SZ>(J.src.leaves[I.src_leaf], lane);
    const uint32_t sa = smem_addr(simg) + RA.off;
    const LeafDesc& LB = J.dst.leaves[I.dst_leaf];
    const uint32_t da = smem_addr(dimg) + LB.sbase + (RUNS ? 0u : 4u * lane);
    const SgAddr GA = RUNS ? sg_addr(LB, V, W) : SgAddr{};
    // word k = lane + 32 m: merged chunk j0 from bit r on (lane src0), and the
    // next merged chunk (lane src1) from bit 0 on, shifted up by CC - r
    uint32_t src0[ROUNDS], src1[ROUNDS], sh[ROUNDS], up[ROUNDS], koff[ROUNDS];
    bool hisel[ROUNDS], mine[ROUNDS];
#pragma unroll
    for (int m = 0; m < ROUNDS; ++m) {
        const uint32_t k = lane + 32u * m;
        koff[m] = RUNS ? sg_word_off(GA, k < (uint32_t)C ? k : 0u) : 128u * m;
        const uint32_t j0 = 32u * k / CC;
        const uint32_t r = 32u * k - j0 * CC;
        src0[m] = (j0 * T) & 31u;
        src1[m] = ((j0 + 1u) * T) & 31u;
        hisel[m] = r >= 32u;
        sh[m] = r & 31u;
        up[m] = CC - r;
        mine[m] = k < (uint32_t)C;
    }

    // Chunks of one lane (T = 1) that are not a whole number of words: the
    // lane writes every word whose first bit lies in its chunk -- one, or two
    // when a second word starts inside -- and the last of them takes its
    // remaining bits from the low bits of the next lane's chunk, fetched with
    // one shuffle.  One shuffle per super-group instead of three per output
    // word, and each word has a single writer.  The words a lane writes are
    // lane constants, in either organisation.  Where 2 to 4 lanes merge a
    // chunk, the shuffle assembly below was measured faster.
    constexpr bool PIECES = NEXT && T == 1;
    const bool holder = (lane % (uint32_t)T) == 0u;
    const uint32_t cs = (lane / (uint32_t)T) * (uint32_t)CC;  // the merged chunk's first bit
    const uint32_t ka0 = (cs + 31u) >> 5;                       // its first word starting inside
    const uint32_t a0 = 32u * ka0 - cs;                         // ... which starts a0 bits into the chunk
    const bool two_a = ((cs + (uint32_t)CC - 1u) >> 5) > ka0;   // a second word starts inside
    const uint32_t up_last = (uint32_t)CC - (two_a ? a0 + 32u : a0);  // the last word's bits from this chunk (1..32)
    const uint32_t pbase = smem_addr(dimg) + LB.sbase;
    const uint32_t off_a0 = RUNS ? sg_word_off(GA, ka0) : 4u * ka0;
    const uint32_t off_last = two_a ? (RUNS ? sg_word_off(GA, ka0 + 1u) : 4u * ka0 + 4u) : off_a0;

    auto body = [&](uint32_t g, auto check_tag) {
        constexpr bool CHECK = decltype(check_tag)::value;
        Elem x[B][V];
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const uint32_t gg = g + b;
            const uint32_t rec0 = 32u * V * gg + (uint32_t)V * lane;
            if (CHECK) {
#pragma unroll
                for (int v = 0; v < V; ++v) x[b][v] = 0;
                if (gg >= g1 || rec0 >= nvalid) continue;
                if (rec0 + V > nvalid) {
#pragma unroll
                    for (int v = 0; v < V; ++v)
                        x[b][v] = rec0 + v < nvalid ? (Elem)lds<S::SZ>(sa + gg * RA.step + v * RA.vstride) : (Elem)0;
                    continue;
                }
            }
            ld_run<V, S::SZ, Elem>(sa + gg * RA.step, RA, x[b]);
        }
        Code c[B][V];
        if constexpr (S::FLOAT) {
            bool any_bad = false;
#pragma unroll
            for (int b = 0; b < B; ++b)
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    bool bd;
                    c[b][v] = (Code)conv_fast<S::LE, S::LM, S::E, S::M>((uint64_t)x[b][v], bd);
                    any_bad |= bd;
                }
            if (__any_sync(0xFFFFFFFFu, any_bad)) {
#pragma unroll
                for (int b = 0; b < B; ++b)
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        bool bd;
                        conv_fast<S::LE, S::LM, S::E, S::M>((uint64_t)x[b][v], bd);
                        if (bd) c[b][v] = (Code)fconv_general((uint64_t)x[b][v], S::LE, S::LM, S::E, S::M);
                    }
            }
        } else {
#pragma unroll
            for (int b = 0; b < B; ++b)
#pragma unroll
                for (int v = 0; v < V; ++v) c[b][v] = (Code)((uint64_t)x[b][v] & S::CODE_MASK);
        }
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const uint32_t gg = g + b;
            if (CHECK && gg >= g1) break;
            Chunk ch = 0;
#pragma unroll
            for (int v = 0; v < V; ++v) ch |= (Chunk)c[b][v] << (v * W);
#pragma unroll
            for (int d = 1; d < T; d *= 2) {
                const uint32_t p = __shfl_down_sync(0xFFFFFFFFu, (uint32_t)ch, d);
                ch |= (Chunk)p << (C * d);
            }
            const uint32_t lo = (uint32_t)ch;
            const uint32_t hi = WIDE ? (uint32_t)((uint64_t)ch >> 32) : 0u;
            if constexpr (PIECES) {
                const uint32_t nlo = __shfl_down_sync(0xFFFFFFFFu, lo, T);  // the next chunk's low bits
                const uint32_t q = pbase + (RUNS ? sg_base(GA, gg) : gg * (uint32_t)(4 * C));
                if (holder) {
                    const uint32_t first = __funnelshift_r(lo, hi, a0);
                    if (two_a) sts<4>(q + off_a0, first);
                    sts<4>(q + off_last, (two_a ? hi >> a0 : first) | shl_c(nlo, up_last));
                }
                continue;
            }
            const uint32_t q = da + (RUNS ? sg_base(GA, gg) : gg * (uint32_t)(4 * C));
#pragma unroll
            for (int m = 0; m < ROUNDS; ++m) {
                const uint32_t a_lo = __shfl_sync(0xFFFFFFFFu, lo, src0[m]);
                const uint32_t a_hi = WIDE ? __shfl_sync(0xFFFFFFFFu, hi, src0[m]) : 0u;
                const uint32_t nx = NEXT ? __shfl_sync(0xFFFFFFFFu, lo, src1[m]) : 0u;
                uint32_t word = __funnelshift_r(hisel[m] ? a_hi : a_lo, hisel[m] ? 0u : a_hi, sh[m]);
                if (NEXT) word |= shl_c(nx, up[m]);
                if (mine[m]) sts<4>(q + koff[m], word);
            }
        }
    };
    const uint32_t gfull = min(g1, max(g0, nvalid / (32u * V)));  // super-groups below hold valid records only
    uint32_t g = g0;
    for (; g + B <= gfull; g += B) body(g, std::false_type{});
    for (; g < g1; g += B) body(g, std::true_type{});
}

template <class S, bool RUNS>
__device__ __noinline__ void stream_unpack(const ItemDesc& I, const JobDesc& J, const uint8_t* simg, uint8_t* dimg,
                                           uint32_t g0, uint32_t g1, uint32_t nvalid)
{
    constexpr int V = S::V, W = S::W, C = S::C, B = S::B;
    constexpr int NW = chunk_read_words<C>();
    static_assert(NW >= 1 && NW <= 3, "a chunk spans at most three words");
    using Elem = typename S::Elem;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t bit = lane * (uint32_t)C;
    const LeafDesc& LA = J.src.leaves[I.src_leaf];
    const SgAddr GA = RUNS ? sg_addr(LA, V, W) : SgAddr{};
    // the lane's chunk: its first word, and its bit in that word (a run holds
    // a whole number of words, so the bit is the same in every organisation)
    uint32_t woff = 4u * (bit >> 5);
    if (RUNS && GA.split) {
        const uint32_t rl = (uint32_t)V * lane;
        const uint32_t run = rl >> GA.lshift;
        woff = run * GA.bstride + 4u * (((rl - (run << GA.lshift)) * (uint32_t)W) >> 5);
    }
    const uint32_t sa = smem_addr(simg) + LA.sbase + woff;
    const uint32_t sh = bit & 31u;
    const LaneRun RB = affine_run<V, S::SZ>(J.dst.leaves[I.dst_leaf], lane);
    const uint32_t da = smem_addr(dimg) + RB.off;
    const bool sgn = I.is_signed != 0;

    auto body = [&](uint32_t g, auto check_tag) {
        constexpr bool CHECK = decltype(check_tag)::value;
        uint64_t c[B][V];
#pragma unroll
        for (int b = 0; b < B; ++b) {
            if (CHECK && g + b >= g1) {  // past the share: nothing to read
#pragma unroll
                for (int v = 0; v < V; ++v) c[b][v] = 0;
                continue;
            }
            const uint32_t p = sa + (RUNS ? sg_base(GA, g + b) : (g + b) * (uint32_t)(4 * C));
            const uint32_t w0 = (uint32_t)lds<4>(p);
            const uint32_t w1 = NW > 1 ? (uint32_t)lds<4>(p + 4u) : 0u;
            const uint32_t w2 = NW > 2 ? (uint32_t)lds<4>(p + 8u) : 0u;
            const uint64_t chunk = ((uint64_t)__funnelshift_r(w1, w2, sh) << 32) | __funnelshift_r(w0, w1, sh);
#pragma unroll
            for (int v = 0; v < V; ++v) c[b][v] = (chunk >> (v * W)) & S::CODE_MASK;
        }
        Elem x[B][V];
        if constexpr (S::FLOAT) {
            bool any_bad = false;
#pragma unroll
            for (int b = 0; b < B; ++b)
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    bool bd;
                    x[b][v] = (Elem)conv_fast<S::E, S::M, S::LE, S::LM>(c[b][v], bd);
                    any_bad |= bd;
                }
            if (__any_sync(0xFFFFFFFFu, any_bad)) {
#pragma unroll
                for (int b = 0; b < B; ++b)
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        bool bd;
                        conv_fast<S::E, S::M, S::LE, S::LM>(c[b][v], bd);
                        if (bd) x[b][v] = (Elem)fconv_general(c[b][v], S::E, S::M, S::LE, S::LM);
                    }
            }
        } else {
            constexpr uint32_t UP = 32u - (uint32_t)W;
#pragma unroll
            for (int b = 0; b < B; ++b)
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const uint32_t u = (uint32_t)c[b][v];
                    x[b][v] = sgn ? (uint32_t)(((int32_t)(u << UP)) >> UP) : u;
                }
        }
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const uint32_t gg = g + b;
            if (CHECK && gg >= g1) break;
            const uint32_t rec0 = 32u * V * gg + (uint32_t)V * lane;
            if (CHECK && rec0 + V > nvalid) {
#pragma unroll
                for (int v = 0; v < V; ++v)
                    if (rec0 + v >= nvalid) x[b][v] = 0;
            }
            st_run<V, S::SZ, Elem>(da + gg * RB.step, RB, x[b]);
        }
    };
    const uint32_t gfull = min(g1, max(g0, nvalid / (32u * V)));
    uint32_t g = g0;
    for (; g + B <= gfull; g += B) body(g, std::false_type{});
    for (; g < g1; g += B) body(g, std::true_type{});
}

// Runs a VALUE item over quads [q0, q1) (128 records each) in the loop of its
// compile-time format (ItemDesc::spec); false when it has none.
// RUNS: the loops that also address AoSoA-organised streams (kernel mode 3).
template <bool RUNS>
__device__ __forceinline__ bool run_spec(const ItemDesc& I, const JobDesc& J, const uint8_t* simg, uint8_t* dimg,
                                         uint32_t q0, uint32_t q1, uint32_t nvalid)
{
    const bool pack = I.sop == S_BITS_INT || I.sop == S_BITS_FLOAT;
    switch (I.spec) {
#define LLGB_SPEC_CASE(id, fl, sz, e, m, w, ao)                                                            \
    case id: {                                                                                             \
        using S = StreamSpec<fl, sz, e, m, w>;                                                             \
        if constexpr (ao && !RUNS) {                                                                       \
            return false;                                                                                  \
        } else {                                                                                           \
            if (pack) stream_pack<S, RUNS>(I, J, simg, dimg, q0 * (4u / S::V), q1 * (4u / S::V), nvalid);\
            else stream_unpack<S, RUNS>(I, J, simg, dimg, q0 * (4u / S::V), q1 * (4u / S::V), nvalid);   \
            return true;                                                                                   \
        }                                                                                                  \
    }
        LLGB_STREAM_SPECS(LLGB_SPEC_CASE)
#undef LLGB_SPEC_CASE
    default: return false;
    }
}

}  // namespace llgb
