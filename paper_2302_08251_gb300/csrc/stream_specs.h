// stream_specs.h -- bit-stream formats with loops specialised at compile time.
//
// BitpackIntSoA and BitpackFloatSoA (Sec. 3 of the paper) take their bit
// count, or exponent and mantissa widths, as parameters that may be known at
// compile time.  The formats listed here -- the integer widths and float
// formats of the benchmarked workloads -- get pack and unpack loops whose
// widths, shifts and conversions are constants; any other format runs the
// loops with run-time widths.  The planner (plan.cpp) marks a VALUE item with
// the entry's id when it moves a 4- or 8-byte leaf of a SoA-like view to or
// from a bit stream of a listed format; the copy kernel (copy_kernel.cuh)
// instantiates one loop per entry and direction: for SoA streams in kernel
// mode 0, for streams organised as AoSoA in kernel mode 3.
#pragma once

#include <stdint.h>

namespace llgb {

// X(id, is_float, leaf bytes, exponent bits, mantissa bits, stream bits, AoSoA only)
//   integers: 4-byte leaves stored in 1, 3, 7, 12, 17 or 31 bits;
//   floats:   f64 or f32 leaves stored as (E, M) with E in {5, 8, 11} and
//             M in {2, 10, 23, 52}; the pairs that are plain f32 or f64
//             element moves (f64 as E8M23 and E11M52, f32 as E8M23) have
//             loops of their own for SoA streams and use these only for
//             streams organised as AoSoA.
#define LLGB_STREAM_SPECS(X)                                                                                       \
    X(1, 0, 4, 0, 0, 1, 0) X(2, 0, 4, 0, 0, 3, 0) X(3, 0, 4, 0, 0, 7, 0) X(4, 0, 4, 0, 0, 12, 0)                    \
    X(5, 0, 4, 0, 0, 17, 0) X(6, 0, 4, 0, 0, 31, 0)                                                                \
    X(7, 1, 8, 5, 2, 8, 0) X(8, 1, 8, 5, 10, 16, 0) X(9, 1, 8, 5, 23, 29, 0) X(10, 1, 8, 5, 52, 58, 0)              \
    X(11, 1, 8, 8, 2, 11, 0) X(12, 1, 8, 8, 10, 19, 0) X(13, 1, 8, 8, 52, 61, 0)                                    \
    X(14, 1, 8, 11, 2, 14, 0) X(15, 1, 8, 11, 10, 22, 0) X(16, 1, 8, 11, 23, 35, 0)                                 \
    X(17, 1, 4, 5, 2, 8, 0) X(18, 1, 4, 5, 10, 16, 0) X(19, 1, 4, 5, 23, 29, 0) X(20, 1, 4, 5, 52, 58, 0)           \
    X(21, 1, 4, 8, 2, 11, 0) X(22, 1, 4, 8, 10, 19, 0) X(23, 1, 4, 8, 52, 61, 0)                                    \
    X(24, 1, 4, 11, 2, 14, 0) X(25, 1, 4, 11, 10, 22, 0) X(26, 1, 4, 11, 23, 35, 0) X(27, 1, 4, 11, 52, 64, 0)      \
    X(28, 1, 8, 8, 23, 32, 1) X(29, 1, 8, 11, 52, 64, 1) X(30, 1, 4, 8, 23, 32, 1)

// Consecutive records each lane takes per super-group of 32 V records, by
// code width alone: codes of at most 64 bits per lane, and for codes under 16
// bits a lane chunk of 32 bits or more, which needs no merging over lanes
// (f64 leaves of such codes then take two 16-byte vectors per lane: measured
// 8-10% faster on their packs than two records per lane merged over two
// lanes, and within 2% on their unpacks).
constexpr int stream_vpl(int /* leaf bytes */, int bits)
{
    return bits >= 32 ? 1 : (bits >= 16 ? 2 : 4);
}

struct StreamSpecInfo {
    int id, is_float, leaf_bytes, exp, man, bits, aosoa_only;
};

constexpr StreamSpecInfo kStreamSpecs[] = {
#define LLGB_SPEC_ROW(id, fl, sz, e, m, w, ao) {id, fl, sz, e, m, w, ao},
    LLGB_STREAM_SPECS(LLGB_SPEC_ROW)
#undef LLGB_SPEC_ROW
};

}  // namespace llgb
