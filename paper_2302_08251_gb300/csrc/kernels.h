// kernels.h -- host-side entry points of the CUDA kernels.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "job.h"

namespace llgb {

// copy.cu
// mode 0: general kernel; 2 / 4: gather kernel of that form (every job of the
// launch must have JobDesc::gather == mode and fit its words per thread).
cudaError_t launch_copy(const CopyArgs& args, int mode, int grid, int threads, size_t smem_bytes,
                        cudaStream_t stream);
int gather_words_per_thread(int mode);
// copy_gather.cu: a job's gather program for CTAs of `consumers` consumer
// threads (JobDesc::program), built on the GPU into `out`, which holds
// gather_program_words(mode, consumers) words.
size_t gather_program_words(int mode, uint32_t consumers);
cudaError_t launch_gather_program(const JobDesc& job, int mode, uint32_t consumers, uint32_t* out,
                                  cudaStream_t stream);
// Raise the copy kernel's dynamic shared memory limit for `mode` to smem_bytes
// (done by launch_copy too; call it before capturing a graph).
cudaError_t prepare_copy(int mode, size_t smem_bytes);
size_t copy_shared_header_bytes();
cudaError_t read_device_status(unsigned* out, bool reset);
// The bounded-wait self-test kernel (one CTA waits limit_ns on an mbarrier
// nothing arrives on, then records LLGB_ERR_TIMEOUT).
cudaError_t launch_wait_selftest(uint64_t limit_ns, unsigned long long* waited_ns, cudaStream_t stream);

// nbody.cu: a particle view.  Leaf f of record i lies at base[f] + off(i),
//   AoS     off(i) = 28 i                       (lanes 1,  bstride 28)
//   SoA     off(i) = 4 i                        (lanes 0xFFFFFFFF: one block)
//   AoSoA   off(i) = (i / L) bstride + (i % L) 4 (lanes L, bstride 28 L)
// lshift / lmask hold log2 L and L - 1 when L is a power of two (AoS and SoA:
// 0 and 0 with bstride 28 and 4).  step_lanes / step_off / wrap_off advance a
// (block, lane) cursor by 32 records without a division: lane += step_lanes,
// offset += step_off, and on passing the last lane, lane -= L and offset +=
// wrap_off.
struct ParticleView {
    uint8_t* base[7];
    uint32_t bstride;
    uint32_t lshift;
    uint32_t lmask;
    uint32_t n;
    uint32_t lanes;
    uint32_t step_lanes;
    uint64_t step_off;
    uint64_t wrap_off;
};

// Address kinds of the index traversal: compile-time AoS, SoA, AoSoA32;
// PV_GENERIC shift / mask (power-of-two lanes); PV_DIV divides by the lane
// count.
enum { PV_AOS = 0, PV_SOA = 1, PV_AOSOA32 = 2, PV_GENERIC = 3, PV_DIV = 4 };

// Traversals (the paper's open point in Sec. 5): INDEX walks the flat record
// index and maps every access through the mapping; BLOCKS nests the walk the
// way the mapping lays records out (blocks, then lanes).
enum { TRAVERSE_INDEX = 0, TRAVERSE_BLOCKS = 1 };

// Access instrumentation of the n-body kernels (Sec. 4): FieldAccessCount
// counters (reads of leaves 0..6, then writes) and Heatmap counters (per
// granule of 2^gshift bytes; leaf f's element of record i is at byte
// boff[f] + offset(i) of its blob, whose counters start at hstart[f]).
struct NbodyInstr {
    unsigned long long* counts;  // 14 counters, or nullptr
    unsigned long long* heat;    // heatmap counters, or nullptr
    uint64_t boff[7];
    uint64_t hstart[7];
    uint32_t gshift;
    int count_mode;              // 1: global atomic per access; 2: per-block counters
};

cudaError_t launch_nbody(const ParticleView& v, int kind, int layout, float eps, float dt, cudaStream_t stream);
// One phase with a chosen traversal: the update (velocities) or the move
// (positions).  `layout` is 0 AoS, 1 SoA, 2 AoSoA.
cudaError_t launch_nbody_update(const ParticleView& v, int kind, int traversal, float eps, float dt,
                                cudaStream_t stream);
cudaError_t launch_nbody_move(const ParticleView& v, int kind, int layout, int traversal, float dt,
                              cudaStream_t stream);
// div: the view is AoSoA with a lane count that is not a power of two.
// FP32 FMA throughput probe: *fmas receives the FMAs the launch performs.
cudaError_t launch_fma_probe(uint32_t iters, float* sink, uint64_t* fmas, cudaStream_t stream);
cudaError_t launch_nbody_instrumented(const ParticleView& v, bool div, const NbodyInstr& ins, float eps, float dt,
                                      cudaStream_t stream);

}  // namespace llgb
