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
// Raise the copy kernel's dynamic shared memory limit for `mode` to smem_bytes
// (done by launch_copy too; call it before capturing a graph).
cudaError_t prepare_copy(int mode, size_t smem_bytes);
size_t copy_shared_header_bytes();
cudaError_t read_device_status(unsigned* out, bool reset);

// nbody.cu: a particle view, leaf f of record i at
//   base[f] + (i >> lshift) * bstride + (i & lmask) * 4.
struct ParticleView {
    uint8_t* base[7];
    uint32_t bstride;
    uint32_t lshift;
    uint32_t lmask;
    uint32_t n;
};

enum { PV_AOS = 0, PV_SOA = 1, PV_AOSOA32 = 2, PV_GENERIC = 3 };

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

cudaError_t launch_nbody(const ParticleView& v, int kind, float eps, float dt, cudaStream_t stream);
cudaError_t launch_nbody_instrumented(const ParticleView& v, const NbodyInstr& ins, float eps, float dt,
                                      cudaStream_t stream);

}  // namespace llgb
