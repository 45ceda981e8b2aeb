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

cudaError_t launch_nbody(const ParticleView& v, int kind, float eps, float dt, cudaStream_t stream);

}  // namespace llgb
