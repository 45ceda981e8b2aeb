// copy_mode0.cu -- kernel mode 0 of the copy kernel: value loops (copy_kernel.cuh).
#include "copy_kernel.cuh"

namespace llgb {

cudaError_t launch_mode0(const CopyArgs& args, int grid, int threads, size_t smem, cudaStream_t stream)
{
    return launch_mode<0>(args, grid, threads, smem, stream);
}

cudaError_t prepare_mode0(size_t smem) { return prepare_mode<0>(smem); }

cudaError_t status_mode0(unsigned* out, bool reset) { return unit_status(out, reset); }

}  // namespace llgb
