// copy_mode3.cu -- kernel mode 3 of the copy kernel: value loops with the
// compile-time stream loops of bit leaves organised as AoSoA (copy_kernel.cuh).
#include "copy_kernel.cuh"

namespace llgb {

cudaError_t launch_mode3(const CopyArgs& args, int grid, int threads, size_t smem, cudaStream_t stream)
{
    return launch_mode<3>(args, grid, threads, smem, stream);
}

cudaError_t prepare_mode3(size_t smem) { return prepare_mode<3>(smem); }

cudaError_t status_mode3(unsigned* out, bool reset) { return unit_status(out, reset); }

}  // namespace llgb
