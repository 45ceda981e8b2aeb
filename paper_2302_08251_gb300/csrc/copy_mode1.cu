// copy_mode1.cu -- kernel mode 1 of the copy kernel: value loops with the
// run-addressed loop of AoSoA-organised bit leaves (copy_kernel.cuh).
#include "copy_kernel.cuh"

namespace llgb {

cudaError_t launch_mode1(const CopyArgs& args, int grid, int threads, size_t smem, cudaStream_t stream)
{
    return launch_mode<1>(args, grid, threads, smem, stream);
}

cudaError_t prepare_mode1(size_t smem) { return prepare_mode<1>(smem); }

cudaError_t status_mode1(unsigned* out, bool reset) { return unit_status(out, reset); }

}  // namespace llgb
