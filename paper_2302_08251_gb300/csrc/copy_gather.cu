// copy_gather.cu -- kernel modes 2 and 4 of the copy kernel: gather programs
// of 2 and 4 source words for jobs made of byte moves (copy_kernel.cuh).
#include "copy_kernel.cuh"

namespace llgb {

cudaError_t launch_gather(const CopyArgs& args, int mode, int grid, int threads, size_t smem, cudaStream_t stream)
{
    return mode == 4 ? launch_mode<4>(args, grid, threads, smem, stream) : launch_mode<2>(args, grid, threads, smem, stream);
}

cudaError_t prepare_gather(int mode, size_t smem) { return mode == 4 ? prepare_mode<4>(smem) : prepare_mode<2>(smem); }

cudaError_t status_gather(unsigned* out, bool reset) { return unit_status(out, reset); }

}  // namespace llgb
