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

size_t gather_program_words(int mode, uint32_t consumers)
{
    const uint32_t K = mode == 4 ? GatherMax<4>::value : GatherMax<2>::value;
    const uint32_t F = mode == 4 ? gather_program_fields<4>() : gather_program_fields<2>();
    return kProgramHeader + (size_t)K * F * consumers;
}

cudaError_t launch_gather_program(const JobDesc& job, int mode, uint32_t consumers, uint32_t* out, cudaStream_t stream)
{
    const uint32_t K = mode == 4 ? GatherMax<4>::value : GatherMax<2>::value;
    const uint32_t threads = 256, blocks = (K * consumers + threads - 1) / threads;
    if (mode == 4)
        gather_program_kernel<4><<<blocks, threads, 0, stream>>>(job, consumers, out);
    else
        gather_program_kernel<2><<<blocks, threads, 0, stream>>>(job, consumers, out);
    return cudaGetLastError();
}

}  // namespace llgb
