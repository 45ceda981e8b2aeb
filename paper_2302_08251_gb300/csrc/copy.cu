// copy.cu -- host dispatch of the copy kernel modes, the device status words
// and the bounded-wait self-test.
//
// The kernel itself is in copy_kernel.cuh; each mode is compiled in its own
// translation unit (copy_mode0.cu, copy_mode1.cu, copy_mode3.cu, copy_gather.cu).
#include "copy_kernel.cuh"

namespace llgb {

// per translation unit (copy_mode0.cu, copy_mode1.cu, copy_gather.cu)
cudaError_t launch_mode0(const CopyArgs& args, int grid, int threads, size_t smem, cudaStream_t stream);
cudaError_t prepare_mode0(size_t smem);
cudaError_t status_mode0(unsigned* out, bool reset);
cudaError_t launch_mode1(const CopyArgs& args, int grid, int threads, size_t smem, cudaStream_t stream);
cudaError_t prepare_mode1(size_t smem);
cudaError_t status_mode1(unsigned* out, bool reset);
cudaError_t launch_mode3(const CopyArgs& args, int grid, int threads, size_t smem, cudaStream_t stream);
cudaError_t prepare_mode3(size_t smem);
cudaError_t status_mode3(unsigned* out, bool reset);
cudaError_t launch_gather(const CopyArgs& args, int mode, int grid, int threads, size_t smem, cudaStream_t stream);
cudaError_t prepare_gather(int mode, size_t smem);
cudaError_t status_gather(unsigned* out, bool reset);

// Self-test of the failure path: one CTA waits, through the copy kernel's
// bounded wait, on an mbarrier that no thread ever arrives on.  The wait
// gives up after limit_ns and the kernel records LLGB_ERR_TIMEOUT in the
// device status word, as a copy kernel does when one of its waits runs out;
// then it returns.  `waited_ns` (may be null) receives the time it waited.
__global__ void wait_selftest_kernel(uint64_t limit_ns, unsigned long long* waited_ns)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint64_t t0 = global_timer_ns();
        const bool completed = mbar_wait_bounded(&bar, 0u, limit_ns);
        const uint64_t t1 = global_timer_ns();
        if (!completed) atomicOr(&g_device_status, (unsigned)LLGB_ERR_TIMEOUT);
        if (waited_ns) *waited_ns = t1 - t0;
    }
}

cudaError_t launch_wait_selftest(uint64_t limit_ns, unsigned long long* waited_ns, cudaStream_t stream)
{
    wait_selftest_kernel<<<1, 32, 0, stream>>>(limit_ns, waited_ns);
    return cudaGetLastError();
}

size_t copy_shared_header_bytes() { return (sizeof(CopyShared) + 15u) & ~size_t(15); }

int gather_words_per_thread(int mode) { return mode == 2 ? GatherMax<2>::value : (mode == 4 ? GatherMax<4>::value : 0); }

cudaError_t prepare_copy(int mode, size_t smem_bytes)
{
    switch (mode) {
    case 1: return prepare_mode1(smem_bytes);
    case 3: return prepare_mode3(smem_bytes);
    case 2:
    case 4: return prepare_gather(mode, smem_bytes);
    default: return prepare_mode0(smem_bytes);
    }
}

cudaError_t launch_copy(const CopyArgs& args, int mode, int grid, int threads, size_t smem_bytes,
                        cudaStream_t stream)
{
    switch (mode) {
    case 1: return launch_mode1(args, grid, threads, smem_bytes, stream);
    case 3: return launch_mode3(args, grid, threads, smem_bytes, stream);
    case 2:
    case 4: return launch_gather(args, mode, grid, threads, smem_bytes, stream);
    default: return launch_mode0(args, grid, threads, smem_bytes, stream);
    }
}

cudaError_t read_device_status(unsigned* out, bool reset)
{
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return e;
    *out = 0;
    if ((e = unit_status(out, reset)) != cudaSuccess) return e;  // this unit: the self-test
    if ((e = status_mode0(out, reset)) != cudaSuccess) return e;
    if ((e = status_mode1(out, reset)) != cudaSuccess) return e;
    if ((e = status_mode3(out, reset)) != cudaSuccess) return e;
    return status_gather(out, reset);
}

}  // namespace llgb
