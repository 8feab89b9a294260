// lp_mixed.cu -- mixed-precision batched simplex with the FP32 condensed
// tableau in shared memory: one CTA per LP (mixed_kernel), one warp per LP
// (mixed_warp_kernel) or persistent CTAs over a list (mixed_queue_kernel).
// The per-LP code (FP32 Steps 1-3, FP64 certificate) is mixed_solve in
// lp_mixed_solve.cuh.  This path has no counterpart in the paper (which is
// FP64 only).

#include "lp_mixed_solve.cuh"

namespace lpb {
namespace {

__global__ void __launch_bounds__(kMaxThreads, 2)
mixed_kernel(const DeviceBatch B, const Tolerances tol, const MixedParams mp, const int32_t* __restrict__ order,
             const FallbackQueues fq, int32_t* __restrict__ diag)
{
    extern __shared__ __align__(16) unsigned char smem[];
    BlockGroup g(reinterpret_cast<long long*>(smem + SmallLayout::red64),
                 reinterpret_cast<unsigned*>(smem + SmallLayout::red32));
    mixed_solve_lp(g, B, tol, mp, order[blockIdx.x], smem + SmallLayout::total, fq, diag);
}

// Persistent CTAs over a list: LP order[idx] for idx taken from an atomic
// counter (0 at launch) until *count is reached.
__global__ void __launch_bounds__(kMaxThreads, 2)
mixed_queue_kernel(const DeviceBatch B, const Tolerances tol, const MixedParams mp, const int32_t* __restrict__ order,
                   const int32_t* __restrict__ count, int32_t* __restrict__ counter, const FallbackQueues fq,
                   int32_t* __restrict__ diag)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int next;
    const int n_items = *count;
    for (;;) {
        if (threadIdx.x == 0) next = atomicAdd(counter, 1);
        __syncthreads();
        const int idx = next;
        __syncthreads();
        if (idx >= n_items) break;
        BlockGroup g(reinterpret_cast<long long*>(smem + SmallLayout::red64),
                     reinterpret_cast<unsigned*>(smem + SmallLayout::red32));
        mixed_solve_lp(g, B, tol, mp, order[idx], smem + SmallLayout::total, fq, diag);
        __syncthreads();
    }
}

// One warp per LP (blockDim = 32): for small tableaux, where a whole CTA per
// LP mostly waits at barriers.
__global__ void __launch_bounds__(32, 32)
mixed_warp_kernel(const DeviceBatch B, const Tolerances tol, const MixedParams mp, const int32_t* __restrict__ order,
                  const FallbackQueues fq, int32_t* __restrict__ diag)
{
    extern __shared__ __align__(16) unsigned char smem[];
    WarpGroup g;
    mixed_solve_lp(g, B, tol, mp, order[blockIdx.x], smem, fq, diag);
}

}  // namespace

cudaError_t mixed_kernel_prepare() {
    cudaError_t err = cudaFuncSetAttribute(mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)(kMaxSmemPerBlock - 1024));
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(mixed_queue_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(kMaxSmemPerBlock - 1024));
    if (err != cudaSuccess) return err;
    return cudaFuncSetAttribute(mixed_warp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(kMaxSmemPerBlock - 1024));
}

cudaError_t launch_mixed(const DeviceBatch& B, const Tolerances& tol, const MixedParams& mp,
                         const int32_t* order, int32_t count, int threads, size_t smem,
                         const FallbackQueues& fq, int32_t* diag, cudaStream_t stream) {
    if (count <= 0) return cudaSuccess;
    if (threads == 32)
        mixed_warp_kernel<<<count, 32, smem, stream>>>(B, tol, mp, order, fq, diag);
    else
        mixed_kernel<<<count, threads, smem, stream>>>(B, tol, mp, order, fq, diag);
    return cudaGetLastError();
}

int mixed_queue_ctas_per_sm(int threads, size_t smem) {
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, mixed_queue_kernel, threads, smem) != cudaSuccess)
        return 1;
    return blocks > 0 ? blocks : 1;
}

cudaError_t launch_mixed_queue(const DeviceBatch& B, const Tolerances& tol, const MixedParams& mp,
                               const int32_t* order, const int32_t* count, int32_t* counter, int ctas, int threads,
                               size_t smem, const FallbackQueues& fq, int32_t* diag, cudaStream_t stream) {
    cudaError_t err = cudaMemsetAsync(counter, 0, sizeof(int32_t), stream);
    if (err != cudaSuccess) return err;
    mixed_queue_kernel<<<ctas, threads, smem, stream>>>(B, tol, mp, order, count, counter, fq, diag);
    return cudaGetLastError();
}

}  // namespace lpb
