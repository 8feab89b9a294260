// lp_mixed_streamed.cu -- mixed-precision simplex for LPs whose FP32 tableau
// exceeds one CTA's shared memory: the same per-LP code as the shared-memory
// kernels (mixed_solve: FP32 Steps 1-3 of Section 3, FP64 certificate), with
// the LP's area (certificate vectors, labels, FP32 tableau) in a global
// workspace slot instead.  Persistent CTAs take LPs from an atomic counter;
// CTA i owns slot i.  The arithmetic of an LP does not depend on where its
// tableau lives or on the number of threads, so the results are bit-identical
// to the shared-memory kernels' (tested).
//
// Compiled with -dlcm=cg (global loads cached in L2 only), like the FP64
// streamed kernel: the tableau is rewritten every pivot and gets no reuse
// from L1.  Two CTAs per SM (64 registers): the kernel waits on L2 latency,
// and twice the warps in flight measured 9% faster than one CTA with 128.

#include "lp_mixed_solve.cuh"

namespace lpb {
namespace {

__global__ void __launch_bounds__(kMixedStreamedThreads, 2)
mixed_streamed_kernel(const DeviceBatch B, const Tolerances tol, const MixedParams mp,
                      const int32_t* __restrict__ order, const int32_t count, unsigned char* workspace,
                      const size_t slot_bytes, int32_t* __restrict__ counter, const FallbackQueues fq,
                      int32_t* __restrict__ diag)
{
    __shared__ __align__(16) unsigned char small[SmallLayout::total];
    __shared__ int next;
    unsigned char* big = workspace + (size_t)blockIdx.x * slot_bytes;
    for (;;) {
        if (threadIdx.x == 0) next = atomicAdd(counter, 1);
        __syncthreads();
        const int idx = next;
        __syncthreads();
        if (idx >= count) break;
        BlockGroup g(reinterpret_cast<long long*>(small + SmallLayout::red64),
                     reinterpret_cast<unsigned*>(small + SmallLayout::red32));
        mixed_solve_lp(g, B, tol, mp, order[idx], big, fq, diag);
        __syncthreads();
    }
}

}  // namespace

int mixed_streamed_ctas_per_sm() {
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, mixed_streamed_kernel, kMixedStreamedThreads, 0) !=
        cudaSuccess)
        return 1;
    return blocks > 0 ? blocks : 1;
}

cudaError_t launch_mixed_streamed(const DeviceBatch& B, const Tolerances& tol, const MixedParams& mp,
                                  const int32_t* order, int32_t count, int slots, unsigned char* workspace,
                                  size_t slot_bytes, int32_t* counter, const FallbackQueues& fq, int32_t* diag,
                                  cudaStream_t stream) {
    if (count <= 0) return cudaSuccess;
    cudaError_t err = cudaMemsetAsync(counter, 0, sizeof(int32_t), stream);
    if (err != cudaSuccess) return err;
    mixed_streamed_kernel<<<slots, kMixedStreamedThreads, 0, stream>>>(B, tol, mp, order, count, workspace,
                                                                        slot_bytes, counter, fq, diag);
    return cudaGetLastError();
}

}  // namespace lpb
