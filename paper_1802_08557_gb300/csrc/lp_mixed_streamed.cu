// lp_mixed_streamed.cu -- mixed-precision simplex for LPs whose FP32 tableau
// exceeds one CTA's shared memory (and the single-launch form, which also
// takes such LPs): the same per-LP code as the shared-memory
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

// A whole mixed-precision batch in one launch (LPB_SCHED_SINGLE): persistent
// CTAs take the LPs order[0 .. count) (longest work first within each part)
// from the atomic `counter`.  Block mode, order[0 .. warp_from): the CTA
// solves each LP with its area in the CTA's shared memory when it fits
// (resident[lp] != 0), else in this CTA's global workspace slot.  Warp mode,
// from the first index >= warp_from a CTA draws: every warp takes its own
// LPs (the small ones, listed last), warp w working in
// smem + w * kMixedSingleWarpArea, claiming its next LP before it solves the
// current one.  The per-LP code is that of the other mixed kernels, so the
// same results.  The FP64 re-solves of the LPs it does not certify stay
// separate launches: they need the whole pass's queues.
__global__ void __launch_bounds__(kMixedSingleThreads, 2)
mixed_single_kernel(const DeviceBatch B, const Tolerances tol, const MixedParams mp,
                    const int32_t* __restrict__ order, const uint8_t* __restrict__ resident, const int32_t count,
                    const int32_t warp_from, unsigned char* workspace, const size_t slot_bytes,
                    int32_t* __restrict__ counter, const FallbackQueues fq, int32_t* __restrict__ diag)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int next;
    unsigned char* slot = workspace ? workspace + (size_t)blockIdx.x * slot_bytes : nullptr;
    int first = count;
    for (;;) {
        if (threadIdx.x == 0) next = atomicAdd(counter, 1);
        __syncthreads();
        const int idx = next;
        __syncthreads();
        if (idx >= count) return;
        if (idx >= warp_from) {
            first = idx;
            break;
        }
        const int lp = order[idx];
        BlockGroup g(reinterpret_cast<long long*>(smem + SmallLayout::red64),
                     reinterpret_cast<unsigned*>(smem + SmallLayout::red32));
        if (resident[lp])
            mixed_solve_lp(g, B, tol, mp, lp, smem + SmallLayout::total, fq, diag);
        else if (slot)
            mixed_solve_lp(g, B, tol, mp, lp, slot, fq, diag);
        else if (threadIdx.x == 0)
            record_internal_error(diag, 7, lp);  // a plan without a slot for a streamed LP
        __syncthreads();
    }
    // warp mode (every thread of the CTA got here with the same `first`)
    const int w = (int)(threadIdx.x >> 5);
    const bool leader = (threadIdx.x & 31) == 0;
    unsigned char* area = smem + (size_t)w * kMixedSingleWarpArea;
    int idx = (w == 0) ? first : __shfl_sync(0xffffffffu, leader ? atomicAdd(counter, 1) : 0, 0);
    while (idx < count) {
        const int nxt = leader ? atomicAdd(counter, 1) : 0;
        WarpGroup g;
        mixed_solve_lp(g, B, tol, mp, order[idx], area, fq, diag);
        idx = __shfl_sync(0xffffffffu, nxt, 0);
    }
}

}  // namespace

cudaError_t mixed_single_prepare(size_t smem) {
    return cudaFuncSetAttribute(mixed_single_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

int mixed_single_ctas_per_sm(size_t smem) {
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, mixed_single_kernel, kMixedSingleThreads, smem) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return blocks;
}

cudaError_t launch_mixed_single(const DeviceBatch& B, const Tolerances& tol, const MixedParams& mp,
                                const int32_t* order, const uint8_t* resident, int32_t count, int32_t warp_from,
                                int ctas, size_t smem, unsigned char* workspace, size_t slot_bytes,
                                int32_t* counter, const FallbackQueues& fq, int32_t* diag, cudaStream_t stream) {
    if (count <= 0) return cudaSuccess;
    // warp mode needs every warp's area
    if (warp_from < count && smem < kMixedSingleSmemCap) return cudaErrorInvalidValue;
    cudaError_t err = cudaMemsetAsync(counter, 0, sizeof(int32_t), stream);
    if (err != cudaSuccess) return err;
    mixed_single_kernel<<<ctas, kMixedSingleThreads, smem, stream>>>(B, tol, mp, order, resident, count, warp_from,
                                                                      workspace, slot_bytes, counter, fq, diag);
    return cudaGetLastError();
}

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
