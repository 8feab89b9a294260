// lp_peaks.cu -- throughput microbenchmarks of the units the solver's kernels
// are bound by: the FP64 FMA pipe, the FP32 FMA pipe and shared-memory
// bandwidth.  They give the denominators of the roofline fractions that the
// benchmark reports for the resident kernels (the copy bandwidth of HBM and
// the BF16 tensor peak are measured elsewhere).  No counterpart in the paper.
//
// Each kernel keeps its data in registers or shared memory, runs long enough
// (milliseconds) for launch overhead to vanish, and writes one value per
// thread so that the compiler keeps the work.

#include <algorithm>

#include "lp_internal.h"
#include "lpbatch.h"

namespace lpb {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kFp64Chains = 8;
constexpr int kFp32Chains = 16;
constexpr int kSmemSlots = 4;  // float4 slots per thread

// Independent FMA chains per thread: a <- a*m + c.  With |m| < 1 and small c
// the values stay bounded and normal.
__global__ void __launch_bounds__(kPeakThreads) peak_fp64_kernel(double* out, int iters, double m, double c) {
    double a[kFp64Chains];
#pragma unroll
    for (int i = 0; i < kFp64Chains; ++i) a[i] = 1.0 + 1e-3 * (threadIdx.x + i);
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int i = 0; i < kFp64Chains; ++i) a[i] = fma(a[i], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kFp64Chains; ++i) s += a[i];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kPeakThreads) peak_fp32_kernel(float* out, int iters, float m, float c) {
    float a[kFp32Chains];
#pragma unroll
    for (int i = 0; i < kFp32Chains; ++i) a[i] = 1.0f + 1e-3f * (threadIdx.x + i);
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int i = 0; i < kFp32Chains; ++i) a[i] = fmaf(a[i], m, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < kFp32Chains; ++i) s += a[i];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// 16-byte shared-memory loads and stores: each thread reads, changes and
// writes back its own slots (no two threads touch one slot), consecutive
// threads on consecutive 16-byte words (no bank conflicts).
__global__ void __launch_bounds__(kPeakThreads) peak_smem_kernel(float* out, int iters) {
    __shared__ float4 buf[kSmemSlots * kPeakThreads];
    const int t = threadIdx.x;
#pragma unroll
    for (int j = 0; j < kSmemSlots; ++j) buf[t + j * kPeakThreads] = make_float4(t, j, 1.0f, 2.0f);
    __syncthreads();
    // explicit ld/st.shared: the compiler may not keep a thread's own slots
    // in registers across the loop
    const unsigned base = static_cast<unsigned>(__cvta_generic_to_shared(&buf[t]));
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int j = 0; j < kSmemSlots; ++j) {
            const unsigned a = base + j * kPeakThreads * 16;
            float4 v;
            asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
            v.x += 1.0f;
            v.w += v.x;
            asm volatile("st.shared.v4.f32 [%0], {%1,%2,%3,%4};" ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                         : "memory");
        }
    }
    __syncthreads();
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < kSmemSlots; ++j) s += buf[t + j * kPeakThreads].w;
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Best time of `reps` launches of `launch` (CUDA events on `s`).
template <typename F>
cudaError_t best_ms(F launch, cudaStream_t s, int reps, float* ms) {
    cudaEvent_t e0, e1;
    cudaError_t err;
    if ((err = cudaEventCreate(&e0))) return err;
    if ((err = cudaEventCreate(&e1))) {
        cudaEventDestroy(e0);
        return err;
    }
    float best = 1e30f;
    launch();  // warm-up
    for (int r = 0; r < reps && !err; ++r) {
        cudaEventRecord(e0, s);
        launch();
        cudaEventRecord(e1, s);
        if ((err = cudaEventSynchronize(e1))) break;
        float t = 0.0f;
        cudaEventElapsedTime(&t, e0, e1);
        best = std::min(best, t);
    }
    if (!err) err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = best;
    return err;
}

}  // namespace
}  // namespace lpb

extern "C" lpb_err lpb_measure_peaks(lpb_peaks* out, void* stream) {
    using namespace lpb;
    api_clear_error();
    if (!out) return api_fail(LPB_EINVAL, "out is NULL");
    *out = lpb_peaks{};
    int dev = 0, sms = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (!err) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err) return api_cuda_fail(err, "device query");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int blocks = sms * 8;  // 2048 threads per SM: every unit busy, latency hidden
    const size_t nthreads = (size_t)blocks * kPeakThreads;
    void* buf = nullptr;
    if ((err = cudaMalloc(&buf, nthreads * sizeof(double)))) return api_cuda_fail(err, "peak buffer");
    const int it64 = 1 << 12, it32 = 1 << 14, itsm = 1 << 13;
    float ms64 = 0, ms32 = 0, mssm = 0;
    err = best_ms([&] { peak_fp64_kernel<<<blocks, kPeakThreads, 0, s>>>((double*)buf, it64, 0.999999, 1e-6); },
                  s, 5, &ms64);
    if (!err)
        err = best_ms([&] { peak_fp32_kernel<<<blocks, kPeakThreads, 0, s>>>((float*)buf, it32, 0.999f, 1e-3f); },
                      s, 5, &ms32);
    if (!err)
        err = best_ms([&] { peak_smem_kernel<<<blocks, kPeakThreads, 0, s>>>((float*)buf, itsm); }, s, 5, &mssm);
    cudaFree(buf);
    if (err) return api_cuda_fail(err, "peak kernels");
    out->fp64_gflops = 2.0 * kFp64Chains * (double)it64 * nthreads / (ms64 * 1e-3) / 1e9;
    out->fp32_gflops = 2.0 * kFp32Chains * (double)it32 * nthreads / (ms32 * 1e-3) / 1e9;
    out->smem_gbs = 2.0 * 16.0 * kSmemSlots * (double)itsm * nthreads / (mssm * 1e-3) / 1e9;
    out->num_sms = sms;
    return LPB_OK;
}
