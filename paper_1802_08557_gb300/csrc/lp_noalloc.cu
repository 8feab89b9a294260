// lp_noalloc.cu -- lp_solve_uniform_noalloc: the streamed FP64 solver for a
// batch of equal-size LPs whose scratch memory comes from a fixed array in
// this module instead of an allocation.
//
// Who needs this: code that may not allocate device memory while it runs --
// for example a caller that owns every byte of the GPU through its own pool, a
// real-time loop that forbids cudaMalloc/cudaFree (they synchronise the device
// and can stall), or an embedding where the allocator is not reachable.  Such a
// caller allocates its inputs and outputs once, up front, and solves with this
// entry point as often as it likes.  The paper has no counterpart; its batches
// are also of one size (Section 4), which is why this entry point takes one m
// and one n.
//
// The scratch array is a file-scope __device__ variable: every GPU that loads
// this library holds its kNoAllocScratchBytes until the process exits.  All
// calls share it and it keeps the previous call's contents, so calls must not
// overlap on the GPU: two calls in flight at once on one device (for example
// on two streams) race on it.  What must start at zero (the work counter) is
// cleared by every call on its stream.

#include <algorithm>
#include <climits>
#include <cmath>

#include "lp_internal.h"
#include "lpbatch.h"

namespace lpb {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;  // 64 MiB

// Scratch: [0, 256) work counter | per-LP descriptors | tableau slots.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// Per-LP descriptors (52 bytes per LP): m, n, order (int32) and a_off, b_off,
// c_off, x_off, y_off (int64).
struct DescPtrs {
    int32_t* m; int32_t* n; int32_t* order;
    int64_t* a_off; int64_t* b_off; int64_t* c_off; int64_t* x_off; int64_t* y_off;
};

DescPtrs carve_descriptors(unsigned char* base, int32_t num_lps) {
    const size_t N = (size_t)num_lps;
    DescPtrs d;
    unsigned char* p = base;
    d.a_off = reinterpret_cast<int64_t*>(p); p += align256(N * 8);
    d.b_off = reinterpret_cast<int64_t*>(p); p += align256(N * 8);
    d.c_off = reinterpret_cast<int64_t*>(p); p += align256(N * 8);
    d.x_off = reinterpret_cast<int64_t*>(p); p += align256(N * 8);
    d.y_off = reinterpret_cast<int64_t*>(p); p += align256(N * 8);
    d.m = reinterpret_cast<int32_t*>(p); p += align256(N * 4);
    d.n = reinterpret_cast<int32_t*>(p); p += align256(N * 4);
    d.order = reinterpret_cast<int32_t*>(p);
    return d;
}

size_t descriptor_bytes(int32_t num_lps) {
    const size_t N = (size_t)num_lps;
    return 5 * align256(N * 8) + 3 * align256(N * 4);
}

// Packed uniform layout: LP k's A at k*m*n, b and y at k*m, c and x at k*n.
__global__ void fill_uniform_descriptors(DescPtrs d, int32_t num_lps, int32_t m, int32_t n) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= num_lps) return;
    d.m[k] = m;
    d.n[k] = n;
    d.order[k] = (int32_t)k;
    d.a_off[k] = k * (int64_t)m * n;
    d.b_off[k] = k * (int64_t)m;
    d.c_off[k] = k * (int64_t)n;
    d.x_off[k] = k * (int64_t)n;
    d.y_off[k] = k * (int64_t)m;
}

// Device address of the scratch array in the current context.  Looked up on
// every call (the lookup allocates nothing): after cudaDeviceReset, or with
// another context current, the module is loaded again and the array can sit
// at another address, so a cached pointer could point at freed or foreign
// memory.
cudaError_t scratch_address(unsigned char** out) {
    void* p = nullptr;
    const cudaError_t err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (err != cudaSuccess) return err;
    *out = static_cast<unsigned char*>(p);
    return cudaSuccess;
}

}  // namespace
}  // namespace lpb

extern "C" lpb_err lp_solve_uniform_noalloc(int32_t num_lps, int32_t m, int32_t n,
                                            const double* A, const double* b, const double* c,
                                            int32_t* status, int32_t* iters, double* obj, double* x, double* y,
                                            const lp_batch_opts* opts, void* stream) {
    using namespace lpb;
    if (num_lps < 1 || m < 1 || n < 1) return LPB_EINVAL;
    if (m > LPB_MAX_DIM || n > LPB_MAX_DIM) return LPB_ETOOBIG;
    if (!A || !b || !c || !status || !iters || !obj || !x) return LPB_EINVAL;
    lp_batch_opts o;
    lpb_default_opts(&o);
    if (opts) o = *opts;
    if (!(o.eps_opt >= 0) || !(o.eps_piv >= 0) || !(o.eps_feas >= 0) || !(o.tau >= 0)) return LPB_EINVAL;
    // Only the FP64 streamed kernel runs here; the mixed-precision path needs
    // its own workspaces and re-solve queues, which this entry point has not.
    if (o.precision != LP_PREC_FP64) return LPB_EINVAL;

    // Room: the counter, the descriptors, and at least one tableau slot sized
    // for the widest phase-I tableau (every row with b_i < 0).
    const size_t slot_bytes = streamed_slot_bytes(m, n, m);
    const size_t desc_bytes = descriptor_bytes(num_lps);
    if (256 + desc_bytes + slot_bytes > kNoAllocScratchBytes) return LPB_ETOOBIG;

    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return LPB_ECUDA;
    unsigned char* base = nullptr;
    if ((err = scratch_address(&base)) != cudaSuccess) return LPB_ECUDA;
    int sms = 0;
    if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return LPB_ECUDA;

    int32_t* counter = reinterpret_cast<int32_t*>(base);
    const DescPtrs d = carve_descriptors(base + 256, num_lps);
    unsigned char* slots_base = base + 256 + desc_bytes;
    int64_t slots = (int64_t)sms * fp64_streamed_ctas_per_sm();
    slots = std::min<int64_t>(slots, num_lps);
    slots = std::min<int64_t>(slots, (int64_t)((kNoAllocScratchBytes - 256 - desc_bytes) / slot_bytes));

    // Same tolerances and screening windows as lp_batch_create.
    Tolerances tol;
    tol.eps_opt = o.eps_opt;
    tol.eps_piv = o.eps_piv;
    tol.eps_feas = o.eps_feas;
    tol.tau = o.tau;
    tol.max_iters = o.max_iters;
    tol.key_window = (o.tau <= std::ldexp(1.0, -33))
                         ? (long long)std::ceil(o.tau * std::ldexp(1.0, 54) * (1.0 + std::ldexp(1.0, -30))) + 4
                         : -1;
    tol.ratio_rel = (float)std::max(std::ldexp(1.0, -12), 8.0 * o.tau);
    tol.ratio_abs = (float)std::max(std::ldexp(1.0, -20), 8.0 * o.tau);

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    fill_uniform_descriptors<<<(num_lps + 255) / 256, 256, 0, s>>>(d, num_lps, m, n);
    if ((err = cudaGetLastError()) != cudaSuccess) return LPB_ECUDA;
    DeviceBatch B{d.m, d.n, d.a_off, d.b_off, d.c_off, d.x_off, d.y_off, A, b, c, status, iters, obj, x, y};
    // launch_fp64_streamed zeroes the counter on `s` before the kernel.
    err = launch_fp64_streamed(B, tol, d.order, num_lps, (int)slots, slots_base, slot_bytes, counter, nullptr, s);
    return err == cudaSuccess ? LPB_OK : LPB_ECUDA;
}
