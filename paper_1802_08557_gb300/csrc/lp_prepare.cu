// lp_prepare.cu -- input checks and per-LP phase-I row counts, run once by
// lp_batch_create to plan the launches (the batch sizing of Algorithm 1 in
// Section 4.1 needs each LP's tableau footprint, Eq. 5).  The check runs on
// the batch's own copy of the inputs and zeroes every non-finite entry it
// counts, so that no kernel after it on the stream sees one, whether or not
// the host has read the count yet.

#include <climits>

#include "lp_internal.h"

namespace lpb {
namespace {

// Counts the non-finite entries of v into *bad and sets them to 0.
__global__ void check_finite_kernel(double* __restrict__ v, int64_t len, unsigned long long* bad) {
    unsigned long long local = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
        const long long bits = __double_as_longlong(v[i]) & LLONG_MAX;
        if (bits >= 0x7FF0000000000000LL) {
            v[i] = 0.0;
            ++local;
        }
    }
    local = __reduce_add_sync(0xffffffffu, (unsigned)local);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(bad, local);
}

// One warp per LP: number of rows with b_i < 0 (rows that get an artificial).
__global__ void count_negative_rhs_kernel(const DeviceBatch B, int32_t num_lps, int32_t* __restrict__ k) {
    const int lane = threadIdx.x & 31;
    const int lp = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (lp >= num_lps) return;
    const int m = B.m[lp];
    const double* bv = B.b + B.b_off[lp];
    int cnt = 0;
    for (int i = lane; i < m; i += 32) cnt += (bv[i] < 0.0) ? 1 : 0;
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    if (lane == 0) k[lp] = cnt;
}

int grid_for(int64_t len, int threads) {
    int64_t g = (len + threads * 4 - 1) / (threads * 4);
    if (g < 1) g = 1;
    if (g > 4096) g = 4096;
    return (int)g;
}

}  // namespace

cudaError_t launch_input_check(double* A, int64_t a_len, double* b, int64_t b_len, double* c, int64_t c_len,
                               unsigned long long* bad, cudaStream_t stream) {
    cudaError_t err = cudaMemsetAsync(bad, 0, sizeof(unsigned long long), stream);
    if (err != cudaSuccess) return err;
    const int t = 256;
    if (a_len > 0) check_finite_kernel<<<grid_for(a_len, t), t, 0, stream>>>(A, a_len, bad);
    if (b_len > 0) check_finite_kernel<<<grid_for(b_len, t), t, 0, stream>>>(b, b_len, bad);
    if (c_len > 0) check_finite_kernel<<<grid_for(c_len, t), t, 0, stream>>>(c, c_len, bad);
    return cudaGetLastError();
}

cudaError_t launch_count_negative_rhs(const DeviceBatch& B, int32_t num_lps, int32_t* k, cudaStream_t stream) {
    const int t = 256;
    const int64_t threads = (int64_t)num_lps * 32;
    count_negative_rhs_kernel<<<(unsigned)((threads + t - 1) / t), t, 0, stream>>>(B, num_lps, k);
    return cudaGetLastError();
}

}  // namespace lpb
