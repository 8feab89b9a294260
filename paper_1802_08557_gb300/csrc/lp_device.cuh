// lp_device.cuh -- device helpers shared by the simplex kernels: exact
// order-preserving integer keys of FP64/FP32 values and block reductions built
// on warp `redux` instructions.
#pragma once

#include <climits>

#include "lp_internal.h"

namespace lpb {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// Internal-consistency failure seen by a kernel: counted in diag[0]; the
// first failure's code and LP index are kept in diag[1], diag[2].  The
// kernel skips the access it was about to make and gives up on the LP.
__device__ __forceinline__ void record_internal_error(int32_t* diag, int code, int lp, int a = 0, int b = 0,
                                                      int c = 0, int d = 0, int e = 0) {
    if (!diag) return;
    if (atomicAdd(diag, 1) == 0) {
        diag[1] = code;
        diag[2] = lp;
        diag[3] = a; diag[4] = b; diag[5] = c; diag[6] = d; diag[7] = e;
    }
}

// Order-preserving map of a (non-NaN) double to a signed 64-bit key:
// a < b  <=>  okey(a) < okey(b);  -0 and +0 map to the same key.
// The keys are built from the two 32-bit words of the double: written on its
// 64-bit pattern, a test of the key can be compiled into an FP64 compare,
// which GB300 issues to its narrow FP64 pipe at the cost of an FMA.
__device__ __forceinline__ long long okey(double v) {
    int hi = __double2hiint(v);
    const unsigned lo = (unsigned)__double2loint(v);
    hi = (hi == INT_MIN && lo == 0u) ? 0 : hi;  // -0 -> +0
    const int s = hi >> 31;                     // all ones for a negative v
    return (long long)(((unsigned long long)(unsigned)(hi ^ (s & INT_MAX)) << 32) |
                       (unsigned long long)(lo ^ (unsigned)s));
}
// v < t, given kt = okey(t) (t not NaN), by integer operations; a NaN v
// counts as below every threshold, so that no check passes on a NaN.
__device__ __forceinline__ bool below_key(double v, long long kt) {
    const unsigned ha = (unsigned)__double2hiint(v) & 0x7FFFFFFFu;
    const bool nan = ha > 0x7FF00000u || (ha == 0x7FF00000u && (unsigned)__double2loint(v) != 0u);
    return nan || okey(v) < kt;
}
// v > t, given kt = okey(t) (t not NaN), by integer operations; false for a NaN v.
__device__ __forceinline__ bool above_key(double v, long long kt) {
    const unsigned ha = (unsigned)__double2hiint(v) & 0x7FFFFFFFu;
    const bool nan = ha > 0x7FF00000u || (ha == 0x7FF00000u && (unsigned)__double2loint(v) != 0u);
    return !nan && okey(v) > kt;
}
__device__ __forceinline__ double kval(long long k) {
    return __longlong_as_double(k ^ ((k >> 63) & LLONG_MAX));
}
// Key of |v| (the plain bit pattern with the sign cleared).
__device__ __forceinline__ long long abskey(double v) {
    return (long long)(((unsigned long long)((unsigned)__double2hiint(v) & 0x7FFFFFFFu) << 32) |
                       (unsigned long long)(unsigned)__double2loint(v));
}

__device__ __forceinline__ long long warp_min_i64(long long v) {
    const int hi = (int)(v >> 32);
    const int mhi = __reduce_min_sync(kFull, hi);
    const unsigned lo = (hi == mhi) ? (unsigned)(v & 0xffffffffLL) : 0xffffffffu;
    const unsigned mlo = __reduce_min_sync(kFull, lo);
    return (long long)(((unsigned long long)(unsigned)mhi << 32) | (unsigned long long)mlo);
}

// Float order key (int32): a < b <=> fkey(a) < fkey(b); -0 and +0 map alike.
__device__ __forceinline__ int fkey(float f) {
    int b = __float_as_int(f);
    b = (b == INT_MIN) ? 0 : b;
    return b ^ ((b >> 31) & INT_MAX);
}
__device__ __forceinline__ float fval(int k) { return __int_as_float(k ^ ((k >> 31) & INT_MAX)); }

// |v| as a float by integer operations only (no FP64-pipe conversion, which
// GB300 issues at the FP64 rate): the double's exponent rebiased and its
// significand truncated to 24 bits, so for |v| in [2^-126, 2^128) the result
// is below |v| by less than 2^-23 relative; 0 gives 0, smaller magnitudes
// give at most 7 * 2^-149, larger ones the largest finite float.
__device__ __forceinline__ float f64_abs_to_f32_trunc(double v) {
    const int hi = __double2hiint(v) & 0x7fffffff;
    const unsigned lo = (unsigned)__double2loint(v);
    const int t = min(max(hi - (896 << 20), 0), 0x0FEFFFFF);
    return __uint_as_float(__funnelshift_l(lo, (unsigned)t, 3));
}
// v as a float, the same truncation with v's sign.
__device__ __forceinline__ float f64_to_f32_trunc(double v) {
    return __uint_as_float(__float_as_uint(f64_abs_to_f32_trunc(v)) | ((unsigned)__double2hiint(v) & 0x80000000u));
}

// Unbiased binary exponent of a double from its bits (-1023 for 0 and subnormals).
__device__ __forceinline__ int dexp(double v) { return (int)((__double_as_longlong(v) >> 52) & 0x7FF) - 1023; }

// Asynchronous 8-byte copy global -> shared (no register staging, so a thread
// can have many in flight); cp_async_wait_all waits for this thread's copies.
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// ---- mbarriers and bulk asynchronous copies (global -> this CTA's shared
// memory), for the streamed kernel's staged update ----
__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// Makes initialised mbarriers visible to the asynchronous proxy.
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// `bytes` (a multiple of 16) from 16-byte aligned global `src` to 16-byte
// aligned shared `dst`; completion counted on `bar`.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
// Wait for the phase of `bar` with the given parity; false after `cycles`
// clock cycles (the copy did not complete).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, long long cycles) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > cycles) return false;
    return true;
}
// Orders this thread's earlier generic-proxy accesses of shared memory before
// later asynchronous-proxy writes to it (reuse of a staging buffer).
__device__ __forceinline__ void fence_proxy_async_shared() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Orders this thread's earlier generic-proxy writes of global memory before
// later asynchronous-proxy reads of it (bulk copies of rows it updated).
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Block-wide reductions over per-warp `redux` results.  Each call writes
// one slot per warp, waits at a barrier, reads every slot, and waits at a
// second barrier before returning, so no later write can overtake a read of
// the same slot whatever the calls that follow.
struct Reducer {
    long long* s64;   // kMaxWarps int64 slots
    unsigned* s32;    // 2 x kMaxWarps uint32 slots (value, count)
    int nw, warp, lane;

    __device__ long long min_i64(long long v) {
        v = warp_min_i64(v);
        if (lane == 0) s64[warp] = v;
        __syncthreads();
        long long r = s64[0];
        for (int w = 1; w < nw; ++w) r = min(r, s64[w]);
        __syncthreads();
        return r;
    }
    __device__ unsigned min_u32(unsigned v) {
        v = __reduce_min_sync(kFull, v);
        if (lane == 0) s32[warp] = v;
        __syncthreads();
        unsigned r = s32[0];
        for (int w = 1; w < nw; ++w) r = min(r, s32[w]);
        __syncthreads();
        return r;
    }
    __device__ int min_i32(int v) {
        return (int)(min_u32((unsigned)v ^ 0x80000000u) ^ 0x80000000u);
    }
    // Block-wide (sum of cnt, min of v).
    __device__ void count_min(unsigned cnt, unsigned v, unsigned& cnt_out, unsigned& v_out) {
        cnt = __reduce_add_sync(kFull, cnt);
        v = __reduce_min_sync(kFull, v);
        if (lane == 0) { s32[warp] = v; s32[kMaxWarps + warp] = cnt; }
        __syncthreads();
        unsigned c = 0, r = 0xffffffffu;
        for (int w = 0; w < nw; ++w) { c += s32[kMaxWarps + w]; r = min(r, s32[w]); }
        __syncthreads();
        cnt_out = c;
        v_out = r;
    }
    // Exclusive prefix count of `flag` over the block (in thread order) and
    // the total; `flag` must be the same for all lanes' view of bal.
    __device__ int prefix_count(bool flag, int& total) {
        const unsigned bal = __ballot_sync(kFull, flag);
        if (lane == 0) s32[warp] = (unsigned)__popc(bal);
        __syncthreads();
        int before = 0, tot = 0;
        for (int w = 0; w < nw; ++w) {
            const int cw = (int)s32[w];
            before += (w < warp) ? cw : 0;
            tot += cw;
        }
        __syncthreads();
        total = tot;
        return before + __popc(bal & ((1u << lane) - 1u));
    }
};


// The thread group that solves one LP, as a CTA: tid/nt index it, sync() is a
// block barrier, reductions are the Reducer's.
struct BlockGroup : Reducer {
    int tid, nt;
    __device__ BlockGroup(long long* s64_, unsigned* s32_)
        : Reducer{s64_, s32_, (int)(blockDim.x >> 5), (int)(threadIdx.x >> 5), (int)(threadIdx.x & 31)},
          tid((int)threadIdx.x), nt((int)blockDim.x) {}
    __device__ void sync() { __syncthreads(); }
};

// The thread group that solves one LP, as a single warp: no block barriers;
// sync() is __syncwarp (which also orders shared-memory accesses among the
// lanes) and every reduction is one or two `redux` instructions.  Each
// reduction starts with __syncwarp so that shared-memory writes made before
// it are visible to every lane after it.
struct WarpGroup {
    int tid, nt, lane, warp, nw;
    __device__ WarpGroup() : tid((int)(threadIdx.x & 31)), nt(32), lane((int)(threadIdx.x & 31)), warp(0), nw(1) {}
    __device__ void sync() { __syncwarp(); }
    __device__ long long min_i64(long long v) {
        __syncwarp();
        return warp_min_i64(v);
    }
    __device__ unsigned min_u32(unsigned v) {
        __syncwarp();
        return __reduce_min_sync(kFull, v);
    }
    __device__ int min_i32(int v) {
        return (int)(min_u32((unsigned)v ^ 0x80000000u) ^ 0x80000000u);
    }
    __device__ void count_min(unsigned cnt, unsigned v, unsigned& cnt_out, unsigned& v_out) {
        __syncwarp();
        const unsigned c = __reduce_add_sync(kFull, cnt);
        const unsigned r = __reduce_min_sync(kFull, v);
        cnt_out = c;
        v_out = r;
    }
    __device__ int prefix_count(bool flag, int& total) {
        __syncwarp();
        const unsigned bal = __ballot_sync(kFull, flag);
        total = __popc(bal);
        return __popc(bal & ((1u << lane) - 1u));
    }
};

}  // namespace
}  // namespace lpb
