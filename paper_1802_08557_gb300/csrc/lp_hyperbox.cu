// lp_hyperbox.cu -- hyperbox LPs (Gurung & Ray, arXiv 1802.08557, Section
// 4.4, Eq. 7): maximise l.x over a box lo <= x <= hi for many directions l.
// The maximiser takes lo_i where l_i < 0 and hi_i otherwise, so each LP is one
// dot product sum_i l_i h_i.
//
// The paper gives each LP a 32-thread block with one working thread.  Here:
//  - dim <= kTileMaxDim: persistent CTAs stride over tiles of `tile_lps`
//    consecutive LPs; each tile (l, and the per-LP boxes when there are any)
//    is staged into shared memory by bulk asynchronous copies (cp.async.bulk,
//    completion counted on an mbarrier), `stages` tiles in flight per CTA.
//    Thread t then owns LP t of the tile: obj = fma over i = 0..dim-1 in index
//    order, h_i chosen by a 32-bit integer sign test (no FP64 compare), the shared
//    box read from shared memory (a broadcast).  x, when asked for, is written
//    by a flat pass over the tile (coalesced stores).  Tiles that are not
//    whole (the last one) or arrays that are not 16-byte aligned are loaded
//    with plain loads instead.
//  - larger dim: one warp per LP, lanes over i, a fixed xor-tree sum.
// Bound: the FP64 pipe (one FMA per 8 bytes of l) for one shared box and no x;
// HBM bandwidth when every LP has its own box or x is written.
//
// Waits on an mbarrier are bounded (kWaitCycles of clock64): a CTA whose copy
// does not complete gives up, writes NaN to the outputs of the tiles it has
// not finished, waits (bounded again) for its other copies and returns.

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>

#include "lp_internal.h"

namespace lpb {
namespace {

constexpr int kTileMaxDim = 64;
constexpr long long kWaitCycles = 2000000000LL;  // ~1 s at 2 GHz
constexpr unsigned kFullMask = 0xffffffffu;

struct HbArgs {
    const double* L;
    const double* lo;
    const double* hi;
    double* obj;
    double* x;
    int64_t num_lps;
    int64_t num_tiles;
    int64_t num_full_tiles;  // tiles that may be bulk-copied (whole, aligned)
    int dim;
    int tile_lps;            // LPs per tile = threads per CTA
    int stages;
    int stage_offset;        // bytes from the start of shared memory
    int stage_bytes;
};

// l < 0 (strictly: -0 is not negative), from the bits, in 32-bit words: on
// GB300 a 64-bit integer compare, like an FP64 compare, is issued to the
// FP64 pipe, where it would cost as much as the FMA it feeds (measured: one
// such test per coordinate halved the kernel's FMA rate).
__device__ __forceinline__ bool is_negative(double v) {
    const unsigned hw = (unsigned)__double2hiint(v);
    const unsigned lw = (unsigned)__double2loint(v);
    return (hw >> 31) != 0u && ((hw << 1) | lw) != 0u;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// Bulk copy global -> this CTA's shared memory; bytes a multiple of 16, both
// addresses 16-byte aligned.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Order this thread's earlier generic-proxy accesses of shared memory before
// later async-proxy (bulk copy) writes to it.
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait for the phase with the given parity; false after kWaitCycles.
__device__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > kWaitCycles) return false;
    return true;
}

template <bool kBoxPerLp>
__global__ void __launch_bounds__(128) hyperbox_tile_kernel(const HbArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);        // one per stage
    double* box = reinterpret_cast<double*>(smem + 64);       // shared box: lo, hi
    const int tid = threadIdx.x, nt = blockDim.x;
    const int dim = a.dim;
    const int S = a.stages;
    const int64_t tile_elems = (int64_t)a.tile_lps * dim;
    const uint32_t tile_bytes = (uint32_t)(tile_elems * 8);

    if (tid == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&bar[s], 1);
        mbar_init_fence();
    }
    if (!kBoxPerLp)
        for (int i = tid; i < dim; i += nt) {
            box[i] = a.lo[i];
            box[dim + i] = a.hi[i];
        }
    __syncthreads();

    auto stage = [&](int s) { return reinterpret_cast<double*>(smem + a.stage_offset + (size_t)s * a.stage_bytes); };
    auto issue = [&](int64_t t, int s) {  // thread 0 only
        double* d = stage(s);
        const int64_t off = t * tile_elems;
        mbar_expect_tx(&bar[s], kBoxPerLp ? 3u * tile_bytes : tile_bytes);
        bulk_load(d, a.L + off, tile_bytes, &bar[s]);
        if (kBoxPerLp) {
            bulk_load(d + tile_elems, a.lo + off, tile_bytes, &bar[s]);
            bulk_load(d + 2 * tile_elems, a.hi + off, tile_bytes, &bar[s]);
        }
    };

    const int64_t t0 = blockIdx.x, step = gridDim.x;
    uint32_t pending = 0;  // stages with a copy issued and not yet waited for (thread 0's view)
    if (tid == 0)
        for (int s = 0; s < S; ++s) {
            const int64_t t = t0 + (int64_t)s * step;
            if (t < a.num_full_tiles) {
                issue(t, s);
                pending |= 1u << s;
            }
        }
    uint32_t phase = 0;  // bit s: parity of the next completion of stage s
    bool ok = true;
    for (int64_t it = 0;; ++it) {
        const int64_t t = t0 + it * step;
        if (t >= a.num_tiles) break;
        const int s = (int)(it % S);
        double* Ls = stage(s);
        const int64_t lp0 = t * a.tile_lps;
        const int count = (int)((a.num_lps - lp0) < a.tile_lps ? (a.num_lps - lp0) : a.tile_lps);
        const int64_t n_el = (int64_t)count * dim;
        if (t < a.num_full_tiles) {
            bool got = ok && mbar_wait(&bar[s], (phase >> s) & 1u);
            got = __syncthreads_and(got) != 0;
            if (got) {
                phase ^= 1u << s;
                pending &= ~(1u << s);
            }
            ok = got;
        } else if (ok) {
            // plain loads: the last (partial) tile, or arrays that are not aligned
            const int64_t g0 = lp0 * dim;
            for (int64_t e = tid; e < n_el; e += nt) {
                Ls[e] = a.L[g0 + e];
                if (kBoxPerLp) {
                    Ls[tile_elems + e] = a.lo[g0 + e];
                    Ls[2 * tile_elems + e] = a.hi[g0 + e];
                }
            }
            __syncthreads();
        }
        if (!ok) {
            // a copy did not complete: no result for this tile
            const double nan = __longlong_as_double(0x7FF8000000000000LL);
            if (tid < count) a.obj[lp0 + tid] = nan;
            if (a.x)
                for (int64_t e = tid; e < n_el; e += nt) a.x[lp0 * dim + e] = nan;
            continue;
        }
        if (tid < count) {
            const double* l = Ls + (size_t)tid * dim;
            const double* lo = kBoxPerLp ? Ls + tile_elems + (size_t)tid * dim : box;
            const double* hi = kBoxPerLp ? Ls + 2 * tile_elems + (size_t)tid * dim : box + dim;
            double acc = 0.0;
#pragma unroll 4
            for (int i = 0; i < dim; ++i) {
                const double li = l[i];
                acc = __fma_rn(li, is_negative(li) ? lo[i] : hi[i], acc);
            }
            a.obj[lp0 + tid] = acc;
        }
        if (a.x) {
            // h, coalesced: element e of the tile is coordinate e mod dim
            const int dstep = nt % dim;
            int i = tid % dim;
            for (int64_t e = tid; e < n_el; e += nt) {
                const double li = Ls[e];
                double h;
                if (kBoxPerLp) h = is_negative(li) ? Ls[tile_elems + e] : Ls[2 * tile_elems + e];
                else h = is_negative(li) ? box[i] : box[dim + i];
                a.x[lp0 * dim + e] = h;
                i += dstep;
                if (i >= dim) i -= dim;
            }
        }
        __syncthreads();  // every thread is done with stage s
        if (tid == 0) {
            const int64_t tn = t + (int64_t)S * step;
            if (tn < a.num_full_tiles) {
                fence_proxy_async();
                issue(tn, s);
                pending |= 1u << s;
            }
        }
    }
    // after a failed wait: let the copies still in flight land before exiting
    if (tid == 0 && !ok)
        for (int s = 0; s < S; ++s)
            if (pending & (1u << s)) mbar_wait(&bar[s], (phase >> s) & 1u);
}

template <bool kBoxPerLp>
__global__ void __launch_bounds__(256) hyperbox_warp_kernel(const HbArgs a) {
    const int lane = threadIdx.x & 31;
    const int dim = a.dim;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = w0; k < a.num_lps; k += nw) {
        const int64_t base = k * dim;
        const double* l = a.L + base;
        const double* lo = kBoxPerLp ? a.lo + base : a.lo;
        const double* hi = kBoxPerLp ? a.hi + base : a.hi;
        double acc = 0.0;
        for (int i = lane; i < dim; i += 32) {
            const double li = l[i];
            const double h = is_negative(li) ? lo[i] : hi[i];
            acc = __fma_rn(li, h, acc);
            if (a.x) a.x[base + i] = h;
        }
        for (int o = 16; o > 0; o >>= 1) acc = __dadd_rn(acc, __shfl_xor_sync(kFullMask, acc, o));
        if (lane == 0) a.obj[k] = acc;
    }
}

int g_num_sms[64] = {};

int num_sms(int device) {
    if (device < 0 || device >= 64) return 152;
    if (g_num_sms[device] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || v <= 0) v = 152;
        g_num_sms[device] = v;
    }
    return g_num_sms[device];
}

}  // namespace

cudaError_t launch_hyperbox(const double* L, const double* lo, const double* hi, bool box_per_lp, double* obj,
                            double* x, int64_t num_lps, int dim, cudaStream_t stream) {
    if (num_lps <= 0) return cudaSuccess;
    int device = 0;
    cudaError_t err = cudaGetDevice(&device);
    if (err != cudaSuccess) return err;
    const int sms = num_sms(device);
    HbArgs a{};
    a.L = L; a.lo = lo; a.hi = hi; a.obj = obj; a.x = x;
    a.num_lps = num_lps;
    a.dim = dim;
    if (dim > kTileMaxDim) {
        const int threads = 256;
        const int64_t blocks = std::min<int64_t>((num_lps + 7) / 8, (int64_t)sms * 8);
        if (box_per_lp) hyperbox_warp_kernel<true><<<(unsigned)blocks, threads, 0, stream>>>(a);
        else hyperbox_warp_kernel<false><<<(unsigned)blocks, threads, 0, stream>>>(a);
        return cudaGetLastError();
    }
    const int arrays = box_per_lp ? 3 : 1;
    a.tile_lps = (dim * arrays <= 96) ? 128 : 64;
    a.stage_bytes = (int)((size_t)a.tile_lps * dim * 8 * arrays);
    a.stages = std::max(2, std::min(4, (48 << 10) / a.stage_bytes));
    a.stage_offset = ((64 + 2 * dim * 8 + 127) / 128) * 128;  // mbarriers, shared box, then the stages
    const size_t smem = (size_t)a.stage_offset + (size_t)a.stages * a.stage_bytes;
    a.num_tiles = (num_lps + a.tile_lps - 1) / a.tile_lps;
    auto aligned = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    const bool bulk = aligned(L) && (!box_per_lp || (aligned(lo) && aligned(hi)));
    a.num_full_tiles = bulk ? num_lps / a.tile_lps : 0;
    auto kernel = box_per_lp ? hyperbox_tile_kernel<true> : hyperbox_tile_kernel<false>;
    if ((err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return err;
    int per_sm = 0;
    if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, a.tile_lps, smem))) return err;
    const int64_t blocks = std::min<int64_t>(a.num_tiles, (int64_t)sms * std::max(1, per_sm));
    kernel<<<(unsigned)blocks, a.tile_lps, smem, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace lpb
