// lp_mlp_tc.cu -- the warm-start network's matrix product on the 5th-generation
// tensor cores: C[M x N] = A[M x K] . B[N x K]^T, BF16 operands (both
// K-major), FP32 accumulation in tensor memory, the fused epilogues of
// lp_mlp_gemm.cuh.  No counterpart in the paper.
//
// Persistent CTAs of 10 warps, one per SM, each taking 128 x 128 output tiles
// tile = blockIdx.x, blockIdx.x + gridDim.x, ... (columns of a row of tiles
// consecutive, so neighbouring CTAs share A's rows in L2):
//  - warp 0, one lane: TMA producer.  Tiles of 128 rows x 64 K-elements of A
//    and of B (128 bytes per row, 128-byte swizzle) are copied by
//    cp.async.bulk.tensor into a ring of 4 stages (5 when the product writes
//    BF16 outputs only, whose epilogue staging is half as wide) that runs across
//    output tiles; each stage's full barrier counts the bytes in, its empty
//    barrier is armed by the MMAs that read it.
//  - warp 1, one lane: MMA issuer.  Four tcgen05.mma (128 x 128 x 16) per
//    stage into one of two 128-column FP32 accumulators in tensor memory
//    (tile i uses accumulator i % 2), a tcgen05.commit per stage to free it
//    and one per tile to hand the accumulator to the epilogue.
//  - warps 2..9: epilogue.  Warp w reads accumulator lanes 32(w%4) .. +31
//    (its rows; a warp may only reach its own quarter of the lanes) and
//    columns 64((w-2)/4) .. +63 with tcgen05.ld, releases the accumulator to
//    the MMA warp, and applies the epilogue with 16-byte stores -- while the
//    MMAs of the next tile run in the other accumulator.  Two warps per lane
//    quarter halve each warp's share of a tile: the epilogue, not the tensor
//    pipe, sets the pace of these K <= 512 products.
// Rows and columns past M, N and K are zero-filled by the TMA unit and not
// stored.  Every wait is bounded (about two seconds of clock) and also ends
// when another role of the CTA has given up: the CTA then counts a fault,
// writes NaN for the tile at hand, waits (bounded) for the copies and MMAs it
// started, frees its tensor memory and returns.
//
// The tensor cores' accumulation is checked against the FP64 product within
// the FP32 accumulation bound (it has matched the mma.sync kernels bit for
// bit on the shapes tested, which nothing here relies on).

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "lp_internal.h"
#include "lp_mlp_gemm.cuh"
#include "lp_tcgen05.h"

namespace lpb {
namespace {

constexpr int kTcM = 128, kTcN = 128, kTcK = 64;
constexpr int kTcEpiWarps = 8, kTcThreads = 64 + 32 * kTcEpiWarps;
constexpr int kTcEpiCols = kTcN / 2;  // columns of a tile per epilogue warp
constexpr uint32_t kTileBytes = kTcM * kTcK * 2;  // 16 KB per operand tile (also for B: kTcN == kTcM)
// Ring depth and epilogue staging, per form.  Per epilogue warp: 32 rows of
// its 64 columns, padded so that a lane's row piece and a row's 16-byte
// chunks fall on distinct banks, then its 64 bias values.  kWide (an FP32
// output C): rows of 256 bytes (272 with padding), 4 stages.  Otherwise
// (BF16 outputs only): rows of 128 bytes (144), which leaves room for a
// fifth stage -- the operand stream is bound by the latency of the TMA loads,
// so more bytes in flight is what speeds it.
template <bool kWide>
struct TcForm {
    static constexpr int kStages = kWide ? 4 : 5;
    static constexpr uint32_t kStageRow = kWide ? 272 : 144, kStageWarp = 32 * kStageRow;
    static constexpr size_t kSmem = 1024 /* alignment slack */ + 2 * kStages * (size_t)kTileBytes +
                                    kTcEpiWarps * kStageWarp + kTcEpiWarps * kTcEpiCols * 4 +
                                    256 /* barriers */;
    static_assert(kSmem <= 227 * 1024, "shared memory of the tcgen05 product");
    static_assert(8 * (2 * kStages + 5) <= 256, "barrier area");
};
constexpr long long kTcWaitCycles = 4000000000LL;  // ~2 s at 2 GHz
constexpr int kTcChunks = kTcEpiCols / 16;  // 16-column chunks per epilogue warp

__device__ int g_tc_faults;  // CTAs that gave up on a wait (read by lp_mlp_tc_faults)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}
// Wait for the phase of parity `parity` to complete: at most ~2 s, and not
// past the moment another role of the CTA raised *fault.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* fault) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*fault) return false;
        if (clock64() - t0 > kTcWaitCycles) {
            *fault = 1;
            return false;
        }
        __nanosleep(32);
    }
    return true;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// 16 columns of this warp's 32 accumulator lanes (no wait: see tmem_wait).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

template <int kEpi, bool kWide>
__global__ void __launch_bounds__(kTcThreads, 1)
gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const GemmArgs g) {
    constexpr int kTcStages = TcForm<kWide>::kStages;
    constexpr uint32_t kStageRow = TcForm<kWide>::kStageRow, kStageWarp = TcForm<kWide>::kStageWarp;
    extern __shared__ uint8_t smem_raw[];
    __shared__ int s_fault;
    __shared__ uint32_t s_tmem;
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;  // 128-byte swizzle atoms need 1024-byte alignment
    const uint32_t a_tiles = base, b_tiles = base + kTcStages * kTileBytes;
    const uint32_t stage_out = base + 2 * kTcStages * kTileBytes;     // epilogue staging, one area per warp
    const uint32_t bias_s = stage_out + kTcEpiWarps * kStageWarp;     // kTcEpiCols floats per epilogue warp
    const uint32_t bars = bias_s + kTcEpiWarps * kTcEpiCols * 4;
    // barriers: full[S], empty[S], acc_full[2], acc_empty[2], mma_done
    auto full = [&](int s) { return bars + 8u * s; };
    auto empty = [&](int s) { return bars + 8u * (kTcStages + s); };
    auto acc_full = [&](int b) { return bars + 8u * (2 * kTcStages + b); };
    auto acc_empty = [&](int b) { return bars + 8u * (2 * kTcStages + 2 + b); };
    const uint32_t mma_done = bars + 8u * (2 * kTcStages + 4);
    volatile int* fault = &s_fault;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk = (g.K + kTcK - 1) / kTcK;
    const int n_tiles = (g.N + kTcN - 1) / kTcN;
    const int tiles = n_tiles * ((g.M + kTcM - 1) / kTcM);

    if (threadIdx.x == 0) {
        s_fault = 0;
        for (int s = 0; s < kTcStages; ++s) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(acc_full(b), 1);
            mbar_init(acc_empty(b), kTcEpiWarps);  // one arrival per epilogue warp
        }
        mbar_init(mma_done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(2 * kTcN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    if (warp == 0) {
        if (lane == 0) {
            int kt = 0;  // k-blocks issued by this CTA: ring position
            for (int t = blockIdx.x; t < tiles && !*fault; t += gridDim.x) {
                const int m0 = (t / n_tiles) * kTcM, n0 = (t % n_tiles) * kTcN;
                for (int kb = 0; kb < nk; ++kb, ++kt) {
                    const int s = kt % kTcStages;
                    if (!mbar_wait(empty(s), ((kt / kTcStages) & 1) ^ 1, fault)) break;
                    mbar_expect_tx(full(s), 2 * kTileBytes);
                    tma_load_2d(a_tiles + s * kTileBytes, &tmA, kb * kTcK, m0, full(s));
                    tma_load_2d(b_tiles + s * kTileBytes, &tmB, kb * kTcK, n0, full(s));
                }
            }
            if (*fault) {
                // let the copies already started land before the CTA can leave
                for (int k = (kt > kTcStages ? kt - kTcStages : 0); k < kt; ++k) {
                    const int s = k % kTcStages;
                    const long long t0 = clock64();
                    while (!mbar_try_wait(full(s), (k / kTcStages) & 1) && clock64() - t0 < kTcWaitCycles) {
                    }
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = tc::idesc_bf16_f32(kTcM, kTcN);
            int kt = 0, i = 0;
            for (int t = blockIdx.x; t < tiles && !*fault; t += gridDim.x, ++i) {
                const int b = i & 1;
                if (!mbar_wait(acc_empty(b), ((i >> 1) & 1) ^ 1, fault)) break;
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(b * kTcN);
                bool ok = true;
                for (int kb = 0; kb < nk; ++kb, ++kt) {
                    const int s = kt % kTcStages;
                    if (!mbar_wait(full(s), (kt / kTcStages) & 1, fault)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
#pragma unroll
                    for (int kk = 0; kk < kTcK / 16; ++kk) {
                        // K-major, 128-byte swizzle: 8-row groups 1024 bytes
                        // apart; a 16-element K step moves the start by 32 bytes
                        const uint64_t ad =
                            tc::smem_desc(a_tiles + s * kTileBytes + kk * 32, 16, 1024, tc::kSwizzle128B);
                        const uint64_t bd =
                            tc::smem_desc(b_tiles + s * kTileBytes + kk * 32, 16, 1024, tc::kSwizzle128B);
                        tc_mma(d, ad, bd, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
                    }
                    tc_commit(empty(s));  // stage s is free once these MMAs have read it
                }
                if (!ok) break;
                tc_commit(acc_full(b));  // tile i's accumulator is complete
            }
            tc_commit(mma_done);  // arrives when every MMA issued above has completed
        }
        __syncwarp();
    } else {
        // epilogue: warp w owns accumulator lanes (rows) 32*(w%4) .. +31 and
        // columns cb .. cb + 63 of the tile
        const int q = warp & 3, ew = warp - 2;
        const int cb = (ew >> 2) * kTcEpiCols;
        uint8_t* my_stage = smem_raw + (stage_out - raw) + (size_t)ew * kStageWarp;
        float* my_bias = reinterpret_cast<float*>(smem_raw + (bias_s - raw)) + ew * kTcEpiCols;
        // the fast path: BF16 rows (and FP32 rows of C) through the warp's
        // staging area, written out as whole contiguous rows; 16-byte aligned
        // rows needed (ldc a multiple of 4, ldh of 8, aligned bases)
        const bool vec = (g.ldc % 4 == 0) && (g.ldh % 8 == 0) &&
                         ((reinterpret_cast<uintptr_t>(g.C) | reinterpret_cast<uintptr_t>(g.pre) |
                           reinterpret_cast<uintptr_t>(g.hbf) | reinterpret_cast<uintptr_t>(g.bias)) & 15u) == 0;
        int i = 0;
        for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++i) {
            const int m0 = (t / n_tiles) * kTcM, n0 = (t % n_tiles) * kTcN;
            const int b = i & 1;
            const bool ok = mbar_wait(acc_full(b), (i >> 1) & 1, fault);
            tc_fence_after();
            uint32_t v[kTcChunks][16];
            if (ok) {
#pragma unroll
                for (int c = 0; c < kTcChunks; ++c)
                    tmem_ld16(tmem + (uint32_t)(b * kTcN) + ((uint32_t)(q * 32) << 16) + (uint32_t)(cb + c * 16), v[c]);
                tmem_wait();
#pragma unroll
                for (int c = 0; c < kTcChunks; ++c)
#pragma unroll
                    for (int j = 0; j < 16; ++j) asm volatile("" : "+r"(v[c][j]));  // the values exist from here on
            }
            // the accumulator is in registers: hand it back to the MMA warp
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acc_empty(b));
            const int row0 = m0 + q * 32, row = row0 + lane;
            const bool full_tile = vec && n0 + kTcN <= g.N && row0 + 32 <= g.M;
            if (full_tile && (kEpi == kEpiBias || kEpi == kEpiBiasReLU)) {
                // the warp's bias columns
                if (lane < kTcEpiCols / 4)
                    reinterpret_cast<float4*>(my_bias)[lane] = reinterpret_cast<const float4*>(g.bias + n0 + cb)[lane];
                __syncwarp();
            }
            if (!ok) {
#pragma unroll
                for (int c = 0; c < kTcChunks; ++c)
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[c][j] = 0x7fc00000u;  // NaN: the tile failed
            }
            // the accumulators as floats, in the same registers
            float (&f)[kTcChunks][16] = *reinterpret_cast<float(*)[kTcChunks][16]>(&v[0][0]);
            if (full_tile) {
                // epilogue arithmetic in registers (as epilogue16 does it)
#pragma unroll
                for (int c = 0; c < kTcChunks; ++c) {
                    if (kEpi == kEpiBias || kEpi == kEpiBiasReLU) {
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const float4 bb = reinterpret_cast<const float4*>(my_bias)[c * 4 + u];
                            f[c][4 * u] = f[c][4 * u] + bb.x; f[c][4 * u + 1] = f[c][4 * u + 1] + bb.y;
                            f[c][4 * u + 2] = f[c][4 * u + 2] + bb.z; f[c][4 * u + 3] = f[c][4 * u + 3] + bb.w;
                        }
                    }
                    if (kEpi == kEpiMaskGrad) {
                        const float* pr = g.pre + (size_t)row * g.ldc + n0 + cb + c * 16;
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const float4 p4 = reinterpret_cast<const float4*>(pr)[u];
                            f[c][4 * u] = (p4.x > 0.0f) ? f[c][4 * u] : 0.0f;
                            f[c][4 * u + 1] = (p4.y > 0.0f) ? f[c][4 * u + 1] : 0.0f;
                            f[c][4 * u + 2] = (p4.z > 0.0f) ? f[c][4 * u + 2] : 0.0f;
                            f[c][4 * u + 3] = (p4.w > 0.0f) ? f[c][4 * u + 3] : 0.0f;
                        }
                    }
                }
                // FP32 rows of C (the warp's 64 columns = 256 bytes) through the staging area
                if (kWide && g.C) {
#pragma unroll
                    for (int c = 0; c < kTcChunks; ++c) {
                        float4* dst = reinterpret_cast<float4*>(my_stage + lane * kStageRow + c * 64);
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            dst[u] = make_float4(f[c][4 * u], f[c][4 * u + 1], f[c][4 * u + 2], f[c][4 * u + 3]);
                    }
                    __syncwarp();
                    // a row is 16 chunks of 16 bytes: 2 rows per warp store
#pragma unroll 4
                    for (int r = 0; r < 32; r += 2) {
                        const int rr = r + (lane >> 4), ch = lane & 15;
                        const uint4 val = *reinterpret_cast<const uint4*>(my_stage + rr * kStageRow + ch * 16);
                        *reinterpret_cast<uint4*>(g.C + (size_t)(row0 + rr) * g.ldc + n0 + cb + ch * 4) = val;
                    }
                    __syncwarp();
                }
                if (kEpi == kEpiBiasReLU || kEpi == kEpiMaskGrad) {
                    // BF16 rows of h (the warp's 64 columns = 128 bytes) through the staging area
#pragma unroll
                    for (int c = 0; c < kTcChunks; ++c) {
                        __nv_bfloat16 hv[16];
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            hv[j] = __float2bfloat16_rn(kEpi == kEpiBiasReLU ? fmaxf(f[c][j], 0.0f) : f[c][j]);
                        uint4* dst = reinterpret_cast<uint4*>(my_stage + lane * kStageRow + c * 32);
                        dst[0] = *reinterpret_cast<const uint4*>(&hv[0]);
                        dst[1] = *reinterpret_cast<const uint4*>(&hv[8]);
                        if (g.hbfT) {
#pragma unroll
                            for (int j = 0; j < 16; ++j) g.hbfT[(size_t)(n0 + cb + c * 16 + j) * g.ldt + row] = hv[j];
                        }
                    }
                    __syncwarp();
                    // a row is 8 chunks of 16 bytes: 4 rows per warp store
#pragma unroll 4
                    for (int r = 0; r < 32; r += 4) {
                        const int rr = r + (lane >> 3), ch = lane & 7;
                        const uint4 val = *reinterpret_cast<const uint4*>(my_stage + rr * kStageRow + ch * 16);
                        *reinterpret_cast<uint4*>(g.hbf + (size_t)(row0 + rr) * g.ldh + n0 + cb + ch * 8) = val;
                    }
                    __syncwarp();
                }
            } else if (row < g.M) {
                // partial tile or unaligned rows: element by element
#pragma unroll
                for (int c = 0; c < kTcChunks; ++c) {
                    const int col0 = n0 + cb + c * 16;
                    if (vec && col0 + 16 <= g.N) {
                        epilogue16<kEpi>(g, row, col0, f[c]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (col0 + j < g.N) epilogue<kEpi>(g, row, col0 + j, f[c][j]);
                    }
                }
            }
            if (!ok) break;
        }
    }
    // teardown: every MMA has completed (mma_done) before the accumulators are freed
    __syncthreads();
    if (warp == 1) {
        if (lane == 0) {
            const long long t0 = clock64();
            while (!mbar_try_wait(mma_done, 0) && clock64() - t0 < kTcWaitCycles) {
            }
            if (*fault) atomicAdd(&g_tc_faults, 1);
        }
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kTcN) : "memory");
    }
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime.
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// 2-D BF16 tensor [rows x k] with row stride ld elements, box 64 x 128, 128-byte swizzle.
bool make_map(CUtensorMap* map, const void* base, int rows, int k, int ld) {
    auto fn = encode_fn();
    if (!fn) return false;
    if ((reinterpret_cast<uintptr_t>(base) & 15u) || ((size_t)ld * 2) % 16 || rows < 1 || k < 1) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)k, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kTcK, (cuuint32_t)kTcM};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int kEpi, bool kWide>
cudaError_t launch_tc(const GemmArgs& g, cudaStream_t s) {
    static_assert(tc::valid_m128_n(kTcN), "instruction shape");
    constexpr size_t kTcSmem = TcForm<kWide>::kSmem;
    CUtensorMap ma, mb;
    if (!make_map(&ma, g.A, g.M, g.K, g.lda) || !make_map(&mb, g.B, g.N, g.K, g.ldb)) return cudaErrorNotSupported;
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(gemm_tc_kernel<kEpi, kWide>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kTcSmem);
    });
    if (attr != cudaSuccess) return attr;
    int dev = 0, sms = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (!err) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err) return err;
    const int64_t tiles = (int64_t)((g.N + kTcN - 1) / kTcN) * ((g.M + kTcM - 1) / kTcM);
    const int grid = (int)std::min<int64_t>(tiles, sms);  // one persistent CTA per SM
    gemm_tc_kernel<kEpi, kWide><<<grid, kTcThreads, kTcSmem, s>>>(ma, mb, g);
    return cudaGetLastError();
}

// the wide form (FP32 staging, 4 stages) when the product writes C
template <int kEpi>
cudaError_t launch_tc(const GemmArgs& g, cudaStream_t s) {
    return g.C ? launch_tc<kEpi, true>(g, s) : launch_tc<kEpi, false>(g, s);
}

}  // namespace

cudaError_t gemm_tc(int epi, const void* args, cudaStream_t s) {
    const GemmArgs& g = *static_cast<const GemmArgs*>(args);
    switch (epi) {
        case kEpiStore: return launch_tc<kEpiStore>(g, s);
        case kEpiBiasReLU: return launch_tc<kEpiBiasReLU>(g, s);
        case kEpiBias: return launch_tc<kEpiBias>(g, s);
        default: return launch_tc<kEpiMaskGrad>(g, s);
    }
}

cudaError_t gemm_tc_faults(int* count) { return cudaMemcpyFromSymbol(count, g_tc_faults, sizeof(int)); }

}  // namespace lpb
