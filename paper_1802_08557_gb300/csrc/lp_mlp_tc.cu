// lp_mlp_tc.cu -- the warm-start network's matrix product on the 5th-generation
// tensor cores: C[M x N] = A[M x K] . B[N x K]^T, BF16 operands (both
// K-major), FP32 accumulation in tensor memory, the fused epilogues of
// lp_mlp_gemm.cuh.  No counterpart in the paper.
//
// One CTA of 4 warps per 128 x 128 output tile:
//  - warp 0, one lane: TMA producer.  Tiles of 128 rows x 64 K-elements of A
//    and of B (128 bytes per row, 128-byte swizzle) are copied by
//    cp.async.bulk.tensor into a ring of kStages stages; each stage's full
//    barrier counts the bytes in, its empty barrier is armed by the MMAs that
//    read it.
//  - warp 1, one lane: MMA issuer.  Four tcgen05.mma (128 x 128 x 16) per
//    stage into one 128-column FP32 accumulator in tensor memory; a
//    tcgen05.commit per stage frees it, a last one signals the epilogue.
//  - all 4 warps: epilogue.  Warp w reads accumulator lanes 32w..32w+31 (rows)
//    with tcgen05.ld, 16 columns at a time, and applies the epilogue.
// Rows and columns past M, N and K are zero-filled by the TMA unit and not
// stored.  Every wait is bounded (about two seconds of clock): on expiry the
// CTA counts a fault, writes NaN for its tile, waits (bounded) for the
// copies and MMAs it started, frees its tensor memory and returns.
//
// The accumulation order inside the tensor core differs from the mma.sync
// kernels', so results agree with them (and with the FP64 reference) within
// the FP32 accumulation bound, not bit for bit.

#include <cuda.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <mutex>

#include "lp_internal.h"
#include "lp_mlp_gemm.cuh"
#include "lp_tcgen05.h"

namespace lpb {
namespace {

constexpr int kTcM = 128, kTcN = 128, kTcK = 64, kTcStages = 3, kTcThreads = 128;
constexpr uint32_t kTileBytes = kTcM * kTcK * 2;  // 16 KB per operand tile (also for B: kTcN == kTcM)
constexpr size_t kTcSmem = 1024 /* alignment slack */ + 2 * kTcStages * (size_t)kTileBytes + 256;
constexpr long long kTcWaitCycles = 4000000000LL;  // ~2 s at 2 GHz

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
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}
// Wait for the phase of parity `parity` to complete, at most ~2 s.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > kTcWaitCycles) return false;
        __nanosleep(64);
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
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <int kEpi>
__global__ void __launch_bounds__(kTcThreads, 1)
gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const GemmArgs g) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;  // 128-byte swizzle atoms need 1024-byte alignment
    const uint32_t a_tiles = base, b_tiles = base + kTcStages * kTileBytes;
    const uint32_t bars = base + 2 * kTcStages * kTileBytes;  // full[S], empty[S], acc, tmem holder
    auto full = [&](int s) { return bars + 8u * s; };
    auto empty = [&](int s) { return bars + 8u * (kTcStages + s); };
    const uint32_t accb = bars + 8u * (2 * kTcStages);
    const uint32_t holder = accb + 8u;
    uint32_t* holder_ptr = reinterpret_cast<uint32_t*>(smem_raw + (holder - raw));

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * kTcM, n0 = blockIdx.x * kTcN;
    const int nk = (g.K + kTcK - 1) / kTcK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kTcStages; ++s) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        mbar_init(accb, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(holder), "r"(kTcN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *holder_ptr;

    __shared__ int s_fault;
    if (threadIdx.x == 0) s_fault = 0;
    __syncthreads();
    int issued = 0;  // k-blocks whose copies the producer started
    if (warp == 0 && lane == 0) {
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % kTcStages;
            if (!mbar_wait(empty(s), ((kb / kTcStages) & 1) ^ 1)) {
                s_fault = 1;
                break;
            }
            mbar_expect_tx(full(s), 2 * kTileBytes);
            tma_load_2d(a_tiles + s * kTileBytes, &tmA, kb * kTcK, m0, full(s));
            tma_load_2d(b_tiles + s * kTileBytes, &tmB, kb * kTcK, n0, full(s));
            ++issued;
        }
    } else if (warp == 1 && lane == 0) {
        constexpr uint32_t idesc = tc::idesc_bf16_f32(kTcM, kTcN);
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % kTcStages;
            if (!mbar_wait(full(s), (kb / kTcStages) & 1)) {
                s_fault = 1;
                break;
            }
            tc_fence_after();
#pragma unroll
            for (int kk = 0; kk < kTcK / 16; ++kk) {
                // K-major, 128-byte swizzle: 8-row groups 1024 bytes apart; the
                // 16-element K step advances the start address by 32 bytes
                const uint64_t ad = tc::smem_desc(a_tiles + s * kTileBytes + kk * 32, 16, 1024, tc::kSwizzle128B);
                const uint64_t bd = tc::smem_desc(b_tiles + s * kTileBytes + kk * 32, 16, 1024, tc::kSwizzle128B);
                tc_mma(tmem, ad, bd, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
            }
            tc_commit(empty(s));  // stage s is free once these MMAs have read it
        }
        tc_commit(accb);  // every MMA issued above has completed
    }
    __syncwarp();
    const bool acc_ok = mbar_wait(accb, 0);
    tc_fence_after();
    const bool fault = !acc_ok || s_fault;
    const int row = m0 + warp * 32 + lane;
    // 16-byte row accesses need ldc (C, pre) and ldh (h) to keep col0 aligned
    const bool vec = (g.ldc % 4 == 0) && (g.ldh % 8 == 0) &&
                     ((reinterpret_cast<uintptr_t>(g.C) | reinterpret_cast<uintptr_t>(g.pre) |
                       reinterpret_cast<uintptr_t>(g.hbf) | reinterpret_cast<uintptr_t>(g.bias)) & 15u) == 0;
    for (int c0 = 0; c0 < kTcN; c0 += 16) {
        uint32_t v[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
        if (row < g.M) {
            const int col0 = n0 + c0;
            if (vec && col0 + 16 <= g.N) {
                float f[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) f[j] = fault ? __int_as_float(0x7fc00000) : __uint_as_float(v[j]);
                epilogue16<kEpi>(g, row, col0, f);
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int col = col0 + j;
                    if (col < g.N)
                        epilogue<kEpi>(g, row, col, fault ? __int_as_float(0x7fc00000) : __uint_as_float(v[j]));
                }
            }
        }
    }
    if (fault && threadIdx.x == 0) {
        atomicAdd(&g_tc_faults, 1);
        // let the copies started for this tile land before the CTA leaves
        for (int kb = (issued > kTcStages ? issued - kTcStages : 0); kb < issued; ++kb)
            mbar_wait(full(kb % kTcStages), (kb / kTcStages) & 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcN) : "memory");
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

template <int kEpi>
cudaError_t launch_tc(const GemmArgs& g, cudaStream_t s) {
    static_assert(tc::valid_m128_n(kTcN), "instruction shape");
    CUtensorMap ma, mb;
    if (!make_map(&ma, g.A, g.M, g.K, g.lda) || !make_map(&mb, g.B, g.N, g.K, g.ldb)) return cudaErrorNotSupported;
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(gemm_tc_kernel<kEpi>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
    });
    if (attr != cudaSuccess) return attr;
    const dim3 grid((g.N + kTcN - 1) / kTcN, (g.M + kTcM - 1) / kTcM);
    gemm_tc_kernel<kEpi><<<grid, kTcThreads, kTcSmem, s>>>(ma, mb, g);
    return cudaGetLastError();
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
