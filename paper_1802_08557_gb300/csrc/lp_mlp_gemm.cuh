// lp_mlp_gemm.cuh -- arguments and fused epilogues of the warm-start
// network's matrix product C[M x N] = A[M x K] . B[N x K]^T (BF16 operands,
// FP32 accumulation), shared by the mma.sync kernels (lp_mlp.cu) and the
// tcgen05 kernel (lp_mlp_tc.cu).
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

namespace lpb {
namespace {

// Epilogue variants of the GEMM.
enum Epi : int {
    kEpiStore = 0,   // C = acc (FP32)
    kEpiBiasReLU,    // pre = acc + bias -> C; h = relu(pre) -> hbf [M x ldh], hbfT [N x ldt]
    kEpiBias,        // C = acc + bias
    kEpiMaskGrad,    // g = acc * (pre > 0) -> C; g -> hbf, hbfT
};

struct GemmArgs {
    const __nv_bfloat16* A;  // [M x K], lda
    const __nv_bfloat16* B;  // [N x K], ldb
    float* C;                // [M x N], ldc
    int M, N, K, lda, ldb, ldc;
    const float* bias;       // [N]
    const float* pre;        // [M x N] (ld = ldc): ReLU mask source
    __nv_bfloat16* hbf;      // [M x ldh]
    __nv_bfloat16* hbfT;     // [N x ldt]
    int ldh, ldt;
};

// Epilogue of one output element (row, col) with accumulator v.
template <int kEpi>
__device__ __forceinline__ void epilogue(const GemmArgs& g, int row, int col, float v) {
    const size_t ci = (size_t)row * g.ldc + col;
    if (kEpi == kEpiStore) {
        g.C[ci] = v;
    } else if (kEpi == kEpiBias) {
        g.C[ci] = v + g.bias[col];
    } else if (kEpi == kEpiBiasReLU) {
        // (inference: no pre-activation and no transposed copy,
        // which only the backward pass reads)
        v = v + g.bias[col];
        if (g.C) g.C[ci] = v;
        const __nv_bfloat16 h = __float2bfloat16_rn(fmaxf(v, 0.0f));
        g.hbf[(size_t)row * g.ldh + col] = h;
        if (g.hbfT) g.hbfT[(size_t)col * g.ldt + row] = h;
    } else {  // kEpiMaskGrad
        v = (g.pre[ci] > 0.0f) ? v : 0.0f;
        g.C[ci] = v;
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        g.hbf[(size_t)row * g.ldh + col] = h;
        g.hbfT[(size_t)col * g.ldt + row] = h;
    }
}

// Epilogue of 16 consecutive columns col0..col0+15 of one row with
// accumulators v[]: the same arithmetic as epilogue() element by element, with
// 16-byte loads and stores of the row-major arrays.  The caller guarantees
// that all 16 columns are inside N and that C, pre (ldc), h (ldh) and bias are
// 16-byte aligned at col0.
template <int kEpi>
__device__ __forceinline__ void epilogue16(const GemmArgs& g, int row, int col0, float (&v)[16]) {
    const size_t ci = (size_t)row * g.ldc + col0;
    if (kEpi == kEpiBias || kEpi == kEpiBiasReLU) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 b = *reinterpret_cast<const float4*>(g.bias + col0 + 4 * q);
            v[4 * q] = v[4 * q] + b.x; v[4 * q + 1] = v[4 * q + 1] + b.y;
            v[4 * q + 2] = v[4 * q + 2] + b.z; v[4 * q + 3] = v[4 * q + 3] + b.w;
        }
    }
    if (kEpi == kEpiMaskGrad) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 p = *reinterpret_cast<const float4*>(g.pre + ci + 4 * q);
            v[4 * q] = (p.x > 0.0f) ? v[4 * q] : 0.0f; v[4 * q + 1] = (p.y > 0.0f) ? v[4 * q + 1] : 0.0f;
            v[4 * q + 2] = (p.z > 0.0f) ? v[4 * q + 2] : 0.0f; v[4 * q + 3] = (p.w > 0.0f) ? v[4 * q + 3] : 0.0f;
        }
    }
    if (g.C) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
            *reinterpret_cast<float4*>(g.C + ci + 4 * q) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    }
    if (kEpi == kEpiBiasReLU || kEpi == kEpiMaskGrad) {
        __nv_bfloat16 h[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) h[j] = __float2bfloat16_rn(kEpi == kEpiBiasReLU ? fmaxf(v[j], 0.0f) : v[j]);
        uint4* dst = reinterpret_cast<uint4*>(g.hbf + (size_t)row * g.ldh + col0);
        dst[0] = *reinterpret_cast<const uint4*>(&h[0]);
        dst[1] = *reinterpret_cast<const uint4*>(&h[8]);
        if (g.hbfT) {
#pragma unroll
            for (int j = 0; j < 16; ++j) g.hbfT[(size_t)(col0 + j) * g.ldt + row] = h[j];
        }
    }
}

}  // namespace

// The product on the tensor cores' tcgen05 path (TMA-staged tiles, TMEM
// accumulator); lp_mlp_tc.cu.  Returns cudaErrorNotSupported when a tensor
// map cannot be made for these arguments (alignment, strides).
cudaError_t gemm_tc(int epi, const void* args, cudaStream_t s);
// CTAs of that kernel that gave up on a bounded wait since the library loaded.
cudaError_t gemm_tc_faults(int* count);

}  // namespace lpb
