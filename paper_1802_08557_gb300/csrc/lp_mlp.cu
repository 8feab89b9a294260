// lp_mlp.cu -- the warm-start network: a 3-layer perceptron (n_in -> h1 ->
// h2 -> n_out, ReLU) trained and run on the GPU by the kernels below.  No
// counterpart in the paper (its solver always starts from the slack basis).
//
// Precision scheme: every matrix product takes BF16 operands (round to
// nearest even) and accumulates in FP32 on the tensor cores; biases,
// pre-activations, the loss and all gradients are FP32; an operand is rounded
// to BF16 only where it enters a product.  Master weights and Adam moments
// are FP32.  The products run on the tcgen05 kernel (lp_mlp_tc.cu: TMA tiles,
// TMEM accumulator); the warp-level mma.sync m16n8k16 kernels below take the
// products it cannot address and serve as selectable reference forms.
//
// Every product is one NT GEMM, C[M x N] = A[M x K] . B[N x K]^T with both
// operands row-major and K contiguous.  To get there the network keeps each
// weight matrix in both orientations (BF16) and writes each activation and
// each gradient both as [batch x width] and as [width x batch]; K dimensions
// are padded to multiples of 32 with zeros, so the GEMM needs no K bound.
//  forward   a1 = x W1^T + b1 ; a2 = h1 W2^T + b2 ; z = h2 W3^T + b3
//  backward  dW3 = g3^T h2 ; dh2 = g3 W3 ; dW2 = g2^T h1 ; dh1 = g2 W2 ; dW1 = g1^T x
// Bias gradients are column sums in a fixed order (one thread per column), the
// loss a fixed-order sum: results do not depend on scheduling.

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "lp_internal.h"
#include "lp_mlp_gemm.cuh"
#include "lpbatch.h"

namespace lpb {

constexpr int kPadK = 32;        // K dimensions are padded to this multiple
constexpr int kInferRows = 131072;  // rows of BF16 activations held for inference chunks

inline int pad_to(int v, int q) { return (v + q - 1) / q * q; }

namespace {

constexpr int kBM = 64, kBN = 64, kBK = 32, kGemmThreads = 128;

__device__ __forceinline__ uint32_t ld_u32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <int kEpi>
__global__ void __launch_bounds__(kGemmThreads) gemm_nt_kernel(const GemmArgs g) {
    __shared__ __align__(16) __nv_bfloat16 As[kBM][kBK + 8];
    __shared__ __align__(16) __nv_bfloat16 Bs[kBN][kBK + 8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int gq = lane >> 2, tq = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.0f;

    for (int k0 = 0; k0 < g.K; k0 += kBK) {
        // tiles: 64 rows x 32 bf16 = 4 x 16-byte chunks per row; 2 chunks per thread per operand
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int idx = tid + c * kGemmThreads;
            const int row = idx >> 2, col = (idx & 3) * 8;
            uint4 va = make_uint4(0, 0, 0, 0), vb = make_uint4(0, 0, 0, 0);
            if (m0 + row < g.M) va = *reinterpret_cast<const uint4*>(g.A + (size_t)(m0 + row) * g.lda + k0 + col);
            if (n0 + row < g.N) vb = *reinterpret_cast<const uint4*>(g.B + (size_t)(n0 + row) * g.ldb + k0 + col);
            *reinterpret_cast<uint4*>(&As[row][col]) = va;
            *reinterpret_cast<uint4*>(&Bs[row][col]) = vb;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kBK; kk += 16) {
            uint32_t a[2][4], b[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm + i * 16 + gq;
                a[i][0] = ld_u32(&As[r][kk + 2 * tq]);
                a[i][1] = ld_u32(&As[r + 8][kk + 2 * tq]);
                a[i][2] = ld_u32(&As[r][kk + 2 * tq + 8]);
                a[i][3] = ld_u32(&As[r + 8][kk + 2 * tq + 8]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int n = wn + j * 8 + gq;
                b[j][0] = ld_u32(&Bs[n][kk + 2 * tq]);
                b[j][1] = ld_u32(&Bs[n][kk + 2 * tq + 8]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
    }

    // epilogue: element (row, col) of fragment (i, j, r)
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int row = m0 + wm + i * 16 + gq + ((r & 2) ? 8 : 0);
                const int col = n0 + wn + j * 8 + 2 * tq + (r & 1);
                if (row < g.M && col < g.N) epilogue<kEpi>(g, row, col, acc[i][j][r]);
            }
}

// The same product for large grids: 128 x 128 tiles over 8 warps (each
// 64 x 32), operands staged by 16-byte cp.async in two stages (the next K
// tile loads while the current one multiplies), fragments by ldmatrix.x4
// from rows padded to 80 bytes (no bank conflicts).  Each output element
// gets the same mma.sync sequence (K ascending in steps of 16) as in
// gemm_nt_kernel, so the results are bit-identical.
constexpr int kTM = 128, kTN = 128, kTK = 32, kTThreads = 256, kTLd = kTK + 8;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    const int bytes = valid ? 16 : 0;  // 0: the 16 bytes are zero-filled
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(gmem), "r"(bytes) : "memory");
}
__device__ __forceinline__ void ldmatrix_x4(uint32_t (&r)[4], const void* smem) {
    const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

template <int kEpi>
__global__ void __launch_bounds__(kTThreads) gemm_nt_tiled_kernel(const GemmArgs g) {
    __shared__ __align__(16) __nv_bfloat16 As[2][kTM][kTLd];
    __shared__ __align__(16) __nv_bfloat16 Bs[2][kTN][kTLd];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m0 = blockIdx.y * kTM, n0 = blockIdx.x * kTN;
    const int wm = (warp >> 2) * 64, wn = (warp & 3) * 32;
    const int gq = lane >> 2, tq = lane & 3;
    float acc[4][4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.0f;
    // one stage: 128 rows x 4 chunks of 16 bytes per operand, 2 chunks of
    // each per thread; rows past M (N) are zero-filled from a valid address
    auto load = [&](int st, int k0) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int idx = tid + c * kTThreads;
            const int row = idx >> 2, col = (idx & 3) * 8;
            const bool va = m0 + row < g.M, vb = n0 + row < g.N;
            cp_async16(&As[st][row][col], g.A + (size_t)(va ? m0 + row : 0) * g.lda + k0 + col, va);
            cp_async16(&Bs[st][row][col], g.B + (size_t)(vb ? n0 + row : 0) * g.ldb + k0 + col, vb);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    const int nk = g.K / kTK;
    load(0, 0);
    for (int kt = 0; kt < nk; ++kt) {
        const int st = kt & 1;
        if (kt + 1 < nk) {
            load(st ^ 1, (kt + 1) * kTK);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kTK; kk += 16) {
            uint32_t a[4][4], b[2][4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
                ldmatrix_x4(a[i], &As[st][wm + i * 16 + (lane & 7) + ((lane >> 3) & 1) * 8][kk + (lane >> 4) * 8]);
#pragma unroll
            for (int jj = 0; jj < 2; ++jj)
                ldmatrix_x4(b[jj], &Bs[st][wn + jj * 16 + (lane & 7) + (lane >> 4) * 8][kk + ((lane >> 3) & 1) * 8]);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint32_t bj[2] = {b[j >> 1][(j & 1) * 2], b[j >> 1][(j & 1) * 2 + 1]};
                    mma_bf16(acc[i][j], a[i], bj);
                }
        }
        __syncthreads();  // this stage is reloaded two tiles later
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int row = m0 + wm + i * 16 + gq + ((r & 2) ? 8 : 0);
                const int col = n0 + wn + j * 8 + 2 * tq + (r & 1);
                if (row < g.M && col < g.N) epilogue<kEpi>(g, row, col, acc[i][j][r]);
            }
}

// Kernel forms of the product (lp_mlp_gemm_bf16's `form`).
enum GemmForm : int { kFormAuto = 0, kFormMma64 = 1, kFormMma128 = 2, kFormTc = 3 };

// 128 x 128 tiles when they give at least one per SM, else 64 x 64 (small
// products, e.g. the weight gradients of one training batch): same results.
template <int kEpi>
cudaError_t gemm(const GemmArgs& a, cudaStream_t s, int form = kFormAuto) {
    if (form == kFormTc || form == kFormAuto) {
        // the tcgen05 kernel; in AUTO the mma.sync kernels take the products
        // it cannot address (no tensor map for these strides or alignment)
        const cudaError_t e = gemm_tc(kEpi, &a, s);
        if (form == kFormTc || e != cudaErrorNotSupported) return e;
    }
    const int64_t big_tiles = (int64_t)((a.N + kTN - 1) / kTN) * ((a.M + kTM - 1) / kTM);
    if (form == kFormMma128 || (form == kFormAuto && big_tiles >= 152)) {
        const dim3 grid((a.N + kTN - 1) / kTN, (a.M + kTM - 1) / kTM);
        gemm_nt_tiled_kernel<kEpi><<<grid, kTThreads, 0, s>>>(a);
    } else {
        const dim3 grid((a.N + kBN - 1) / kBN, (a.M + kBM - 1) / kBM);
        gemm_nt_kernel<kEpi><<<grid, kGemmThreads, 0, s>>>(a);
    }
    return cudaGetLastError();
}

// x (FP32 [batch x n_in]) -> (x - mean) * inv_std as BF16, [batch x ld] and
// transposed [n_in x ldT] (xbT null: inference, no transposed copy); padding
// columns/rows were zeroed at allocation and rows batch..ldT-1 of the
// transposed copy are zeroed here.
__global__ void features_kernel(const float* __restrict__ x, int batch, int n_in, const float* __restrict__ mean,
                                const float* __restrict__ inv_std, __nv_bfloat16* __restrict__ xb, int ld,
                                __nv_bfloat16* __restrict__ xbT, int ldT) {
    if (!xbT) {
        const int64_t total = (int64_t)batch * n_in;
        for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
             e += (int64_t)gridDim.x * blockDim.x) {
            const int r = (int)(e / n_in), c = (int)(e - (int64_t)r * n_in);
            xb[(size_t)r * ld + c] = __float2bfloat16_rn((x[e] - mean[c]) * inv_std[c]);
        }
        return;
    }
    const int64_t total = (int64_t)ldT * n_in;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / n_in), c = (int)(e - (int64_t)r * n_in);
        __nv_bfloat16 v = __float2bfloat16_rn(0.0f);
        if (r < batch) {
            v = __float2bfloat16_rn((x[(size_t)r * n_in + c] - mean[c]) * inv_std[c]);
            xb[(size_t)r * ld + c] = v;
        }
        xbT[(size_t)c * ldT + r] = v;
    }
}

// Weighted BCE: g3 = w (sigmoid(z) - y) / (batch n_out), as FP32 and BF16 (both
// orientations); per-row loss sums (fixed order) into row_loss[batch].
__global__ void loss_grad_kernel(const float* __restrict__ z, const float* __restrict__ y, int batch, int n_out,
                                 float pos_weight, float* __restrict__ g, __nv_bfloat16* __restrict__ gb, int ldb,
                                 __nv_bfloat16* __restrict__ gbT, int ldT, double* __restrict__ row_loss) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= ldT) return;
    const double inv = 1.0 / ((double)batch * n_out);
    double sum = 0.0;
    for (int c = 0; c < n_out; ++c) {
        float gv = 0.0f;
        if (r < batch) {
            const size_t i = (size_t)r * n_out + c;
            const double zz = z[i], yy = y[i];
            const double w = yy * pos_weight + (1.0 - yy);
            const double sp_neg = (zz > 0.0) ? log1p(exp(-zz)) : -zz + log1p(exp(zz));  // softplus(-z)
            const double sp_pos = sp_neg + zz;                                           // softplus(z)
            sum += w * (yy * sp_neg + (1.0 - yy) * sp_pos);
            const double sig = 1.0 / (1.0 + exp(-zz));
            gv = (float)(w * (sig - yy) * inv);
            g[i] = gv;
            gb[(size_t)r * ldb + c] = __float2bfloat16_rn(gv);
        }
        gbT[(size_t)c * ldT + r] = __float2bfloat16_rn(gv);
    }
    if (r < batch) row_loss[r] = sum * inv;
}

// Column sums of g [batch x n] (stride ld) in row order: one thread per column.
__global__ void colsum_kernel(const float* __restrict__ g, int batch, int n, int ld, float* __restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    double s = 0.0;
    for (int r = 0; r < batch; ++r) s += g[(size_t)r * ld + c];
    out[c] = (float)s;
}

// Fixed-order sum of row_loss -> *out (one thread).
__global__ void sum_kernel(const double* __restrict__ v, int n, double* __restrict__ out) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += v[i];
    *out = s;
}

// Adam on one parameter array (FP32 master p, moments m, v; gradient gr), then
// the BF16 copies: wb [rows x ldw] and wbT [cols x ldwT] (null for biases).
__global__ void adam_kernel(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ gr, int64_t count, int cols, float lr, float beta1, float beta2,
                            float eps, float c1, float c2, __nv_bfloat16* __restrict__ wb, int ldw,
                            __nv_bfloat16* __restrict__ wbT, int ldwT) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const double g = gr[i];
        const double mm = beta1 * (double)m[i] + (1.0 - beta1) * g;
        const double vv = beta2 * (double)v[i] + (1.0 - beta2) * g * g;
        const double step = lr * (mm / c1) / (sqrt(vv / c2) + eps);
        const float np = (float)((double)p[i] - step);
        p[i] = np;
        m[i] = (float)mm;
        v[i] = (float)vv;
        if (wb) {
            const int r = (int)(i / cols), c = (int)(i - (int64_t)r * cols);
            const __nv_bfloat16 b = __float2bfloat16_rn(np);
            wb[(size_t)r * ldw + c] = b;
            wbT[(size_t)c * ldwT + r] = b;
        }
    }
}

// BF16 copies of a weight matrix [rows x cols] (FP32) in both orientations.
__global__ void weights_bf16_kernel(const float* __restrict__ w, int rows, int cols, __nv_bfloat16* __restrict__ wb,
                                    int ldw, __nv_bfloat16* __restrict__ wbT, int ldwT) {
    const int64_t total = (int64_t)rows * cols;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / cols), c = (int)(i - (int64_t)r * cols);
        const __nv_bfloat16 b = __float2bfloat16_rn(w[i]);
        wb[(size_t)r * ldw + c] = b;
        wbT[(size_t)c * ldwT + r] = b;
    }
}

// Columns [from, to) of a [rows x ld] BF16 matrix set to zero (the batch
// padding of the transposed activations, which the weight-gradient products
// sum over).
__global__ void zero_cols_kernel(__nv_bfloat16* __restrict__ buf, int rows, int ld, int from, int to) {
    const int w = to - from;
    const int64_t total = (int64_t)rows * w;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / w), c = from + (int)(i - (int64_t)r * w);
        buf[(size_t)r * ld + c] = __float2bfloat16_rn(0.0f);
    }
}

// Input statistics (lp_mlp_fit_scaling), two deterministic passes: per
// column chunk sums of x (pass 0) or of (x - mean)^2 (pass 1) in FP64 over
// rows [chunk*rows_per_chunk, ...), thread (tx, ty) of a 32 x 8 block taking
// column blockIdx.x*32 + tx and every 8th row; partials [chunks x n] in a
// fixed order, then reduce_columns_kernel sums them in chunk order.
constexpr int kStatRows = 8;
__global__ void column_partials_kernel(const float* __restrict__ x, int64_t rows, int n, int64_t rows_per_chunk,
                                       const double* __restrict__ mean, double* __restrict__ partial) {
    __shared__ double red[kStatRows][32];
    const int c = blockIdx.x * 32 + threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.y * rows_per_chunk;
    const int64_t r1 = min(rows, r0 + rows_per_chunk);
    double acc = 0.0;
    if (c < n) {
        const double mu = mean ? mean[c] : 0.0;
        for (int64_t r = r0 + threadIdx.y; r < r1; r += kStatRows) {
            const double v = (double)x[r * n + c];
            acc = mean ? __fma_rn(v - mu, v - mu, acc) : acc + v;
        }
    }
    red[threadIdx.y][threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.y == 0 && c < n) {
        double s = 0.0;
        for (int i = 0; i < kStatRows; ++i) s += red[i][threadIdx.x];
        partial[(size_t)blockIdx.y * n + c] = s;
    }
}

// mean (pass 0) or 1/std (pass 1; 1 for a constant feature) from the partials.
__global__ void reduce_columns_kernel(const double* __restrict__ partial, int chunks, int n, int64_t rows,
                                      double* __restrict__ mean, float* __restrict__ mean32,
                                      float* __restrict__ inv_std, int pass) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    double s = 0.0;
    for (int k = 0; k < chunks; ++k) s += partial[(size_t)k * n + c];
    if (pass == 0) {
        mean[c] = s / (double)rows;
        mean32[c] = (float)(s / (double)rows);
    } else {
        const double sd = sqrt(s / (double)rows);
        inv_std[c] = sd > 0.0 ? (float)(1.0 / sd) : 1.0f;
    }
}

// h = bf16(relu(a)) of given pre-activations a [batch x n] (FP32), as the
// forward epilogue writes it: hb [batch x ldh] and hbT [n x ldt] (rows
// batch..ldt-1 of hbT zeroed: the batch padding of the weight-gradient sums).
__global__ void relu_bf16_kernel(const float* __restrict__ a, int batch, int n, __nv_bfloat16* __restrict__ hb,
                                 int ldh, __nv_bfloat16* __restrict__ hbT, int ldt) {
    const int64_t total = (int64_t)ldt * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / n), c = (int)(e - (int64_t)r * n);
        __nv_bfloat16 h = __float2bfloat16_rn(0.0f);
        if (r < batch) {
            h = __float2bfloat16_rn(fmaxf(a[(size_t)r * n + c], 0.0f));
            hb[(size_t)r * ldh + c] = h;
        }
        hbT[(size_t)c * ldt + r] = h;
    }
}

inline unsigned grid_for(int64_t n, int threads = 256) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, 152 * 16));
}

}  // namespace

// ---- the model ---------------------------------------------------------------

struct MlpLayer {
    int in, out, in_pad, out_pad;       // K of the forward product and of dX
    float *W, *b, *mW, *vW, *mb, *vb, *gW, *gb;
    __nv_bfloat16 *Wb, *WbT;            // [out x in_pad], [in x out_pad]
};

struct MlpModel {
    int n_in, h1, h2, n_out, max_batch, train_batch, bpad;
    MlpLayer L[3];
    float *mean, *inv_std;
    // activations: xb, h1b, h2b for max_batch rows (the inference chunk), the
    // rest (training only) for bpad rows
    __nv_bfloat16 *xb, *xbT, *h1b, *h1bT, *h2b, *h2bT, *g3b, *g3bT, *g2b, *g2bT, *g1b, *g1bT;
    float *a1, *a2, *z, *g3, *g2, *g1, *tmp;
    double *row_loss, *loss;
    int64_t step = 0;
    std::vector<void*> allocs;
};

namespace {

template <typename T>
cudaError_t zalloc(MlpModel* m, T** p, size_t count) {
    void* v = nullptr;
    cudaError_t err = cudaMalloc(&v, std::max<size_t>(count, 1) * sizeof(T));
    if (err != cudaSuccess) return err;
    m->allocs.push_back(v);
    *p = static_cast<T*>(v);
    return cudaMemset(v, 0, std::max<size_t>(count, 1) * sizeof(T));
}

}  // namespace

cudaError_t mlp_alloc(MlpModel* m) {
    cudaError_t e;
    const int dims[4] = {m->n_in, m->h1, m->h2, m->n_out};
    for (int l = 0; l < 3; ++l) {
        MlpLayer& L = m->L[l];
        L.in = dims[l];
        L.out = dims[l + 1];
        L.in_pad = pad_to(L.in, kPadK);
        L.out_pad = pad_to(L.out, kPadK);
        const size_t nw = (size_t)L.out * L.in;
        if ((e = zalloc(m, &L.W, nw)) || (e = zalloc(m, &L.b, L.out)) || (e = zalloc(m, &L.mW, nw)) ||
            (e = zalloc(m, &L.vW, nw)) || (e = zalloc(m, &L.mb, L.out)) || (e = zalloc(m, &L.vb, L.out)) ||
            (e = zalloc(m, &L.gW, nw)) || (e = zalloc(m, &L.gb, L.out)) ||
            (e = zalloc(m, &L.Wb, (size_t)L.out * L.in_pad)) || (e = zalloc(m, &L.WbT, (size_t)L.in * L.out_pad)))
            return e;
    }
    const size_t B = (size_t)m->bpad;
    const size_t BI = (size_t)std::max(m->max_batch, m->bpad);
    const int in_pad = m->L[0].in_pad, h1p = m->L[1].in_pad, h2p = m->L[2].in_pad, outp = m->L[2].out_pad;
    if ((e = zalloc(m, &m->mean, m->n_in)) || (e = zalloc(m, &m->inv_std, m->n_in)) ||
        (e = zalloc(m, &m->xb, BI * in_pad)) || (e = zalloc(m, &m->xbT, (size_t)m->n_in * B)) ||
        (e = zalloc(m, &m->h1b, BI * h1p)) || (e = zalloc(m, &m->h1bT, (size_t)m->h1 * B)) ||
        (e = zalloc(m, &m->h2b, BI * h2p)) || (e = zalloc(m, &m->h2bT, (size_t)m->h2 * B)) ||
        (e = zalloc(m, &m->g3b, B * outp)) || (e = zalloc(m, &m->g3bT, (size_t)m->n_out * B)) ||
        (e = zalloc(m, &m->g2b, B * h2p)) || (e = zalloc(m, &m->g2bT, (size_t)m->h2 * B)) ||
        (e = zalloc(m, &m->g1b, B * h1p)) || (e = zalloc(m, &m->g1bT, (size_t)m->h1 * B)) ||
        (e = zalloc(m, &m->a1, B * m->h1)) || (e = zalloc(m, &m->a2, B * m->h2)) ||
        (e = zalloc(m, &m->z, B * m->n_out)) || (e = zalloc(m, &m->g3, B * m->n_out)) ||
        (e = zalloc(m, &m->g2, B * m->h2)) || (e = zalloc(m, &m->g1, B * m->h1)) ||
        (e = zalloc(m, &m->tmp, B * std::max(m->h1, m->h2))) || (e = zalloc(m, &m->row_loss, B)) ||
        (e = zalloc(m, &m->loss, 1)))
        return e;
    return cudaSuccess;
}

void mlp_free(MlpModel* m) {
    for (void* p : m->allocs) cudaFree(p);
    m->allocs.clear();
}

cudaError_t mlp_refresh_bf16(MlpModel* m, cudaStream_t s) {
    for (int l = 0; l < 3; ++l) {
        const MlpLayer& L = m->L[l];
        weights_bf16_kernel<<<grid_for((int64_t)L.out * L.in), 256, 0, s>>>(L.W, L.out, L.in, L.Wb, L.in_pad, L.WbT,
                                                                             L.out_pad);
    }
    return cudaGetLastError();
}

// Forward pass for `batch` rows of raw features x (FP32, device).  With
// logits != null the logits are copied there ([batch x n_out], FP32).
cudaError_t mlp_forward(MlpModel* m, const float* x, int batch, float* logits, cudaStream_t s) {
    cudaError_t e;
    const int bT = pad_to(batch, kPadK);
    const bool infer = logits != nullptr;  // only the BF16 activations and the logits are written
    features_kernel<<<grid_for((int64_t)bT * m->n_in), 256, 0, s>>>(x, batch, m->n_in, m->mean, m->inv_std, m->xb,
                                                                      m->L[0].in_pad, infer ? nullptr : m->xbT, bT);
    if ((e = cudaGetLastError())) return e;
    GemmArgs g{};
    // layer 1
    g.A = m->xb; g.lda = m->L[0].in_pad; g.B = m->L[0].Wb; g.ldb = m->L[0].in_pad;
    g.M = batch; g.N = m->h1; g.K = m->L[0].in_pad; g.C = infer ? nullptr : m->a1; g.ldc = m->h1;
    g.bias = m->L[0].b;
    g.hbf = m->h1b; g.ldh = m->L[1].in_pad; g.hbfT = infer ? nullptr : m->h1bT; g.ldt = bT;
    if ((e = gemm<kEpiBiasReLU>(g, s))) return e;
    // layer 2
    g = GemmArgs{};
    g.A = m->h1b; g.lda = m->L[1].in_pad; g.B = m->L[1].Wb; g.ldb = m->L[1].in_pad;
    g.M = batch; g.N = m->h2; g.K = m->L[1].in_pad; g.C = infer ? nullptr : m->a2; g.ldc = m->h2;
    g.bias = m->L[1].b;
    g.hbf = m->h2b; g.ldh = m->L[2].in_pad; g.hbfT = infer ? nullptr : m->h2bT; g.ldt = bT;
    if ((e = gemm<kEpiBiasReLU>(g, s))) return e;
    // layer 3
    g = GemmArgs{};
    g.A = m->h2b; g.lda = m->L[2].in_pad; g.B = m->L[2].Wb; g.ldb = m->L[2].in_pad;
    g.M = batch; g.N = m->n_out; g.K = m->L[2].in_pad; g.C = logits ? logits : m->z; g.ldc = m->n_out;  // logits: inference
    g.bias = m->L[2].b;
    if ((e = gemm<kEpiBias>(g, s))) return e;
    if (!infer && bT > batch) {
        zero_cols_kernel<<<grid_for((int64_t)m->h1 * (bT - batch)), 256, 0, s>>>(m->h1bT, m->h1, bT, batch, bT);
        zero_cols_kernel<<<grid_for((int64_t)m->h2 * (bT - batch)), 256, 0, s>>>(m->h2bT, m->h2, bT, batch, bT);
        zero_cols_kernel<<<grid_for((int64_t)m->h2 * (bT - batch)), 256, 0, s>>>(m->g2bT, m->h2, bT, batch, bT);
        zero_cols_kernel<<<grid_for((int64_t)m->h1 * (bT - batch)), 256, 0, s>>>(m->g1bT, m->h1, bT, batch, bT);
    }
    return cudaGetLastError();
}

// Backward pass from the forward values a1, a2 (pre-activations) and z
// (logits), with the BF16 activations (x, h1, h2, both orientations) already
// in the model's buffers; gradients into L[l].gW / gb; loss into m->loss.
cudaError_t mlp_backward_from(MlpModel* m, const float* y, int batch, float pos_weight, const float* a1,
                              const float* a2, const float* z, cudaStream_t s) {
    cudaError_t e;
    const int bT = pad_to(batch, kPadK);
    loss_grad_kernel<<<(bT + 127) / 128, 128, 0, s>>>(z, y, batch, m->n_out, pos_weight, m->g3, m->g3b,
                                                      m->L[2].out_pad, m->g3bT, bT, m->row_loss);
    sum_kernel<<<1, 1, 0, s>>>(m->row_loss, batch, m->loss);
    if ((e = cudaGetLastError())) return e;
    GemmArgs g{};
    // dW3 = g3^T h2 : [n_out x h2], K = batch
    g.A = m->g3bT; g.lda = bT; g.B = m->h2bT; g.ldb = bT; g.M = m->n_out; g.N = m->h2; g.K = bT;
    g.C = m->L[2].gW; g.ldc = m->h2;
    if ((e = gemm<kEpiStore>(g, s))) return e;
    colsum_kernel<<<(m->n_out + 127) / 128, 128, 0, s>>>(m->g3, batch, m->n_out, m->n_out, m->L[2].gb);
    // g2 = (g3 W3) * [a2 > 0] : [batch x h2], K = n_out (B operand = W3^T [h2 x out_pad])
    g = GemmArgs{};
    g.A = m->g3b; g.lda = m->L[2].out_pad; g.B = m->L[2].WbT; g.ldb = m->L[2].out_pad; g.M = batch; g.N = m->h2;
    g.K = m->L[2].out_pad; g.C = m->g2; g.ldc = m->h2; g.pre = a2; g.hbf = m->g2b; g.ldh = m->L[2].in_pad;
    g.hbfT = m->g2bT; g.ldt = bT;
    if ((e = gemm<kEpiMaskGrad>(g, s))) return e;
    // dW2 = g2^T h1
    g = GemmArgs{};
    g.A = m->g2bT; g.lda = bT; g.B = m->h1bT; g.ldb = bT; g.M = m->h2; g.N = m->h1; g.K = bT;
    g.C = m->L[1].gW; g.ldc = m->h1;
    if ((e = gemm<kEpiStore>(g, s))) return e;
    colsum_kernel<<<(m->h2 + 127) / 128, 128, 0, s>>>(m->g2, batch, m->h2, m->h2, m->L[1].gb);
    // g1 = (g2 W2) * [a1 > 0]
    g = GemmArgs{};
    g.A = m->g2b; g.lda = m->L[1].out_pad; g.B = m->L[1].WbT; g.ldb = m->L[1].out_pad; g.M = batch; g.N = m->h1;
    g.K = m->L[1].out_pad; g.C = m->g1; g.ldc = m->h1; g.pre = a1; g.hbf = m->g1b; g.ldh = m->L[1].in_pad;
    g.hbfT = m->g1bT; g.ldt = bT;
    if ((e = gemm<kEpiMaskGrad>(g, s))) return e;
    // dW1 = g1^T x
    g = GemmArgs{};
    g.A = m->g1bT; g.lda = bT; g.B = m->xbT; g.ldb = bT; g.M = m->h1; g.N = m->n_in; g.K = bT;
    g.C = m->L[0].gW; g.ldc = m->n_in;
    if ((e = gemm<kEpiStore>(g, s))) return e;
    colsum_kernel<<<(m->h1 + 127) / 128, 128, 0, s>>>(m->g1, batch, m->h1, m->h1, m->L[0].gb);
    return cudaGetLastError();
}

// Forward + backward; gradients into L[l].gW / gb; loss into m->loss.
cudaError_t mlp_backward(MlpModel* m, const float* x, const float* y, int batch, float pos_weight, cudaStream_t s) {
    cudaError_t e;
    if ((e = mlp_forward(m, x, batch, nullptr, s))) return e;
    return mlp_backward_from(m, y, batch, pos_weight, m->a1, m->a2, m->z, s);
}

// The backward pass at given forward values (layer-wise checks of the
// backward kernels): x's BF16 copies by the features kernel, h1 and h2 as
// bf16(relu(a)) in both orientations, then mlp_backward_from on a1, a2, z.
cudaError_t mlp_backward_at(MlpModel* m, const float* x, const float* a1, const float* a2, const float* z,
                            const float* y, int batch, float pos_weight, cudaStream_t s) {
    cudaError_t e;
    const int bT = pad_to(batch, kPadK);
    features_kernel<<<grid_for((int64_t)bT * m->n_in), 256, 0, s>>>(x, batch, m->n_in, m->mean, m->inv_std, m->xb,
                                                                      m->L[0].in_pad, m->xbT, bT);
    relu_bf16_kernel<<<grid_for((int64_t)bT * m->h1), 256, 0, s>>>(a1, batch, m->h1, m->h1b, m->L[1].in_pad,
                                                                     m->h1bT, bT);
    relu_bf16_kernel<<<grid_for((int64_t)bT * m->h2), 256, 0, s>>>(a2, batch, m->h2, m->h2b, m->L[2].in_pad,
                                                                     m->h2bT, bT);
    if (bT > batch) {
        zero_cols_kernel<<<grid_for((int64_t)m->h2 * (bT - batch)), 256, 0, s>>>(m->g2bT, m->h2, bT, batch, bT);
        zero_cols_kernel<<<grid_for((int64_t)m->h1 * (bT - batch)), 256, 0, s>>>(m->g1bT, m->h1, bT, batch, bT);
    }
    if ((e = cudaGetLastError())) return e;
    return mlp_backward_from(m, y, batch, pos_weight, a1, a2, z, s);
}

// One product through a chosen kernel form (lp_mlp_gemm_bf16).
cudaError_t mlp_gemm_dispatch(int epi, int form, const GemmArgs& g, cudaStream_t s) {
    switch (epi) {
        case kEpiStore: return gemm<kEpiStore>(g, s, form);
        case kEpiBiasReLU: return gemm<kEpiBiasReLU>(g, s, form);
        case kEpiBias: return gemm<kEpiBias>(g, s, form);
        default: return gemm<kEpiMaskGrad>(g, s, form);
    }
}

cudaError_t mlp_adam(MlpModel* m, float lr, cudaStream_t s) {
    ++m->step;
    const float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
    const float c1 = (float)(1.0 - std::pow(0.9, (double)m->step));
    const float c2 = (float)(1.0 - std::pow(0.999, (double)m->step));
    for (int l = 0; l < 3; ++l) {
        MlpLayer& L = m->L[l];
        const int64_t nw = (int64_t)L.out * L.in;
        adam_kernel<<<grid_for(nw), 256, 0, s>>>(L.W, L.mW, L.vW, L.gW, nw, L.in, lr, beta1, beta2, eps, c1, c2,
                                                  L.Wb, L.in_pad, L.WbT, L.out_pad);
        adam_kernel<<<grid_for(L.out), 256, 0, s>>>(L.b, L.mb, L.vb, L.gb, L.out, 1, lr, beta1, beta2, eps, c1, c2,
                                                     nullptr, 0, nullptr, 0);
    }
    return cudaGetLastError();
}

}  // namespace lpb

// ---- C ABI ---------------------------------------------------------------------

struct lp_mlp {
    int device = 0;
    lpb::MlpModel m;
};

namespace {

using lpb::api_fail;
using lpb::api_cuda_fail;

// He-uniform weights, rounded to BF16-representable values (splitmix64 stream).
float bf16_round_host(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7F800000u) == 0x7F800000u) return f;
    u = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}

uint64_t splitmix64(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

int64_t param_count(const lpb::MlpModel& m) {
    int64_t n = 0;
    for (const lpb::MlpLayer& L : m.L) n += (int64_t)L.out * L.in + L.out;
    return n;
}

bool on_device(const void* p, int dev) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeManaged || (at.type == cudaMemoryTypeDevice && at.device == dev);
}

class Dev {
  public:
    explicit Dev(int d) {
        cudaGetDevice(&prev_);
        if (prev_ != d) cudaSetDevice(d);
        d_ = d;
    }
    ~Dev() {
        if (prev_ != d_) cudaSetDevice(prev_);
    }

  private:
    int prev_ = 0, d_ = 0;
};

lpb_err copy_params(lp_mlp* net, float* host, bool to_host) {
    Dev guard(net->device);
    size_t off = 0;
    for (lpb::MlpLayer& L : net->m.L) {
        const size_t nw = (size_t)L.out * L.in;
        cudaError_t e = to_host ? cudaMemcpy(host + off, L.W, nw * 4, cudaMemcpyDeviceToHost)
                                : cudaMemcpy(L.W, host + off, nw * 4, cudaMemcpyHostToDevice);
        if (e) return api_cuda_fail(e, "parameter copy");
        off += nw;
        e = to_host ? cudaMemcpy(host + off, L.b, (size_t)L.out * 4, cudaMemcpyDeviceToHost)
                    : cudaMemcpy(L.b, host + off, (size_t)L.out * 4, cudaMemcpyHostToDevice);
        if (e) return api_cuda_fail(e, "parameter copy");
        off += L.out;
    }
    if (!to_host) {
        // new weights: Adam restarts, BF16 copies refreshed
        for (lpb::MlpLayer& L : net->m.L) {
            const size_t nw = (size_t)L.out * L.in;
            cudaMemset(L.mW, 0, nw * 4);
            cudaMemset(L.vW, 0, nw * 4);
            cudaMemset(L.mb, 0, (size_t)L.out * 4);
            cudaMemset(L.vb, 0, (size_t)L.out * 4);
        }
        net->m.step = 0;
        cudaError_t e = lpb::mlp_refresh_bf16(&net->m, nullptr);
        if (!e) e = cudaDeviceSynchronize();
        if (e) return api_cuda_fail(e, "weight refresh");
    }
    return LPB_OK;
}

}  // namespace

namespace lpb {

void mlp_shape(const lp_mlp* net, int* n_in, int* n_out, int* device) {
    *n_in = net->m.n_in;
    *n_out = net->m.n_out;
    *device = net->device;
}

}  // namespace lpb

extern "C" {

lpb_err lp_mlp_create(lp_mlp** out, int32_t n_in, int32_t n_h1, int32_t n_h2, int32_t n_out, int32_t max_batch,
                      uint64_t seed) {
    lpb::api_clear_error();
    if (!out) return api_fail(LPB_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_in < 1 || n_h1 < 1 || n_h2 < 1 || n_out < 1 || max_batch < 1)
        return api_fail(LPB_EINVAL, "layer widths and max_batch must be >= 1");
    if (n_in > LPB_MAX_MLP_WIDTH || n_h1 > LPB_MAX_MLP_WIDTH || n_h2 > LPB_MAX_MLP_WIDTH ||
        n_out > LPB_MAX_MLP_WIDTH || max_batch > LPB_MAX_MLP_BATCH)
        return api_fail(LPB_ETOOBIG, "a layer width or max_batch exceeds the limit");
    lp_mlp* net = new lp_mlp();
    cudaGetDevice(&net->device);
    lpb::MlpModel& m = net->m;
    m.n_in = n_in; m.h1 = n_h1; m.h2 = n_h2; m.n_out = n_out;
    // BF16 activations for at least kInferRows rows, so that inference runs
    // in large chunks (whole-GPU GEMMs) even when training batches are small;
    // the training buffers for max_batch rows only
    m.max_batch = std::max<int>(max_batch, lpb::kInferRows);
    m.train_batch = max_batch;
    m.bpad = lpb::pad_to(max_batch, lpb::kPadK);
    cudaError_t e = lpb::mlp_alloc(&m);
    if (e) {
        lpb::mlp_free(&m);
        delete net;
        return e == cudaErrorMemoryAllocation ? api_fail(LPB_ENOMEM, "network buffers") : api_cuda_fail(e, "network buffers");
    }
    // He-uniform initial weights, zero biases; identity input scaling
    std::vector<float> p((size_t)param_count(m));
    uint64_t st = seed;
    size_t off = 0;
    for (const lpb::MlpLayer& L : m.L) {
        const double lim = std::sqrt(6.0 / L.in);
        for (int64_t i = 0; i < (int64_t)L.out * L.in; ++i) {
            const double u = (double)(splitmix64(st) >> 11) * (1.0 / 9007199254740992.0);
            p[off++] = bf16_round_host((float)((2.0 * u - 1.0) * lim));
        }
        for (int i = 0; i < L.out; ++i) p[off++] = 0.0f;
    }
    std::vector<float> zero(n_in, 0.0f), one(n_in, 1.0f);
    if ((e = cudaMemcpy(m.mean, zero.data(), n_in * 4, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(m.inv_std, one.data(), n_in * 4, cudaMemcpyHostToDevice))) {
        lpb::mlp_free(&m);
        delete net;
        return api_cuda_fail(e, "input scaling");
    }
    lpb_err r = copy_params(net, p.data(), false);
    if (r != LPB_OK) {
        lpb::mlp_free(&m);
        delete net;
        return r;
    }
    *out = net;
    return LPB_OK;
}

lpb_err lp_mlp_num_params(const lp_mlp* net, int64_t* count) {
    if (!net || !count) return api_fail(LPB_EINVAL, "net or count is NULL");
    *count = param_count(net->m);
    return LPB_OK;
}

lpb_err lp_mlp_set_params(lp_mlp* net, const float* params) {
    lpb::api_clear_error();
    if (!net || !params) return api_fail(LPB_EINVAL, "net or params is NULL");
    return copy_params(net, const_cast<float*>(params), false);
}

lpb_err lp_mlp_get_params(lp_mlp* net, float* params) {
    lpb::api_clear_error();
    if (!net || !params) return api_fail(LPB_EINVAL, "net or params is NULL");
    return copy_params(net, params, true);
}

lpb_err lp_mlp_set_scaling(lp_mlp* net, const float* mean, const float* inv_std) {
    lpb::api_clear_error();
    if (!net || !mean || !inv_std) return api_fail(LPB_EINVAL, "net, mean or inv_std is NULL");
    Dev guard(net->device);
    cudaError_t e;
    if ((e = cudaMemcpy(net->m.mean, mean, (size_t)net->m.n_in * 4, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(net->m.inv_std, inv_std, (size_t)net->m.n_in * 4, cudaMemcpyHostToDevice)))
        return api_cuda_fail(e, "input scaling");
    return LPB_OK;
}

lpb_err lp_mlp_fit_scaling(lp_mlp* net, const float* x, int64_t rows, void* stream) {
    lpb::api_clear_error();
    if (!net || !x) return api_fail(LPB_EINVAL, "net or x is NULL");
    if (rows < 1) return api_fail(LPB_EINVAL, "rows must be >= 1");
    Dev guard(net->device);
    if (!on_device(x, net->device)) return api_fail(LPB_EINVAL, "x must be device memory of the network's device");
    const int n = net->m.n_in;
    const int64_t per_chunk = std::max<int64_t>(4096, (rows + 1023) / 1024);
    const int chunks = (int)((rows + per_chunk - 1) / per_chunk);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double *partial = nullptr, *mean = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&partial, (size_t)chunks * n * sizeof(double), s);
    if (!e) e = cudaMallocAsync((void**)&mean, (size_t)n * sizeof(double), s);
    if (!e) {
        const dim3 grid((n + 31) / 32, chunks), block(32, lpb::kStatRows);
        lpb::column_partials_kernel<<<grid, block, 0, s>>>(x, rows, n, per_chunk, nullptr, partial);
        lpb::reduce_columns_kernel<<<(n + 127) / 128, 128, 0, s>>>(partial, chunks, n, rows, mean, net->m.mean,
                                                                   nullptr, 0);
        lpb::column_partials_kernel<<<grid, block, 0, s>>>(x, rows, n, per_chunk, mean, partial);
        lpb::reduce_columns_kernel<<<(n + 127) / 128, 128, 0, s>>>(partial, chunks, n, rows, nullptr, nullptr,
                                                                   net->m.inv_std, 1);
        e = cudaGetLastError();
    }
    if (partial) cudaFreeAsync(partial, s);
    if (mean) cudaFreeAsync(mean, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) return api_cuda_fail(e, "input statistics");
    return LPB_OK;
}

lpb_err lp_mlp_get_scaling(lp_mlp* net, float* mean, float* inv_std) {
    lpb::api_clear_error();
    if (!net || !mean || !inv_std) return api_fail(LPB_EINVAL, "net, mean or inv_std is NULL");
    Dev guard(net->device);
    cudaError_t e;
    if ((e = cudaMemcpy(mean, net->m.mean, (size_t)net->m.n_in * 4, cudaMemcpyDeviceToHost)) ||
        (e = cudaMemcpy(inv_std, net->m.inv_std, (size_t)net->m.n_in * 4, cudaMemcpyDeviceToHost)))
        return api_cuda_fail(e, "input scaling");
    return LPB_OK;
}

lpb_err lp_mlp_forward(lp_mlp* net, const float* x, int64_t batch, float* logits, void* stream) {
    lpb::api_clear_error();
    if (!net || !x || !logits) return api_fail(LPB_EINVAL, "net, x or logits is NULL");
    if (batch < 0) return api_fail(LPB_EINVAL, "batch must be >= 0");
    if (batch == 0) return LPB_OK;
    Dev guard(net->device);
    if (!on_device(x, net->device) || !on_device(logits, net->device))
        return api_fail(LPB_EINVAL, "x and logits must be device memory of the network's device");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    lpb::MlpModel& m = net->m;
    for (int64_t r0 = 0; r0 < batch; r0 += m.max_batch) {
        const int nb = (int)std::min<int64_t>(m.max_batch, batch - r0);
        cudaError_t e = lpb::mlp_forward(&m, x + r0 * m.n_in, nb, logits + r0 * m.n_out, s);
        if (e) return api_cuda_fail(e, "network forward");
    }
    return LPB_OK;
}

lpb_err lp_mlp_train_step(lp_mlp* net, const float* x, const float* y, int32_t batch, float lr, float pos_weight,
                          double* loss, void* stream) {
    lpb::api_clear_error();
    if (!net || !x || !y) return api_fail(LPB_EINVAL, "net, x or y is NULL");
    if (batch < 1 || batch > net->m.train_batch) return api_fail(LPB_EINVAL, "batch must be in [1, max_batch]");
    if (!(lr > 0.0f) || !(pos_weight > 0.0f)) return api_fail(LPB_EINVAL, "lr and pos_weight must be > 0");
    Dev guard(net->device);
    if (!on_device(x, net->device) || !on_device(y, net->device))
        return api_fail(LPB_EINVAL, "x and y must be device memory of the network's device");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if ((e = lpb::mlp_backward(&net->m, x, y, batch, pos_weight, s)) || (e = lpb::mlp_adam(&net->m, lr, s)))
        return api_cuda_fail(e, "training step");
    if (loss) {
        if ((e = cudaMemcpyAsync(loss, net->m.loss, sizeof(double), cudaMemcpyDeviceToHost, s)) ||
            (e = cudaStreamSynchronize(s)))
            return api_cuda_fail(e, "loss");
    }
    return LPB_OK;
}

}  // extern "C"

namespace {

// Gradients of the last backward pass (parameter layout) and its loss to the host.
lpb_err copy_gradients(lp_mlp* net, float* grads, double* loss) {
    cudaError_t e;
    size_t off = 0;
    for (lpb::MlpLayer& L : net->m.L) {
        const size_t nw = (size_t)L.out * L.in;
        if ((e = cudaMemcpy(grads + off, L.gW, nw * 4, cudaMemcpyDeviceToHost))) return api_cuda_fail(e, "gradients");
        off += nw;
        if ((e = cudaMemcpy(grads + off, L.gb, (size_t)L.out * 4, cudaMemcpyDeviceToHost)))
            return api_cuda_fail(e, "gradients");
        off += L.out;
    }
    if (loss && (e = cudaMemcpy(loss, net->m.loss, sizeof(double), cudaMemcpyDeviceToHost)))
        return api_cuda_fail(e, "loss");
    return LPB_OK;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" {

lpb_err lp_mlp_gradients(lp_mlp* net, const float* x, const float* y, int32_t batch, float pos_weight, float* grads,
                         double* loss, void* stream) {
    lpb::api_clear_error();
    if (!net || !x || !y || !grads) return api_fail(LPB_EINVAL, "net, x, y or grads is NULL");
    if (batch < 1 || batch > net->m.train_batch) return api_fail(LPB_EINVAL, "batch must be in [1, max_batch]");
    if (!(pos_weight > 0.0f)) return api_fail(LPB_EINVAL, "pos_weight must be > 0");
    Dev guard(net->device);
    if (!on_device(x, net->device) || !on_device(y, net->device))
        return api_fail(LPB_EINVAL, "x and y must be device memory of the network's device");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = lpb::mlp_backward(&net->m, x, y, batch, pos_weight, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) return api_cuda_fail(e, "forward/backward");
    return copy_gradients(net, grads, loss);
}

lpb_err lp_mlp_gradients_at(lp_mlp* net, const float* x, const float* a1, const float* a2, const float* z,
                            const float* y, int32_t batch, float pos_weight, float* grads, double* loss,
                            void* stream) {
    lpb::api_clear_error();
    if (!net || !x || !a1 || !a2 || !z || !y || !grads) return api_fail(LPB_EINVAL, "a pointer argument is NULL");
    if (batch < 1 || batch > net->m.train_batch) return api_fail(LPB_EINVAL, "batch must be in [1, max_batch]");
    if (!(pos_weight > 0.0f)) return api_fail(LPB_EINVAL, "pos_weight must be > 0");
    Dev guard(net->device);
    for (const void* p : {(const void*)x, (const void*)a1, (const void*)a2, (const void*)z, (const void*)y})
        if (!on_device(p, net->device))
            return api_fail(LPB_EINVAL, "x, a1, a2, z and y must be device memory of the network's device");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = lpb::mlp_backward_at(&net->m, x, a1, a2, z, y, batch, pos_weight, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) return api_cuda_fail(e, "backward");
    return copy_gradients(net, grads, loss);
}

lpb_err lp_mlp_gemm_bf16(int32_t epilogue, int32_t form, int32_t M, int32_t N, int32_t K, const uint16_t* A,
                         int32_t lda, const uint16_t* B, int32_t ldb, float* C, int32_t ldc, const float* bias,
                         const float* pre, uint16_t* h, int32_t ldh, uint16_t* hT, int32_t ldt, void* stream) {
    lpb::api_clear_error();
    if (epilogue < LPB_EPI_STORE || epilogue > LPB_EPI_MASK_GRAD) return api_fail(LPB_EINVAL, "unknown epilogue");
    if (form < LPB_GEMM_AUTO || form > LPB_GEMM_TC) return api_fail(LPB_EINVAL, "unknown kernel form");
    if (M < 1 || N < 1 || K < 1 || K % 32 != 0) return api_fail(LPB_EINVAL, "M, N >= 1 and K a positive multiple of 32");
    if (M > LPB_MAX_MLP_BATCH * 8 || N > LPB_MAX_MLP_BATCH * 8 || K > LPB_MAX_MLP_BATCH * 8)
        return api_fail(LPB_ETOOBIG, "a dimension exceeds the limit");
    if (!A || !B || lda < K || ldb < K || lda % 8 != 0 || ldb % 8 != 0 || !aligned16(A) || !aligned16(B))
        return api_fail(LPB_EINVAL, "A and B: 16-byte aligned, lda and ldb >= K and multiples of 8");
    const bool need_c = epilogue != LPB_EPI_BIAS_RELU;
    const bool need_bias = epilogue == LPB_EPI_BIAS || epilogue == LPB_EPI_BIAS_RELU;
    const bool need_h = epilogue == LPB_EPI_BIAS_RELU || epilogue == LPB_EPI_MASK_GRAD;
    if ((need_c && !C) || (C && ldc < N) || (need_bias && !bias) || (epilogue == LPB_EPI_MASK_GRAD && (!pre || !C)))
        return api_fail(LPB_EINVAL, "C (ldc >= N), bias or pre missing for this epilogue");
    if ((need_h && (!h || ldh < N)) || (epilogue == LPB_EPI_MASK_GRAD && !hT) || (hT && ldt < M))
        return api_fail(LPB_EINVAL, "h (ldh >= N) or hT (ldt >= M) missing for this epilogue");
    int dev = 0;
    cudaGetDevice(&dev);
    for (const void* p : {(const void*)A, (const void*)B, (const void*)C, (const void*)bias, (const void*)pre,
                          (const void*)h, (const void*)hT})
        if (p && !on_device(p, dev)) return api_fail(LPB_EINVAL, "arrays must be device memory of the current device");
    lpb::GemmArgs g{};
    g.A = reinterpret_cast<const __nv_bfloat16*>(A);
    g.B = reinterpret_cast<const __nv_bfloat16*>(B);
    g.C = C;
    g.M = M; g.N = N; g.K = K; g.lda = lda; g.ldb = ldb; g.ldc = ldc;
    g.bias = need_bias ? bias : nullptr;
    g.pre = epilogue == LPB_EPI_MASK_GRAD ? pre : nullptr;
    g.hbf = need_h ? reinterpret_cast<__nv_bfloat16*>(h) : nullptr;
    g.hbfT = need_h ? reinterpret_cast<__nv_bfloat16*>(hT) : nullptr;
    g.ldh = ldh; g.ldt = ldt;
    const cudaError_t e = lpb::mlp_gemm_dispatch(epilogue, form, g, static_cast<cudaStream_t>(stream));
    if (e == cudaErrorNotSupported) return api_fail(LPB_EINVAL, "no tensor map for these operands");
    if (e) return api_cuda_fail(e, "product");
    return LPB_OK;
}

lpb_err lp_mlp_tc_faults(int32_t* count) {
    lpb::api_clear_error();
    if (!count) return api_fail(LPB_EINVAL, "count is NULL");
    int c = 0;
    const cudaError_t e = lpb::gemm_tc_faults(&c);
    if (e) return api_cuda_fail(e, "fault counter");
    *count = c;
    return LPB_OK;
}

lpb_err lp_mlp_destroy(lp_mlp* net) {
    if (!net) return LPB_OK;
    {
        Dev guard(net->device);
        cudaDeviceSynchronize();
        lpb::mlp_free(&net->m);
    }
    delete net;
    return LPB_OK;
}

}  // extern "C"
