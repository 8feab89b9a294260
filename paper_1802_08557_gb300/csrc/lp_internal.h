// lp_internal.h -- declarations shared by the host API (lp_api.cu) and the
// solver kernels.  Not part of the public ABI (see include/lpbatch.h).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include <string>

#include "lpbatch.h"

namespace lpb {

// Device-side view of a batch: per-LP sizes and element offsets, the data,
// and the result arrays (Section 4.1: tableau data in global memory).
struct DeviceBatch {
    const int32_t* m;
    const int32_t* n;
    const int64_t* a_off;
    const int64_t* b_off;
    const int64_t* c_off;
    const int64_t* x_off;  // prefix sums of n
    const int64_t* y_off;  // prefix sums of m
    const double* A;
    const double* b;
    const double* c;
    int32_t* status;
    int32_t* iters;
    double* obj;
    double* x;
    double* y;  // may be null
};

struct Tolerances {
    double eps_opt;
    double eps_piv;
    double eps_feas;
    double tau;
    int32_t max_iters;  // <= 0: 50*(m+n)
    // Screening windows derived from tau on the host (see tie_screen_* in
    // lp_api.cu): an upper bound on the tie window of Step 1 in units of the
    // FP64 key (< 0: always take the exact FP64 path), and the relative /
    // absolute FP32 windows of the Step 2 ratio screen.
    long long key_window;
    float ratio_rel;
    float ratio_abs;
};

// Per-LP outcome codes (same values as lp_status in include/lpbatch.h).
enum : int32_t { kOptimal = 0, kInfeasible = 1, kUnbounded = 2, kIterLimit = 3, kNumerical = 4 };

constexpr int kMaxThreads = 512;
constexpr int kMaxWarps = kMaxThreads / 32;
constexpr size_t kMaxSmemPerBlock = 227 * 1024;  // opt-in dynamic shared memory per CTA on sm_103

// Per-LP working storage of the FP64 simplex kernels.  The small part
// (reduction scratch) is always in shared memory.  The big part holds the
// condensed (Tucker) tableau -- R = m+1 (+1 phase-I row) rows x LD >= n+k+1
// columns, column 0 = right-hand side, then the non-basic variables -- plus
// per-row / per-column arrays.  It lives in shared memory for the resident
// kernel and in a global-memory workspace slot for the streamed kernel.  The
// k-independent arrays come first, so the kernel can place them before it has
// counted the k rows with b_i < 0.
struct SmallLayout {
    static constexpr size_t red64 = 0;                                   // 2 x kMaxWarps int64
    static constexpr size_t red32 = red64 + 2 * kMaxWarps * 8;           // 6 x kMaxWarps uint32
    static constexpr size_t total = red32 + 6 * kMaxWarps * 4;
};

struct BigLayout {
    int R, LD;
    size_t rkey, row_var, neg;   // k-independent
    size_t T, colE, col_var;     // k-dependent
    size_t total;
};

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

// streamed = false: odd row stride (column reads hit distinct shared-memory
// banks); streamed = true: rows padded to 32 bytes (aligned global sectors).
__host__ __device__ inline BigLayout big_layout(int m, int n, int k, bool streamed) {
    BigLayout L;
    L.R = m + 1 + (k > 0 ? 1 : 0);
    L.LD = streamed ? ((n + k + 1 + 3) & ~3) : ((n + k + 1) | 1);
    size_t o = 0;
    L.rkey = o;    o += align16((size_t)m * sizeof(long long));
    L.row_var = o; o += align16((size_t)m * sizeof(int));
    L.neg = o;     o += align16((size_t)m * sizeof(int));
    L.T = o;       o += align16((size_t)L.R * (size_t)L.LD * sizeof(double));
    L.colE = o;    o += align16((size_t)L.R * sizeof(double));
    L.col_var = o; o += align16((size_t)L.LD * sizeof(int));
    L.total = o;
    return L;
}

// Dynamic shared memory of the resident kernel for one LP.
__host__ __device__ inline size_t resident_smem_bytes(int m, int n, int k) {
    return SmallLayout::total + big_layout(m, n, k, false).total;
}

// Global workspace bytes of one streamed slot (256-byte aligned).
__host__ __device__ inline size_t streamed_slot_bytes(int m, int n, int k) {
    return (big_layout(m, n, k, true).total + 255) & ~size_t(255);
}

// Shared-memory layout of the mixed-precision kernel (after SmallLayout):
// FP64 certification vectors (x_B; y, which also holds the ray of an
// unbounded LP; the residual), the FP32 copy zf of the vector being refined
// (converted once per refinement step instead of once per use) and per-row
// arrays first (k-independent), then the FP32 condensed tableau (R x LD
// floats, LD a multiple of 4), its pivot-column copy colE (after the simplex:
// the FP32 copy of the residual) and the column labels.
struct MixedLayout {
    int R, LD;
    size_t scal, xb, yv, res, zf, row_var, neg, spos, slist, nbl;  // k-independent
    size_t T, colE, col_var;                           // k-dependent
    size_t total;
};

__host__ __device__ inline MixedLayout mixed_layout(int m, int n, int k) {
    MixedLayout L;
    L.R = m + 1 + (k > 0 ? 1 : 0);
    L.LD = (n + k + 1 + 3) & ~3;  // 16-byte rows for the quad update
    const size_t mn = (size_t)(m > n ? m : n);
    size_t o = 0;
    L.scal = o;    o += 32;  // broadcast scalars (objective, ray slope, Farkas gap)
    L.xb = o;      o += align16((size_t)m * 8);
    L.yv = o;      o += align16((size_t)m * 8);
    L.res = o;     o += align16(mn * 8);
    L.zf = o;      o += align16((size_t)m * 4);
    L.row_var = o; o += align16((size_t)m * 4);
    L.neg = o;     o += align16((size_t)m * 4);
    L.spos = o;    o += align16((size_t)m * 4);
    L.slist = o;   o += align16((size_t)m * 4);
    L.nbl = o;     o += align16((size_t)m * 4);
    L.T = o;       o += align16((size_t)L.R * (size_t)L.LD * 4);
    L.colE = o;    o += align16((size_t)L.R * 4);
    L.col_var = o; o += align16((size_t)L.LD * 4);
    L.total = o;
    return L;
}

__host__ __device__ inline size_t mixed_smem_bytes(int m, int n, int k) {
    return SmallLayout::total + mixed_layout(m, n, k).total;
}

// Tolerances of the FP32 simplex and of the FP64 certificate.
struct MixedParams {
    float eps_opt32, eps_piv32, eps_feas32;
    double cert_tol;     // primal (x scaled by max(1,|b|_inf)) and dual feasibility tolerance
    double conv_tol;     // refinement: every residual <= conv_tol * (|rhs| + |B||z|) ...
    double fwd_tol;      // ... and the last correction <= fwd_tol * max(|z_i|, fwd_floor * max|z|)
    double fwd_floor;    // (components far below the largest are judged against it)
    int32_t max_refine;  // refinement steps per vector
};

// Where the mixed-precision kernels put the LPs they do not certify: an LP
// whose FP64 tableau fits one CTA (resident_smem_bytes <= kMaxSmemPerBlock -
// 1 KiB) is appended to q (length *len, capacity cap), any other to qbig (the
// FP64 streamed re-solve).  The lengths are zeroed by the caller before the
// first mixed launch of a solve; a null queue or a full one records internal
// error 4 and reports the LP LP_NUMERICAL.
struct FallbackQueues {
    int32_t* q;
    int32_t* len;
    int32_t cap;
    int32_t* qbig;
    int32_t* lenbig;
    int32_t capbig;
};

cudaError_t mixed_kernel_prepare();
// One CTA per LP of order[0..count) (one warp per LP when threads == 32):
// FP32 simplex in shared memory, FP64 certificate; uncertified LPs to fq.
// diag: 3 int32 (count, first code, first LP) of internal-consistency
// failures (see record_internal_error); may be null.
cudaError_t launch_mixed(const DeviceBatch& B, const Tolerances& tol, const MixedParams& mp,
                         const int32_t* order, int32_t count, int threads, size_t smem,
                         const FallbackQueues& fq, int32_t* diag, cudaStream_t stream);

// Launchers (lp_fp64_simplex.cu).
constexpr int kStreamedThreads = 512;
// Shared memory of a streamed FP64 LP's staged rank-1 update (the rings of
// bulk-copied tableau chunks and the pivot row and column copies): the
// streamed kernel's dynamic shared memory, and the least the single-launch
// kernel gets when its batch has streamed LPs.  Enough for R + LD up to
// ~2,000 doubles; larger LPs take the plain update loop.
constexpr size_t kStreamStageBytes = 88 * 1024;
cudaError_t fp64_kernels_prepare();
// diag: 8 int32 internal-consistency record (see record_internal_error), or null.
cudaError_t launch_fp64_resident(const DeviceBatch& B, const Tolerances& tol, const int32_t* order,
                                 int32_t count, int threads, size_t smem, int32_t* diag, cudaStream_t stream);
// Persistent CTAs (grid = slots) take LPs of `order` from the atomic `counter`
// (must be 0 at launch); each CTA keeps its tableau in workspace slot
// blockIdx.x of `slot_bytes` bytes.
// count_dev (or null): a device-side length of `order`, read at launch and
// capped at `count`.
cudaError_t launch_fp64_streamed(const DeviceBatch& B, const Tolerances& tol, const int32_t* order,
                                 int32_t count, int slots, unsigned char* workspace, size_t slot_bytes,
                                 int32_t* counter, int32_t* diag, cudaStream_t stream,
                                 const int32_t* count_dev = nullptr);
// CTAs of the streamed kernel that fit on one SM.
cudaError_t fp64_single_prepare(size_t smem);
int fp64_single_ctas_per_sm(size_t smem);
cudaError_t launch_fp64_single(const DeviceBatch& B, const Tolerances& tol, const int32_t* order,
                               const uint8_t* resident, int32_t count, int ctas, size_t smem,
                               unsigned char* workspace, size_t slot_bytes, int32_t* counter, int32_t* diag,
                               cudaStream_t stream);
int fp64_streamed_ctas_per_sm();
// Resident kernel over a device-side LP list (persistent CTAs, atomic
// `counter` zeroed on `stream` before the launch).  `smem` must cover every
// listed LP's resident_smem_bytes and stay below kMaxSmemPerBlock - 1 KiB.
cudaError_t launch_fp64_resident_queue(const DeviceBatch& B, const Tolerances& tol, const int32_t* queue,
                                       const int32_t* queue_len, int32_t queue_cap, int32_t num_lps,
                                       int32_t* counter, int32_t* diag, int ctas, int threads,
                                       size_t smem, cudaStream_t stream);
int fp64_resident_queue_ctas_per_sm(int threads, size_t smem);

// Checks (lp_api.cu helpers in lp_prepare.cu): counts non-finite values of
// A, b, c into *bad and the rows with b_i < 0 of every LP into k[].
// FP64 simplex of one LP on a thread-block cluster of C CTAs (lp_cluster.cu):
// rows split over the CTAs' shared memory, rp rows each; row labels, column
// labels and exchange slots in every CTA.
struct ClusterLayout {
    int rp, LD;
    size_t row_var, neg, xch, col_var, T, prow, ob, colE, rkey, total;
};

constexpr size_t kClusterXchBytes = 128;  // exchange slots of one CTA (lp_cluster.cu)

__host__ __device__ inline ClusterLayout cluster_layout(int m, int n, int k, int C) {
    ClusterLayout L;
    const int R = m + 1 + (k > 0 ? 1 : 0);
    L.rp = (R + C - 1) / C;
    L.LD = (n + k + 1) | 1;
    size_t o = SmallLayout::total;
    L.row_var = o; o += align16((size_t)(m + 2) * 4);
    L.neg = o;     o += align16((size_t)m * 4);
    L.xch = o;     o += kClusterXchBytes;
    L.col_var = o; o += align16((size_t)L.LD * 4);
    L.T = o;       o += align16((size_t)L.rp * L.LD * 8);
    L.prow = o;    o += align16((size_t)L.LD * 8);
    L.ob = o;      o += align16((size_t)L.LD * 8);
    L.colE = o;    o += align16((size_t)L.rp * 8);
    L.rkey = o;    o += align16((size_t)L.rp * 8);
    L.total = o;
    return L;
}

constexpr int kMaxClusterCtas = 16;
size_t cluster_smem_bytes(int m, int n, int k, int C);
cudaError_t cluster_kernel_prepare();
int cluster_max_active(int C, size_t smem);
// count_dev (or null): a device-side length of `order`, read at launch and
// capped at `count`.
cudaError_t launch_fp64_cluster(const DeviceBatch& B, const Tolerances& tol, const int32_t* order, int32_t count,
                                int C, int clusters, size_t smem, int32_t* counter, int32_t* diag,
                                cudaStream_t stream, const int32_t* count_dev = nullptr);

// Persistent form of the mixed-precision kernel: CTAs take order[idx] for idx
// from an atomic counter (zeroed here) until *count.
cudaError_t launch_mixed_queue(const DeviceBatch& B, const Tolerances& tol, const MixedParams& mp,
                               const int32_t* order, const int32_t* count, int32_t* counter, int ctas, int threads,
                               size_t smem, const FallbackQueues& fq, int32_t* diag, cudaStream_t stream);
int mixed_queue_ctas_per_sm(int threads, size_t smem);

// Mixed precision with the FP32 tableau in a global workspace slot
// (lp_mixed_streamed.cu), for LPs whose FP32 tableau exceeds one CTA's shared
// memory: persistent CTAs of kMixedStreamedThreads threads take LPs of
// order[0..count) from `counter` (zeroed here); CTA i works in slot i of
// `slot_bytes` bytes (at least mixed_layout(m, n, k).total of every listed LP,
// a multiple of 256).  Results are bit-identical to the shared-memory kernels.
constexpr int kMixedStreamedThreads = 512;
// LPB_SCHED_SINGLE with mixed precision: one persistent launch of CTAs of this
// many threads (two per SM).  order[0 .. warp_from) are solved one per CTA,
// each LP's area in shared memory up to kMixedSingleSmemCap (resident[lp]),
// else in the CTA's global workspace slot; order[warp_from .. count) -- LPs
// the default plan gives one warp, with an area of at most
// kMixedSingleWarpArea -- one per warp, warp w of a CTA working in
// smem + w * kMixedSingleWarpArea (the CTA's shared memory is then
// kMixedSingleSmemCap).
constexpr int kMixedSingleThreads = 256;
constexpr size_t kMixedSingleSmemCap = 110 * 1024;
constexpr size_t kMixedSingleWarpArea = kMixedSingleSmemCap / (kMixedSingleThreads / 32);
static_assert(kMixedSingleWarpArea % 128 == 0, "warp areas of the single launch must stay 128-byte aligned");
cudaError_t mixed_single_prepare(size_t smem);
int mixed_single_ctas_per_sm(size_t smem);
cudaError_t launch_mixed_single(const DeviceBatch& B, const Tolerances& tol, const MixedParams& mp,
                                const int32_t* order, const uint8_t* resident, int32_t count, int32_t warp_from,
                                int ctas, size_t smem, unsigned char* workspace, size_t slot_bytes,
                                int32_t* counter, const FallbackQueues& fq, int32_t* diag, cudaStream_t stream);
cudaError_t launch_mixed_streamed(const DeviceBatch& B, const Tolerances& tol, const MixedParams& mp,
                                  const int32_t* order, int32_t count, int slots, unsigned char* workspace,
                                  size_t slot_bytes, int32_t* counter, const FallbackQueues& fq, int32_t* diag,
                                  cudaStream_t stream);
int mixed_streamed_ctas_per_sm();

// Learned warm start (lp_warm.cu): features [num_lps x (m+n)] = (b, c) as
// FP32; the restricted-LP solve and FP64 check of each LP from the network's
// logits (uncertified LPs appended to fb_queue); labels [num_lps x m] = 1 where
// an optimal LP's dual y_i > 0.
cudaError_t launch_warm_features(const DeviceBatch& B, int32_t num_lps, int32_t m, int32_t n, float* x,
                                 cudaStream_t s);
cudaError_t launch_warm(const DeviceBatch& B, const float* logits, int32_t num_lps, int32_t m, int32_t n,
                        int32_t kmax, int32_t max_rounds, int32_t max_iters, float threshold, double eps_opt,
                        double eps_piv, double cert_tol, int32_t* fb_queue, int32_t* fb_len, int32_t fb_cap,
                        const int32_t* queue, const int32_t* queue_len, int32_t* ov_queue, int32_t* ov_len,
                        int32_t* certified, int32_t* rounds, int32_t* diag, cudaStream_t s);
cudaError_t launch_warm_labels(const DeviceBatch& B, int32_t num_lps, int32_t m, float* labels, cudaStream_t s);
// Input and output widths and the device of a warm-start network.
void mlp_shape(const lp_mlp* net, int* n_in, int* n_out, int* device);

// Error reporting of the C ABI: records the text returned by lpb_last_error
// (per host thread) and returns the code.
lpb_err api_fail(lpb_err e, const std::string& msg);
lpb_err api_cuda_fail(cudaError_t err, const char* what);
void api_clear_error();

// Hyperbox LPs (Section 4.4, Eq. 7): obj[k] = max of L[k].x over the box
// (lo, hi shared when !box_per_lp, else one box per LP laid out like L); x
// (optional) the maximiser.  Device pointers; asynchronous on `stream`.
cudaError_t launch_hyperbox(const double* L, const double* lo, const double* hi, bool box_per_lp, double* obj,
                            double* x, int64_t num_lps, int dim, cudaStream_t stream);

// Input check of a batch's own device copies of A, b, c: *bad = the number of
// non-finite entries, each of which is set to 0.
cudaError_t launch_input_check(double* A, int64_t a_len, double* b, int64_t b_len, double* c, int64_t c_len,
                               unsigned long long* bad, cudaStream_t stream);
// k[lp] = the number of rows of LP lp with b_i < 0 (rows that get an artificial).
cudaError_t launch_count_negative_rhs(const DeviceBatch& B, int32_t num_lps, int32_t* k, cudaStream_t stream);

}  // namespace lpb
