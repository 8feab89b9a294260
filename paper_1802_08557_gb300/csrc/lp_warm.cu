// lp_warm.cu -- learned warm start: the warm-start network predicts which
// constraints are active at the optimum; the LP restricted to those rows is
// solved and its optimum checked against the full LP in FP64.  No counterpart
// in the paper (its solver always starts from the slack basis, Section 3).
//
// Per LP (one CTA):
//  1. R = rows whose logit exceeds the threshold (capacity kmax);
//  2. the restricted LP  max c^T x  s.t.  A_R x <= b_R, x >= 0  (all n columns,
//     |R| rows) is solved by the simplex method of Section 3 (Steps 1-3, slack
//     basis; b_R >= 0 is required, there is no phase I here);
//  3. its optimum x (and duals y_R) is checked on the full LP in FP64 from the
//     original data: every row A_i x <= b_i + tol_p, y_R >= -tol_d, every
//     reduced cost A_R^T y_R - c >= -tol_d, and c^T x = b_R^T y_R within 1e-9.
//     Together these prove x optimal for the full LP (y = y_R on R, 0 off R is
//     dual feasible and complementary);
//  4. rows the optimum violates are added to R and step 2 runs again
//     (constraint generation: the simplex continues from the proposal until
//     the restricted optimum is feasible); an unbounded restricted LP adds the
//     rows that bound its ray.  With R outgrowing kmax rows the LP goes to the
//     overflow queue when one is given (the host runs a second pass with a
//     larger kmax over it); after max_rounds rounds, with b_R < 0, when a
//     check fails, or overflowing without that queue, it goes to the queue of
//     the cold FP64 solve, which decides it.
// Tolerances: tol_p = cert_tol * max(1, max|b|), tol_d = cert_tol * max(1, max|c|).

#include <algorithm>
#include <climits>

#include "lp_device.cuh"
#include "lp_internal.h"

namespace lpb {
namespace {

constexpr int kWarmThreads = 128;

struct WarmArgs {
    DeviceBatch B;
    const float* logits;   // [num_lps x m]
    int32_t num_lps, m, n, kmax, max_rounds, max_iters;
    float threshold;       // logit threshold
    double eps_opt, eps_piv, cert_tol;
    int32_t* fb_queue;
    int32_t* fb_len;
    int32_t fb_cap;
    const int32_t* queue;      // non-null: solve the LPs queue[0 .. *queue_len) (else LP = CTA index)
    const int32_t* queue_len;
    int32_t* ov_queue;         // non-null: LPs whose restricted LP outgrows kmax rows go here
    int32_t* ov_len;           //   (capacity fb_cap) instead of to the cold queue
    int32_t* certified;    // count of LPs certified here
    int32_t* rounds;       // total restricted solves
    int32_t* diag;
};

__global__ void __launch_bounds__(kWarmThreads) warm_features_kernel(DeviceBatch B, int32_t num_lps, int32_t m,
                                                                      int32_t n, float* __restrict__ x) {
    const int64_t w = (int64_t)m + n;
    const int64_t total = (int64_t)num_lps * w;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = e / w;
        const int i = (int)(e - k * w);
        x[e] = (i < m) ? (float)B.b[B.b_off[k] + i] : (float)B.c[B.c_off[k] + (i - m)];
    }
}

// Dynamic shared memory of the warm kernel.
struct WarmLayout {
    int LD;  // tableau row stride (doubles)
    size_t rows, inR, col_var, row_var, T, colE, rkey, xv, yv, total;
};

__host__ __device__ inline WarmLayout warm_layout(int m, int n, int kmax) {
    WarmLayout L;
    L.LD = (n + 1) | 1;
    size_t o = SmallLayout::total;
    L.rows = o;    o += align16((size_t)kmax * 4);
    L.inR = o;     o += align16((size_t)m * 4);
    L.col_var = o; o += align16((size_t)(n + 1) * 4);
    L.row_var = o; o += align16((size_t)kmax * 4);
    L.T = o;       o += align16((size_t)(kmax + 1) * L.LD * 8);
    L.colE = o;    o += align16((size_t)(kmax + 1) * 8);
    L.rkey = o;    o += align16((size_t)(kmax + 1) * 8);
    L.xv = o;      o += align16((size_t)n * 8);
    L.yv = o;      o += align16((size_t)kmax * 8);
    L.total = o;
    return L;
}

// One LP of the warm solve (the whole CTA).
__device__ __forceinline__ void warm_one(const WarmArgs& a, const int lp) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x, nt = blockDim.x;
    Reducer red{reinterpret_cast<long long*>(smem + SmallLayout::red64),
                reinterpret_cast<unsigned*>(smem + SmallLayout::red32), nt >> 5, tid >> 5, tid & 31};
    const int m = a.m, n = a.n, kmax = a.kmax;
    const WarmLayout L = warm_layout(m, n, kmax);
    int* rows = reinterpret_cast<int*>(smem + L.rows);
    int* inR = reinterpret_cast<int*>(smem + L.inR);
    int* col_var = reinterpret_cast<int*>(smem + L.col_var);
    int* row_var = reinterpret_cast<int*>(smem + L.row_var);
    double* T = reinterpret_cast<double*>(smem + L.T);
    double* colE = reinterpret_cast<double*>(smem + L.colE);
    long long* rkey = reinterpret_cast<long long*>(smem + L.rkey);  // Step 2 ratio keys
    __shared__ double s_rinv;
    double* xv = reinterpret_cast<double*>(smem + L.xv);
    double* yv = reinterpret_cast<double*>(smem + L.yv);
    const int LD = L.LD;
    const double* __restrict__ A = a.B.A + a.B.a_off[lp];
    const double* __restrict__ bv = a.B.b + a.B.b_off[lp];
    const double* __restrict__ cv = a.B.c + a.B.c_off[lp];
    const float* lg = a.logits + (size_t)lp * m;

    // tolerances from the data
    long long bk = 0x3FF0000000000000LL, ck = 0x3FF0000000000000LL;  // 1.0
    for (int i = tid; i < m; i += nt) bk = max(bk, abskey(bv[i]));
    for (int j = tid; j < n; j += nt) ck = max(ck, abskey(cv[j]));
    const double tol_p = a.cert_tol * __longlong_as_double(-red.min_i64(-bk));
    const double tol_d = a.cert_tol * __longlong_as_double(-red.min_i64(-ck));
    // thresholds of the checks as order keys: the checks compare by integer
    // operations (an FP64 compare takes the FP64 pipe, which bounds this
    // kernel); a NaN never passes
    const long long k_neg_tol_p = okey(-tol_p), k_tol_p = okey(tol_p), k_neg_tol_d = okey(-tol_d);
    const long long k_eps_piv = okey(a.eps_piv), k_zero = 0;
    const long long k_neg_eps_opt = okey(-a.eps_opt), k_huge = okey(1e300);

    // 1. predicted rows, ascending
    int k = 0;
    for (int i0 = 0; i0 < m; i0 += nt) {
        const int i = i0 + tid;
        const bool sel = (i < m) && (lg[i] > a.threshold);
        int tot;
        const int pos = k + red.prefix_count(sel, tot);
        if (i < m) inR[i] = sel ? 1 : 0;
        if (sel && pos < kmax) rows[pos] = i;
        k += tot;
    }
    __syncthreads();
    bool ok = k <= kmax;
    bool overflow = !ok;  // the rows outgrew kmax (the only failure a larger kmax can cure)
    int iters = 0, round = 0;
    bool certified = false;
    while (ok && !certified) {
        if (round >= a.max_rounds) { ok = false; break; }
        ++round;
        // ---- 2. restricted tableau: rows R (slack basis), columns 1..n structurals
        unsigned negb = 0, dummy;
        for (int r = tid; r < k; r += nt) negb += below_key(bv[rows[r]], k_zero) ? 1u : 0u;
        red.count_min(negb, 0u, negb, dummy);
        if (negb) { ok = false; break; }
        for (int j = tid; j <= n; j += nt) col_var[j] = j - 1;  // column j holds structural j-1 (0: RHS)
        for (int r = tid; r < k; r += nt) row_var[r] = n + r;   // slack of restricted row r
        {
            // rows R of [b | A] in one flat pass (all loads of a thread in flight)
            const int W = n + 1;
            int r = tid / W, j = tid - (tid / W) * W;
            const int dr = nt / W, dj = nt - dr * W;
            for (int idx = tid; idx < k * W; idx += nt) {
                T[(size_t)r * LD + j] = (j == 0) ? bv[rows[r]] : A[(size_t)rows[r] * n + j - 1];
                r += dr;
                j += dj;
                if (j >= W) { j -= W; ++r; }
            }
        }
        {
            double* To = T + (size_t)k * LD;
            for (int j = tid; j <= n; j += nt) To[j] = (j == 0) ? 0.0 : -cv[j - 1];
        }
        __syncthreads();
        int status = -1, e_unb = -1;
        const double* To = T + (size_t)k * LD;
        while (status < 0) {
            // Step 1: most negative reduced cost; exact ties to the lowest label
            long long loc = LLONG_MAX;
            for (int j = 1 + tid; j <= n; j += nt) loc = min(loc, okey(To[j]));
            const long long dmin = red.min_i64(loc);
            if (!(dmin < k_neg_eps_opt)) { status = 0; break; }
            unsigned esel = 0xFFFFFFFFu;
            for (int j = 1 + tid; j <= n; j += nt)
                if (okey(To[j]) == dmin) esel = min(esel, ((unsigned)col_var[j] << 16) | (unsigned)j);
            esel = red.min_u32(esel);
            const int e = (int)(esel & 0xFFFFu);
            if (e < 1 || e > n) { status = 4; break; }
            // Step 2: minimum ratio over rows with t_re > eps_piv; exact ties to
            // the lowest row.  FP32 screen first (operands truncated to FP32
            // by integer operations, rows with an operand outside [2^-100,
            // 2^100] always candidates, window 2^-12 relative + 2^-20
            // absolute: far wider than the screen's error); exact FP64
            // ratios only when more than one row survives.  The row is the
            // plain rule's in every case; the FP64 divides it saves are most
            // of this kernel's FP64-pipe time besides the update.
            int floc = INT_MAX;
            for (int r = tid; r <= k; r += nt) {
                const double t = T[(size_t)r * LD + e];
                colE[r] = t;
                long long code = LLONG_MAX;  // not eligible
                if (r < k && above_key(t, k_eps_piv)) {
                    const double beta = T[(size_t)r * LD];
                    const int et = dexp(t), eb = dexp(beta);
                    if (et >= -100 && et <= 100 && (abskey(beta) == 0 || (eb >= -100 && eb <= 100))) {
                        const int fk = fkey(__fdividef(f64_to_f32_trunc(beta), f64_to_f32_trunc(t)));
                        code = fk;
                        floc = min(floc, fk);
                    } else {
                        code = LLONG_MIN;  // unscreened: always a candidate
                    }
                }
                rkey[r] = code;
            }
            const int fmin = red.min_i32(floc);  // barrier: rkey, colE complete
            long long fwin = LLONG_MIN;
            if (fmin != INT_MAX) {
                const float fm = fval(fmin);
                fwin = fkey(fm + __fmaf_rn(0x1p-12f, fabsf(fm), 0x1p-20f));
            }
            unsigned lcnt = 0, lsel = 0xFFFFFFFFu;
            for (int r = tid; r < k; r += nt) {
                const long long code = rkey[r];
                if (code == LLONG_MIN || (code != LLONG_MAX && code <= fwin)) {
                    ++lcnt;
                    lsel = min(lsel, (unsigned)r);
                }
            }
            red.count_min(lcnt, lsel, lcnt, lsel);
            if (lcnt == 0) { status = 2; e_unb = e; break; }
            if (lcnt > 1) {
                // several candidates: their exact ratios, the exact rule
                long long rl = LLONG_MAX;
                for (int r = tid; r < k; r += nt) {
                    const long long code = rkey[r];
                    long long rk = LLONG_MAX;
                    if (code == LLONG_MIN || (code != LLONG_MAX && code <= fwin))
                        rk = okey(__ddiv_rn(T[(size_t)r * LD], colE[r]));
                    rkey[r] = rk;
                    rl = min(rl, rk);
                }
                const long long rmin = red.min_i64(rl);
                unsigned sel = 0xFFFFFFFFu;
                for (int r = tid; r < k; r += nt)
                    if (rkey[r] == rmin) sel = min(sel, (unsigned)r);
                lsel = red.min_u32(sel);
            }
            const int l = (int)lsel;
            if (l < 0 || l >= k || abskey(colE[l]) >= k_huge) { status = 4; break; }
            if (iters >= a.max_iters) { status = 3; break; }
            // Step 3: pivot row times one reciprocal (the restricted LP only
            // proposes the rows; its optimum is checked on the full LP below),
            // computed once and shared: a warp's FP64 instruction costs the
            // whole warp's pipe time
            if (tid == 0) s_rinv = __drcp_rn(colE[l]);
            __syncthreads();
            const double rinv = s_rinv;
            double* Tl = T + (size_t)l * LD;
            for (int j = tid; j <= n; j += nt) Tl[j] = (j == e) ? rinv : __dmul_rn(Tl[j], rinv);
            if (tid == 0) {
                const int ev = col_var[e];
                col_var[e] = row_var[l];
                row_var[l] = ev;
            }
            __syncthreads();
            {
                // every other row, over the (k+1) x (n+1) elements in one flat
                // pass (no idle lanes at row ends)
                const int W = n + 1;
                int r = tid / W, j = tid - (tid / W) * W;
                const int dr = nt / W, dj = nt - dr * W;
                for (int idx = tid; idx < (k + 1) * W; idx += nt) {
                    if (r != l) {
                        double* t = T + (size_t)r * LD + j;
                        *t = __fma_rn(-colE[r], Tl[j], (j == e) ? 0.0 : *t);
                    }
                    r += dr;
                    j += dj;
                    if (j >= W) { j -= W; ++r; }
                }
            }
            __syncthreads();
            ++iters;
        }
        if (status == 3 || status == 4) { ok = false; break; }
        // restricted solution: x on basic structurals, y_R from slack columns
        for (int j = tid; j < n; j += nt) xv[j] = 0.0;
        for (int r = tid; r < k; r += nt) yv[r] = 0.0;
        __syncthreads();
        for (int r = tid; r < k; r += nt) {
            const int v = row_var[r];
            if ((unsigned)v < (unsigned)n) xv[v] = T[(size_t)r * LD];
        }
        for (int j = 1 + tid; j <= n; j += nt) {
            const int v = col_var[j];
            if (v >= n && v < n + k) yv[v - n] = To[j];
        }
        __syncthreads();
        unsigned add = 0, first;
        if (status == 2) {
            // unbounded restricted LP: add the rows that bound its ray d
            // (d_e = 1 for the entering structural, d_v = -t_re for basic structurals)
            const int ve = col_var[e_unb];
            for (int i = tid; i < m; i += nt) {
                if (inR[i]) continue;
                double s = ((unsigned)ve < (unsigned)n) ? A[(size_t)i * n + ve] : 0.0;
                for (int r = 0; r < k; ++r) {
                    const int v = row_var[r];
                    if ((unsigned)v < (unsigned)n) s = __fma_rn(-A[(size_t)i * n + v], T[(size_t)r * LD + e_unb], s);
                }
                const bool bound = above_key(s, k_tol_p);
                inR[i] = bound ? 2 : 0;  // 2: to be added
                add += bound ? 1u : 0u;
            }
            red.count_min(add, 0u, add, first);
            if (add == 0) { ok = false; break; }
        } else {
            // ---- 3. checks on the full LP in FP64, from the original data
            unsigned bad = 0;
            for (int i = tid; i < m; i += nt) {
                double s = bv[i];
                for (int r = 0; r < k; ++r) {
                    const int v = row_var[r];
                    if ((unsigned)v < (unsigned)n) s = __fma_rn(-A[(size_t)i * n + v], xv[v], s);
                }
                const bool viol = below_key(s, k_neg_tol_p);
                if (!inR[i]) {
                    inR[i] = viol ? 2 : 0;
                    add += viol ? 1u : 0u;
                } else {
                    bad += viol ? 1u : 0u;  // a restricted row must hold already
                }
            }
            for (int r = tid; r < k; r += nt) bad += below_key(yv[r], k_neg_tol_d) ? 1u : 0u;
            for (int j = tid; j < n; j += nt) {
                double d = -cv[j];
                for (int r = 0; r < k; ++r) d = __fma_rn(A[(size_t)rows[r] * n + j], yv[r], d);
                bad += below_key(d, k_neg_tol_d) ? 1u : 0u;
            }
            unsigned tot_add;
            red.count_min(add, 0u, tot_add, first);
            red.count_min(bad, 0u, bad, first);
            add = tot_add;
            if (bad) { ok = false; break; }
            if (add == 0) {
                // strong duality (warp 0, fixed order)
                __shared__ double s_gap[2];
                if (tid < 32) {
                    double px = 0.0, dy = 0.0;
                    for (int j = tid; j < n; j += 32) px = __fma_rn(cv[j], xv[j], px);
                    for (int r = tid; r < k; r += 32) dy = __fma_rn(bv[rows[r]], yv[r], dy);
                    for (int o = 16; o > 0; o >>= 1) {
                        px = __dadd_rn(px, __shfl_xor_sync(kFull, px, o));
                        dy = __dadd_rn(dy, __shfl_xor_sync(kFull, dy, o));
                    }
                    if (tid == 0) { s_gap[0] = px; s_gap[1] = dy; }
                }
                __syncthreads();
                const double px = s_gap[0], dy = s_gap[1];
                if (!(fabs(px - dy) <= a.cert_tol * fmax(1.0, fabs(px)))) { ok = false; break; }
                certified = true;
                if (tid == 0) {
                    a.B.status[lp] = kOptimal;
                    a.B.iters[lp] = iters;
                    a.B.obj[lp] = px;
                }
                break;
            }
        }
        // ---- 4. grow R by the marked rows (ascending), if there is room
        if (k + (int)add > kmax) {
            ok = false;
            overflow = true;
            break;
        }
        for (int i0 = 0; i0 < m; i0 += nt) {
            const int i = i0 + tid;
            const bool sel = (i < m) && (inR[i] == 2);
            int tot;
            const int pos = k + red.prefix_count(sel, tot);
            if (sel) {
                rows[pos] = i;
                inR[i] = 1;
            }
            k += tot;
        }
        __syncthreads();
    }
    if (tid == 0) atomicAdd(a.rounds, round);
    if (certified) {
        double* x = a.B.x + a.B.x_off[lp];
        for (int j = tid; j < n; j += nt) x[j] = xv[j];
        if (a.B.y) {
            double* y = a.B.y + a.B.y_off[lp];
            for (int i = tid; i < m; i += nt) y[i] = 0.0;
            __syncthreads();
            for (int r = tid; r < k; r += nt) y[rows[r]] = yv[r];
        }
        if (tid == 0) atomicAdd(a.certified, 1);
    } else if (tid == 0) {
        const bool retry = overflow && a.ov_queue != nullptr;
        const int pos = atomicAdd(retry ? a.ov_len : a.fb_len, 1);
        if (pos < a.fb_cap) (retry ? a.ov_queue : a.fb_queue)[pos] = lp;
        else record_internal_error(a.diag, 4, lp);
    }
}

// One CTA per LP of the batch, or (a.queue) persistent CTAs over the LPs of a
// device-side queue, whose length only the device knows.
__global__ void __launch_bounds__(kWarmThreads) warm_kernel(const WarmArgs a) {
    const int count = a.queue ? min(*a.queue_len, a.fb_cap) : min(a.num_lps, (int)blockIdx.x + 1);
    for (int qi = blockIdx.x; qi < count; qi += gridDim.x) {
        const int lp = a.queue ? a.queue[qi] : qi;
        if ((unsigned)lp >= (unsigned)a.num_lps) {
            if (threadIdx.x == 0) record_internal_error(a.diag, 9, lp);
            continue;
        }
        warm_one(a, lp);
        __syncthreads();  // the next LP reuses the shared memory
    }
}

__global__ void warm_labels_kernel(DeviceBatch B, int32_t num_lps, int32_t m, float* __restrict__ labels) {
    const int64_t total = (int64_t)num_lps * m;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = e / m;
        const int i = (int)(e - k * m);
        labels[e] = (B.status[k] == kOptimal && B.y[B.y_off[k] + i] > 0.0) ? 1.0f : 0.0f;
    }
}

}  // namespace

cudaError_t launch_warm_labels(const DeviceBatch& B, int32_t num_lps, int32_t m, float* labels, cudaStream_t s) {
    const int64_t total = (int64_t)num_lps * m;
    const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 32);
    warm_labels_kernel<<<blocks, 256, 0, s>>>(B, num_lps, m, labels);
    return cudaGetLastError();
}

size_t warm_smem_bytes(int m, int n, int kmax) { return warm_layout(m, n, kmax).total; }

cudaError_t launch_warm_features(const DeviceBatch& B, int32_t num_lps, int32_t m, int32_t n, float* x,
                                 cudaStream_t s) {
    const int64_t total = (int64_t)num_lps * (m + n);
    const unsigned blocks = (unsigned)std::min<int64_t>((total + kWarmThreads - 1) / kWarmThreads, 152 * 64);
    warm_features_kernel<<<blocks, kWarmThreads, 0, s>>>(B, num_lps, m, n, x);
    return cudaGetLastError();
}

cudaError_t launch_warm(const DeviceBatch& B, const float* logits, int32_t num_lps, int32_t m, int32_t n,
                        int32_t kmax, int32_t max_rounds, int32_t max_iters, float threshold, double eps_opt,
                        double eps_piv, double cert_tol, int32_t* fb_queue, int32_t* fb_len, int32_t fb_cap,
                        const int32_t* queue, const int32_t* queue_len, int32_t* ov_queue, int32_t* ov_len,
                        int32_t* certified, int32_t* rounds, int32_t* diag, cudaStream_t s) {
    if (num_lps <= 0) return cudaSuccess;
    WarmArgs a{};
    a.queue = queue; a.queue_len = queue_len; a.ov_queue = ov_queue; a.ov_len = ov_len;
    a.B = B; a.logits = logits; a.num_lps = num_lps; a.m = m; a.n = n; a.kmax = kmax;
    a.max_rounds = max_rounds; a.max_iters = max_iters; a.threshold = threshold;
    a.eps_opt = eps_opt; a.eps_piv = eps_piv; a.cert_tol = cert_tol;
    a.fb_queue = fb_queue; a.fb_len = fb_len; a.fb_cap = fb_cap; a.certified = certified; a.rounds = rounds;
    a.diag = diag;
    const size_t smem = warm_smem_bytes(m, n, kmax);
    cudaError_t err = cudaFuncSetAttribute(warm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int grid = num_lps;
    if (queue) {
        // one wave of persistent CTAs over the queue
        int dev = 0, sms = 0, per_sm = 0;
        if ((err = cudaGetDevice(&dev)) || (err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) ||
            (err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, warm_kernel, kWarmThreads, smem)))
            return err;
        grid = std::min<int>(num_lps, sms * std::max(1, per_sm));
    }
    warm_kernel<<<grid, kWarmThreads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace lpb
