// lp_fp64_resident.cu -- FP64 dense simplex with the tableau resident in
// shared memory, one CTA per LP.
//
// Method: Gurung & Ray, "Simultaneous Solving of Batched Linear Programs on a
// GPU" (arXiv 1802.08557).  Section 4.1 assigns one CUDA block per LP; Section
// 4.2 parallelises Step 1 (entering variable) and Step 2 (leaving variable) as
// reductions and Step 3 (pivot) over the tableau elements.  Differences from
// the paper's kernel (which kept the full tableau in global memory and used
// shared/global tree reductions):
//  - the condensed (Tucker) tableau is kept: one column per NON-basic
//    variable plus the right-hand side (column 0).  A pivot swaps the labels of
//    the entering column and the leaving row.  Basic columns of the paper's
//    full tableau are unit vectors and carry no information;
//  - the tableau lives in shared memory for the whole solve; global memory is
//    touched only to read A, b, c and write the results;
//  - reductions are warp `redux` instructions on 64-bit order-preserving
//    integer keys of the FP64 values (exact, no FP64-pipe compares);
//  - phase I runs in the same kernel (the paper launches twice, Section 5).
//
// Arithmetic is the oracle's, operation for operation, so that both reach the
// same pivot sequence: ratio = rhs / t (IEEE divide), pivot row = row / PE
// (IEEE divide), update t_ij = fma(-t_ie, r_j, t_ij), tie window
// v + tau*max(1,|v|) as a product followed by a sum.  This file is compiled
// with --fmad=false and only uses the _rn intrinsics for FP64 arithmetic.

#include <climits>

#include "lp_internal.h"

namespace lpb {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// Order-preserving map of a (non-NaN) double to a signed 64-bit key:
// a < b  <=>  okey(a) < okey(b);  -0 and +0 map to the same key.
__device__ __forceinline__ long long okey(double v) {
    long long b = __double_as_longlong(v);
    b = (b == LLONG_MIN) ? 0LL : b;
    return b ^ ((b >> 63) & LLONG_MAX);
}
__device__ __forceinline__ double kval(long long k) {
    return __longlong_as_double(k ^ ((k >> 63) & LLONG_MAX));
}
// Key of |v| (the plain bit pattern with the sign cleared).
__device__ __forceinline__ long long abskey(double v) { return __double_as_longlong(v) & LLONG_MAX; }

// Tie window of Steps 1 and 2: v + tau * max(1, |v|) (product, then sum).
__device__ __forceinline__ double tie_threshold(double v, double tau) {
    const long long ab = abskey(v);
    const double s = (ab < 0x3FF0000000000000LL) ? 1.0 : __longlong_as_double(ab);
    return __dadd_rn(v, __dmul_rn(tau, s));
}

__device__ __forceinline__ long long warp_min_i64(long long v) {
    const int hi = (int)(v >> 32);
    const int mhi = __reduce_min_sync(kFull, hi);
    const unsigned lo = (hi == mhi) ? (unsigned)(v & 0xffffffffLL) : 0xffffffffu;
    const unsigned mlo = __reduce_min_sync(kFull, lo);
    return (long long)(((unsigned long long)(unsigned)mhi << 32) | (unsigned long long)mlo);
}

// Block-wide minima.  `scratch` alternates between two halves so that a
// buffer is never rewritten before every thread has read it.
struct Reducer {
    long long* s64;
    unsigned* s32;
    int nw, warp, lane;
    int b64 = 0, b32 = 0;

    __device__ long long min_i64(long long v) {
        v = warp_min_i64(v);
        long long* s = s64 + b64 * kMaxWarps;
        b64 ^= 1;
        if (lane == 0) s[warp] = v;
        __syncthreads();
        long long r = s[0];
        for (int w = 1; w < nw; ++w) r = min(r, s[w]);
        return r;
    }
    __device__ unsigned min_u32(unsigned v) {
        v = __reduce_min_sync(kFull, v);
        unsigned* s = s32 + b32 * kMaxWarps;
        b32 ^= 1;
        if (lane == 0) s[warp] = v;
        __syncthreads();
        unsigned r = s[0];
        for (int w = 1; w < nw; ++w) r = min(r, s[w]);
        return r;
    }
};

struct Tab {
    double* T;        // R x LD, row-major; column 0 = right-hand side
    double* colE;     // copy of the pivot column
    int* col_var;     // variable of each column (1..Cvar live)
    int* row_var;     // basic variable of each constraint row
    int LD;
};

// Step 3 (Section 3.1, Listing 1) on the condensed tableau: divide pivot row
// l by PE = colE[l], then t_ij <- fma(-t_ie, r_j, t_ij) for every other active
// row.  In column e (which now holds the leaving variable) the old entry of the
// paper's full tableau is the unit column of a basic variable, i.e. 0 off the
// pivot row and 1 on it, so r_e = 1/PE and t_ie <- fma(-t_ie, r_e, 0).
// colE[0..Ract) must hold column e on entry.
__device__ __forceinline__ void pivot(Tab& tb, int Ract, int Cact, int l, int e) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int LD = tb.LD;
    double* __restrict__ T = tb.T;
    const double* __restrict__ colE = tb.colE;
    const double pe = colE[l];
    double* Tl = T + (size_t)l * LD;
    for (int j = tid; j < Cact; j += nt) {
        const double v = (j == e) ? 1.0 : Tl[j];
        Tl[j] = __ddiv_rn(v, pe);
    }
    if (tid == 0) {
        const int ev = tb.col_var[e];
        tb.col_var[e] = tb.row_var[l];
        tb.row_var[l] = ev;
    }
    __syncthreads();
    const int total = (Ract - 1) * Cact;
    int ii = tid / Cact;
    int jj = tid - ii * Cact;
    const int di = nt / Cact;
    const int dj = nt - di * Cact;
    for (int idx = tid; idx < total; idx += nt) {
        const int r = ii + (ii >= l ? 1 : 0);
        double* t = T + (size_t)r * LD + jj;
        const double old = (jj == e) ? 0.0 : *t;
        *t = __fma_rn(-colE[r], Tl[jj], old);
        ii += di;
        jj += dj;
        if (jj >= Cact) { jj -= Cact; ++ii; }
    }
    __syncthreads();
}

// A retired artificial (it just left the basis and may never re-enter) sits
// in column e: move the last live column into its place and shrink.
__device__ __forceinline__ void retire_column(Tab& tb, int Ract, int e, int& Cvar) {
    const int tid = threadIdx.x, nt = blockDim.x;
    if (e != Cvar) {
        for (int r = tid; r < Ract; r += nt) {
            double* row = tb.T + (size_t)r * tb.LD;
            row[e] = row[Cvar];
        }
        if (tid == 0) tb.col_var[e] = tb.col_var[Cvar];
    }
    --Cvar;
    __syncthreads();
}

__global__ void __launch_bounds__(kMaxThreads)
fp64_resident_kernel(const DeviceBatch B, const Tolerances tol, const int32_t* __restrict__ order)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lp = order[blockIdx.x];
    const int m = B.m[lp];
    const int n = B.n[lp];
    const int nm = n + m;
    const double* __restrict__ A = B.A + B.a_off[lp];
    const double* __restrict__ bv = B.b + B.b_off[lp];
    const double* __restrict__ cv = B.c + B.c_off[lp];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;

    // k-independent part of the layout (k = 0 gives the same offsets)
    const ResidentLayout L0 = resident_layout(m, n, 0);
    Reducer red{reinterpret_cast<long long*>(smem + L0.red64), reinterpret_cast<unsigned*>(smem + L0.red32),
                nw, warp, lane};
    long long* rkey = reinterpret_cast<long long*>(smem + L0.rkey);
    int* row_var = reinterpret_cast<int*>(smem + L0.row_var);
    int* neg = reinterpret_cast<int*>(smem + L0.neg);

    // ---- Tableau build (the host-side fill of Section 4.1, done here) -----
    // Rows with b_i < 0 are negated and get an artificial (two-phase method,
    // Section 3); they are ranked in ascending row order.
    int k = 0;
    for (int i0 = 0; i0 < m; i0 += nt) {
        const int i = i0 + tid;
        const bool isneg = (i < m) && (bv[i] < 0.0);
        const unsigned bal = __ballot_sync(kFull, isneg);
        if (lane == 0) red.s32[warp] = (unsigned)__popc(bal);
        __syncthreads();
        int before = 0, tot = 0;
        for (int w = 0; w < nw; ++w) {
            const int cw = (int)red.s32[w];
            before += (w < warp) ? cw : 0;
            tot += cw;
        }
        if (i < m) {
            if (isneg) {
                const int r = k + before + __popc(bal & ((1u << lane) - 1u));
                neg[r] = i;
                row_var[i] = nm + r;
            } else {
                row_var[i] = n + i;
            }
        }
        k += tot;
        __syncthreads();
    }

    const ResidentLayout L = resident_layout(m, n, k);
    Tab tb;
    tb.T = reinterpret_cast<double*>(smem + L.T);
    tb.colE = reinterpret_cast<double*>(smem + L.colE);
    tb.col_var = reinterpret_cast<int*>(smem + L.col_var);
    tb.row_var = row_var;
    tb.LD = L.LD;
    const int LD = L.LD;
    double* __restrict__ T = tb.T;
    int Cvar = n + k;  // live variable columns 1..Cvar

    for (int j = tid; j <= Cvar; j += nt)
        tb.col_var[j] = (j == 0) ? -1 : (j <= n ? j - 1 : n + neg[j - 1 - n]);
    for (int i = warp; i < m; i += nw) {
        const bool isneg = row_var[i] >= nm;
        const double* Ai = A + (size_t)i * n;
        double* Ti = T + (size_t)i * LD;
        for (int j = lane; j <= Cvar; j += 32) {
            double v;
            if (j == 0) v = bv[i];
            else if (j <= n) v = Ai[j - 1];
            else v = (neg[j - 1 - n] == i) ? 1.0 : 0.0;
            Ti[j] = isneg ? -v : v;
        }
    }
    {
        double* Tm = T + (size_t)m * LD;
        for (int j = tid; j <= Cvar; j += nt) Tm[j] = (j >= 1 && j <= n) ? -cv[j - 1] : 0.0;
    }
    long long bmax_key = 0x3FF0000000000000LL;  // 1.0
    for (int i = tid; i < m; i += nt) bmax_key = max(bmax_key, abskey(bv[i]));
    bmax_key = -red.min_i64(-bmax_key);  // also orders the fills above
    if (k > 0) {
        // auxiliary objective: maximise -(sum of artificials), priced out by
        // subtracting every negated row in ascending row order
        double* Tw = T + (size_t)(m + 1) * LD;
        for (int j = tid; j <= Cvar; j += nt) {
            double w = 0.0;
            for (int t = 0; t < k; ++t) w = __dsub_rn(w, T[(size_t)neg[t] * LD + j]);
            Tw[j] = w;
        }
        __syncthreads();
    }

    const long long key_neg_eps_opt = okey(-tol.eps_opt);
    const long long key_eps_piv = okey(tol.eps_piv);
    const int max_iters = tol.max_iters > 0 ? tol.max_iters : 50 * (m + n);
    int iters = 0;
    int status = -1;
    int phase = (k > 0) ? 1 : 2;
    int yrow = m;

    while (status < 0) {
        const int orow = (phase == 1) ? m + 1 : m;
        const int Ract = (phase == 1) ? m + 2 : m + 1;
        const double* Trow = T + (size_t)orow * LD;

        // ---- Step 1: entering variable (most negative reduced cost) -------
        long long dloc = LLONG_MAX;
        for (int j = 1 + tid; j <= Cvar; j += nt)
            if (tb.col_var[j] < nm) dloc = min(dloc, okey(Trow[j]));
        const long long dmin = red.min_i64(dloc);
        if (dmin >= key_neg_eps_opt) {
            if (phase == 2) { status = kOptimal; break; }
            // ---- end of phase I (Section 3, two-phase method) -------------
            const double wstar = -T[(size_t)(m + 1) * LD];
            if (wstar > __dmul_rn(tol.eps_feas, __longlong_as_double(bmax_key))) {
                status = kInfeasible;
                yrow = m + 1;
                break;
            }
            // drive artificials still basic (at level 0) out of the basis on
            // the lowest non-artificial column with |t_ij| > eps_piv
            for (int i = 0; i < m && status < 0; ++i) {
                if (row_var[i] < nm) continue;
                const double* Ti = T + (size_t)i * LD;
                unsigned sel = 0xffffffffu;
                for (int j = 1 + tid; j <= Cvar; j += nt)
                    if (tb.col_var[j] < nm && abskey(Ti[j]) > key_eps_piv)
                        sel = min(sel, ((unsigned)tb.col_var[j] << 16) | (unsigned)j);
                sel = red.min_u32(sel);
                if (sel == 0xffffffffu) continue;  // redundant row
                if (iters >= max_iters) { status = kIterLimit; break; }
                const int e = (int)(sel & 0xffffu);
                for (int r = tid; r < m + 1; r += nt) tb.colE[r] = T[(size_t)r * LD + e];
                __syncthreads();
                pivot(tb, m + 1, Cvar + 1, i, e);
                ++iters;
                if (tb.col_var[e] >= nm) retire_column(tb, m + 1, e, Cvar);
            }
            phase = 2;
            continue;
        }
        long long kthr = 0;
        if (lane == 0) kthr = okey(tie_threshold(kval(dmin), tol.tau));
        kthr = __shfl_sync(kFull, kthr, 0);
        unsigned esel = 0xffffffffu;
        for (int j = 1 + tid; j <= Cvar; j += nt) {
            const int v = tb.col_var[j];
            if (v < nm && okey(Trow[j]) <= kthr) esel = min(esel, ((unsigned)v << 16) | (unsigned)j);
        }
        esel = red.min_u32(esel);
        const int e = (int)(esel & 0xffffu);

        // ---- Step 2: leaving row (minimum ratio rhs_i / t_ie, t_ie > eps) --
        long long rloc = LLONG_MAX;
        for (int i = tid; i < Ract; i += nt) {
            const double t = T[(size_t)i * LD + e];
            tb.colE[i] = t;
            if (i < m) {
                long long rk = LLONG_MAX;
                if (okey(t) > key_eps_piv) rk = okey(__ddiv_rn(T[(size_t)i * LD], t));
                rkey[i] = rk;
                rloc = min(rloc, rk);
            }
        }
        const long long rmin = red.min_i64(rloc);
        if (rmin == LLONG_MAX) {
            status = (phase == 2) ? kUnbounded : kNumerical;
            break;
        }
        long long rthr = 0;
        if (lane == 0) rthr = okey(tie_threshold(kval(rmin), tol.tau));
        rthr = __shfl_sync(kFull, rthr, 0);
        unsigned lsel = 0xffffffffu;
        for (int i = tid; i < m; i += nt)
            if (rkey[i] <= rthr) lsel = min(lsel, (unsigned)i);
        const int l = (int)red.min_u32(lsel);
        if (abskey(tb.colE[l]) >= 0x7FF0000000000000LL) { status = kNumerical; break; }
        if (iters >= max_iters) { status = kIterLimit; break; }

        // ---- Step 3: pivot ---------------------------------------------------
        pivot(tb, Ract, Cvar + 1, l, e);
        ++iters;
        if (tb.col_var[e] >= nm) retire_column(tb, Ract, e, Cvar);
    }

    // ---- results: x (basic rows -> rhs, non-basic -> 0), y (slack reduced
    // costs of row `yrow`), objective corner, status, pivots -----------------
    double* __restrict__ x = B.x + B.x_off[lp];
    double* __restrict__ y = B.y ? B.y + B.y_off[lp] : nullptr;
    const double* Ty = T + (size_t)yrow * LD;
    for (int j = 1 + tid; j <= Cvar; j += nt) {
        const int v = tb.col_var[j];
        if (v < n) x[v] = 0.0;
        else if (v < nm && y) y[v - n] = Ty[j];
    }
    for (int i = tid; i < m; i += nt) {
        const int v = row_var[i];
        if (v < n) x[v] = T[(size_t)i * LD];
        else if (v < nm && y) y[v - n] = 0.0;
    }
    if (tid == 0) {
        B.status[lp] = status;
        B.iters[lp] = iters;
        B.obj[lp] = T[(size_t)m * LD];
    }
}

}  // namespace

cudaError_t fp64_resident_prepare() {
    return cudaFuncSetAttribute(fp64_resident_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kMaxSmemPerBlock);
}

cudaError_t launch_fp64_resident(const DeviceBatch& B, const Tolerances& tol, const int32_t* order,
                                 int32_t count, int threads, size_t smem, cudaStream_t stream) {
    if (count <= 0) return cudaSuccess;
    fp64_resident_kernel<<<count, threads, smem, stream>>>(B, tol, order);
    return cudaGetLastError();
}

}  // namespace lpb
