// lp_mixed_solve.cuh -- one LP on an FP32 condensed tableau, then the FP64
// certificate of the basis the FP32 run ended on (mixed_solve); included by
// the shared-memory kernels (lp_mixed.cu) and by the streamed kernel
// (lp_mixed_streamed.cu), whose tableau lives in a global workspace slot.
//
// The paper's method (Gurung & Ray, arXiv 1802.08557, Section 3: Steps 1-3 on
// the tableau, two-phase method; Section 4: one CTA per LP) is run with FP32
// tableau arithmetic: on GB300 the FP32 pipe is ~64x faster than the FP64 pipe.
// The FP32 run only proposes a basis.  The answer comes from FP64:
//  - B^-1 is read off the FP32 tableau (the column of slack n+c in the
//    condensed tableau is B^-1 e_c; a basic slack's is a unit vector);
//  - x_B = B^-1 b and y^T = c_B^T B^-1 are refined in FP64: residual in FP64
//    from the original A, b, c, correction through the FP32 B^-1, until the
//    correction is below conv_tol relative;
//  - the certificate is checked in FP64: x_B >= -tol (primal), y >= -tol and
//    A^T y - c >= -tol on non-basic structurals (dual), c^T x = b^T y;
//    for an unbounded claim, a refined ray d (d >= -tol, c^T d > 0) from a
//    primal-feasible point.
//  - an infeasible claim gets a Farkas certificate from the phase-I basis.
// An LP whose claim is not certified (or that ends at the iteration limit or
// in breakdown) is appended to a device queue and solved again by an FP64
// kernel (FallbackQueues: the one-CTA kernel when its FP64 tableau fits, else
// the streamed one).  So every reported optimum comes from an FP64 basic
// solution of a basis proven optimal to cert_tol.
//
// This path has no counterpart in the paper (which is FP64 only).

#pragma once

#include <climits>

#include "lp_device.cuh"
#include "lp_internal.h"

namespace lpb {
namespace {

__device__ __forceinline__ float fabs32(float v) { return __int_as_float(__float_as_int(v) & INT_MAX); }

// 64-bit key: signed `hi` compared first, then unsigned `lo`.
__device__ __forceinline__ long long pack_key(int hi, unsigned lo) {
    return (long long)(((unsigned long long)(unsigned)hi << 32) | (unsigned long long)lo);
}

// Rows per batch of the pivot update (all loads of a batch issued before its
// stores).  Measured on 50x50 LPs: deeper batches, two quads per thread and
// step, deeper unrolling of the loops that read A, or a larger register budget
// for the one-warp kernel were all slower (larger code or spills, same
// latency-bound issue rate).
constexpr int kPivotBatch = 4;

struct Tab32 {
    float* T;
    float* colE;
    int* col_var;
    int* row_var;
    int LD;
};

// Thread layout of the pivot update over quads of 4 columns: thread tid takes
// quads q0, q0 + qstep, ... and rows r0, r0 + rg, ...  It depends only on the
// number of active columns, so it is recomputed only when that changes.
struct QuadMap {
    int cact, q0, qstep, r0, rg;
};

__device__ __forceinline__ QuadMap quad_map(int tid, int nt, int Cact) {
    QuadMap m;
    m.cact = Cact;
    const int nq = (Cact + 3) >> 2;
    if (nq >= nt) {
        m.q0 = tid; m.qstep = nt; m.r0 = 0; m.rg = 1;
    } else {
        m.rg = nt / nq;
        m.r0 = tid / nq;
        m.q0 = tid - m.r0 * nq; m.qstep = nq;
        if (m.r0 >= m.rg) m.q0 = nq;  // idle in the update
    }
    return m;
}

// Step 3 in FP32; G is the thread group that owns the LP (BlockGroup or
// WarpGroup).  Returns the variable that left the basis, read between the two
// barriers, where nothing writes it.
//  phase A: pivot row l times 1/PE (its column e becomes 1/PE); column e of
//           every other row set to 0, so that the uniform update of phase B
//           gives fma(-t_ie, 1/PE, 0) = -t_ie/PE there (the leaving variable's
//           column);
//  phase B: t_rj = fma(-t_re, r_j, t_rj) for r != l over quads of 4 columns
//           (16-byte loads and stores; LD is a multiple of 4), kPivotBatch
//           rows per batch with every load of a batch issued before its
//           stores.
//  Columns of the last quad beyond Cact are padding: updated, never read.
template <class G>
__device__ __forceinline__ int pivot32(G& g, Tab32& tb, int Ract, int Cact, int l, int e, const QuadMap& qm) {
    const int tid = g.tid, nt = g.nt;
    const int LD = tb.LD;
    float* T = tb.T;
    const float* colE = tb.colE;
    const float rinv = __frcp_rn(colE[l]);
    float* Tl = T + l * LD;
    for (int j = tid; j < Cact; j += nt) Tl[j] = (j == e) ? rinv : __fmul_rn(Tl[j], rinv);
    for (int r = tid; r < Ract; r += nt)
        if (r != l) T[r * LD + e] = 0.0f;
    if (tid == 0) {
        const int ev = tb.col_var[e];
        tb.col_var[e] = tb.row_var[l];
        tb.row_var[l] = ev;
    }
    g.sync();
    const int left = tb.col_var[e];
    const int nq = (Cact + 3) >> 2;
    const int qstep = qm.qstep, r0 = qm.r0, rg = qm.rg;
    constexpr int kB = kPivotBatch;
    for (int q = qm.q0; q < nq; q += qstep) {
        const float4 p = *reinterpret_cast<const float4*>(Tl + 4 * q);
        float* base = T + 4 * q;
        int r = r0;
        for (; r + (kB - 1) * rg < Ract; r += kB * rg) {
            float4 v[kB];
            float c[kB];
#pragma unroll
            for (int u = 0; u < kB; ++u) {
                v[u] = *reinterpret_cast<const float4*>(base + (r + u * rg) * LD);
                c[u] = -colE[r + u * rg];
            }
#pragma unroll
            for (int u = 0; u < kB; ++u) {
                v[u].x = __fmaf_rn(c[u], p.x, v[u].x); v[u].y = __fmaf_rn(c[u], p.y, v[u].y);
                v[u].z = __fmaf_rn(c[u], p.z, v[u].z); v[u].w = __fmaf_rn(c[u], p.w, v[u].w);
            }
#pragma unroll
            for (int u = 0; u < kB; ++u)
                if (r + u * rg != l) *reinterpret_cast<float4*>(base + (r + u * rg) * LD) = v[u];
        }
        for (; r < Ract; r += rg) {
            float4* a0 = reinterpret_cast<float4*>(base + r * LD);
            float4 v0 = *a0;
            const float c0 = -colE[r];
            v0.x = __fmaf_rn(c0, p.x, v0.x); v0.y = __fmaf_rn(c0, p.y, v0.y);
            v0.z = __fmaf_rn(c0, p.z, v0.z); v0.w = __fmaf_rn(c0, p.w, v0.w);
            if (r != l) *a0 = v0;
        }
    }
    g.sync();
    return left;
}

template <class G>
__device__ __forceinline__ void retire_column32(G& g, Tab32& tb, int Ract, int e, int& Cvar) {
    const int tid = g.tid, nt = g.nt;
    if (e != Cvar) {
        for (int r = tid; r < Ract; r += nt) {
            float* row = tb.T + r * tb.LD;
            row[e] = row[Cvar];
        }
        if (tid == 0) tb.col_var[e] = tb.col_var[Cvar];
    }
    --Cvar;
    g.sync();
}

// Lanes per output of the certificate's long sums (residuals and corrections
// over all m rows for a few outputs): a power of two from m alone, so that the
// arithmetic of an LP does not depend on the launch form; 1 below m = 64.
__device__ __forceinline__ int split_width(int m) {
    int p = 1;
    while (p < 32 && m >= 64 * p) p <<= 1;
    return p;
}

// Sum over the P consecutive lanes of a split group (butterfly; every lane of
// the group ends with the same value).  All 32 lanes of the warp must call it.
__device__ __forceinline__ double group_sum(double v, int P) {
    for (int off = P >> 1; off > 0; off >>= 1) v = __dadd_rn(v, __shfl_xor_sync(kFull, v, off));
    return v;
}
__device__ __forceinline__ float group_sum(float v, int P) {
    for (int off = P >> 1; off > 0; off >>= 1) v = __fadd_rn(v, __shfl_xor_sync(kFull, v, off));
    return v;
}

template <class G, bool kSplit>
__device__ __forceinline__ void mixed_solve(G& g, const DeviceBatch& B, const Tolerances& tol, const MixedParams& mp,
                                            const int lp, unsigned char* big, const FallbackQueues& fq,
                                            int32_t* diag);

// mixed_solve with the split chosen from the LP's m (the same in every form).
template <class G>
__device__ __forceinline__ void mixed_solve_lp(G& g, const DeviceBatch& B, const Tolerances& tol,
                                               const MixedParams& mp, const int lp, unsigned char* big,
                                               const FallbackQueues& fq, int32_t* diag) {
    if (split_width(B.m[lp]) > 1)
        mixed_solve<G, true>(g, B, tol, mp, lp, big, fq, diag);
    else
        mixed_solve<G, false>(g, B, tol, mp, lp, big, fq, diag);
}

// max |v| over the group (FP64), as a double.
template <class G>
__device__ __forceinline__ double block_absmax(G& g, double v) {
    return __longlong_as_double(-g.min_i64(-abskey(v)));
}

// One LP on the FP32 tableau, then its FP64 certificate.  `big` is the
// LP's shared-memory area (mixed_layout); G is the group of threads that owns
// the LP.  kSplit: the certificate's long sums are split over
// split_width(m) > 1 lanes (else P = 1 at compile time, plain loops).
template <class G, bool kSplit>
__device__ __forceinline__ void mixed_solve(G& g, const DeviceBatch& B, const Tolerances& tol, const MixedParams& mp,
                                            const int lp, unsigned char* big, const FallbackQueues& fq,
                                            int32_t* diag)
{
    const int m = B.m[lp];
    const int n = B.n[lp];
    const int nm = n + m;
    const double* __restrict__ A = B.A + B.a_off[lp];
    const double* __restrict__ bv = B.b + B.b_off[lp];
    const double* __restrict__ cv = B.c + B.c_off[lp];
    const int tid = g.tid, nt = g.nt;
    const int lane = g.lane, warp = g.warp;

    const MixedLayout L0 = mixed_layout(m, n, 0);
    double* scal = reinterpret_cast<double*>(big + L0.scal);  // values broadcast from warp 0
    double& s_obj = scal[0];
    double& s_cd = scal[1];
    double& s_gamma = scal[2];
    double* xb = reinterpret_cast<double*>(big + L0.xb);
    double* yv = reinterpret_cast<double*>(big + L0.yv);
    double* dv = yv;  // the ray of an unbounded LP; y is only refined for optimal and infeasible ones
    double* res = reinterpret_cast<double*>(big + L0.res);
    float* zf = reinterpret_cast<float*>(big + L0.zf);  // FP32 copy of the vector being refined
    int* row_var = reinterpret_cast<int*>(big + L0.row_var);
    int* neg = reinterpret_cast<int*>(big + L0.neg);
    int* spos = reinterpret_cast<int*>(big + L0.spos);
    int* slist = reinterpret_cast<int*>(big + L0.slist);
    // non-basic slacks c in increasing order, packed (column position << 16) | c
    int* nbl = reinterpret_cast<int*>(big + L0.nbl);

    {
        // every 128-byte line of this LP's A requested into L2 at once, so the
        // build's loads below find it there instead of each waiting on HBM
        const char* a0 = reinterpret_cast<const char*>(A);
        const size_t bytes = (size_t)m * (size_t)n * 8;
        for (size_t off = (size_t)tid * 128; off < bytes; off += (size_t)nt * 128)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(a0 + off));
    }
    // ---- tableau build (FP32), rows with b_i < 0 negated (two-phase) -------
    int k = 0;
    for (int i0 = 0; i0 < m; i0 += nt) {
        const int i = i0 + tid;
        const bool isneg = (i < m) && (bv[i] < 0.0);
        int tot;
        const int r = k + g.prefix_count(isneg, tot);
        if (i < m) {
            if (isneg) {
                neg[r] = i;
                row_var[i] = nm + r;
            } else {
                row_var[i] = n + i;
            }
        }
        k += tot;
    }
    g.sync();  // neg[] and row_var[] are read by other threads below
    const MixedLayout L = mixed_layout(m, n, k);
    Tab32 tb;
    tb.T = reinterpret_cast<float*>(big + L.T);
    tb.colE = reinterpret_cast<float*>(big + L.colE);
    tb.col_var = reinterpret_cast<int*>(big + L.col_var);
    tb.row_var = row_var;
    tb.LD = L.LD;
    const int LD = L.LD;
    float* rf = tb.colE;  // FP32 copy of the certificate's residual (colE is dead after the simplex)
    float* T = tb.T;  // the tableau is written through several pointers: no restrict
    int Cvar = n + k;

    for (int j = tid; j <= Cvar; j += nt)
        tb.col_var[j] = (j == 0) ? -1 : (j <= n ? j - 1 : n + neg[j - 1 - n]);
    // FP32 range: every nonzero |a_ij|, |b_i|, |c_j| within [2^-60, 2^60]
    auto outside = [](double v) {
        const long long a = abskey(v);
        return a != 0 && (a < 0x3C30000000000000LL || a > 0x43B0000000000000LL);
    };
    unsigned out_of_range = 0;
    {
        // A into rows 0..m-1, columns 1..n: one flat pass over the LP's A with
        // several independent loads in flight per thread (measured: 16-byte
        // pair loads and 8-deep unrolling were not faster)
        const int mn = m * n;
        const int di = nt / n, dj = nt - di * n;
        int i = tid / n, j = tid - i * n;
#pragma unroll 4
        for (int idx = tid; idx < mn; idx += nt) {
            const double a = A[idx];
            out_of_range += outside(a) ? 1u : 0u;
            const float v = __double2float_rn(a);
            T[i * LD + 1 + j] = (row_var[i] >= nm) ? -v : v;
            i += di;
            j += dj;
            if (j >= n) { j -= n; ++i; }
        }
    }
    // column 0 (b) and the slack columns of the negated rows
    for (int i = warp; i < m; i += g.nw) {
        const bool isneg = row_var[i] >= nm;
        float* Ti = T + i * LD;
        for (int t = lane; t <= k; t += 32) {
            const int j = (t == 0) ? 0 : n + t;
            const float v = (t == 0) ? __double2float_rn(bv[i]) : ((neg[t - 1] == i) ? 1.0f : 0.0f);
            Ti[j] = isneg ? -v : v;
        }
    }
    {
        float* Tm = T + m * LD;
        for (int j = tid; j <= Cvar; j += nt) Tm[j] = (j >= 1 && j <= n) ? -__double2float_rn(cv[j - 1]) : 0.0f;
    }
    long long bkey = 0x3FF0000000000000LL, ckey = 0x3FF0000000000000LL;  // 1.0
    for (int i = tid; i < m; i += nt) {
        bkey = max(bkey, abskey(bv[i]));
        out_of_range += outside(bv[i]) ? 1u : 0u;
    }
    for (int j = tid; j < n; j += nt) {
        ckey = max(ckey, abskey(cv[j]));
        out_of_range += outside(cv[j]) ? 1u : 0u;
    }
    const double bmax = __longlong_as_double(-g.min_i64(-bkey));  // barrier: fills done
    const double cmax = __longlong_as_double(-g.min_i64(-ckey));
    {
        unsigned dummy;
        g.count_min(out_of_range, 0u, out_of_range, dummy);
    }
    if (k > 0) {
        float* Tw = T + (m + 1) * LD;
        for (int j = tid; j <= Cvar; j += nt) {
            float w = 0.0f;
            for (int t = 0; t < k; ++t) w = __fsub_rn(w, T[neg[t] * LD + j]);
            Tw[j] = w;
        }
        g.sync();
    }

    // ---- FP32 simplex (Steps 1-3, two-phase) ----------------------------
    const int key_neg_eps_opt = fkey(-mp.eps_opt32);
    const int max_iters = tol.max_iters > 0 ? tol.max_iters : 50 * (m + n);
    int iters = 0;
    int status = -1;
    int phase = (k > 0) ? 1 : 2;
    int e_unb = -1;
    QuadMap qm = quad_map(tid, nt, Cvar + 1);
    if (out_of_range) status = kNumerical;  // straight to the FP64 kernel

    while (status < 0) {
        const int orow = (phase == 1) ? m + 1 : m;
        const int Ract = (phase == 1) ? m + 2 : m + 1;
        const float* Trow = T + orow * LD;
        bool end_phase1 = false;
        // Step 1, one pass: min over (key of d_j, variable label) packed in 64
        // bits -- the most negative reduced cost, exact ties to the lowest label
        long long dloc = LLONG_MAX;
        for (int j = 1 + tid; j <= Cvar; j += nt) {
            const int v = tb.col_var[j];
            if (v < nm) dloc = min(dloc, pack_key(fkey(Trow[j]), ((unsigned)v << 16) | (unsigned)j));
        }
        const long long dsel = g.min_i64(dloc);
        const int dmin = (int)(dsel >> 32);
        if (dsel == LLONG_MAX || dmin >= key_neg_eps_opt) {
            if (phase == 2) { status = kOptimal; break; }
            end_phase1 = true;
        } else {
            const int e = (int)(dsel & 0xffff);
            if (e < 1 || e > Cvar) {
                if (tid == 0) record_internal_error(diag, 1, lp, dmin, 0, iters, phase, (int)(dsel & 0xffffffff));
                status = kNumerical;
                break;
            }
            // Step 2, one pass: min over (key of ratio, row)
            long long rloc = LLONG_MAX;
            for (int i = tid; i < Ract; i += nt) {
                const float t = T[i * LD + e];
                tb.colE[i] = t;
                if (i < m && t > mp.eps_piv32)
                    rloc = min(rloc, pack_key(fkey(__fdividef(T[i * LD], t)), (unsigned)i));
            }
            const long long rsel = g.min_i64(rloc);
            if (rsel == LLONG_MAX) {
                if (phase == 2) {
                    status = kUnbounded;
                    e_unb = e;
                    break;
                }
                // phase I cannot be unbounded: in FP32 this is rounding noise
                // in the auxiliary row; end phase I (the certificate decides)
                end_phase1 = true;
            } else {
                const int l = (int)(rsel & 0xffffffff);
                if (l < 0 || l >= m) {
                    if (tid == 0) record_internal_error(diag, 2, lp, (int)(rsel >> 32), 0, iters, phase, l);
                    status = kNumerical;
                    break;
                }
                if (!isfinite(tb.colE[l])) { status = kNumerical; break; }
                if (iters >= max_iters) { status = kIterLimit; break; }
                if (qm.cact != Cvar + 1) qm = quad_map(tid, nt, Cvar + 1);
                const int left = pivot32(g, tb, Ract, Cvar + 1, l, e, qm);
                ++iters;
                if (left >= nm) retire_column32(g, tb, Ract, e, Cvar);
            }
        }
        if (end_phase1) {
            const float wstar = -T[(m + 1) * LD];
            if (wstar > mp.eps_feas32 * (float)bmax) { status = kInfeasible; break; }
            for (int i = 0; i < m && status < 0; ++i) {
                if (row_var[i] < nm) continue;
                const float* Ti = T + i * LD;
                unsigned sel = 0xffffffffu;
                for (int j = 1 + tid; j <= Cvar; j += nt)
                    if (tb.col_var[j] < nm && fabs32(Ti[j]) > mp.eps_piv32)
                        sel = min(sel, ((unsigned)tb.col_var[j] << 16) | (unsigned)j);
                sel = g.min_u32(sel);
                if (sel == 0xffffffffu) continue;
                if (iters >= max_iters) { status = kIterLimit; break; }
                const int e = (int)(sel & 0xffffu);
                if (e < 1 || e > Cvar) {
                    if (tid == 0) record_internal_error(diag, 1, lp, 0, 0, iters, phase, (int)sel);
                    status = kNumerical;
                    break;
                }
                for (int r = tid; r < m + 1; r += nt) tb.colE[r] = T[r * LD + e];
                g.sync();
                if (qm.cact != Cvar + 1) qm = quad_map(tid, nt, Cvar + 1);
                const int left = pivot32(g, tb, m + 1, Cvar + 1, i, e, qm);
                ++iters;
                if (left >= nm) retire_column32(g, tb, m + 1, e, Cvar);
            }
            phase = 2;
        }
    }

    // ---- labels must name variables: a corrupted one would become a wild
    // global index below (self-check; the LP is then re-solved in FP64) -----
    {
        unsigned badl = 0, dummy;
        const unsigned nvar = (unsigned)(nm + k);
        for (int i = tid; i < m; i += nt) badl += ((unsigned)row_var[i] >= nvar) ? 1u : 0u;
        for (int j = 1 + tid; j <= Cvar; j += nt) badl += ((unsigned)tb.col_var[j] >= nvar) ? 1u : 0u;
        g.count_min(badl, 0u, badl, dummy);
        if (badl) {
            if (tid == 0) record_internal_error(diag, 6, lp, (int)badl, status, iters, phase, Cvar);
            status = kNumerical;
        }
    }

    // ---- FP64 certificate ---------------------------------------------------
    bool ok = (status == kOptimal || status == kUnbounded);
    int s = 0;    // basic structurals
    int nnb = 0;  // non-basic slacks (the columns of B^-1 that are not unit vectors)
    // nbl from a complete spos (after a barrier); ends with a barrier
    auto build_nbl = [&]() {
        int cnt = 0;
        for (int c0 = 0; c0 < m; c0 += nt) {
            const int c = c0 + tid;
            const int p = (c < m) ? spos[c] : 0;
            int tot;
            const int pos = cnt + g.prefix_count(p > 0, tot);
            if (p > 0) nbl[pos] = (int)(((unsigned)p << 16) | (unsigned)c);  // p <= n + k, c < m: 16 bits each
            cnt += tot;
        }
        g.sync();
        return cnt;
    };
    const int P = kSplit ? split_width(m) : 1;
    const int sgid = tid / P, sq = tid - (tid / P) * P, sgroups = nt / P;
    if (ok) {
        unsigned nart = 0, dummy;
        for (int i = tid; i < m; i += nt) nart += (row_var[i] >= nm) ? 1u : 0u;
        g.count_min(nart, 0u, nart, dummy);
        ok = (nart == 0);
    }
    if (ok) {
        // where each slack is: column position (> 0) or -(basic row + 1)
        for (int j = 1 + tid; j <= Cvar; j += nt) {
            const int v = tb.col_var[j];
            if (v >= n && v < nm) spos[v - n] = j;
        }
        // compacted list of the rows whose basic variable is structural
        for (int i0 = 0; i0 < m; i0 += nt) {
            const int i = i0 + tid;
            const int v = (i < m) ? row_var[i] : -1;
            if (i < m && v >= n && v < nm) spos[v - n] = -(i + 1);
            const bool st = (i < m) && (v < n);
            int tot;
            const int pos = s + g.prefix_count(st, tot);
            if (st) slist[pos] = i;
            s += tot;
        }
        // every slack must be placed exactly once: a live column or a basic row
        unsigned badpos = 0, dummy;
        for (int c = tid; c < m; c += nt) {
            const int p = spos[c];
            badpos += (p == 0 || p > Cvar || -p - 1 >= m) ? 1u : 0u;
        }
        g.count_min(badpos, 0u, badpos, dummy);
        if (badpos) {
            if (tid == 0) record_internal_error(diag, 3, lp);
            ok = false;
        }
        nnb = build_nbl();
        for (int i = tid; i < m; i += nt) xb[i] = (double)T[i * LD];
        g.sync();
    }
    const double tol_p = mp.cert_tol * bmax;
    const double tol_d = mp.cert_tol * cmax;

    // Refine  B z = rhs  (z by tableau row), rhs = b or -(column of rhs_var):
    // z += B^-1 r with the residual r in FP64 from the original data and B^-1
    // the FP32 one of the tableau.  Converged when the residual the last
    // correction was computed from is within conv_tol of |rhs_c| +
    // sum |B_c,i| |z_i| (backward error) and that correction moved no
    // component by more than fwd_tol of max(|z_i|, fwd_floor max|z|) (forward
    // error: an ill-conditioned basis stalls and is left to the FP64 re-solve).
    // The tolerance tests run in FP32 on magnitudes: |a| of A by integer
    // operations (f64_abs_to_f32_trunc; A is range-checked), z and r through
    // their FP32 copies zf, rf, converted once where they are written.
    const float conv_tol32 = (float)mp.conv_tol, fwd_tol32 = (float)mp.fwd_tol;
    auto refine = [&](double* z, int rhs_var, bool& conv) {
        conv = false;
        double zloc = 0.0;
        for (int i = tid; i < m; i += nt) {
            zloc = (abskey(z[i]) > abskey(zloc)) ? z[i] : zloc;
            zf[i] = fabs32(__double2float_rn(z[i]));
        }
        const float zfloor = (float)mp.fwd_floor * __double2float_ru(block_absmax(g, zloc));  // barrier: zf complete
        for (int it = 0; it <= mp.max_refine; ++it) {
            unsigned bad = 0;
            for (int c = tid; c < m; c += nt) {
                double r;
                if (rhs_var < 0) r = bv[c];
                else r = (rhs_var < n) ? -A[(size_t)c * n + rhs_var] : ((rhs_var - n == c) ? -1.0 : 0.0);
                float mag = f64_abs_to_f32_trunc(r);  // b, A or 1: range-checked
                const double* Ac = A + (size_t)c * n;
#pragma unroll 4
                for (int t = 0; t < s; ++t) {
                    const int i = slist[t];
                    const double a = Ac[row_var[i]];
                    r = __fma_rn(-a, z[i], r);
                    mag = __fmaf_rn(f64_abs_to_f32_trunc(a), zf[i], mag);
                }
                const int p = spos[c];
                if (p < 0) {
                    r = __dsub_rn(r, z[-p - 1]);
                    mag = __fadd_rn(mag, zf[-p - 1]);
                }
                res[c] = r;
                const float r32 = __double2float_rn(r);
                rf[c] = r32;
                bad += (!(fabs32(r32) <= conv_tol32 * mag) || isinf(mag)) ? 1u : 0u;
            }
            g.sync();
            unsigned fwdbad = 0;
            for (int i = tid; i < m; i += nt) {
                float acc = 0.0f;
                const float* Ti = T + i * LD;
#pragma unroll 4
                for (int u = 0; u < nnb; ++u) {
                    const int pc = nbl[u];
                    acc = __fmaf_rn(Ti[(unsigned)pc >> 16], rf[pc & 0xffff], acc);
                }
                const int v = row_var[i];
                // the correction: B^-1 r (FP32), plus r_c exactly for a basic slack
                const double d = (v >= n) ? __dadd_rn((double)acc, res[v - n]) : (double)acc;
                const double znew = __dadd_rn(z[i], d);
                z[i] = znew;
                const float zn32 = fabs32(__double2float_rn(znew));
                zf[i] = zn32;
                fwdbad += (!(fabs32(__double2float_rn(d)) <= fwd_tol32 * fmaxf(zn32, zfloor))) ? 1u : 0u;
            }
            unsigned tot, dummy;
            g.count_min(bad + (fwdbad << 16), 0u, tot, dummy);
            if (tot == 0) { conv = true; break; }
        }
    };

    if (ok) {
        bool conv;
        refine(xb, -1, conv);
        // primal feasibility of the basic solution
        unsigned bad = 0, dummy;
        for (int i = tid; i < m; i += nt) bad += (xb[i] < -tol_p) ? 1u : 0u;
        g.count_min(bad, 0u, bad, dummy);
        ok = conv && bad == 0;
    }
    if (ok && status == kOptimal) {
        // dual: y_c = reduced cost of slack c; refine  y^T B = c_B^T
        for (int c = tid; c < m; c += nt) {
            const int p = spos[c];
            yv[c] = (p > 0) ? (double)T[m * LD + p] : 0.0;
        }
        g.sync();
        bool conv = false;
        double yloc = 0.0;
        for (int c = tid; c < m; c += nt) {
            yloc = (abskey(yv[c]) > abskey(yloc)) ? yv[c] : yloc;
            zf[c] = __double2float_rn(yv[c]);  // y in FP32 (signed: the dual screen uses it)
        }
        const float yfloor = (float)mp.fwd_floor * __double2float_ru(block_absmax(g, yloc));  // barrier: zf complete
        for (int it = 0; it <= mp.max_refine; ++it) {
            // rho_i = c_(v_i) - y^T col(v_i) for each basic variable (by tableau row)
            // (split over P lanes per basic variable, rows c = q, q + P, ...)
            unsigned bad = 0;
            for (int t0 = 0; t0 < s; t0 += sgroups) {
                const int t = t0 + sgid;
                const bool act = t < s;
                const int i = act ? slist[t] : 0;
                const int v = act ? row_var[i] : 0;
                double r = (act && sq == 0) ? cv[v] : 0.0;
                float mag = (act && sq == 0) ? f64_abs_to_f32_trunc(r) : 0.0f;
                if (act) {
#pragma unroll 4
                    for (int c = sq; c < m; c += P) {
                        const double a = A[(size_t)c * n + v];
                        r = __fma_rn(-yv[c], a, r);
                        mag = __fmaf_rn(f64_abs_to_f32_trunc(a), fabs32(zf[c]), mag);
                    }
                }
                r = group_sum(r, P);
                mag = group_sum(mag, P);
                if (act && sq == 0) {
                    res[i] = r;
                    const float r32 = __double2float_rn(r);
                    rf[i] = r32;
                    bad += (!(fabs32(r32) <= conv_tol32 * mag) || isinf(mag)) ? 1u : 0u;
                }
            }
            for (int i = tid; i < m; i += nt) {
                const int v = row_var[i];
                if (v >= n) {
                    res[i] = -yv[v - n];
                    rf[i] = -zf[v - n];
                    bad += (abskey(yv[v - n]) != 0) ? 1u : 0u;
                }
            }
            g.sync();
            // corrections of the non-basic slacks (B^-1 columns), split over
            // P lanes each; parked in zf[c], which is rewritten below
            for (int u0 = 0; u0 < nnb; u0 += sgroups) {
                const int u = u0 + sgid;
                const bool act = u < nnb;
                const int pc = act ? nbl[u] : 0;
                float acc = 0.0f;
                if (act) {
                    const float* Tp = T + ((unsigned)pc >> 16);
#pragma unroll 4
                    for (int i = sq; i < m; i += P) acc = __fmaf_rn(rf[i], Tp[i * LD], acc);
                }
                acc = group_sum(acc, P);
                if (act && sq == 0) zf[pc & 0xffff] = acc;
            }
            g.sync();
            unsigned fwdbad = 0;
            for (int c = tid; c < m; c += nt) {
                const int p = spos[c];
                const double d = (p > 0) ? (double)zf[c] : res[-p - 1];
                const double ynew = __dadd_rn(yv[c], d);
                yv[c] = ynew;
                const float yn32 = __double2float_rn(ynew);
                zf[c] = yn32;
                fwdbad += (!(fabs32(__double2float_rn(d)) <= fwd_tol32 * fmaxf(fabs32(yn32), yfloor))) ? 1u : 0u;
            }
            unsigned tot, dummy;
            g.count_min(bad + (fwdbad << 16), 0u, tot, dummy);
            if (tot == 0) { conv = true; break; }
        }
        // dual feasibility: y >= -tol and A^T y - c >= -tol on non-basic
        // structurals; each reduced cost is screened in FP32 (y from zf,
        // rounded; a truncated by f64_to_f32_trunc, < 2^-23 relative) with an
        // error bound and computed in FP64 only when the screen cannot decide
        unsigned bad = 0, dummy;
        for (int c = tid; c < m; c += nt) bad += (yv[c] < -tol_d) ? 1u : 0u;
        // (split over P lanes per column like the residuals)
        for (int j0 = 0; j0 < Cvar; j0 += sgroups) {
            const int j = 1 + j0 + sgid;
            const int v = (j <= Cvar) ? tb.col_var[j] : n;
            const bool act = v < n;
            float d32 = (act && sq == 0) ? -f64_to_f32_trunc(cv[v]) : 0.0f;
            float mag = fabs32(d32);
            if (act) {
#pragma unroll 4
                for (int c = sq; c < m; c += P) {
                    const float a = f64_to_f32_trunc(A[(size_t)c * n + v]);
                    const float yc = zf[c];
                    d32 = __fmaf_rn(yc, a, d32);
                    mag = __fmaf_rn(fabs32(yc), fabs32(a), mag);
                }
            }
            d32 = group_sum(d32, P);
            mag = group_sum(mag, P);
            // |d32 - d| <= (m/P + log2 P + 2) * 2^-23 * (|c| + sum |y||a|):
            // the conversions 1.5 * 2^-23, at most m/P + log2 P roundings of
            // 2^-24 in sequence; (m + 2) * 2^-23 * mag covers it with mag's
            // own roundings
            const bool undecided = act && (!(d32 - (float)(m + 2) * 1.2e-7f * mag >= -(float)tol_d) || isinf(mag));
            if (__any_sync(kFull, undecided)) {
                double d = (undecided && sq == 0) ? -cv[v] : 0.0;
                if (undecided) {
#pragma unroll 4
                    for (int c = sq; c < m; c += P) d = __fma_rn(yv[c], A[(size_t)c * n + v], d);
                }
                d = group_sum(d, P);
                if (undecided && sq == 0) bad += (d < -tol_d) ? 1u : 0u;
            }
        }
        g.count_min(bad, 0u, bad, dummy);
        ok = conv && bad == 0;
    }
    if (ok && status == kUnbounded) {
        // ray: entering variable up by 1, basic variables by d = -B^-1 a_e
        const int ve = tb.col_var[e_unb];
        for (int i = tid; i < m; i += nt) dv[i] = -(double)T[i * LD + e_unb];
        g.sync();
        bool conv;
        refine(dv, ve, conv);
        double loc = 0.0;
        for (int i = tid; i < m; i += nt) loc = (abskey(dv[i]) > abskey(loc)) ? dv[i] : loc;
        const double dmax = block_absmax(g, loc);
        unsigned bad = 0, dummy;
        for (int i = tid; i < m; i += nt) bad += (dv[i] < -mp.cert_tol * fmax(1.0, dmax)) ? 1u : 0u;
        g.count_min(bad, 0u, bad, dummy);
        // objective increase along the ray (warp 0, fixed order)
        if (warp == 0) {
            double part = 0.0;
            for (int t = lane; t < s; t += 32) {
                const int i = slist[t];
                part = __fma_rn(cv[row_var[i]], dv[i], part);
            }
            for (int o = 16; o > 0; o >>= 1) part = __dadd_rn(part, __shfl_xor_sync(kFull, part, o));
            if (lane == 0) s_cd = __dadd_rn(part, (ve < n) ? cv[ve] : 0.0);
        }
        g.sync();
        ok = conv && bad == 0 && s_cd > mp.cert_tol * fmax(1.0, dmax) * cmax;
    }

    // ---- infeasible: Farkas certificate from the phase-I basis ---------------
    // y_c = reduced cost of slack c in the phase-I row (0 when basic) is the
    // multiplier vector of phase I's dual: y >= 0, A^T y >= 0, b^T y = -w* < 0,
    // and y_i <= 1 on the negated rows.  It is refined in FP64 so that y^T B
    // equals phase I's costs on the basis (0 for structurals and slacks; y_i = 1
    // on a row whose artificial is basic), then checked: y >= 0, A^T y >= 0 to
    // rounding, and gamma = -b^T y with gamma / max(y on negated rows) above
    // 1e-6 max(1, max|b|).  That quotient bounds the phase-I optimum from below
    // (sum of artificials >= gamma / max y_neg for every x >= 0), so the FP64
    // rule (infeasible when the phase-I optimum exceeds 1e-9 max(1, max|b|))
    // reaches the same status.  Otherwise the LP goes to the FP64 re-solve.
    bool farkas = false;
    if (status == kInfeasible && k > 0) {
        int sf = 0;
        for (int j = 1 + tid; j <= Cvar; j += nt) {
            const int v = tb.col_var[j];
            if (v >= n && v < nm) spos[v - n] = j;
        }
        for (int i0 = 0; i0 < m; i0 += nt) {
            const int i = i0 + tid;
            const int v = (i < m) ? row_var[i] : -1;
            if (i < m && v >= n && v < nm) spos[v - n] = -(i + 1);
            const bool st = (i < m) && (v < n);
            int tot;
            const int pos = sf + g.prefix_count(st, tot);
            if (st) slist[pos] = i;
            sf += tot;
        }
        unsigned badpos = 0, dummy;
        for (int c = tid; c < m; c += nt) {
            const int p = spos[c];
            badpos += (p == 0 || p > Cvar || -p - 1 >= m) ? 1u : 0u;
        }
        g.count_min(badpos, 0u, badpos, dummy);
        if (badpos == 0) {
            nnb = build_nbl();
            const float* Tw = T + (m + 1) * LD;
            for (int c = tid; c < m; c += nt) {
                const int p = spos[c];
                yv[c] = (p > 0) ? (double)Tw[p] : 0.0;
            }
            g.sync();
            for (int it = 0; it < 4; ++it) {
                // residual of y^T B = c_B (phase-I costs), one entry per tableau
                // row (split over P lanes per basic structural)
                for (int t0 = 0; t0 < sf; t0 += sgroups) {
                    const int t = t0 + sgid;
                    const bool act = t < sf;
                    const int v = act ? row_var[slist[t]] : 0;
                    double r = 0.0;
                    if (act) {
#pragma unroll 4
                        for (int c = sq; c < m; c += P) r = __fma_rn(-yv[c], A[(size_t)c * n + v], r);
                    }
                    r = group_sum(r, P);
                    if (act && sq == 0) {
                        res[slist[t]] = r;
                        rf[slist[t]] = __double2float_rn(r);
                    }
                }
                for (int i = tid; i < m; i += nt) {
                    const int v = row_var[i];
                    double r;
                    if (v >= n && v < nm) r = -yv[v - n];
                    else if (v >= nm) r = __dsub_rn(yv[neg[v - nm]], 1.0);
                    else continue;
                    res[i] = r;
                    rf[i] = __double2float_rn(r);
                }
                g.sync();
                // corrections of the non-basic slacks, split over P lanes each
                for (int u0 = 0; u0 < nnb; u0 += sgroups) {
                    const int u = u0 + sgid;
                    const bool act = u < nnb;
                    const int pc = act ? nbl[u] : 0;
                    float acc = 0.0f;
                    if (act) {
                        const float* Tp = T + ((unsigned)pc >> 16);
#pragma unroll 4
                        for (int i = sq; i < m; i += P) acc = __fmaf_rn(rf[i], Tp[i * LD], acc);
                    }
                    acc = group_sum(acc, P);
                    if (act && sq == 0) zf[pc & 0xffff] = acc;
                }
                g.sync();
                for (int c = tid; c < m; c += nt) {
                    const int p = spos[c];
                    const double d = (p > 0) ? (double)zf[c] : res[-p - 1];
                    yv[c] = __dadd_rn(yv[c], d);
                }
                g.sync();
            }
            // checks: y >= 0 (tiny negatives clamped), A^T y >= 0 to rounding
            unsigned bad = 0;
            for (int c = tid; c < m; c += nt) {
                const double yc = yv[c];
                bad += (yc < -1e-9) ? 1u : 0u;
                if (yc < 0.0) yv[c] = 0.0;
            }
            g.count_min(bad, 0u, bad, dummy);
            for (int j = tid; j < n; j += nt) {
                double gj = 0.0, sc = 0.0;
#pragma unroll 4
                for (int c = 0; c < m; ++c) {
                    const double a = A[(size_t)c * n + j];
                    gj = __fma_rn(yv[c], a, gj);
                    sc = __fma_rn(yv[c], fabs(a), sc);
                }
                bad += (gj < -1e-12 * sc) ? 1u : 0u;
            }
            double yneg = 0.0;
            for (int t = tid; t < k; t += nt) yneg = fmax(yneg, yv[neg[t]]);
            const double ymax_neg = block_absmax(g, yneg);
            g.count_min(bad, 0u, bad, dummy);
            if (warp == 0) {
                double part = 0.0;
                for (int c = lane; c < m; c += 32) part = __fma_rn(-bv[c], yv[c], part);
                for (int o = 16; o > 0; o >>= 1) part = __dadd_rn(part, __shfl_xor_sync(kFull, part, o));
                if (lane == 0) s_gamma = part;
            }
            g.sync();
            farkas = bad == 0 && ymax_neg > 0.0 && s_gamma > 1e-6 * bmax * ymax_neg;
        }
    }
    if (farkas) {
        double* __restrict__ x = B.x + B.x_off[lp];
        for (int j = tid; j < n; j += nt) x[j] = 0.0;
        if (B.y) {
            double* __restrict__ y = B.y + B.y_off[lp];
            for (int c = tid; c < m; c += nt) y[c] = yv[c];
        }
        if (tid == 0) {
            B.status[lp] = kInfeasible;
            B.iters[lp] = iters;
            B.obj[lp] = 0.0;
        }
        return;
    }

    if (!ok) {
        if (tid == 0) {
            // FP64 re-solve in one CTA when its FP64 tableau fits, else streamed
            const bool fits = resident_smem_bytes(m, n, k) <= kMaxSmemPerBlock - 1024;
            int32_t* q = fits ? fq.q : fq.qbig;
            int32_t* len = fits ? fq.len : fq.lenbig;
            const int32_t cap = fits ? fq.cap : fq.capbig;
            const int pos = q ? atomicAdd(len, 1) : cap;
            if (pos < cap) {
                q[pos] = lp;
            } else {
                record_internal_error(diag, 4, lp);
                B.status[lp] = kNumerical;
            }
        }
        return;
    }

    // ---- certified: FP64 outputs ------------------------------------------------
    double* __restrict__ x = B.x + B.x_off[lp];
    double* __restrict__ y = B.y ? B.y + B.y_off[lp] : nullptr;
    for (int j = 1 + tid; j <= Cvar; j += nt) {
        const int v = tb.col_var[j];
        if ((unsigned)v < (unsigned)n) x[v] = 0.0;
    }
    for (int i = tid; i < m; i += nt) {
        const int v = row_var[i];
        if ((unsigned)v < (unsigned)n) x[v] = xb[i];
    }
    if (y) {
        for (int c = tid; c < m; c += nt) {
            if (status == kOptimal) {
                y[c] = yv[c];
            } else {
                const int p = spos[c];
                y[c] = (p > 0) ? (double)T[m * LD + p] : 0.0;
            }
        }
    }
    if (warp == 0) {
        double part = 0.0;
        for (int t = lane; t < s; t += 32) {
            const int i = slist[t];
            part = __fma_rn(cv[row_var[i]], xb[i], part);
        }
        for (int o = 16; o > 0; o >>= 1) part = __dadd_rn(part, __shfl_xor_sync(kFull, part, o));
        if (lane == 0) s_obj = part;
    }
    g.sync();
    if (tid == 0) {
        B.status[lp] = status;
        B.iters[lp] = iters;
        B.obj[lp] = s_obj;
    }
}

}  // namespace
}  // namespace lpb
