// lp_cluster.cu -- FP64 simplex of one LP on a thread-block cluster: the
// condensed tableau (Section 3.1) is split by rows over the cluster's CTAs and
// kept in their shared memory for the whole solve (distributed shared memory),
// for tableaux larger than one CTA's shared memory.  Same rules and the same
// FP64 operations as the single-CTA kernel (Steps 1-3, two-phase method, tie
// windows, drive-out), so the results are bit-identical to it and to the
// oracle.  The paper keeps such tableaux in global memory (Section 4).
//
// Row r of the tableau lives in CTA r / rp (rp rows per CTA).  Column data
// (labels, the count of live columns) and the row labels are replicated in
// every CTA and updated identically.  One pivot:
//   A. every CTA copies the objective row from its owner (DSMEM) and runs
//      Step 1 on the copy (identical data -> identical entering column e);
//   B. Step 2, screened as in the one-CTA kernel: FP32 ratio keys of each
//      CTA's rows -> exchange slot, cluster barrier 1, cluster minimum and
//      window; each CTA counts its candidates, computes their exact ratios,
//      and normalizes its lowest candidate row into its pivot-row buffer
//      (speculatively) -> slot, barrier 2.  One candidate in the cluster (the
//      common case) is the exact answer and its buffer is ready; several take
//      the exact rule (one more exchange) and, if the buffered row is not the
//      chosen one, its owner normalizes again behind one more barrier;
//   C. every CTA copies the pivot row from the owner's buffer and updates its
//      own rows (and retires an artificial column); barrier 3.
// So a pivot costs three cluster barriers in the common case.
// Exchange slots alternate between pivots, so a slot is only rewritten after
// every reader has passed a later barrier.  Every branch depends on replicated
// values or on values read after a barrier, so all CTAs of a cluster take the
// same path through every barrier.
// Persistent: rank 0 of each cluster takes the next LP from an atomic counter.

#include <cooperative_groups.h>

#include <algorithm>
#include <climits>

#include "lp_device.cuh"
#include "lp_internal.h"

namespace cg = cooperative_groups;

namespace lpb {
namespace {

constexpr int kClusterThreads = 512;

// Tie window of Steps 1 and 2: v + tau * max(1, |v|) (product, then sum).
__device__ __forceinline__ double tie_thr(double v, double tau) {
    const long long ab = abskey(v);
    const double s = (ab < 0x3FF0000000000000LL) ? 1.0 : __longlong_as_double(ab);
    return __dadd_rn(v, __dmul_rn(tau, s));
}

// Exchange slots in shared memory (two of each, alternating).
struct Xch {
    long long fmin[2];  // Step 2: this CTA's minimum screened ratio key
    long long rmin[2];  // Step 2: minimum exact ratio key over this CTA's candidates
    unsigned cnt[2];    // Step 2: candidates in this CTA
    unsigned sel[2];    // lowest candidate row (Step 2) / selected column (drive-out)
    unsigned sel2[2];   // Step 2, several candidates: lowest row within the exact window
    unsigned pad[2];
    double pe[2];       // pivot element of `sel`
};
static_assert(sizeof(Xch) <= kClusterXchBytes, "exchange slots exceed their shared-memory region");

__device__ __forceinline__ void build_and_solve(cg::cluster_group& cl, const int C, const int q,
                                                const DeviceBatch& B, const Tolerances& tol, const int lp,
                                                unsigned char* smem, int32_t* diag) {
    const int m = B.m[lp];
    const int n = B.n[lp];
    const int nm = n + m;
    const double* __restrict__ A = B.A + B.a_off[lp];
    const double* __restrict__ bv = B.b + B.b_off[lp];
    const double* __restrict__ cv = B.c + B.c_off[lp];
    const int tid = threadIdx.x, nt = blockDim.x;
    Reducer red{reinterpret_cast<long long*>(smem + SmallLayout::red64),
                reinterpret_cast<unsigned*>(smem + SmallLayout::red32), nt >> 5, tid >> 5, tid & 31};
    const ClusterLayout L0 = cluster_layout(m, n, 0, C);
    int* row_var = reinterpret_cast<int*>(smem + L0.row_var);
    int* neg = reinterpret_cast<int*>(smem + L0.neg);
    Xch* xch = reinterpret_cast<Xch*>(smem + L0.xch);

    // ---- negated rows, ranked (every CTA, identically) -------------------
    int k = 0;
    for (int i0 = 0; i0 < m; i0 += nt) {
        const int i = i0 + tid;
        const bool isneg = (i < m) && (bv[i] < 0.0);
        int tot;
        const int r = k + red.prefix_count(isneg, tot);
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
    __syncthreads();
    const ClusterLayout L = cluster_layout(m, n, k, C);
    const int LD = L.LD, rp = L.rp;
    int* col_var = reinterpret_cast<int*>(smem + L.col_var);
    double* T = reinterpret_cast<double*>(smem + L.T);       // this CTA's rows
    double* prow = reinterpret_cast<double*>(smem + L.prow); // pivot-row buffer (read by the others)
    double* ob = reinterpret_cast<double*>(smem + L.ob);     // local copy of a remote row
    double* colE = reinterpret_cast<double*>(smem + L.colE);
    long long* rkey = reinterpret_cast<long long*>(smem + L.rkey);
    const int R = m + 1 + (k > 0 ? 1 : 0);
    const int r_lo = q * rp;
    const int nrow = max(0, min(R, r_lo + rp) - r_lo);
    int Cvar = n + k;
    // row r of the cluster's tableau, wherever it lives
    auto row_ptr = [&](int r) -> double* { return cl.map_shared_rank(T, r / rp) + (size_t)(r % rp) * LD; };

    for (int j = tid; j <= Cvar; j += nt) col_var[j] = (j == 0) ? -1 : (j <= n ? j - 1 : n + neg[j - 1 - n]);
    {
        // this CTA's constraint rows: A in one flat pass (several independent
        // loads in flight per thread), then b and the slack columns
        const int rows_a = max(0, min(m, r_lo + rp) - r_lo);
        const int64_t cnt = (int64_t)rows_a * n;
        const double* Ab = A + (size_t)r_lo * n;
        int lr = (n > 0) ? tid / n : 0, j = tid - lr * n;
        const int dl = nt / n, dj = nt - dl * n;
        for (int64_t idx = tid; idx < cnt; idx += nt) {
            cp_async8(T + (size_t)lr * LD + 1 + j, Ab + idx);
            lr += dl;
            j += dj;
            if (j >= n) { j -= n; ++lr; }
        }
        cp_async_wait_all();
        __syncthreads();
        if (k > 0)  // negated rows (b_i < 0)
            for (int64_t idx = tid; idx < cnt; idx += nt) {
                const int l2 = (int)(idx / n), j2 = (int)(idx - (int64_t)l2 * n);
                if (row_var[r_lo + l2] >= nm) T[(size_t)l2 * LD + 1 + j2] = -T[(size_t)l2 * LD + 1 + j2];
            }
        for (int lr2 = 0; lr2 < rows_a; ++lr2) {
            const int r = r_lo + lr2;
            const bool isneg = row_var[r] >= nm;
            double* Tr = T + (size_t)lr2 * LD;
            for (int t = tid; t <= k; t += nt) {
                const int jj = (t == 0) ? 0 : n + t;
                const double v = (t == 0) ? bv[r] : ((neg[t - 1] == r) ? 1.0 : 0.0);
                Tr[jj] = isneg ? -v : v;
            }
        }
        if (m >= r_lo && m < r_lo + rp) {
            double* Tm = T + (size_t)(m - r_lo) * LD;
            for (int jj = tid; jj <= Cvar; jj += nt) Tm[jj] = (jj >= 1 && jj <= n) ? -cv[jj - 1] : 0.0;
        }
    }
    long long bmax_key = 0x3FF0000000000000LL;  // 1.0
    for (int i = tid; i < m; i += nt) bmax_key = max(bmax_key, abskey(bv[i]));
    bmax_key = -red.min_i64(-bmax_key);
    cl.sync();  // every constraint row built
    if (k > 0 && (m + 1) / rp == q) {
        // auxiliary objective: subtract every negated row in ascending order
        double* Tw = T + (size_t)((m + 1) - r_lo) * LD;
        for (int j = tid; j <= Cvar; j += nt) {
            double w = 0.0;
            for (int t = 0; t < k; ++t) w = __dsub_rn(w, row_ptr(neg[t])[j]);
            Tw[j] = w;
        }
    }
    cl.sync();

    const long long key_neg_eps_opt = okey(-tol.eps_opt);
    const long long key_eps_piv = okey(tol.eps_piv);
    const int max_iters = tol.max_iters > 0 ? tol.max_iters : 50 * (m + n);
    int iters = 0, status = -1, phase = (k > 0) ? 1 : 2, yrow = m, xs = 0;

    // Pivot on row l, column e over rows < Ract.  With `ready`, the owner of
    // row l has already written the normalized row into its buffer; otherwise
    // it normalizes now and a barrier publishes the buffer.  Returns the label
    // of the leaving variable.
    auto pivot = [&](int l, int e, int Ract, bool ready) -> int {
        const int Cact = Cvar + 1;
        const int ql = l / rp;
        if (q == ql) {
            double* Tl = T + (size_t)(l - r_lo) * LD;
            if (!ready) {
                const double pe = colE[l - r_lo];
                for (int j = tid; j < Cact; j += nt) prow[j] = __ddiv_rn((j == e) ? 1.0 : Tl[j], pe);
                __syncthreads();
            }
            for (int j = tid; j < Cact; j += nt) Tl[j] = prow[j];
        }
        if (tid == 0) {
            const int ev = col_var[e];
            col_var[e] = row_var[l];
            row_var[l] = ev;
        }
        if (!ready) cl.sync();  // the pivot row is published
        const double* src = cl.map_shared_rank(prow, ql);
        for (int j = tid; j < Cact; j += nt) ob[j] = src[j];
        __syncthreads();
        const int left = col_var[e];
        const int rows = max(0, min(Ract, r_lo + rp) - r_lo);
        // this CTA's rows except the pivot row, element by element with the
        // (row, column) position stepped incrementally (no division per element)
        const int lloc = (q == ql) ? l - r_lo : rows;  // local index of the pivot row (rows: not here)
        const int total = (rows - (lloc < rows ? 1 : 0)) * Cact;
        int ii = tid / Cact, jj = tid - ii * Cact;
        const int di = nt / Cact, dj = nt - di * Cact;
        for (int idx = tid; idx < total; idx += nt) {
            const int lr = ii + (ii >= lloc ? 1 : 0);
            double* t = T + (size_t)lr * LD + jj;
            *t = __fma_rn(-colE[lr], ob[jj], (jj == e) ? 0.0 : *t);
            ii += di;
            jj += dj;
            if (jj >= Cact) { jj -= Cact; ++ii; }
        }
        __syncthreads();
        if (left >= nm) {
            // a retired artificial: the last live column moves into e
            if (e != Cvar)
                for (int lr = tid; lr < rows; lr += nt) {
                    double* row = T + (size_t)lr * LD;
                    row[e] = row[Cvar];
                }
            if (tid == 0 && e != Cvar) col_var[e] = col_var[Cvar];
            --Cvar;
            __syncthreads();
        }
        cl.sync();  // every row updated
        return left;
    };

    while (status < 0) {
        const int orow = (phase == 1) ? m + 1 : m;
        const int Ract = (phase == 1) ? m + 2 : m + 1;
        // ---- A: objective row copy, Step 1 ------------------------------
        {
            const double* src = row_ptr(orow);
            for (int j = tid; j <= Cvar; j += nt) ob[j] = src[j];
            __syncthreads();
        }
        long long dloc = LLONG_MAX;
        for (int j = 1 + tid; j <= Cvar; j += nt)
            if (col_var[j] < nm) dloc = min(dloc, okey(ob[j]));
        const long long dmin = red.min_i64(dloc);
        if (dmin >= key_neg_eps_opt) {
            if (phase == 2) { status = kOptimal; break; }
            const double wstar = -ob[0];
            if (wstar > __dmul_rn(tol.eps_feas, __longlong_as_double(bmax_key))) {
                status = kInfeasible;
                yrow = m + 1;
                break;
            }
            // drive artificials still basic out of the basis
            for (int i = 0; i < m && status < 0; ++i) {
                if (row_var[i] < nm) continue;
                const int qi = i / rp;
                if (q == qi) {
                    const double* Ti = T + (size_t)(i - r_lo) * LD;
                    unsigned sel = 0xffffffffu;
                    for (int j = 1 + tid; j <= Cvar; j += nt)
                        if (col_var[j] < nm && abskey(Ti[j]) > key_eps_piv)
                            sel = min(sel, ((unsigned)col_var[j] << 16) | (unsigned)j);
                    sel = red.min_u32(sel);
                    if (tid == 0) xch->sel[xs] = sel;
                }
                cl.sync();
                const unsigned sel = cl.map_shared_rank(xch, qi)->sel[xs];
                xs ^= 1;
                if (sel == 0xffffffffu) continue;  // redundant row
                if (iters >= max_iters) { status = kIterLimit; break; }
                const int e = (int)(sel & 0xffffu);
                for (int lr = tid; lr < nrow; lr += nt)
                    if (r_lo + lr < m + 1) colE[lr] = T[(size_t)lr * LD + e];
                __syncthreads();
                pivot(i, e, m + 1, false);
                ++iters;
            }
            phase = 2;
            continue;
        }
        const long long kthr = okey(tie_thr(kval(dmin), tol.tau));
        unsigned esel = 0xffffffffu;
        for (int j = 1 + tid; j <= Cvar; j += nt) {
            const int v = col_var[j];
            if (v < nm && okey(ob[j]) <= kthr) esel = min(esel, ((unsigned)v << 16) | (unsigned)j);
        }
        esel = red.min_u32(esel);
        const int e = (int)(esel & 0xffffu);
        if (e < 1 || e > Cvar) {
            if (tid == 0 && q == 0) record_internal_error(diag, 1, lp, e, Cvar, iters, phase, 0);
            status = kNumerical;
            break;
        }
        // ---- B: Step 2.  FP32 screen of this CTA's rows (rows whose operands
        // leave [2^-100, 2^100] are always candidates), cluster minimum, window
        // max(2^-12, 8 tau) relative + max(2^-20, 8 tau) absolute (far wider
        // than the screen's error: operands truncated to FP32 by integer
        // operations, < 2^-23 relative each, no FP64-pipe conversion, and the
        // approximate divide); one candidate in the cluster is the exact
        // answer, several get the exact rule on their exact ratios.
        int floc = INT_MAX;
        for (int lr = tid; lr < nrow; lr += nt) {
            const int r = r_lo + lr;
            if (r >= Ract) continue;
            const double t = T[(size_t)lr * LD + e];
            colE[lr] = t;
            long long code = LLONG_MAX;  // not eligible
            if (r < m && okey(t) > key_eps_piv) {
                const double beta = T[(size_t)lr * LD];
                const int et = dexp(t), eb = dexp(beta);
                const bool safe = et >= -100 && et <= 100 && (abskey(beta) == 0 || (eb >= -100 && eb <= 100));
                if (safe) {
                    const int fk = fkey(__fdividef(f64_to_f32_trunc(beta), f64_to_f32_trunc(t)));
                    code = fk;
                    floc = min(floc, fk);
                } else {
                    code = LLONG_MIN;
                }
            }
            rkey[lr] = code;
        }
        floc = red.min_i32(floc);
        if (tid == 0) xch->fmin[xs] = floc;
        cl.sync();  // 1
        int fmin = INT_MAX;
        for (int qq = 0; qq < C; ++qq) fmin = min(fmin, (int)cl.map_shared_rank(xch, qq)->fmin[xs]);
        long long fwin = LLONG_MIN;
        if (fmin != INT_MAX) {
            const float fm = fval(fmin);
            fwin = fkey(fm + __fmaf_rn(tol.ratio_rel, fabsf(fm), tol.ratio_abs));
        }
        unsigned lcnt = 0, lsel = 0xffffffffu;
        for (int lr = tid; lr < nrow; lr += nt) {
            const long long code = rkey[lr];
            if (r_lo + lr < m && (code == LLONG_MIN || (code != LLONG_MAX && code <= fwin))) {
                ++lcnt;
                lsel = min(lsel, (unsigned)(r_lo + lr));
            }
        }
        red.count_min(lcnt, lsel, lcnt, lsel);
        // exact ratio keys of this CTA's candidates (every other row: none),
        // so that rkey no longer holds screen keys in any CTA
        long long rloc = LLONG_MAX;
        for (int lr = tid; lr < nrow; lr += nt) {
            const long long code = rkey[lr];
            long long rk = LLONG_MAX;
            if (r_lo + lr < m && (code == LLONG_MIN || (code != LLONG_MAX && code <= fwin)))
                rk = okey(__ddiv_rn(T[(size_t)lr * LD], colE[lr]));
            rkey[lr] = rk;
            rloc = min(rloc, rk);
        }
        if (lcnt > 0) rloc = red.min_i64(rloc);
        // speculative: the lowest candidate row, normalized, into the buffer
        if (lcnt > 0) {
            const int lr = (int)lsel - r_lo;
            const double pe = colE[lr];
            const double* Tl = T + (size_t)lr * LD;
            for (int j = tid; j <= Cvar; j += nt) prow[j] = __ddiv_rn((j == e) ? 1.0 : Tl[j], pe);
        }
        if (tid == 0) {
            xch->cnt[xs] = lcnt;
            xch->sel[xs] = lsel;
            xch->rmin[xs] = rloc;
            xch->pe[xs] = (lcnt > 0) ? colE[lsel - r_lo] : 0.0;
        }
        cl.sync();  // 2
        unsigned total = 0, l = 0xffffffffu;
        double pe = 0.0;
        long long rmin = LLONG_MAX;
        for (int qq = 0; qq < C; ++qq) {
            const Xch* xo = cl.map_shared_rank(xch, qq);
            const unsigned c = xo->cnt[xs];
            total += c;
            if (c > 0 && xo->sel[xs] < l) { l = xo->sel[xs]; pe = xo->pe[xs]; }
            rmin = min(rmin, xo->rmin[xs]);
        }
        bool ready = true;
        if (total == 0) {
            xs ^= 1;
            status = (phase == 2) ? kUnbounded : kNumerical;
            break;
        }
        if (total > 1) {
            // exact rule over the candidates: lowest row within the tie window
            // of the minimum exact ratio
            const long long rthr = okey(tie_thr(kval(rmin), tol.tau));
            unsigned s2 = 0xffffffffu;
            for (int lr = tid; lr < nrow; lr += nt)
                if (r_lo + lr < m && rkey[lr] <= rthr) s2 = min(s2, (unsigned)(r_lo + lr));
            s2 = red.min_u32(s2);
            if (tid == 0) xch->sel2[xs] = s2;
            cl.sync();
            l = 0xffffffffu;
            for (int qq = 0; qq < C; ++qq) l = min(l, cl.map_shared_rank(xch, qq)->sel2[xs]);
            // the owner's buffer holds its lowest candidate: ready if that is l
            ready = false;
            if (l < (unsigned)m) {
                const Xch* xo = cl.map_shared_rank(xch, (int)l / rp);
                ready = xo->cnt[xs] > 0 && xo->sel[xs] == l;
                pe = ready ? xo->pe[xs] : 0.0;
            }
        }
        xs ^= 1;
        if (l >= (unsigned)m) {
            if (tid == 0 && q == 0) record_internal_error(diag, 2, lp, (int)l, (int)total, iters, phase, e);
            status = kNumerical;
            break;
        }
        if (!ready) pe = cl.map_shared_rank(colE, (int)l / rp)[l - ((int)l / rp) * rp];
        if (abskey(pe) >= 0x7FF0000000000000LL) { status = kNumerical; break; }
        if (iters >= max_iters) { status = kIterLimit; break; }
        pivot((int)l, e, Ract, ready);
        ++iters;
    }

    // ---- labels must name variables (replicated: the same decision everywhere)
    {
        unsigned badl = 0, dummy;
        const unsigned nvar = (unsigned)(nm + k);
        for (int i = tid; i < m; i += nt) badl += ((unsigned)row_var[i] >= nvar) ? 1u : 0u;
        for (int j = 1 + tid; j <= Cvar; j += nt) badl += ((unsigned)col_var[j] >= nvar) ? 1u : 0u;
        red.count_min(badl, 0u, badl, dummy);
        if (badl) {
            if (tid == 0 && q == 0) {
                record_internal_error(diag, 6, lp, (int)badl, status, iters, phase, Cvar);
                B.status[lp] = kNumerical;
                B.iters[lp] = iters;
            }
            return;
        }
    }
    // ---- results (each CTA its rows; rank 0 the non-basic structurals) -----
    double* __restrict__ x = B.x + B.x_off[lp];
    double* __restrict__ y = B.y ? B.y + B.y_off[lp] : nullptr;
    if (q == 0)
        for (int j = 1 + tid; j <= Cvar; j += nt) {
            const int v = col_var[j];
            if ((unsigned)v < (unsigned)n) x[v] = 0.0;
        }
    if (y && yrow / rp == q) {
        const double* Ty = T + (size_t)(yrow - r_lo) * LD;
        for (int j = 1 + tid; j <= Cvar; j += nt) {
            const int v = col_var[j];
            if (v >= n && v < nm) y[v - n] = Ty[j];
        }
    }
    for (int lr = tid; lr < nrow; lr += nt) {
        const int r = r_lo + lr;
        if (r >= m) continue;
        const int v = row_var[r];
        if ((unsigned)v < (unsigned)n) x[v] = T[(size_t)lr * LD];
        else if (v >= n && v < nm && y) y[v - n] = 0.0;
    }
    if (tid == 0 && m / rp == q) B.obj[lp] = T[(size_t)(m - r_lo) * LD];
    if (tid == 0 && q == 0) {
        B.status[lp] = status;
        B.iters[lp] = iters;
    }
}

__global__ void __launch_bounds__(kClusterThreads, 1)
fp64_cluster_kernel(const DeviceBatch B, const Tolerances tol, const int32_t* __restrict__ order, const int32_t count,
                    const int32_t* __restrict__ count_dev, int32_t* __restrict__ counter, int32_t* __restrict__ diag)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_next;
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks();
    const int q = (int)cl.block_rank();
    const int n_items = count_dev ? min(*count_dev, count) : count;
    for (;;) {
        if (q == 0 && threadIdx.x == 0) s_next = atomicAdd(counter, 1);
        cl.sync();
        const int idx = *cl.map_shared_rank(&s_next, 0);
        cl.sync();  // every CTA has read it (and left the previous LP's rows)
        if (idx >= n_items) break;
        build_and_solve(cl, C, q, B, tol, order[idx], smem, diag);
    }
}

}  // namespace

size_t cluster_smem_bytes(int m, int n, int k, int C) { return cluster_layout(m, n, k, C).total; }

cudaError_t cluster_kernel_prepare() {
    cudaError_t err = cudaFuncSetAttribute(fp64_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)(kMaxSmemPerBlock - 1024));
    if (err != cudaSuccess) return err;
    return cudaFuncSetAttribute(fp64_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

// Clusters of `C` CTAs that can be resident at once with `smem` bytes each
// (0: this cluster shape cannot run).
int cluster_max_active(int C, size_t smem) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)C, 1, 1);
    cfg.blockDim = dim3(kClusterThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, fp64_cluster_kernel, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

cudaError_t launch_fp64_cluster(const DeviceBatch& B, const Tolerances& tol, const int32_t* order, int32_t count,
                                int C, int clusters, size_t smem, int32_t* counter, int32_t* diag,
                                cudaStream_t stream, const int32_t* count_dev) {
    if (count <= 0) return cudaSuccess;
    cudaError_t err = cudaMemsetAsync(counter, 0, sizeof(int32_t), stream);
    if (err != cudaSuccess) return err;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)(C * clusters), 1, 1);
    cfg.blockDim = dim3(kClusterThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fp64_cluster_kernel, B, tol, order, count, count_dev, counter, diag);
}

}  // namespace lpb
