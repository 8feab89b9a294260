// lp_fp64_simplex.cu -- FP64 dense simplex, one CTA per LP: the tableau is
// resident in shared memory when it fits (fp64_resident_kernel) and streamed
// through a global-memory workspace slot otherwise (fp64_streamed_kernel,
// persistent CTAs taking LPs from an atomic counter).  Both run the same
// per-LP code (solve_one).
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
//  - the tableau lives in shared memory for the whole solve (global memory is
//    touched only to read A, b, c and write the results), or, above one CTA's
//    shared memory, in a global workspace slot whose rank-1 update streams
//    through shared-memory rings filled by bulk asynchronous copies;
//  - reductions are warp `redux` instructions on 64-bit order-preserving
//    integer keys of the FP64 values (exact, no FP64-pipe compares);
//  - phase I runs in the same kernel (the paper launches twice, Section 5);
//  - Steps 1 and 2 screen their candidates without FP64 arithmetic (the FP64
//    pipe of GB300 is ~60x slower than FP32 and a warp FP64 instruction costs
//    the whole warp's pipe time whatever its active mask): Step 1 bounds the tie
//    window of the minimum reduced cost in units of the integer key, Step 2
//    bounds the ratios in FP32 with a window wider than every FP32 rounding
//    error.  When the screen leaves exactly one candidate it is the exact
//    answer; otherwise the exact FP64 rule runs on the candidates.  The result
//    is the same as the plain rule's in every case.
//
// Arithmetic is the oracle's, operation for operation, so that both reach the
// same pivot sequence: ratio = rhs / t (IEEE divide), pivot row = row / PE
// (IEEE divide), update t_ij = fma(-t_ie, r_j, t_ij), tie window
// v + tau*max(1,|v|) as a product followed by a sum.  This file is compiled
// with --fmad=false and only uses the _rn intrinsics for FP64 arithmetic.

#include <climits>

#include "lp_device.cuh"
#include "lp_internal.h"

namespace lpb {
namespace {

// Tie window of Steps 1 and 2: v + tau * max(1, |v|) (product, then sum).
__device__ __forceinline__ double tie_threshold(double v, double tau) {
    const long long ab = abskey(v);
    const double s = (ab < 0x3FF0000000000000LL) ? 1.0 : __longlong_as_double(ab);
    return __dadd_rn(v, __dmul_rn(tau, s));
}

// Upper bound, in units of okey, of okey(thr) - okey(v) where thr is the tie
// threshold v + tau*max(1,|v|) of a negative v (Step 1).  `wb` >=
// tau*2^54*(1+2^-53) + 1.5 is precomputed on the host (< 0: no bound).  The
// interval (v, thr] lies in v's binade or the one below (tau|v| < |v|/2), where
// doubles are spaced at least 2^(E-53) apart, E = exponent of v:
//   E >= 0: thr - v <= tau*2^(E+1)*(1+2^-53) + half an ulp  -> <= wb keys;
//   E <  0: thr - v <= tau*(1+2^-53) + half an ulp          -> <= wb << (-E-1).
__device__ __forceinline__ unsigned long long step1_window(long long kmin, long long wb) {
    if (wb < 0) return ~0ull;
    const int E = dexp(kval(kmin));
    if (E >= 0) return (unsigned long long)wb;
    const int sh = -E - 1;
    if (sh > 30) return ~0ull;
    return (unsigned long long)wb << sh;
}

// ---- Staged update of the streamed kernel ----------------------------------
// The rank-1 update of a tableau in global memory is bound by the bytes it
// keeps in flight.  Each warp streams its share of the rows through a ring of
// kStageDepth chunks of kStageChunkPairs column pairs in shared memory, filled
// by bulk asynchronous copies (cp.async.bulk, completion on one mbarrier per
// chunk) that one lane issues kStageDepth chunks ahead; the pivot row and the
// pivot column are read from shared-memory copies.  The FMA of every element
// is the one of the plain loop, so the results are the same bit for bit.
constexpr int kStageChunkPairs = 96;  // 1.5 KB per chunk: 3 pairs per lane
constexpr int kStageDepth = 3;
constexpr long long kStageWaitCycles = 2000000000LL;  // ~1 s at 2 GHz

// A CTA's shared memory for the staged update: a flag word, the mbarriers and
// rings of every warp, the pivot-row copy (LD doubles), then the pivot-column
// copy (R doubles) of the LP being solved.  Everything but the column copy
// sits at offsets that depend only on the number of warps.
__host__ __device__ inline size_t stage_rings(int nwarps) {
    return (16 + (size_t)nwarps * kStageDepth * 8 + 127) & ~size_t(127);
}
__host__ __device__ inline size_t stage_prow(int nwarps) {
    return stage_rings(nwarps) + (size_t)nwarps * kStageDepth * kStageChunkPairs * 16;
}
__host__ __device__ inline size_t stage_colE(int nwarps, int LD) { return stage_prow(nwarps) + align16((size_t)LD * 8); }
__host__ __device__ inline size_t stage_total(int nwarps, int R, int LD) {
    return stage_colE(nwarps, LD) + align16((size_t)R * 8);
}

// The staged path of one LP: `base` of the staging area (null: the plain
// loop) and the parities of the warp's chunk mbarriers (bit s: parity of the
// next completion of chunk s, warp-uniform).  The flag word at `base`: 1 a
// copy did not complete (LP abandoned); 2 one may still be in flight.
struct Staging {
    unsigned char* base;
    unsigned phase;
};
__device__ __forceinline__ uint64_t* stage_bars(unsigned char* base) {
    return reinterpret_cast<uint64_t*>(base + 16) + (threadIdx.x >> 5) * kStageDepth;
}

struct Tab {
    double* T;        // R x LD, row-major; column 0 = right-hand side
    double* colE;     // copy of the pivot column
    int* col_var;     // variable of each column (1..Cvar live)
    int* row_var;     // basic variable of each constraint row
    int LD;
};

// Phase B of Step 3 for a tableau in global memory, through the staging
// rings: chunk c covers row ii = c / cpr (skipping the pivot row l) and pairs
// [p0, p0 + len) of it; warp w takes chunks w, w + nw, ...  The pivot row is
// read from the staging area's copy, column e from tb.colE (shared memory on this path).
// The pair beyond an odd Cact is padding (updated, never read).  A copy that
// does not complete within kStageWaitCycles abandons the update: the flag
// word is set (the caller reports the LP as numerical) after the warp has waited,
// bounded again, for its other copies.
__device__ __noinline__ unsigned staged_update(const Staging st, const Tab tb, int Ract, int Cact, int l, int e) {
    unsigned phase = st.phase;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int LD = tb.LD;
    uint64_t* bar = stage_bars(st.base);
    double2* ring = reinterpret_cast<double2*>(st.base + stage_rings(nw)) + (size_t)warp * kStageDepth * kStageChunkPairs;
    const int Cp = (Cact + 1) >> 1;
    const int cpr = (Cp + kStageChunkPairs - 1) / kStageChunkPairs;
    const int total = (Ract - 1) * cpr;
    const double2* P2 = reinterpret_cast<const double2*>(st.base + stage_prow(nw));
    auto chunk = [&](int c, int& r, int& p0, int& len) {
        const int ii = c / cpr;
        const int piece = c - ii * cpr;
        r = ii + (ii >= l ? 1 : 0);
        p0 = piece * kStageChunkPairs;
        len = min(kStageChunkPairs, Cp - p0);
    };
    auto issue = [&](int c, int s) {  // lane 0
        int r, p0, len;
        chunk(c, r, p0, len);
        const unsigned bytes = (unsigned)len * 16u;
        mbar_expect_tx(&bar[s], bytes);
        bulk_load(ring + s * kStageChunkPairs, tb.T + (size_t)r * LD + 2 * p0, bytes, &bar[s]);
    };
    unsigned pending = 0;  // chunks issued and not yet waited for (warp-uniform)
    for (int s = 0; s < kStageDepth; ++s) {
        const int c = warp + s * nw;
        if (c < total) {
            if (lane == 0) issue(c, s);
            pending |= 1u << s;
        }
    }
    bool ok = true;
    for (int it = 0;; ++it) {
        const int c = warp + it * nw;
        if (c >= total) break;
        const int s = it % kStageDepth;
        ok = __all_sync(kFull, mbar_wait_bounded(&bar[s], (phase >> s) & 1u, kStageWaitCycles));
        if (!ok) break;
        phase ^= 1u << s;
        pending &= ~(1u << s);
        int r, p0, len;
        chunk(c, r, p0, len);
        const double cr = -tb.colE[r];
        const double2* src = ring + s * kStageChunkPairs;
        double2* dst = reinterpret_cast<double2*>(tb.T + (size_t)r * LD) + p0;
        for (int q = lane; q < len; q += 32) {
            const double2 old = src[q];
            const double2 p = P2[p0 + q];
            const int j = 2 * (p0 + q);
            double2 v;
            v.x = __fma_rn(cr, p.x, (j == e) ? 0.0 : old.x);
            v.y = __fma_rn(cr, p.y, (j + 1 == e) ? 0.0 : old.y);
            dst[q] = v;
        }
        __syncwarp();
        const int cn = c + kStageDepth * nw;
        if (cn < total) {
            if (lane == 0) {
                fence_proxy_async_shared();  // the warp's reads of chunk s before the copy over it
                issue(cn, s);
            }
            pending |= 1u << s;
        }
    }
    if (!ok) {
        // let the copies still in flight land before the rings are reused
        bool drained = true;
        for (int s = 0; s < kStageDepth; ++s)
            if (pending & (1u << s)) {
                drained = mbar_wait_bounded(&bar[s], (phase >> s) & 1u, kStageWaitCycles) && drained;
                phase ^= 1u << s;
            }
        if (lane == 0) atomicMax(reinterpret_cast<int*>(st.base), drained ? 1 : 2);
    }
    return phase;
}

// Step 3 (Section 3.1, Listing 1) on the condensed tableau: divide pivot row
// l by PE = colE[l], then t_ij <- fma(-t_ie, r_j, t_ij) for every other active
// row.  In column e (which now holds the leaving variable) the old entry of the
// paper's full tableau is the unit column of a basic variable, i.e. 0 off the
// pivot row and 1 on it, so r_e = 1/PE and t_ie <- fma(-t_ie, r_e, 0).
// colE[0..Ract) must hold column e on entry.  Returns the variable that left
// the basis (now the label of column e), read by every thread between the two
// barriers, where nothing writes it.
// kPairs (the streamed kernel: rows 32-byte aligned in global memory, LD a
// multiple of 4): the update takes two adjacent columns per thread with
// 16-byte loads and stores -- the same FMA for every element, so the same
// results; the pair beyond an odd Cact is padding (updated, never read).
// The barrier of the thread group that owns the LP: the CTA, or (kWarp: a
// one-warp CTA) the warp -- no block barrier, shared-memory writes ordered by
// __syncwarp.
template <bool kWarp>
__device__ __forceinline__ void group_sync() {
    if (kWarp) __syncwarp();
    else __syncthreads();
}

template <bool kPairs = false, bool kWarp = false>
__device__ __forceinline__ int pivot(Tab& tb, int Ract, int Cact, int l, int e, Staging* st = nullptr) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int LD = tb.LD;
    double* T = tb.T;
    const double* colE = tb.colE;
    const double pe = colE[l];
    double* Tl = T + (size_t)l * LD;
    const bool staged = kPairs && st != nullptr && st->base != nullptr;
    double* prow = staged ? reinterpret_cast<double*>(st->base + stage_prow(nt >> 5)) : nullptr;
    for (int j = tid; j < Cact; j += nt) {
        const double v = (j == e) ? 1.0 : Tl[j];
        const double q = __ddiv_rn(v, pe);
        Tl[j] = q;
        if (staged) prow[j] = q;
    }
    if (tid == 0) {
        const int ev = tb.col_var[e];
        tb.col_var[e] = tb.row_var[l];
        tb.row_var[l] = ev;
    }
    group_sync<kWarp>();
    const int left = tb.col_var[e];
    if (staged) {
        st->phase = staged_update(*st, tb, Ract, Cact, l, e);
        fence_proxy_async_global();  // this thread's stores before later bulk reads of them
        group_sync<kWarp>();
        return left;
    }
    if (kPairs) {
        const int Cp = (Cact + 1) >> 1;
        const int total = (Ract - 1) * Cp;
        int ii = tid / Cp;
        int jp = tid - ii * Cp;
        const int di = nt / Cp;
        const int dj = nt - di * Cp;
        const double2* Tl2 = reinterpret_cast<const double2*>(Tl);
        for (int idx = tid; idx < total; idx += nt) {
            const int r = ii + (ii >= l ? 1 : 0);
            double2* t = reinterpret_cast<double2*>(T + (size_t)r * LD) + jp;
            const double2 old = *t;
            const double2 p = Tl2[jp];
            const double c = -colE[r];
            double2 v;
            v.x = __fma_rn(c, p.x, (2 * jp == e) ? 0.0 : old.x);
            v.y = __fma_rn(c, p.y, (2 * jp + 1 == e) ? 0.0 : old.y);
            *t = v;
            ii += di;
            jp += dj;
            if (jp >= Cp) { jp -= Cp; ++ii; }
        }
        group_sync<kWarp>();
        return left;
    }
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
    group_sync<kWarp>();
    return left;
}

// A retired artificial (it just left the basis and may never re-enter) sits
// in column e: move the last live column into its place and shrink.
// `fence`: the tableau is read by bulk copies later (staged streamed update).
template <bool kWarp = false>
__device__ __forceinline__ void retire_column(Tab& tb, int Ract, int e, int& Cvar, bool fence = false) {
    const int tid = threadIdx.x, nt = blockDim.x;
    if (e != Cvar) {
        for (int r = tid; r < Ract; r += nt) {
            double* row = tb.T + (size_t)r * tb.LD;
            row[e] = row[Cvar];
        }
        if (tid == 0) tb.col_var[e] = tb.col_var[Cvar];
    }
    --Cvar;
    if (fence) fence_proxy_async_global();
    group_sync<kWarp>();
}

// One LP, Steps 1-3 until it halts.  `small` is shared memory
// (SmallLayout); `big` is shared memory (resident) or a global workspace slot
// (streamed), laid out by big_layout.  `stage` (streamed only, may be null):
// `stage_bytes` of this CTA's shared memory for the staged update, used when
// the LP's stage_total fits.
template <bool kStreamed, bool kWarp = false>
__device__ __forceinline__ void solve_one(const DeviceBatch& B, const Tolerances& tol, const int lp,
                                          unsigned char* small, unsigned char* big, int32_t* diag,
                                          unsigned char* stage = nullptr, size_t stage_bytes = 0)
{
    const int m = B.m[lp];
    const int n = B.n[lp];
    const int nm = n + m;
    const double* __restrict__ A = B.A + B.a_off[lp];
    const double* __restrict__ bv = B.b + B.b_off[lp];
    const double* __restrict__ cv = B.c + B.c_off[lp];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;

    // k-independent part of the layout (k = 0 gives the same offsets)
    const BigLayout L0 = big_layout(m, n, 0, kStreamed);
    // the group's reductions: block-wide through the scratch in `small`, or
    // (kWarp) `redux` within the one warp
    auto make_red = [&]() {
        if constexpr (kWarp) {
            return WarpGroup();
        } else {
            return Reducer{reinterpret_cast<long long*>(small + SmallLayout::red64),
                           reinterpret_cast<unsigned*>(small + SmallLayout::red32), nw, warp, lane};
        }
    };
    auto red = make_red();
    long long* rkey = reinterpret_cast<long long*>(big + L0.rkey);
    int* row_var = reinterpret_cast<int*>(big + L0.row_var);
    int* neg = reinterpret_cast<int*>(big + L0.neg);

    // ---- Tableau build (the host-side fill of Section 4.1, done here) -----
    // Rows with b_i < 0 are negated and get an artificial (two-phase method,
    // Section 3); they are ranked in ascending row order.
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
    group_sync<kWarp>();  // neg[] and row_var[] are read by other threads below

    const BigLayout L = big_layout(m, n, k, kStreamed);
    Tab tb;
    tb.T = reinterpret_cast<double*>(big + L.T);
    tb.colE = reinterpret_cast<double*>(big + L.colE);
    tb.col_var = reinterpret_cast<int*>(big + L.col_var);
    tb.row_var = row_var;
    tb.LD = L.LD;
    const int LD = L.LD;
    double* T = tb.T;  // the tableau is written through several pointers: no restrict
    int Cvar = n + k;  // live variable columns 1..Cvar
    Staging stg{nullptr, 0u};
    if (kStreamed && stage != nullptr) {
        if (tid == 0) *reinterpret_cast<int*>(stage) = 0;  // the flag word (read after the barriers below)
        if (stage_total(nw, L.R, L.LD) <= stage_bytes) {
            stg.base = stage;
            tb.colE = reinterpret_cast<double*>(stage + stage_colE(nw, L.LD));  // pivot column in shared memory
            if (lane == 0) {
                for (int q = 0; q < kStageDepth; ++q) mbar_init(&stage_bars(stage)[q], 1);
                mbar_init_fence();
            }
        }
    }
    const bool staged = kStreamed && stg.base != nullptr;
    // the barriers are invalidated before their memory can serve another LP
    // (unless a copy may still be in flight: the kernel then stops)
    auto release_staging = [&]() {
        if (staged && lane == 0 && *reinterpret_cast<volatile int*>(stage) != 2)
            for (int q = 0; q < kStageDepth; ++q) mbar_inval(&stage_bars(stage)[q]);
    };

    for (int j = tid; j <= Cvar; j += nt)
        tb.col_var[j] = (j == 0) ? -1 : (j <= n ? j - 1 : n + neg[j - 1 - n]);
    {
        // A into rows 0..m-1, columns 1..n: one flat pass with several
        // independent loads in flight per thread; then b and the slack columns
        const int64_t cnt = (int64_t)m * n;
        int i = tid / n, j = tid - i * n;
        const int di = nt / n, dj = nt - di * n;
        if (!kStreamed) {
            // shared-memory tableau: asynchronous copies, all in flight at once,
            // then the negated rows in place
            for (int64_t idx = tid; idx < cnt; idx += nt) {
                cp_async8(T + (size_t)i * LD + 1 + j, A + idx);
                i += di;
                j += dj;
                if (j >= n) { j -= n; ++i; }
            }
            cp_async_wait_all();
            group_sync<kWarp>();
            if (k > 0)
                for (int64_t idx = tid; idx < cnt; idx += nt) {
                    const int i2 = (int)(idx / n), j2 = (int)(idx - (int64_t)i2 * n);
                    if (row_var[i2] >= nm) T[(size_t)i2 * LD + 1 + j2] = -T[(size_t)i2 * LD + 1 + j2];
                }
        } else {
#pragma unroll 4
            for (int64_t idx = tid; idx < cnt; idx += nt) {
                const double v = A[idx];
                T[(size_t)i * LD + 1 + j] = (row_var[i] >= nm) ? -v : v;
                i += di;
                j += dj;
                if (j >= n) { j -= n; ++i; }
            }
        }
        for (int r = warp; r < m; r += nw) {
            const bool isneg = row_var[r] >= nm;
            double* Tr = T + (size_t)r * LD;
            for (int t = lane; t <= k; t += 32) {
                const int jj = (t == 0) ? 0 : n + t;
                const double v = (t == 0) ? bv[r] : ((neg[t - 1] == r) ? 1.0 : 0.0);
                Tr[jj] = isneg ? -v : v;
            }
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
        group_sync<kWarp>();
    }

    if (staged) fence_proxy_async_global();  // the build's stores before bulk reads of them
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
                group_sync<kWarp>();
                const int left = pivot<kStreamed, kWarp>(tb, m + 1, Cvar + 1, i, e, &stg);
                ++iters;
                if (staged && *reinterpret_cast<volatile int*>(stage)) { status = kNumerical; break; }
                if (left >= nm) retire_column<kWarp>(tb, m + 1, e, Cvar, staged);
            }
            phase = 2;
            continue;
        }
        // screen: columns whose key lies within the tie-window bound of dmin
        const unsigned long long win = step1_window(dmin, tol.key_window);
        unsigned ecnt = 0, esel = 0xffffffffu;
        for (int j = 1 + tid; j <= Cvar; j += nt) {
            const int v = tb.col_var[j];
            if (v < nm && (unsigned long long)okey(Trow[j]) - (unsigned long long)dmin <= win) {
                ++ecnt;
                esel = min(esel, ((unsigned)v << 16) | (unsigned)j);
            }
        }
        red.count_min(ecnt, esel, ecnt, esel);
        if (ecnt > 1) {
            // several candidates: the exact rule (lowest label within the window)
            const long long kthr = okey(tie_threshold(kval(dmin), tol.tau));
            unsigned sel = 0xffffffffu;
            for (int j = 1 + tid; j <= Cvar; j += nt) {
                const int v = tb.col_var[j];
                if (v < nm && okey(Trow[j]) <= kthr) sel = min(sel, ((unsigned)v << 16) | (unsigned)j);
            }
            esel = red.min_u32(sel);
        }
        const int e = (int)(esel & 0xffffu);

        // ---- Step 2: leaving row (minimum ratio rhs_i / t_ie, t_ie > eps) --
        // FP32 screen: rows with both operands in [2^-100, 2^100] (or rhs 0)
        // get a float ratio; the others are always candidates.  The operands
        // are truncated to FP32 by integer operations (< 2^-23 relative
        // each): a hardware conversion would take the FP64 pipe, which bounds
        // this kernel.  The window (far wider than the screen's error) is
        // set below.
        int floc = INT_MAX;
        for (int i = tid; i < Ract; i += nt) {
            const double t = T[(size_t)i * LD + e];
            tb.colE[i] = t;
            if (i < m) {
                long long code = LLONG_MAX;  // not eligible
                if (okey(t) > key_eps_piv) {
                    const double beta = T[(size_t)i * LD];
                    const int et = dexp(t), eb = dexp(beta);
                    const bool safe = et >= -100 && et <= 100 && (abskey(beta) == 0 || (eb >= -100 && eb <= 100));
                    if (safe) {
                        const int fk = fkey(__fdividef(f64_to_f32_trunc(beta), f64_to_f32_trunc(t)));
                        code = fk;
                        floc = min(floc, fk);
                    } else {
                        code = LLONG_MIN;  // unscreened: always a candidate
                    }
                }
                rkey[i] = code;
            }
        }
        const int fmin = red.min_i32(floc);
        long long fwin = LLONG_MIN;
        if (fmin != INT_MAX) {
            const float fm = fval(fmin);
            fwin = fkey(fm + __fmaf_rn(tol.ratio_rel, fabsf(fm), tol.ratio_abs));
        }
        unsigned lcnt = 0, lsel = 0xffffffffu;
        for (int i = tid; i < m; i += nt) {
            const long long code = rkey[i];
            if (code == LLONG_MIN || (code != LLONG_MAX && code <= fwin)) {
                ++lcnt;
                lsel = min(lsel, (unsigned)i);
            }
        }
        red.count_min(lcnt, lsel, lcnt, lsel);
        if (lcnt == 0) {
            status = (phase == 2) ? kUnbounded : kNumerical;
            break;
        }
        if (lcnt > 1) {
            // several candidates: exact ratios of the candidates, exact rule
            long long rloc = LLONG_MAX;
            for (int i = tid; i < m; i += nt) {
                const long long code = rkey[i];
                long long rk = LLONG_MAX;
                if (code == LLONG_MIN || (code != LLONG_MAX && code <= fwin))
                    rk = okey(__ddiv_rn(T[(size_t)i * LD], tb.colE[i]));
                rkey[i] = rk;
                rloc = min(rloc, rk);
            }
            const long long rmin = red.min_i64(rloc);
            const long long rthr = okey(tie_threshold(kval(rmin), tol.tau));
            unsigned sel = 0xffffffffu;
            for (int i = tid; i < m; i += nt)
                if (rkey[i] <= rthr) sel = min(sel, (unsigned)i);
            lsel = red.min_u32(sel);
        }
        const int l = (int)lsel;
        if (abskey(tb.colE[l]) >= 0x7FF0000000000000LL) { status = kNumerical; break; }
        if (iters >= max_iters) { status = kIterLimit; break; }

        // ---- Step 3: pivot ---------------------------------------------------
        const int left = pivot<kStreamed, kWarp>(tb, Ract, Cvar + 1, l, e, &stg);
        ++iters;
        if (staged && *reinterpret_cast<volatile int*>(stage)) {
            if (tid == 0) record_internal_error(diag, 8, lp, iters);  // a bulk copy did not complete
            status = kNumerical;
            break;
        }
        if (left >= nm) retire_column<kWarp>(tb, Ract, e, Cvar, staged);
    }

    // ---- labels must name variables (self-check before they index global
    // memory); a failure is recorded and the LP reported as LP_NUMERICAL ----
    {
        unsigned badl = 0, dummy;
        const unsigned nvar = (unsigned)(nm + k);
        for (int i = tid; i < m; i += nt) badl += ((unsigned)row_var[i] >= nvar) ? 1u : 0u;
        for (int j = 1 + tid; j <= Cvar; j += nt) badl += ((unsigned)tb.col_var[j] >= nvar) ? 1u : 0u;
        red.count_min(badl, 0u, badl, dummy);
        if (badl) {
            if (tid == 0) {
                record_internal_error(diag, 6, lp, (int)badl, status, iters, phase, Cvar);
                B.status[lp] = kNumerical;
                B.iters[lp] = iters;
            }
            release_staging();
            return;
        }
    }

    // ---- results: x (basic rows -> rhs, non-basic -> 0), y (slack reduced
    // costs of row `yrow`), objective corner, status, pivots -----------------
    double* __restrict__ x = B.x + B.x_off[lp];
    double* __restrict__ y = B.y ? B.y + B.y_off[lp] : nullptr;
    const double* Ty = T + (size_t)yrow * LD;
    for (int j = 1 + tid; j <= Cvar; j += nt) {
        const int v = tb.col_var[j];
        if ((unsigned)v < (unsigned)n) x[v] = 0.0;
        else if (v >= n && v < nm && y) y[v - n] = Ty[j];
    }
    for (int i = tid; i < m; i += nt) {
        const int v = row_var[i];
        if ((unsigned)v < (unsigned)n) x[v] = T[(size_t)i * LD];
        else if (v >= n && v < nm && y) y[v - n] = 0.0;
    }
    if (tid == 0) {
        B.status[lp] = status;
        B.iters[lp] = iters;
        B.obj[lp] = T[(size_t)m * LD];
    }
    release_staging();
}

__global__ void __launch_bounds__(kMaxThreads, 2)
fp64_resident_kernel(const DeviceBatch B, const Tolerances tol, const int32_t* __restrict__ order,
                     int32_t* __restrict__ diag)
{
    extern __shared__ __align__(16) unsigned char smem[];
    solve_one<false>(B, tol, order[blockIdx.x], smem, smem + SmallLayout::total, diag);
}

// One warp per LP (blockDim = 32), the form of the groups of small tableaux:
// the same per-LP code with warp barriers and `redux` reductions instead of
// block barriers and shared-memory round trips; the same arithmetic.
__global__ void __launch_bounds__(32, 32)
fp64_warp_kernel(const DeviceBatch B, const Tolerances tol, const int32_t* __restrict__ order,
                 int32_t* __restrict__ diag)
{
    extern __shared__ __align__(16) unsigned char smem[];
    solve_one<false, true>(B, tol, order[blockIdx.x], smem, smem + SmallLayout::total, diag);
}

// Resident kernel over a device-side list: persistent CTAs take the LPs
// queue[0 .. *queue_len) through the atomic `counter` (0 at launch).  Used for
// the LPs the mixed-precision kernel hands back.
__global__ void __launch_bounds__(kMaxThreads, 2)
fp64_resident_queue_kernel(const DeviceBatch B, const Tolerances tol, const int32_t* __restrict__ queue,
                           const int32_t* __restrict__ queue_len, const int32_t queue_cap, const int32_t num_lps,
                           int32_t* __restrict__ counter, int32_t* __restrict__ diag)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int next;
    const int count = min(*queue_len, queue_cap);
    for (;;) {
        if (threadIdx.x == 0) next = atomicAdd(counter, 1);
        __syncthreads();
        const int idx = next;
        __syncthreads();
        if (idx >= count) break;
        const int lp = queue[idx];
        if (lp < 0 || lp >= num_lps) {
            if (threadIdx.x == 0) record_internal_error(diag, 5, lp);
            continue;
        }
        solve_one<false>(B, tol, lp, smem, smem + SmallLayout::total, diag);
        __syncthreads();
    }
}


__global__ void __launch_bounds__(kStreamedThreads, 2)
fp64_streamed_kernel(const DeviceBatch B, const Tolerances tol, const int32_t* __restrict__ order,
                     const int32_t count, const int32_t* __restrict__ count_dev, unsigned char* workspace,
                     const size_t slot_bytes, int32_t* __restrict__ counter, int32_t* __restrict__ diag,
                     const size_t stage_bytes)
{
    __shared__ __align__(16) unsigned char small[SmallLayout::total];
    __shared__ int next;
    extern __shared__ __align__(128) unsigned char stage[];
    unsigned char* big = workspace + (size_t)blockIdx.x * slot_bytes;
    const int n_items = count_dev ? min(*count_dev, count) : count;
    for (;;) {
        if (threadIdx.x == 0) next = atomicAdd(counter, 1);
        __syncthreads();
        const int idx = next;
        __syncthreads();
        if (idx >= n_items) break;
        solve_one<true>(B, tol, order[idx], small, big, diag, stage_bytes ? stage : nullptr, stage_bytes);
        __syncthreads();
        // a bulk copy that may still be in flight into the rings: take no more LPs
        if (stage_bytes && *reinterpret_cast<volatile int*>(stage) == 2) break;
    }
}

// A whole batch in one launch: persistent CTAs take the LPs order[0 ..
// count) (longest work first) from the atomic `counter` and solve each with
// the tableau in this CTA's shared memory when it fits (resident[lp] != 0),
// else in this CTA's global workspace slot -- the same per-LP code as the
// resident and streamed kernels, so the same results.
__global__ void __launch_bounds__(kStreamedThreads, 2)
fp64_single_kernel(const DeviceBatch B, const Tolerances tol, const int32_t* __restrict__ order,
                   const uint8_t* __restrict__ resident, const int32_t count, unsigned char* workspace,
                   const size_t slot_bytes, int32_t* __restrict__ counter, int32_t* __restrict__ diag,
                   const size_t smem_bytes)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int next;
    unsigned char* slot = workspace ? workspace + (size_t)blockIdx.x * slot_bytes : nullptr;
    for (;;) {
        if (threadIdx.x == 0) next = atomicAdd(counter, 1);
        __syncthreads();
        const int idx = next;
        __syncthreads();
        if (idx >= count) break;
        const int lp = order[idx];
        if (resident[lp]) {
            solve_one<false>(B, tol, lp, smem, smem + SmallLayout::total, diag);
        } else if (slot) {
            // the CTA's shared memory beyond the reduction scratch stages the update
            unsigned char* stage = smem + SmallLayout::total;
            solve_one<true>(B, tol, lp, smem, slot, diag, stage, smem_bytes - SmallLayout::total);
            __syncthreads();
            if (*reinterpret_cast<volatile int*>(stage) == 2) break;  // a copy may still be in flight
        } else if (threadIdx.x == 0) {
            record_internal_error(diag, 7, lp);  // a plan without a slot for a streamed LP
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t fp64_kernels_prepare() {
    cudaError_t err = cudaFuncSetAttribute(fp64_resident_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)kMaxSmemPerBlock);
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(fp64_warp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmemPerBlock);
    if (err != cudaSuccess) return err;
    return cudaFuncSetAttribute(fp64_resident_queue_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(kMaxSmemPerBlock - 1024));
}

int fp64_resident_queue_ctas_per_sm(int threads, size_t smem) {
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fp64_resident_queue_kernel, threads, smem) != cudaSuccess)
        return 1;
    return blocks > 0 ? blocks : 1;
}

cudaError_t launch_fp64_resident_queue(const DeviceBatch& B, const Tolerances& tol, const int32_t* queue,
                                       const int32_t* queue_len, int32_t queue_cap, int32_t num_lps,
                                       int32_t* counter, int32_t* diag, int ctas, int threads,
                                       size_t smem, cudaStream_t stream) {
    cudaError_t err = cudaMemsetAsync(counter, 0, sizeof(int32_t), stream);
    if (err != cudaSuccess) return err;
    fp64_resident_queue_kernel<<<ctas, threads, smem, stream>>>(B, tol, queue, queue_len, queue_cap, num_lps,
                                                                counter, diag);
    return cudaGetLastError();
}

cudaError_t fp64_streamed_prepare() {
    return cudaFuncSetAttribute(fp64_streamed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kStreamStageBytes);
}

int fp64_streamed_ctas_per_sm() {
    int blocks = 0;
    if (fp64_streamed_prepare() != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fp64_streamed_kernel, kStreamedThreads,
                                                      kStreamStageBytes) != cudaSuccess)
        return 1;
    return blocks > 0 ? blocks : 1;
}

cudaError_t launch_fp64_streamed(const DeviceBatch& B, const Tolerances& tol, const int32_t* order,
                                 int32_t count, int slots, unsigned char* workspace, size_t slot_bytes,
                                 int32_t* counter, int32_t* diag, cudaStream_t stream, const int32_t* count_dev) {
    if (count <= 0) return cudaSuccess;
    cudaError_t err = cudaMemsetAsync(counter, 0, sizeof(int32_t), stream);
    if (err != cudaSuccess) return err;
    if ((err = fp64_streamed_prepare()) != cudaSuccess) return err;
    fp64_streamed_kernel<<<slots, kStreamedThreads, kStreamStageBytes, stream>>>(
        B, tol, order, count, count_dev, workspace, slot_bytes, counter, diag, kStreamStageBytes);
    return cudaGetLastError();
}

// fp64_single_kernel: the largest dynamic shared memory that still lets
// `per_sm` CTAs share an SM, and how many do at a given size.
cudaError_t fp64_single_prepare(size_t smem) {
    return cudaFuncSetAttribute(fp64_single_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

int fp64_single_ctas_per_sm(size_t smem) {
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fp64_single_kernel, kStreamedThreads, smem) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return blocks;
}

cudaError_t launch_fp64_single(const DeviceBatch& B, const Tolerances& tol, const int32_t* order,
                               const uint8_t* resident, int32_t count, int ctas, size_t smem,
                               unsigned char* workspace, size_t slot_bytes, int32_t* counter, int32_t* diag,
                               cudaStream_t stream) {
    if (count <= 0) return cudaSuccess;
    cudaError_t err = cudaMemsetAsync(counter, 0, sizeof(int32_t), stream);
    if (err != cudaSuccess) return err;
    fp64_single_kernel<<<ctas, kStreamedThreads, smem, stream>>>(B, tol, order, resident, count, workspace,
                                                                  slot_bytes, counter, diag, smem);
    return cudaGetLastError();
}

cudaError_t launch_fp64_resident(const DeviceBatch& B, const Tolerances& tol, const int32_t* order,
                                 int32_t count, int threads, size_t smem, int32_t* diag, cudaStream_t stream) {
    if (count <= 0) return cudaSuccess;
    if (threads == 32)
        fp64_warp_kernel<<<count, 32, smem, stream>>>(B, tol, order, diag);
    else
        fp64_resident_kernel<<<count, threads, smem, stream>>>(B, tol, order, diag);
    return cudaGetLastError();
}

}  // namespace lpb
