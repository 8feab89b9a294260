/*
 * simplex_oracle.c -- plain CPU FP64 reference of the dense two-phase simplex
 * method of "Simultaneous Solving of Batched Linear Programs on a GPU"
 * (Gurung & Ray, arXiv 1802.08557).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle the CUDA solver is checked
 * against.  Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark may load it; the solver itself never calls it and shares no code,
 * header or constant with it.
 *
 * What it computes (Section 3 of the paper):
 *   maximize  sum_j c_j x_j                         (Eq. 1)
 *   s.t.      sum_j a_ij x_j <= b_i,  i = 1..m      (Eq. 2)
 *             x_j >= 0,               j = 1..n      (Eq. 3)
 * by the tableau simplex method with Dantzig's entering rule (Step 1), the
 * minimum-ratio leaving rule (Step 2) and the pivot operation (Step 3,
 * NewPivotRow = OldPivotRow / PE, NewRow_ij = OldRow_ij - PivotCol_i *
 * NewPivotRow_j), starting from the slack basis (Eq. 4) and running the
 * two-phase method (auxiliary LP minimising the sum of artificials) when
 * some b_i < 0.
 *
 * Layout: the paper's full tableau of Section 3.1 -- one row per constraint
 * plus the objective row, one column per structural, slack and artificial
 * variable, plus the right-hand side; the index of each row's basic variable
 * is kept beside it (the paper's first auxiliary column).  A second objective
 * row carries the auxiliary (phase-I) objective while phase I runs.
 *
 * Readings of points the paper leaves open (the CUDA solver takes the same):
 *  - Sign convention: the objective row holds reduced costs d_j, initially
 *    -c_j; the most negative d_j enters; the ratio is beta_i / t_ie over rows
 *    with t_ie > eps_piv.  This is the paper's "maximum of the last row" and
 *    "b_i / -a_ie" with the row stored negated.
 *  - Optimal when every eligible d_j >= -eps_opt.
 *  - Ties: the minimum m* is found first; then the LOWEST variable index
 *    (entering) or LOWEST row index (leaving) whose value is <= m* +
 *    tau*max(1,|m*|) is taken.
 *  - Zero ratios are allowed (the paper's "minimum positive" would break
 *    degenerate pivots).
 *  - One artificial per row with b_i < 0 (that row is negated first); an
 *    artificial never (re-)enters the basis.
 *  - The original objective row is carried through phase I as an extra row,
 *    which performs the paper's "restore the objective by substitution"
 *    incrementally.
 *  - Phase-I row = 0 for non-artificials, 1 for artificials, minus each
 *    negated row in ascending row order.
 *  - Infeasible when the phase-I optimum w* > eps_feas*max(1, max_i |b_i|).
 *    Otherwise every artificial still basic is pivoted out on the lowest
 *    indexed non-artificial column with |t_ij| > eps_piv (such pivots count as
 *    iterations); if none exists the row is redundant and stays as it is.
 *  - Every pivot of both phases counts toward max_iters.
 *  - Arithmetic is IEEE binary64, round-to-nearest; the update uses fma();
 *    this file must be compiled with -ffp-contract=off so that no other
 *    expression is contracted.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "simplex_oracle.h"

typedef struct {
    int m, n, k;      /* constraints, structural variables, artificials */
    int nvar;         /* n + m + k variables */
    int ncol;         /* nvar + 1: last column is the right-hand side */
    int nrow;         /* m + 1, plus 1 while the phase-I row exists */
    double *t;        /* nrow x ncol, row-major */
    int *basis;       /* basic variable of each constraint row */
    char *is_basic;   /* per variable */
} tableau;

#define T(tb, i, j) ((tb)->t[(size_t)(i) * (size_t)(tb)->ncol + (size_t)(j)])

/* Tie window of Step 1 / Step 2: v* + tau * max(1, |v*|), evaluated as a
 * product followed by a sum (two roundings). */
static double tie_threshold(double vmin, double tau)
{
    double s = fabs(vmin);
    if (s < 1.0) s = 1.0;
    double w = tau * s;
    return vmin + w;
}

static int is_artificial(const tableau *tb, int var) { return var >= tb->n + tb->m; }

/* Step 1 (Section 3.1): entering variable from objective row `orow`.
 * Returns -1 when no eligible reduced cost is below -eps_opt. */
static int pick_entering(const tableau *tb, int orow, const oracle_opts *o)
{
    int found = 0;
    double dmin = 0.0;
    for (int j = 0; j < tb->nvar; ++j) {
        if (tb->is_basic[j] || is_artificial(tb, j)) continue;
        double d = T(tb, orow, j);
        if (!found || d < dmin) { dmin = d; found = 1; }
    }
    if (!found || !(dmin < -o->eps_opt)) return -1;
    double thr = tie_threshold(dmin, o->tau);
    for (int j = 0; j < tb->nvar; ++j) {
        if (tb->is_basic[j] || is_artificial(tb, j)) continue;
        if (T(tb, orow, j) <= thr) return j;
    }
    return -1; /* unreachable: dmin itself satisfies the test */
}

/* Step 2 (Section 3.1): leaving row for entering column e.
 * Returns -1 when no row has t_ie > eps_piv (unbounded direction). */
static int pick_leaving(const tableau *tb, int e, const oracle_opts *o)
{
    const int rhs = tb->ncol - 1;
    int found = 0;
    double rmin = 0.0;
    for (int i = 0; i < tb->m; ++i) {
        double a = T(tb, i, e);
        if (!(a > o->eps_piv)) continue;
        double r = T(tb, i, rhs) / a;
        if (!found || r < rmin) { rmin = r; found = 1; }
    }
    if (!found) return -1;
    double thr = tie_threshold(rmin, o->tau);
    for (int i = 0; i < tb->m; ++i) {
        double a = T(tb, i, e);
        if (!(a > o->eps_piv)) continue;
        double r = T(tb, i, rhs) / a;
        if (r <= thr) return i;
    }
    return -1; /* unreachable */
}

/* Step 3 (Section 3.1 and Listing 1): pivot on (l, e) over the first
 * `nrow_active` rows.  The pivot row is divided by the pivot element, then
 * every other row i gets t_ij <- t_ij - t_ie * r_j (one fused multiply-add). */
static void pivot(tableau *tb, int l, int e, int nrow_active)
{
    const double pe = T(tb, l, e);
    for (int j = 0; j < tb->ncol; ++j) T(tb, l, j) = T(tb, l, j) / pe;
    for (int i = 0; i < nrow_active; ++i) {
        if (i == l) continue;
        const double f = T(tb, i, e);
        for (int j = 0; j < tb->ncol; ++j)
            T(tb, i, j) = fma(-f, T(tb, l, j), T(tb, i, j));
    }
    tb->is_basic[tb->basis[l]] = 0;
    tb->basis[l] = e;
    tb->is_basic[e] = 1;
}

/* Build the tableau of Section 3.1 from (A, b, c): slack basis (Eq. 4);
 * rows with b_i < 0 negated and given an artificial (two-phase method). */
static int build(tableau *tb, int m, int n, const double *A, const double *b, const double *c)
{
    int k = 0;
    for (int i = 0; i < m; ++i) if (b[i] < 0.0) ++k;
    tb->m = m; tb->n = n; tb->k = k;
    tb->nvar = n + m + k;
    tb->ncol = tb->nvar + 1;
    tb->nrow = m + 1 + (k > 0 ? 1 : 0);
    tb->t = (double *)calloc((size_t)tb->nrow * (size_t)tb->ncol, sizeof(double));
    tb->basis = (int *)malloc(sizeof(int) * (size_t)(m > 0 ? m : 1));
    tb->is_basic = (char *)calloc((size_t)tb->nvar + 1, 1);
    if (!tb->t || !tb->basis || !tb->is_basic) return -1;
    const int rhs = tb->ncol - 1;
    int a = 0;
    for (int i = 0; i < m; ++i) {
        for (int j = 0; j < n; ++j) T(tb, i, j) = A[(size_t)i * (size_t)n + (size_t)j];
        T(tb, i, n + i) = 1.0;
        T(tb, i, rhs) = b[i];
        if (b[i] < 0.0) {
            for (int j = 0; j < tb->ncol; ++j) T(tb, i, j) = -T(tb, i, j);
            int av = n + m + a;
            T(tb, i, av) = 1.0;
            tb->basis[i] = av;
            ++a;
        } else {
            tb->basis[i] = n + i;
        }
        tb->is_basic[tb->basis[i]] = 1;
    }
    /* objective row: reduced costs -c_j of the slack basis, value 0 */
    for (int j = 0; j < n; ++j) T(tb, m, j) = -c[j];
    if (k > 0) {
        /* auxiliary objective: maximise -(sum of artificials); price out the
         * basic artificials by subtracting each negated row in ascending order */
        const int w = m + 1;
        for (int j = 0; j < tb->ncol; ++j) T(tb, w, j) = is_artificial(tb, j) && j < tb->nvar ? 1.0 : 0.0;
        for (int i = 0; i < m; ++i) {
            if (!is_artificial(tb, tb->basis[i])) continue;
            for (int j = 0; j < tb->ncol; ++j) T(tb, w, j) = T(tb, w, j) - T(tb, i, j);
        }
    }
    return 0;
}

static void release(tableau *tb)
{
    free(tb->t); free(tb->basis); free(tb->is_basic);
}

/* Simplex loop of Section 3.1 (Steps 1-3 until the halt condition) on
 * objective row `orow`, updating the first `nrow_active` rows. */
static int run_phase(tableau *tb, int orow, int nrow_active, const oracle_opts *o,
                     int max_iters, int *iters, int *entering_out)
{
    for (;;) {
        int e = pick_entering(tb, orow, o);
        if (e < 0) return OR_OPTIMAL;
        int l = pick_leaving(tb, e, o);
        if (l < 0) { *entering_out = e; return OR_UNBOUNDED; }
        if (!isfinite(T(tb, l, e))) return OR_NUMERICAL;
        if (*iters >= max_iters) return OR_ITER_LIMIT;
        pivot(tb, l, e, nrow_active);
        ++*iters;
    }
}

int oracle_solve(int32_t m, int32_t n, const double *A, const double *b, const double *c,
                 const oracle_opts *opts, oracle_result *res, double *x, double *y, double *cert)
{
    oracle_opts o;
    oracle_default_opts(&o);
    if (opts) o = *opts;
    if (m < 1 || n < 1 || !A || !b || !c || !res || !x) return -1;
    const int max_iters = o.max_iters > 0 ? o.max_iters : 50 * (m + n);

    tableau tb;
    memset(&tb, 0, sizeof tb);
    if (build(&tb, m, n, A, b, c) != 0) { release(&tb); return -2; }
    const int rhs = tb.ncol - 1;

    int iters = 0, entering = -1, status;
    int p1_iters = 0;
    int yrow = m;  /* row whose slack entries are reported as y */
    if (tb.k > 0) {
        status = run_phase(&tb, m + 1, m + 2, &o, max_iters, &iters, &entering);
        p1_iters = iters;
        if (status == OR_UNBOUNDED) status = OR_NUMERICAL; /* phase I is bounded by 0 */
        if (status == OR_OPTIMAL) {
            double bmax = 1.0;
            for (int i = 0; i < m; ++i) if (fabs(b[i]) > bmax) bmax = fabs(b[i]);
            double wstar = -T(&tb, m + 1, rhs);
            if (wstar > o.eps_feas * bmax) {
                status = OR_INFEASIBLE;
                yrow = m + 1;
            } else {
                /* drive zero-level artificials out of the basis */
                for (int i = 0; i < m && status == OR_OPTIMAL; ++i) {
                    if (!is_artificial(&tb, tb.basis[i])) continue;
                    int jsel = -1;
                    for (int j = 0; j < n + m; ++j) {
                        if (tb.is_basic[j]) continue;
                        if (fabs(T(&tb, i, j)) > o.eps_piv) { jsel = j; break; }
                    }
                    if (jsel < 0) continue; /* redundant row */
                    if (iters >= max_iters) { status = OR_ITER_LIMIT; break; }
                    pivot(&tb, i, jsel, m + 1);
                    ++iters;
                }
                p1_iters = iters;
                if (status == OR_OPTIMAL) /* the phase-I row is no longer updated */
                    status = run_phase(&tb, m, m + 1, &o, max_iters, &iters, &entering);
            }
        }
    } else {
        status = run_phase(&tb, m, m + 1, &o, max_iters, &iters, &entering);
    }

    /* extraction */
    for (int j = 0; j < n; ++j) x[j] = 0.0;
    for (int i = 0; i < m; ++i) if (tb.basis[i] < n) x[tb.basis[i]] = T(&tb, i, rhs);
    if (y) for (int i = 0; i < m; ++i) y[i] = T(&tb, yrow, n + i);
    res->status = status;
    res->iters = iters;
    res->phase1_iters = p1_iters;
    res->obj = T(&tb, m, rhs);
    res->phase1_obj = tb.k > 0 ? T(&tb, m + 1, rhs) : 0.0;
    res->num_artificial = tb.k;
    res->entering = entering;
    if (cert) {
        /* unbounded ray: d_e = 1, basic structurals move by -t_ie */
        for (int j = 0; j < n; ++j) cert[j] = 0.0;
        if (status == OR_UNBOUNDED && entering >= 0) {
            if (entering < n) cert[entering] = 1.0;
            for (int i = 0; i < m; ++i)
                if (tb.basis[i] < n) cert[tb.basis[i]] = -T(&tb, i, entering);
        }
    }
    release(&tb);
    return 0;
}

void oracle_default_opts(oracle_opts *o)
{
    o->eps_opt = 1e-9;
    o->eps_piv = 1e-9;
    o->eps_feas = 1e-9;
    o->tau = 1e-12;
    o->max_iters = 0;
}

int oracle_solve_batch(int32_t num_lps, const int32_t *m, const int32_t *n,
                       const int64_t *a_off, const double *A,
                       const int64_t *b_off, const double *b,
                       const int64_t *c_off, const double *c,
                       const int64_t *x_off, const int64_t *y_off,
                       const oracle_opts *opts,
                       int32_t *status, int32_t *iters, double *obj, double *x, double *y)
{
    for (int32_t k = 0; k < num_lps; ++k) {
        oracle_result r;
        int rc = oracle_solve(m[k], n[k], A + a_off[k], b + b_off[k], c + c_off[k], opts, &r,
                              x + x_off[k], y ? y + y_off[k] : NULL, NULL);
        if (rc != 0) return rc;
        status[k] = r.status;
        iters[k] = r.iters;
        obj[k] = r.obj;
    }
    return 0;
}
