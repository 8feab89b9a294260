/*
 * simplex_oracle.h -- interface of the CPU FP64 reference simplex (test
 * infrastructure only; see simplex_oracle.c).  The CUDA solver does not
 * include this header.
 */
#ifndef SIMPLEX_ORACLE_H
#define SIMPLEX_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Per-LP outcome codes. */
enum { OR_OPTIMAL = 0, OR_INFEASIBLE = 1, OR_UNBOUNDED = 2, OR_ITER_LIMIT = 3, OR_NUMERICAL = 4 };

typedef struct {
    double eps_opt;   /* optimal when every eligible reduced cost >= -eps_opt */
    double eps_piv;   /* a row takes part in the ratio test when t_ie > eps_piv */
    double eps_feas;  /* infeasible when phase-I optimum > eps_feas*max(1,|b|_inf) */
    double tau;       /* relative tie window of both argmins */
    int32_t max_iters;/* <= 0: 50*(m+n) */
} oracle_opts;

typedef struct {
    int32_t status;
    int32_t iters;          /* all pivots, both phases */
    int32_t phase1_iters;   /* pivots of phase I, drive-out included */
    int32_t num_artificial; /* rows with b_i < 0 */
    int32_t entering;       /* entering variable at unbounded detection, else -1 */
    double obj;             /* objective-row corner of the final tableau */
    double phase1_obj;      /* phase-I row corner (-(sum of artificials)) */
} oracle_result;

void oracle_default_opts(oracle_opts *o);

/* Solve one LP: A is m x n row-major, b has m, c has n entries.
 * x (n entries) receives the final basic solution; y (m entries, may be NULL)
 * the reduced costs of the slack variables (LP duals; Farkas multipliers when
 * infeasible); cert (n entries, may be NULL) the unbounded ray.
 * Returns 0, or a negative value for bad arguments / out of memory. */
int oracle_solve(int32_t m, int32_t n, const double *A, const double *b, const double *c,
                 const oracle_opts *opts, oracle_result *res, double *x, double *y, double *cert);

/* Loop of oracle_solve over a batch laid out by element offsets. */
int oracle_solve_batch(int32_t num_lps, const int32_t *m, const int32_t *n,
                       const int64_t *a_off, const double *A,
                       const int64_t *b_off, const double *b,
                       const int64_t *c_off, const double *c,
                       const int64_t *x_off, const int64_t *y_off,
                       const oracle_opts *opts,
                       int32_t *status, int32_t *iters, double *obj, double *x, double *y);

#ifdef __cplusplus
}
#endif
#endif
