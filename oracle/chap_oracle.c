/*
 * chap_oracle.c -- plain CPU oracle for the best-shift tabu search of
 * "CHAP: A Hybrid GPU-CPU Heuristic for MIP", Sec. 3.1.
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the CPU-baseline leg
 * of the benchmark are the only callers.  This file shares no code, header,
 * table or helper with the CUDA library; it is deliberately slow and literal.
 *
 * What it computes (all arithmetic in IEEE double, no fused multiply-add):
 *
 *  - Row normalisation (Sec. 3.1, "Memory Considerations", second point): every
 *    original row becomes one or two "<=" rows in a canonical order: a "<=" row
 *    stays (a, b); a ">=" row becomes (-a, -b); an "=" row becomes (a, b)
 *    followed by (-a, -b).  Weights, residuals and violation counts live on
 *    these normalised rows.
 *
 *  - Violation: a normalised row is violated when r = ybar - b > eps.  eps is 0
 *    on integral rows (integer coefficients, integer rhs, only integer or
 *    binary variables with finite bounds, magnitudes below 2^52) and
 *    feas_tol * max(1, |b|) otherwise.  The paper states no tolerance; this is
 *    the reading used on both sides.
 *
 *  - Penalty p_ij and score s_j (Sec. 3.1, "Scoring Functions"): for a move of
 *    x_j from xbar_j to c, with ybar_i and y_ij recomputed from scratch,
 *        sat -> viol: -w,  viol -> sat: +w,
 *        viol -> viol and y < ybar: +w/2,  viol -> viol and y > ybar: -w/2,
 *        otherwise 0.
 *    Scores are returned in half-weight units (an int64 "s_half" = 2 s).
 *
 *  - Best shift (Eq. best_move) over the candidate set of Sec. 3.1: the finite
 *    bounds l_j, u_j and every breakpoint lying in [l_j, u_j].  For a continuous
 *    variable the breakpoint is t_ij = (b_i - sum_{k!=j} a_ik xbar_k) / a_ij;
 *    a row that is satisfied with |r| <= eps is "tight" and its breakpoint is
 *    xbar_j itself, which is never a candidate.  For an integer variable it is
 *    the same quotient with b_i replaced by b_i + eps, rounded down when
 *    a_ij > 0 and up when a_ij < 0 (Algorithm 1, breakpoint step): the last
 *    integer at which the row is still satisfied within the tolerance (eps = 0
 *    on integral rows gives the paper's formula unchanged).  Binary variables
 *    have the single flip candidate 1 - xbar_j (Sec. 3.1, "Best Shift Moves").
 *
 *  - Tabu and aspiration (the framework the paper builds on; its rules are not
 *    restated there, the reading used here is): after a move at iteration k
 *    that increases x_j, decreases of x_j are tabu while iter < k + 1 + tenure,
 *    and symmetrically.  A tabu candidate is still admissible when
 *    nviol + dnviol < best_nviol (aspiration).
 *
 *  - Per variable: the admissible candidate with the largest score, ties broken
 *    by the smallest |c - xbar_j| and then the smaller c.  If that score is not
 *    positive, the answer is the incumbent with score 0.  Over all variables:
 *    the largest score, ties broken by the lowest variable index.
 *
 *  - One tabu iteration: apply the selected move; when no variable has a
 *    positive admissible score, add 1 to the weight of every violated
 *    normalised row instead.  Either way the iteration counter advances.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#pragma STDC FP_CONTRACT OFF

#define ORC_BIN 0
#define ORC_INT 1
#define ORC_CONT 2
#define ORC_LE 0
#define ORC_GE 1
#define ORC_EQ 2

typedef struct {
    int32_t n, m;       /* original sizes */
    int32_t mn;         /* number of normalised rows */
    const int64_t *row_ptr;
    const int32_t *col_idx;
    const double *row_val;
    const int64_t *col_ptr;
    const int32_t *row_idx;
    const double *lb, *ub;
    const uint8_t *vtype;
    /* normalised rows */
    int32_t *nr_orig;   /* original row of normalised row k */
    double *nr_sign;    /* +1 or -1 */
    double *nr_rhs;     /* sign * b */
    double *nr_eps;     /* 0 on integral rows */
    int32_t *first_nr;  /* first normalised row of original row i */
    int32_t *num_nr;    /* 1 or 2 */
    uint8_t *row_int;   /* original row i is integral (eps = 0) */
    double feas_tol;
} orc_t;

static int is_integer_value(double v) { return isfinite(v) && floor(v) == v; }

void orc_destroy(orc_t *h)
{
    if (!h) return;
    free(h->nr_orig);
    free(h->nr_sign);
    free(h->nr_rhs);
    free(h->nr_eps);
    free(h->first_nr);
    free(h->num_nr);
    free(h->row_int);
    free(h);
}

/* The arrays passed here must stay alive for the lifetime of the handle. */
orc_t *orc_create(int32_t n, int32_t m,
                  const int64_t *row_ptr, const int32_t *col_idx, const double *row_val,
                  const int64_t *col_ptr, const int32_t *row_idx,
                  const double *lb, const double *ub, const double *rhs,
                  const uint8_t *vtype, const uint8_t *sense, double feas_tol)
{
    orc_t *h = (orc_t *)calloc(1, sizeof(orc_t));
    if (!h) return NULL;
    h->n = n; h->m = m;
    h->row_ptr = row_ptr; h->col_idx = col_idx; h->row_val = row_val;
    h->col_ptr = col_ptr; h->row_idx = row_idx;
    h->lb = lb; h->ub = ub; h->vtype = vtype;
    int32_t mn = 0;
    for (int32_t i = 0; i < m; ++i) mn += (sense[i] == ORC_EQ) ? 2 : 1;
    h->mn = mn;
    h->nr_orig = (int32_t *)malloc(sizeof(int32_t) * (size_t)(mn > 0 ? mn : 1));
    h->nr_sign = (double *)malloc(sizeof(double) * (size_t)(mn > 0 ? mn : 1));
    h->nr_rhs = (double *)malloc(sizeof(double) * (size_t)(mn > 0 ? mn : 1));
    h->nr_eps = (double *)malloc(sizeof(double) * (size_t)(mn > 0 ? mn : 1));
    h->first_nr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    h->num_nr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    h->row_int = (uint8_t *)malloc((size_t)(m > 0 ? m : 1));
    h->feas_tol = feas_tol;
    if (!h->nr_orig || !h->nr_sign || !h->nr_rhs || !h->nr_eps || !h->first_nr || !h->num_nr || !h->row_int) {
        orc_destroy(h);
        return NULL;
    }
    const double lim = 4503599627370496.0; /* 2^52 */
    int32_t k = 0;
    for (int32_t i = 0; i < m; ++i) {
        /* integral row test */
        int integral = is_integer_value(rhs[i]) && fabs(rhs[i]) <= lim;
        double mag = fabs(rhs[i]);
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1] && integral; ++e) {
            double a = row_val[e];
            int32_t j = col_idx[e];
            if (!is_integer_value(a) || fabs(a) > 2147483647.0) integral = 0;
            else if (vtype[j] == ORC_CONT) integral = 0;
            else if (!isfinite(lb[j]) || !isfinite(ub[j])) integral = 0;
            else {
                double bnd = fabs(lb[j]) > fabs(ub[j]) ? fabs(lb[j]) : fabs(ub[j]);
                mag += fabs(a) * bnd;
                if (!(mag <= lim)) integral = 0;
            }
        }
        h->first_nr[i] = k;
        h->row_int[i] = (uint8_t)integral;
        double eps = integral ? 0.0 : feas_tol * (fabs(rhs[i]) > 1.0 ? fabs(rhs[i]) : 1.0);
        if (sense[i] == ORC_LE || sense[i] == ORC_EQ) {
            h->nr_orig[k] = i; h->nr_sign[k] = 1.0; h->nr_rhs[k] = rhs[i]; h->nr_eps[k] = eps; ++k;
        }
        if (sense[i] == ORC_GE || sense[i] == ORC_EQ) {
            h->nr_orig[k] = i; h->nr_sign[k] = -1.0; h->nr_rhs[k] = -rhs[i]; h->nr_eps[k] = eps; ++k;
        }
        h->num_nr[i] = k - h->first_nr[i];
    }
    return h;
}

int32_t orc_num_norm_rows(const orc_t *h) { return h->mn; }

/* Integral flag of every normalised row (1 when eps == 0 by the integral-row rule). */
void orc_norm_row_info(const orc_t *h, int32_t *orig, double *sign, double *rhs, double *eps)
{
    for (int32_t k = 0; k < h->mn; ++k) {
        if (orig) orig[k] = h->nr_orig[k];
        if (sign) sign[k] = h->nr_sign[k];
        if (rhs) rhs[k] = h->nr_rhs[k];
        if (eps) eps[k] = h->nr_eps[k];
    }
}

/* ybar_k = sum over the row of (sign * a) * x, in CSR order. */
static double activity(const orc_t *h, int32_t k, const double *x)
{
    int32_t i = h->nr_orig[k];
    double s = h->nr_sign[k];
    double y = 0.0;
    for (int64_t e = h->row_ptr[i]; e < h->row_ptr[i + 1]; ++e) {
        double a = s * h->row_val[e];
        double t = a * x[h->col_idx[e]];
        y = y + t;
    }
    return y;
}

/* sum_{k != j} (sign * a_k) * x_k in CSR order, and the coefficient of j. */
static double activity_without(const orc_t *h, int32_t k, const double *x, int32_t j, double *a_j)
{
    int32_t i = h->nr_orig[k];
    double s = h->nr_sign[k];
    double y = 0.0;
    *a_j = 0.0;
    for (int64_t e = h->row_ptr[i]; e < h->row_ptr[i + 1]; ++e) {
        double a = s * h->row_val[e];
        if (h->col_idx[e] == j) { *a_j = a; continue; }
        double t = a * x[h->col_idx[e]];
        y = y + t;
    }
    return y;
}

/* Residual r_k = ybar_k - b_k of every normalised row; returns the number violated. */
int64_t orc_residuals(const orc_t *h, const double *x, double *r, uint8_t *viol)
{
    int64_t nv = 0;
    for (int32_t k = 0; k < h->mn; ++k) {
        double rk = activity(h, k, x) - h->nr_rhs[k];
        int v = rk > h->nr_eps[k];
        if (r) r[k] = rk;
        if (viol) viol[k] = (uint8_t)v;
        nv += v;
    }
    return nv;
}

/* Score (half units) and violation-count change of moving x_j from xbar_j to c,
 * every activity recomputed from scratch (Sec. 3.1, Scoring Functions). */
static void score_of(const orc_t *h, int32_t j, double c, const double *x, const int32_t *w,
                     int64_t *s_half, int32_t *dnviol)
{
    int64_t s = 0;
    int32_t dc = 0;
    for (int64_t e = h->col_ptr[j]; e < h->col_ptr[j + 1]; ++e) {
        int32_t i = h->row_idx[e];
        for (int32_t q = 0; q < h->num_nr[i]; ++q) {
            int32_t k = h->first_nr[i] + q;
            double a_j;
            double ybar = activity(h, k, x);
            double y = activity_without(h, k, x, j, &a_j);
            double ac = a_j * c;
            y = y + ac;
            double r0 = ybar - h->nr_rhs[k];
            double r1 = y - h->nr_rhs[k];
            int v0 = r0 > h->nr_eps[k];
            int v1 = r1 > h->nr_eps[k];
            int64_t wk = w[k];
            if (!v0 && v1) s -= 2 * wk;
            else if (v0 && !v1) s += 2 * wk;
            else if (v0 && v1 && y < ybar) s += wk;
            else if (v0 && v1 && y > ybar) s -= wk;
            dc += v1 - v0;
        }
    }
    *s_half = s;
    *dnviol = dc;
}

typedef struct {
    int have;
    double c;
    int64_t s;
    int32_t dc;
} best_t;

static void consider(best_t *b, double xbar, double c, int64_t s, int32_t dc)
{
    if (!b->have) { b->have = 1; b->c = c; b->s = s; b->dc = dc; return; }
    if (s > b->s) { b->c = c; b->s = s; b->dc = dc; return; }
    if (s < b->s) return;
    double d_new = fabs(c - xbar), d_old = fabs(b->c - xbar);
    if (d_new < d_old || (d_new == d_old && c < b->c)) { b->c = c; b->s = s; b->dc = dc; }
}

static void eval_candidate(const orc_t *h, int32_t j, double c, const double *x, const int32_t *w,
                           const int64_t *tabu_inc, const int64_t *tabu_dec, int64_t iter,
                           int64_t nviol, int64_t best_nviol, best_t *best)
{
    double xbar = x[j];
    if (c == xbar) return;
    if (c < h->lb[j] || c > h->ub[j]) return;
    int64_t s;
    int32_t dc;
    score_of(h, j, c, x, w, &s, &dc);
    int tabu = (c > xbar) ? (iter < tabu_inc[j]) : (iter < tabu_dec[j]);
    int admissible = !tabu || (nviol + (int64_t)dc < best_nviol);
    if (admissible) consider(best, xbar, c, s, dc);
}

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* Best shift of one variable (Eq. best_move on the candidate set above): the
 * candidate values are collected, sorted and deduplicated, then each distinct
 * value is scored from scratch. */
static void best_shift_var(const orc_t *h, int32_t j, const double *x, const int32_t *w,
                           const int64_t *tabu_inc, const int64_t *tabu_dec, int64_t iter,
                           int64_t nviol, int64_t best_nviol,
                           double *xhat, int64_t *s_half, int32_t *dnviol)
{
    best_t best = {0, 0.0, 0, 0};
    double xbar = x[j];
    if (h->vtype[j] == ORC_BIN) {
        eval_candidate(h, j, 1.0 - xbar, x, w, tabu_inc, tabu_dec, iter, nviol, best_nviol, &best);
    } else {
        int64_t len = h->col_ptr[j + 1] - h->col_ptr[j];
        double *cand = (double *)malloc(sizeof(double) * (size_t)(4 * len + 2));
        int64_t nc = 0;
        if (cand) {
            if (isfinite(h->lb[j])) cand[nc++] = h->lb[j];
            if (isfinite(h->ub[j])) cand[nc++] = h->ub[j];
            for (int64_t e = h->col_ptr[j]; e < h->col_ptr[j + 1]; ++e) {
                int32_t i = h->row_idx[e];
                for (int32_t q = 0; q < h->num_nr[i]; ++q) {
                    int32_t k = h->first_nr[i] + q;
                    double a_j;
                    double rest = activity_without(h, k, x, j, &a_j);
                    double t;
                    if (h->vtype[j] == ORC_INT) {
                        double bt = h->nr_rhs[k] + h->nr_eps[k];
                        t = (bt - rest) / a_j;
                        t = (a_j > 0.0) ? floor(t) : ceil(t);
                    } else {
                        double r = activity(h, k, x) - h->nr_rhs[k];
                        int viol = r > h->nr_eps[k];
                        if (!viol && fabs(r) <= h->nr_eps[k]) continue; /* tight: breakpoint is xbar */
                        t = (h->nr_rhs[k] - rest) / a_j;
                    }
                    cand[nc++] = t + 0.0;
                }
            }
            qsort(cand, (size_t)nc, sizeof(double), cmp_double);
            for (int64_t q = 0; q < nc; ++q) {
                if (q > 0 && cand[q] == cand[q - 1]) continue;
                eval_candidate(h, j, cand[q], x, w, tabu_inc, tabu_dec, iter, nviol, best_nviol, &best);
            }
            free(cand);
        }
    }
    if (best.have && best.s > 0) {
        *xhat = best.c; *s_half = best.s; *dnviol = best.dc;
    } else {
        *xhat = xbar; *s_half = 0; *dnviol = 0;
    }
}

/* Best shift of the variables vars[0..nv) (all variables when vars == NULL). */
void orc_best_shift(const orc_t *h, const double *x, const int32_t *w,
                    const int64_t *tabu_inc, const int64_t *tabu_dec, int64_t iter,
                    int64_t nviol, int64_t best_nviol,
                    const int32_t *vars, int32_t nv,
                    double *xhat, int64_t *s_half, int32_t *dnviol, int32_t nthreads)
{
    int32_t count = vars ? nv : h->n;
#ifdef _OPENMP
    /* the thread count applies to this call only */
    const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
#endif
    for (int32_t q = 0; q < count; ++q) {
        int32_t j = vars ? vars[q] : q;
        best_shift_var(h, j, x, w, tabu_inc, tabu_dec, iter, nviol, best_nviol,
                       &xhat[q], &s_half[q], &dnviol[q]);
    }
    (void)nthreads;
}

/* Number of threads OpenMP would use for the calls above. */
int32_t orc_max_threads(void)
{
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Run n_iters tabu iterations from the given state (updated in place).
 * Per iteration k, move_var[k] gets the moved variable (-1 for a weight
 * update), move_val[k] its new value, move_s[k] the score in half units and
 * nviol_after[k] the violation count afterwards.  Stops early once nviol == 0
 * when stop_at_feasible is set; returns the number of iterations done.
 */
/*
 * Objective cutoff (Sec. 3.2: the best known objective is imposed as a cutoff
 * constraint so that the search looks for improving solutions).  Original row
 * `row`, given as "<=", holds the objective; y = its activity at x.  When an
 * iteration ends with no violated normalised row, x is a solution: y becomes
 * the best objective, x is copied to x_best and the row's rhs becomes y - d,
 * d = delta on an integral row and max(delta, 4 feas_tol max(1, |y|))
 * otherwise (so that the tightened row is violated beyond its tolerance), with
 * eps recomputed from the new rhs.  The violation record best_nviol restarts
 * from the count of the tightened problem (a reading: the paper does not say).
 */
typedef struct {
    int32_t row;
    double delta;
    double obj;        /* best objective found (out) */
    int64_t count;     /* solutions recorded (in/out) */
    int64_t best_iter; /* iteration at whose end the best one was recorded (in/out) */
    double *x_best;    /* [n] (out) */
} orc_cut_t;

static void tighten(orc_t *h, orc_cut_t *cut, const double *x, int64_t it)
{
    int32_t k = h->first_nr[cut->row];
    double y = activity(h, k, x);
    double d = cut->delta;
    double eps = 0.0;
    if (!h->row_int[cut->row]) {
        double dmin = 4.0 * h->feas_tol * (fabs(y) > 1.0 ? fabs(y) : 1.0);
        if (d < dmin) d = dmin;
    }
    double b = y - d;
    if (!h->row_int[cut->row]) eps = h->feas_tol * (fabs(b) > 1.0 ? fabs(b) : 1.0);
    h->nr_rhs[k] = b;
    h->nr_eps[k] = eps;
    cut->obj = y;
    cut->count += 1;
    cut->best_iter = it;
    memcpy(cut->x_best, x, sizeof(double) * (size_t)h->n);
}

static int64_t run_loop(orc_t *h, double *x, int32_t *w, int64_t *tabu_inc, int64_t *tabu_dec,
                        int64_t *iter, int64_t *best_nviol, int32_t tenure, int64_t n_iters,
                        int32_t stop_at_feasible, orc_cut_t *cut, int32_t *move_var, double *move_val,
                        int64_t *move_s, int64_t *nviol_after, int32_t nthreads);

int64_t orc_run(const orc_t *h, double *x, int32_t *w, int64_t *tabu_inc, int64_t *tabu_dec,
                int64_t *iter, int64_t *best_nviol, int32_t tenure, int64_t n_iters,
                int32_t stop_at_feasible, int32_t *move_var, double *move_val, int64_t *move_s,
                int64_t *nviol_after, int32_t nthreads)
{
    /* without a cutoff the handle is only read */
    return run_loop((orc_t *)h, x, w, tabu_inc, tabu_dec, iter, best_nviol, tenure, n_iters,
                    stop_at_feasible, NULL, move_var, move_val, move_s, nviol_after, nthreads);
}

/*
 * orc_run under the objective cutoff on original row cut_row (a "<=" row):
 * never stops at feasibility; cut_obj, cut_count, cut_iter and x_best[n] are
 * updated at every recorded solution (cut_count and cut_iter carry over from
 * the caller).  The row's rhs stays tightened in the handle afterwards
 * (read it with orc_norm_row_info).
 */
int64_t orc_run_cutoff(orc_t *h, double *x, int32_t *w, int64_t *tabu_inc, int64_t *tabu_dec,
                       int64_t *iter, int64_t *best_nviol, int32_t tenure, int64_t n_iters,
                       int32_t cut_row, double cut_delta, double *cut_obj, int64_t *cut_count,
                       int64_t *cut_iter, double *x_best, int32_t *move_var, double *move_val,
                       int64_t *move_s, int64_t *nviol_after, int32_t nthreads)
{
    orc_cut_t cut = {cut_row, cut_delta, *cut_obj, *cut_count, *cut_iter, x_best};
    int64_t done = run_loop(h, x, w, tabu_inc, tabu_dec, iter, best_nviol, tenure, n_iters, 0, &cut,
                            move_var, move_val, move_s, nviol_after, nthreads);
    *cut_obj = cut.obj;
    *cut_count = cut.count;
    *cut_iter = cut.best_iter;
    return done;
}

static int64_t run_loop(orc_t *h, double *x, int32_t *w, int64_t *tabu_inc, int64_t *tabu_dec,
                        int64_t *iter, int64_t *best_nviol, int32_t tenure, int64_t n_iters,
                        int32_t stop_at_feasible, orc_cut_t *cut, int32_t *move_var, double *move_val,
                        int64_t *move_s, int64_t *nviol_after, int32_t nthreads)
{
    int32_t n = h->n;
    double *xhat = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    int64_t *sh = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int32_t *dc = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    double *r = (double *)malloc(sizeof(double) * (size_t)(h->mn > 0 ? h->mn : 1));
    uint8_t *viol = (uint8_t *)malloc((size_t)(h->mn > 0 ? h->mn : 1));
    int64_t done = 0;
    if (!xhat || !sh || !dc || !r || !viol) goto out;
    for (int64_t k = 0; k < n_iters; ++k) {
        int64_t nviol = orc_residuals(h, x, r, viol);
        if (stop_at_feasible && nviol == 0) break;
        orc_best_shift(h, x, w, tabu_inc, tabu_dec, *iter, nviol, *best_nviol, NULL, 0,
                       xhat, sh, dc, nthreads);
        int32_t bj = -1;
        int64_t bs = 0;
        for (int32_t j = 0; j < n; ++j)
            if (sh[j] > bs) { bs = sh[j]; bj = j; }
        if (bj >= 0) {
            double old = x[bj];
            x[bj] = xhat[bj];
            if (xhat[bj] > old) tabu_dec[bj] = *iter + 1 + tenure;
            else tabu_inc[bj] = *iter + 1 + tenure;
        } else {
            for (int32_t q = 0; q < h->mn; ++q)
                if (viol[q]) w[q] += 1;
        }
        *iter += 1;
        int64_t after = orc_residuals(h, x, NULL, NULL);
        if (after < *best_nviol) *best_nviol = after;
        if (cut && after == 0) {
            tighten(h, cut, x, *iter);
            after = orc_residuals(h, x, NULL, NULL);
            *best_nviol = after;
        }
        if (move_var) move_var[k] = bj;
        if (move_val) move_val[k] = bj >= 0 ? x[bj] : 0.0;
        if (move_s) move_s[k] = bj >= 0 ? bs : 0;
        if (nviol_after) nviol_after[k] = after;
        ++done;
        if (stop_at_feasible && after == 0) break;
    }
out:
    free(xhat); free(sh); free(dc); free(r); free(viol);
    return done;
}
