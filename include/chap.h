/*
 * chap.h -- C ABI of the GB300 best-shift tabu search library (libchap.so).
 *
 * The library evaluates, for every variable of a MIP at the current assignment,
 * its best shift move (Sec. 3.1 "Best Shift Moves", Eq. best_move, Algorithm 1
 * of "CHAP: A Hybrid GPU-CPU Heuristic for MIP"), picks the best admissible move
 * under tabu and aspiration rules, and applies it with an incremental update of
 * the row residuals (Sec. 3.1 "Memory Considerations").  Every step runs in
 * hand-written CUDA kernels for sm_103a; there is no CPU fallback.
 *
 * Conventions shared by every entry point
 *  - Status codes only; no exception or abort crosses the ABI.  After an error
 *    chap_last_error(handle) gives a message valid until the next call on that
 *    handle.
 *  - Streams: every device operation is ordered on the CUDA stream given to
 *    chap_bs_create (NULL = the legacy default stream).  Calls that return host
 *    data synchronise that stream before returning; calls with device outputs
 *    do not.
 *  - Memory: chap_bs_create copies everything it needs; the caller keeps
 *    ownership of every buffer it passes.  Output buffers are caller-owned and
 *    live in host or device memory as the `mem` argument says.
 *  - Values cross the ABI as doubles; integer values are exact below 2^53.
 *  - Normalised rows (Sec. 3.1, "Memory Considerations", second point): every
 *    original row i is turned into "<=" rows, in this canonical order: a "<="
 *    row gives (a_i, b_i); a ">=" row gives (-a_i, -b_i); an "=" row gives
 *    (a_i, b_i) and then (-a_i, -b_i).  Constraint weights w and violation
 *    counts are per normalised row; m_norm = m + (number of "=" rows).
 *  - Violation of a normalised row: r = a.x - b > eps, where eps = 0 on an
 *    integral row (integer coefficients below 2^31 in magnitude, integer rhs,
 *    only binary/integer variables with finite bounds, and sum |a| max(|l|,|u|)
 *    + |b| <= 2^52) and eps = feas_tol * max(1, |b|) on any other row.
 *    Integral rows keep their residual in exact int64 arithmetic.
 *  - Scores are int64 counts of half weights ("score_half" = 2 * s_j with s_j of
 *    Sec. 3.1 "Scoring Functions"), so integer weights give exact scores.
 */
#ifndef CHAP_H
#define CHAP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define CHAP_API __attribute__((visibility("default")))
#else
#define CHAP_API
#endif

typedef int32_t chap_status;
enum {
    CHAP_OK = 0,
    CHAP_E_INVALID = 1,     /* bad argument or malformed problem */
    CHAP_E_OOM = 2,         /* device or host allocation failed */
    CHAP_E_CUDA = 3,        /* a CUDA runtime call failed */
    CHAP_E_TIMEOUT = 4,     /* a bounded device-side wait ran out */
    CHAP_E_STATE = 5,       /* call not valid in the handle's current state */
    CHAP_E_UNSUPPORTED = 6  /* valid input outside what the library handles */
};

enum { CHAP_VAR_BIN = 0, CHAP_VAR_INT = 1, CHAP_VAR_CONT = 2 };
enum { CHAP_ROW_LE = 0, CHAP_ROW_GE = 1, CHAP_ROW_EQ = 2 };
enum { CHAP_MEM_HOST = 0, CHAP_MEM_DEVICE = 1 };

/*
 * The MIP of Sec. 3.1: min c^T x s.t. each row (<=, >=, =) b, l <= x <= u,
 * x_j integer for binary/integer j.  All arrays are HOST memory.
 *  row_ptr[m+1], col_idx[nnz], row_val[nnz]: CSR of A, column indices strictly
 *      increasing inside each row.
 *  col_ptr[n+1], row_idx[nnz], col_val[nnz]: CSC of the same A, row indices
 *      strictly increasing inside each column; must equal the CSR transposed.
 *  lb[n], ub[n]: bounds (+-infinity allowed for integer/continuous variables;
 *      a binary variable's bounds must lie in {0, 1}; integer bounds integral).
 *  obj[n] (may be NULL: zeros), rhs[m] (finite), vtype[n] (CHAP_VAR_*),
 *  sense[m] (CHAP_ROW_*).
 */
typedef struct chap_problem {
    int32_t n, m;
    int64_t nnz;
    const int64_t *row_ptr;
    const int32_t *col_idx;
    const double *row_val;
    const int64_t *col_ptr;
    const int32_t *row_idx;
    const double *col_val;
    const double *lb, *ub, *obj, *rhs;
    const uint8_t *vtype, *sense;
} chap_problem;

/*
 * Options.  feas_tol: tolerance of non-integral rows (default 1e-9).
 * tenure: after a move at iteration k that increases x_j, decreasing x_j is tabu
 * while iter < k + 1 + tenure, and symmetrically (default 10).  max_iters: limit
 * of chap_tabu_run (default 1000).  graph_iters: iterations recorded in one CUDA
 * graph replay (default 64).  stop_at_feasible: chap_tabu_run stops at the first
 * iteration that leaves no violated row (default 1).  lazy_binary (create time,
 * default 0): selective re-evaluation of the binary flip scores (the lazy
 * scheme Sec. 3.1 attributes to earlier GPU heuristics, "Memory
 * Considerations"): the flip score and violation change of every binary
 * variable are kept on the device and recomputed only for the variables of
 * rows whose residual changed (the rows of the moved column); a weight update,
 * a new state or a tightened cutoff recomputes all of them.  Tabu and
 * aspiration are applied to the kept values at every iteration, so every
 * result equals the full pass; the non-binary columns are evaluated in full
 * at every iteration either way.  bin_kernel (create time): how the binary
 * flips are scored in a full pass: column by column (1; a group of lanes per
 * column gathers its rows' states), row by row (2; Sec. 3.1 "Memory
 * Considerations", third point: each row state read once for all its binary
 * entries, the flip terms added into shared-memory column accumulators of a
 * thread-block cluster), or chosen by the library (0, default: column by
 * column, measured faster on the workloads here).
 */
typedef struct chap_options {
    double feas_tol;
    int32_t tenure;
    int32_t graph_iters;
    int64_t max_iters;
    int32_t stop_at_feasible;
    int32_t lazy_binary;
    int32_t static_scratch_only; /* create time, default 0: see chap_bs_best_shift_static_scratch */
    int32_t shard_rank;          /* create time: column shard of this handle (see chap_bs_move_record) */
    int32_t shard_count;         /* create time, default 0 or 1: the handle evaluates every column */
    int32_t bin_kernel;          /* create time: binary flips 0 automatic, 1 column-wise, 2 row-wise, 3 row-blocked */
    int32_t bin_block_rows;      /* create time: rows of one row block of bin_kernel 3 (0: 8192; 1..8192) */
    int32_t reserved;
} chap_options;

/* One move.  var = -1 means "no admissible variable has a positive score": the
 * iteration instead adds 1 to the weight of every violated normalised row. */
typedef struct chap_move {
    int32_t var;
    int32_t dnviol;        /* change of the number of violated normalised rows */
    int64_t score_half;    /* 2 * s_j of the move */
    double old_value;
    double new_value;
} chap_move;

typedef struct chap_tabu_result {
    int64_t iters;            /* iterations run by this call */
    int64_t moves;            /* of which applied moves (the rest updated weights) */
    int64_t feasible_iter;    /* iteration count at which nviol first reached 0, else -1 */
    int64_t final_nviol;
    int64_t best_nviol;
    double seconds;           /* wall time of the call */
    double time_to_feasible_s;/* device time from the call's start to feasibility, else -1 */
    double objective;         /* c^T x at return */
} chap_tabu_result;

/* Sizes and layout facts of a handle (all counts after normalisation). */
typedef struct chap_info {
    int32_t n, m, m_norm;
    int32_t n_bin, n_int, n_cont, n_fixed;
    int64_t nnz, nnz_int_rows, nnz_fp_rows;
    int64_t bytes_per_pass;   /* algorithmic bytes one best-shift pass reads/writes */
    int32_t eval_blocks;      /* CTAs of one best-shift pass */
    int32_t n_hist_cols;      /* columns on the multi-CTA histogram path */
    int32_t launches_per_step;/* kernel launches of one tabu iteration (chap_bs_step) */
    int32_t grid_bin;         /* CTAs of the persistent binary-flip kernel (0: no binary column) */
    int32_t grid_nb;          /* CTAs of the persistent short-column kernel (0: none) */
    int64_t bytes_bin;        /* algorithmic bytes of one launch of the binary-flip kernel */
    int64_t bytes_nb;         /* algorithmic bytes of one launch of the short-column kernel */
    int64_t bytes_cta;        /* ... of the CTA-sort kernel (long non-integer columns) */
    int64_t bytes_hist;       /* ... of the counting-sort kernel (long integer columns) */
    int32_t bin_lanes;        /* lanes that score one binary column (2, 4, 8 or 16) */
    int32_t nb_lanes;         /* lanes that score one short non-binary column (4 or 8) */
    int32_t n_long_cols;      /* columns on the multi-CTA merge-sort path (lists over 8192 entries) */
    int32_t n_cta_cols;       /* columns on the one-CTA shared-memory sort path (129..8192 entries) */
    int32_t bin_rows;         /* 1: binary flips scored row-wise (clusters over column blocks) */
    int32_t bin_row_blocks;   /* > 0: binary flips row-blocked over this many row blocks (bin_kernel 3) */
} chap_info;

CHAP_API void chap_options_default(chap_options *opts);

/*
 * Validate the problem, normalise its rows and copy everything to device
 * memory owned by the handle, then set the state to x0 = clamp(0, l, u), unit
 * weights, no tabu, iteration 0.  opts may be NULL (defaults).  stream is a
 * cudaStream_t (NULL = legacy default stream).  Returns CHAP_E_INVALID for
 * inconsistent CSR/CSC, unsorted or out-of-range indices, NaN or infinite
 * coefficients or rhs, l > u, binary bounds outside {0,1}, fractional integer
 * bounds; CHAP_E_UNSUPPORTED when more than 2^31 - 1 nonzeros or rows;
 * CHAP_E_OOM when a device allocation fails (everything allocated so far is
 * released).  Testing hook: with the environment variable
 * CHAP_FAIL_ALLOC_AFTER=N set, the device allocation after the first N of
 * this call fails.
 * Ref: Sec. 3.1 (problem form, normalisation), Algorithm 1 (inputs).
 */
CHAP_API chap_status chap_bs_create(const chap_problem *prob, const chap_options *opts,
                                    void *stream, struct chap_bs **out);

/* Free every device and host resource of the handle (NULL is accepted). */
CHAP_API chap_status chap_bs_destroy(struct chap_bs *h);

CHAP_API chap_status chap_bs_info(const struct chap_bs *h, chap_info *info);

/*
 * Kernel timing (measurement aid; no counterpart in the paper).  With
 * enable != 0 the following chap_bs_best_shift / chap_bs_step calls record CUDA
 * events on each kernel's own stream around every evaluation kernel and the
 * selection (never inside chap_tabu_run's graph).  chap_bs_kernel_ms then
 * synchronises the handle's stream and writes the durations of the last
 * profiled pass in milliseconds: ms[0] binary flips, ms[1] short non-binary
 * columns, ms[2] CTA-sorted columns and long lists (merge sort), ms[3]
 * counting-sorted columns, ms[4] selection (0 for a kernel the instance does
 * not launch).  ms has 5
 * elements (host).  CHAP_E_STATE when no profiled pass ran since enabling.
 */
CHAP_API chap_status chap_bs_profile(struct chap_bs *h, int32_t enable);
CHAP_API chap_status chap_bs_kernel_ms(struct chap_bs *h, float *ms);

/*
 * Set the assignment and weights, reset tabu stamps and the iteration counter
 * to 0, recompute every residual from scratch (row sums in CSR order) and set
 * best_nviol = nviol.  x[n] may be NULL (x0); w[m_norm] may be NULL (all 1).
 * x must lie in the bounds and be integral on binary/integer variables;
 * weights must be >= 1.  mem: CHAP_MEM_HOST or CHAP_MEM_DEVICE for x and w.
 */
CHAP_API chap_status chap_bs_set_state(struct chap_bs *h, const double *x, const int32_t *w, int32_t mem);

/*
 * Full checkpoint restore: like chap_bs_set_state, plus the tabu stamps
 * tabu_inc[n] / tabu_dec[n] (an increase / decrease of x_j is tabu while
 * iter < stamp), the iteration counter and best_nviol.  Host memory.
 */
CHAP_API chap_status chap_bs_set_checkpoint(struct chap_bs *h, const double *x, const int32_t *w,
                                            const int64_t *tabu_inc, const int64_t *tabu_dec,
                                            int64_t iter, int64_t best_nviol);

/*
 * Read the state back.  Any pointer may be NULL.  x[n], w[m_norm],
 * tabu_inc[n], tabu_dec[n] in `mem` memory; scalars[6] = {iter, nviol,
 * best_nviol, feasible_iter, moves, weight_updates} always host, the last two
 * counted since the last chap_bs_set_state / chap_bs_set_checkpoint.
 * Synchronises the stream when any host output is requested.
 */
CHAP_API chap_status chap_bs_get_state(struct chap_bs *h, double *x, int32_t *w, int64_t *tabu_inc,
                                       int64_t *tabu_dec, int64_t *scalars, int32_t mem);

/*
 * Residuals r = a.x - b of the normalised rows as doubles (exact on integral
 * rows), r[m_norm] in `mem` memory.
 */
CHAP_API chap_status chap_bs_residuals(struct chap_bs *h, double *r, int32_t mem);

/*
 * One best-shift pass at the current state (Sec. 3.1 "Best Shift Moves",
 * Algorithm 1; binary variables: the flip): for every variable j the
 * admissible value with the largest score, ties broken by the smallest
 * |x - xbar_j| and then the smaller x; (xbar_j, 0, 0) when no admissible value
 * has a positive score.  Candidates are the finite bounds and the breakpoints.
 * Admissible: not tabu at the current iteration, or nviol + dnviol < best_nviol
 * (aspiration).  Outputs, each optional (NULL): xhat[n], score_half[n],
 * dnviol[n] in `mem` memory; best (host) = the move of the largest score, ties
 * broken by the lowest variable index, var = -1 when no score is positive.
 */
CHAP_API chap_status chap_bs_best_shift(struct chap_bs *h, double *xhat, int64_t *score_half,
                                        int32_t *dnviol, chap_move *best, int32_t mem);

/*
 * Apply one move x_var <- new_value with the incremental residual update
 * r_i += a_ij (new - old) on the rows of column var (Sec. 3.1, "Memory
 * Considerations", first point), stamp the reverse direction tabu for
 * `tenure` iterations and advance the iteration counter.  var = -1 instead adds
 * 1 to the weight of every violated normalised row (and advances the counter).
 * new_value must be in the domain of var and differ from its current value.
 */
CHAP_API chap_status chap_bs_apply(struct chap_bs *h, int32_t var, double new_value);

/*
 * Same pass and outputs as chap_bs_best_shift, but the long integer columns
 * sorted by the multi-CTA counting sort use a fixed scratch compiled into the
 * library (a file-scope device array: 65536 bins, 256 columns, 1.5 MiB held by
 * every GPU that loads the library until the process exits) instead of the
 * handle's own scratch.  No counterpart in the paper.  It is for callers that
 * cannot give each handle device memory for this scratch: many handles kept
 * under a fixed device-memory budget, or a memory pool that owns the device
 * and hands out nothing per handle.  Create such handles with
 * chap_options.static_scratch_only = 1: they then hold no counting-sort
 * scratch of their own, and every other call that runs a pass
 * (chap_bs_best_shift, chap_bs_step, chap_tabu_run, chap_bs_refresh_features,
 * chap_learned_run) returns CHAP_E_STATE when the instance has counting-sorted
 * columns (n_hist_cols > 0).  The call allocates nothing; its first call on a
 * device resolves the scratch's address with that device current (make it
 * before any stream capture); concurrent first calls from several host threads
 * are serialised.  The scratch starts at zero and every pass leaves it at
 * zero; it is shared by all handles of the process, so passes through it must
 * not overlap on the GPU (same or different handles, any streams): overlapping
 * calls race.  CHAP_E_UNSUPPORTED (with a message) when the instance needs more
 * than 65536 bins or 256 columns.  Arguments as chap_bs_best_shift.
 */
CHAP_API chap_status chap_bs_best_shift_static_scratch(struct chap_bs *h, double *xhat, int64_t *score_half,
                                                       int32_t *dnviol, chap_move *best, int32_t mem);

/*
 * Column-sharded pass over several GPUs (Sec. 3.1: the pass is independent per
 * variable, so its columns can be split; one GPU per process, see DESIGN).
 * A handle created with chap_options.shard_count = K > 1 and shard_rank = k
 * stores the whole instance (every column, for the incremental update of the
 * apply) and replicated state, but its best-shift pass evaluates only shard k:
 * every K-th column of each column class (round robin over the class order).
 * Its chap_bs_best_shift then gives the shard's best move (per-variable
 * outputs of the other columns: the incumbent, score 0).  One iteration of the
 * sharded search: every rank runs chap_bs_best_shift (device outputs or none),
 * writes its move record with chap_bs_move_record, the K records are
 * exchanged (an all-gather of 32 bytes per rank, e.g. NCCL), and every rank
 * calls chap_bs_apply_records with all K records in rank order: the record of
 * the largest score wins (ties: the lowest variable; no positive score on any
 * rank: the weight update), so every rank applies the same move and the state
 * stays replicated.  chap_bs_step, chap_tabu_run and the learned driver
 * return CHAP_E_STATE on a sharded handle.
 *
 * chap_bs_move_record: the move selected by the handle's last pass into rec
 *   (host or device memory as mem says; stream-ordered, synchronises for host).
 * chap_bs_apply_records: reduces recs[0..k) (host or device; 1 <= k <= 1024)
 *   on the device and applies the winner like chap_bs_apply (or the weight
 *   update).  CHAP_E_INVALID for a host record naming a variable out of range.
 */
typedef struct chap_move_record {
    int64_t score_half;    /* <= 0: no move on this shard */
    int32_t var;           /* -1 when no move */
    int32_t dnviol;
    double new_value;
    double old_value;
} chap_move_record;

CHAP_API chap_status chap_bs_move_record(struct chap_bs *h, chap_move_record *rec, int32_t mem);
CHAP_API chap_status chap_bs_apply_records(struct chap_bs *h, const chap_move_record *recs, int32_t k, int32_t mem);

/* One full tabu iteration: best-shift pass, selection, then apply or weight update.
 * out (host, optional) receives the move taken. */
CHAP_API chap_status chap_bs_step(struct chap_bs *h, chap_move *out);

/*
 * Run the tabu search from the current state: iterations are recorded into a
 * CUDA graph of opts->graph_iters iterations (Sec. 3.1, "Kernel
 * Specialization", last point) and replayed until no row is violated (when
 * stop_at_feasible) or opts->max_iters iterations have run in this call.
 * opts may be NULL (the create options).  result (host) is filled on success.
 */
CHAP_API chap_status chap_tabu_run(struct chap_bs *h, const chap_options *opts, chap_tabu_result *result);

/*
 * Objective cutoff (Sec. 3.2, "Solution Pool": each heuristic imposes the best
 * known objective as a cutoff constraint so that the search looks for improving
 * solutions).  Row `row` of the problem, given with sense "<=", holds the
 * objective: its activity y = a_row . x is the objective value (build it as
 * c^T x <= B with B at least the largest value over the bounds so that it
 * starts satisfied, or the incumbent's objective minus delta).  While the
 * cutoff is on, every iteration that ends with no violated row records the
 * current x as a solution of objective y (copied to the handle's best-solution
 * buffer on the device) and tightens the row's rhs to y - delta, which
 * violates it again; best_nviol restarts from that count (the tightened
 * problem's record) and chap_tabu_run does not stop at feasibility.
 * delta: on an integral row an integer in [1, 2^31); on another row any
 * positive value, raised on the device to at least 4 feas_tol max(1, |y|) so
 * that the tightened row is violated beyond its tolerance.  row = -1 switches
 * the cutoff off (delta ignored).  Stream-ordered; a state already feasible
 * when the cutoff is set is recorded at the end of the next iteration.
 * CHAP_E_INVALID: row out of range or not a "<=" row, bad delta.
 */
CHAP_API chap_status chap_bs_set_cutoff(struct chap_bs *h, int32_t row, double delta);

typedef struct chap_cutoff_info {
    int64_t solutions;      /* solutions recorded since the cutoff was set */
    int64_t best_iter;      /* iteration at whose end the best one was recorded (-1: none) */
    double best_objective;  /* its objective (row activity); NaN when none */
    double rhs;             /* current rhs of the cutoff row */
    int32_t row;            /* the cutoff row, -1 when off */
    int32_t reserved;
} chap_cutoff_info;

/*
 * Read the cutoff state (info, host) and optionally the best solution
 * x_best[n] in `mem` memory (unchanged contents when no solution was
 * recorded).  Synchronises the stream.
 */
CHAP_API chap_status chap_bs_get_cutoff(struct chap_bs *h, chap_cutoff_info *info, double *x_best, int32_t mem);

/*
 * Batched tabu chains (growth path; Sec. 3.1, "Parallel Tabu Search Instances").
 * Many independent chains over several instances advance together: one
 * evaluation launch covers every (chain, 32-column tile), then one apply CTA
 * per chain and one weight-bump launch (or the three phases in one persistent
 * launch, see chap_batch_set_persistent); K iterations are captured into one
 * CUDA graph and replayed.  Each chain follows exactly the single-handle
 * iteration (chap_bs_step) of its instance with its own tenure, from
 * x0 = 0, unit weights, no tabu.  Supported instances: every variable binary,
 * every row integral (integer coefficients and rhs), fewer than 2^22 variables.
 *
 * chap_batch_create: probs[n_probs] (host arrays, as chap_bs_create);
 *   chain_prob[n_chains] the instance of each chain, chain_tenure[n_chains] its
 *   tenure.  CHAP_E_UNSUPPORTED for an instance outside the supported class.
 * chap_batch_run: advances every chain by up to max_iters iterations (stops a
 *   chain at its first nviol = 0 when stop_at_feasible), graph_iters iterations
 *   per graph replay; res[n_chains] (host, optional) receives per-chain
 *   counters (chap_chain_result), *seconds (optional) the wall time.
 * chap_batch_autotune: times every schedule (lanes per column 2 / 4 / 8 / 16 x
 *   CTAs per SM 2 / 4 / 8 x three launches per iteration or one persistent
 *   launch) for `iters` iterations from the initial state, keeps the fastest
 *   (chosen[3] host, optional: lanes, CTAs per SM, persistent) and restores the
 *   initial state.
 * chap_batch_autotune_mode: the same over one schedule only (mode 0: three
 *   launches per iteration, 1: persistent, -1: both).
 * chap_batch_set_schedule: sets lanes per column and CTAs per SM explicitly.
 * chap_batch_set_persistent: on = 1 runs each graph segment of K iterations as
 *   one persistent cooperative launch (every CTA resident) whose phases (eval,
 *   apply, bump) are separated by software grid barriers; on = 0 uses three
 *   launches per iteration.  barrier_limit_ns > 0 bounds each barrier wait
 *   (default 2 s; 0 keeps the current bound): a wait that runs out ends the
 *   launch, chap_batch_run returns CHAP_E_TIMEOUT and the chains' state is
 *   invalid until chap_batch_reset.  Default: persistent.
 * The incumbents x of every chain are bitsets (one bit per variable); every
 *   launch carries an L2 access-policy window that keeps them persisting in L2
 *   (Sec. 3.1, "Memory Considerations", fourth point); the batch raises the
 *   process's persisting-L2 set-aside to their size while it lives.
 * chap_batch_reset: every chain back to its initial state.
 * chap_batch_get_x: x of one chain (host double[n of its instance]).
 */
typedef struct chap_chain_result {
    int64_t iters, moves, feasible_iter, final_nviol, best_nviol;
    double time_to_feasible_s;  /* device time from the run's start, else -1 */
} chap_chain_result;

CHAP_API chap_status chap_batch_create(const chap_problem *probs, int32_t n_probs, const int32_t *chain_prob,
                                       const int32_t *chain_tenure, int32_t n_chains, void *stream,
                                       struct chap_batch **out);
CHAP_API chap_status chap_batch_destroy(struct chap_batch *b);
CHAP_API chap_status chap_batch_run(struct chap_batch *b, int64_t max_iters, int32_t stop_at_feasible,
                                    int32_t graph_iters, chap_chain_result *res, double *seconds);
CHAP_API chap_status chap_batch_autotune(struct chap_batch *b, int32_t iters, int32_t *chosen);
CHAP_API chap_status chap_batch_autotune_mode(struct chap_batch *b, int32_t iters, int32_t mode, int32_t *chosen);
CHAP_API chap_status chap_batch_set_schedule(struct chap_batch *b, int32_t lanes_per_column, int32_t ctas_per_sm);
CHAP_API chap_status chap_batch_set_persistent(struct chap_batch *b, int32_t on, int64_t barrier_limit_ns);
CHAP_API chap_status chap_batch_reset(struct chap_batch *b);
CHAP_API chap_status chap_batch_get_x(struct chap_batch *b, int32_t chain, double *x);
CHAP_API const char *chap_batch_last_error(const struct chap_batch *b);

/*
 * Learned move proposal (growth path; no counterpart in the paper).  A network
 * 12 -> 64 -> 64 -> 1 with ReLU predicts every variable's best-shift score from
 * 12 features; the exact best-shift evaluation then runs on the k variables
 * with the largest predictions (ties: lower index) and a full exact pass every
 * exact_every iterations supplies that iteration's move and judges the
 * proposal (a miss: the exact best score exceeds the best score in the
 * proposed subset).  Moves are always chosen by exact scores.
 *
 * Parameters: CHAP_MLP_PARAMS values in the order W1 [12 x 64] (row-major,
 * input x output), b1 [64], W2 [64 x 64], b2 [64], w3 [64], b3; BF16 (uint16
 * bits) for inference, FP32 masters for training.  Features per variable (BF16,
 * row-major [n x 12]): x/(u-l), (x-l)/(u-l), (u-x)/(u-l), min(tabu age,64)/64,
 * share of the column's halves that are violated, their share of sum w|a|,
 * last exact score / (1 + max |score|), iterations since the exact pass / 50,
 * log2(1 + column length)/16, is_binary, is_integer, c_j / max|c|.
 *
 * chap_bs_refresh_features: exact pass at the current state (scores and the
 *   column features recorded for the proposal; no move).
 * chap_bs_features: features of the current state into feat (device, may be
 *   NULL) and the last exact scores scaled by 1/(1 + max|score|) into target
 *   (device float[n], may be NULL): one training pair per variable.
 * chap_bs_propose: features, predictions (pred: device float[n], may be NULL)
 *   and the k selected variables (list: device int32[k], may be NULL).
 * chap_learned_run: the learned tabu loop from the current state;
 *   propose_every: iterations between two proposals.  Between exact passes
 *   the proposed binary variables are scored by their flips and the proposed
 *   non-binary columns with at most 128 breakpoint entries by Algorithm 1
 *   (exact scores); longer columns are moved only at the exact passes.
 * chap_mlp_forward: y[n] = network(x[n x 12]) (device pointers).
 * chap_mlp_loss_grad: adds the gradient of mean((y - t)^2) over the n rows to
 *   grad[CHAP_MLP_PARAMS] and the sum of squared errors to loss[0] (device).
 * chap_mlp_adam: one Adam step (beta 0.9 / 0.999, eps 1e-8) of the FP32
 *   masters w32 with moments m, v from grad (cleared), writing the BF16 copy.
 */
#define CHAP_MLP_PARAMS 5057
typedef struct chap_learned_options {
    int32_t topk, exact_every, propose_every, stop_at_feasible;
    int64_t max_iters;
} chap_learned_options;
typedef struct chap_learned_result {
    int64_t iters, moves, feasible_iter, final_nviol, best_nviol, exact_passes, misses;
    double seconds, time_to_feasible_s;
} chap_learned_result;

CHAP_API chap_status chap_bs_refresh_features(struct chap_bs *h);
CHAP_API chap_status chap_bs_features(struct chap_bs *h, uint16_t *feat, float *target);
CHAP_API chap_status chap_bs_propose(struct chap_bs *h, const uint16_t *weights, int32_t k, int32_t *list, float *pred);
CHAP_API chap_status chap_learned_run(struct chap_bs *h, const uint16_t *weights, const chap_learned_options *lo,
                                      chap_learned_result *res);
CHAP_API chap_status chap_mlp_forward(const uint16_t *weights, const uint16_t *x, int64_t n, float *y, void *stream);
CHAP_API chap_status chap_mlp_loss_grad(const uint16_t *weights, const uint16_t *x, const float *target, int64_t n,
                                        float *grad, float *loss, void *stream);
CHAP_API chap_status chap_mlp_adam(float *w32, uint16_t *wbf, float *m, float *v, float *grad, int32_t step, float lr,
                                   void *stream);

CHAP_API const char *chap_status_str(chap_status s);
CHAP_API const char *chap_last_error(const struct chap_bs *h);

#ifdef __cplusplus
}
#endif
#endif /* CHAP_H */
