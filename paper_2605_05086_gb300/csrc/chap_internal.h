// Internal layout shared by the host code (capi.cu) and the kernels (kernels.cu).
//
// Device layout (all arrays owned by one handle):
//  - Physical rows: one per original row, stored in "<=" orientation: ">=" rows
//    are negated once at create time; an "=" row is stored once as (a, b) and
//    evaluated as its two normalised halves (a, b) and (-a, -b) (Sec. 3.1,
//    "Memory Considerations", second point), which avoids storing its nonzeros
//    twice.
//  - RowState (32 B = one sector per nonzero gather): the residual
//    r = a.x - b of the first half (int64 on integral rows, IEEE double bits on
//    the others), the integer weights of both halves (w2 = -1 for a single row)
//    and, on non-integral rows, the margins eps - r and eps + r, so that every
//    violation test of the flip and breakpoint code is a sign or ordered-key
//    comparison (no FP64 arithmetic per nonzero; GB300's FP64 rate is low).
//    Storing r instead of the activity is the paper's first memory point.
//  - Two CSC matrices: CSC_I holds the nonzeros of integral rows (int32 row,
//    int32 coefficient: 8 B/nnz), CSC_F those of the other rows (int32 row,
//    double coefficient: 12 B/nnz).  Columns are stored in evaluation order
//    var_list (binary columns first, then each non-binary class), so the
//    binary pass streams one contiguous range; position q (var_list[q] = j,
//    vpos[j] = q) owns ci_ptr[q]..ci_ptr[q+1] and cf_ptr[q]..cf_ptr[q+1], the
//    rows of one normalised half first and the "=" rows (two halves) from
//    ci_eq[q] / cf_eq[q] on, so that the kernels run the second-half code only
//    where it has work.  The
//    arithmetic type of a nonzero is known from the matrix it sits in, so no
//    per-row flag is gathered.
//  - CSR (double) of the physical rows, used only to recompute residuals from
//    scratch when a state is set.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/chap.h"

namespace chap {

constexpr int kVarBin = 0, kVarInt = 1, kVarCont = 2;

struct __align__(32) RowState {
    long long r;  // int64 residual or the bits of a double residual
    int w1;       // weight of the first normalised half
    int w2;       // weight of the second half of an "=" row, -1 otherwise
    double m1;    // non-integral rows: eps - r  (first half violated  <=> m1 < 0)
    double m2;    // non-integral rows: eps + r  (second half violated <=> m2 < 0)
};

// Best move of a CTA (or of the whole pass): larger s wins, then lower var.
struct __align__(8) Cand {
    long long s;   // score in half-weight units; <= 0 means "no move"
    int var;       // 0x7fffffff when empty
    int dc;        // change of the number of violated normalised rows
    double xhat;
};

// Device control block of one handle.
struct __align__(16) Ctl {
    long long iter;
    long long nviol;
    long long best_nviol;
    long long feasible_iter;
    long long max_iter;        // kernels do nothing once iter >= max_iter
    long long moves;
    long long bumps;
    long long nviol_delta;     // accumulated by the apply CTAs of one iteration
    unsigned long long t_start_ns;
    unsigned long long t_feas_ns;
    // move chosen by the selection of the current iteration
    long long mv_s;
    double mv_new;
    double mv_old;
    int mv_var;
    int mv_dc;
    int done;                  // set when the run's stop condition holds
    int stop_at_feasible;
    int error;
    unsigned int apply_ticket;
    unsigned int select_ticket;
    int pad;
    // Largest admissible score found so far in the current pass (0 between
    // passes): a lower bound of the move's score, against which the
    // short-column kernel skips the sort of columns that cannot reach it.
    long long pass_best;
    // Objective cutoff (Sec. 3.2, the best known objective imposed as a
    // constraint): active when cut_on != 0.  Row cut_row holds the objective
    // as a "<=" row; whenever an iteration ends with no violated row, its
    // activity is recorded as the best objective and its rhs tightened to that
    // value minus the required improvement.
    int cut_on;
    int cut_row;
    int cut_int;               // the cutoff row is integral (int64 residual, eps = 0)
    int pad2;
    double cut_rhs;            // current rhs of the cutoff row
    double cut_delta;          // required improvement
    double cut_tol;            // feasibility tolerance (non-integral row: eps = tol * max(1, |rhs|))
    double cut_obj;            // objective of the best solution found
    long long cut_count;       // solutions recorded
    long long cut_iter;        // iteration that produced the best one
    // Selective re-evaluation of the binary flip scores (active when lz_on):
    // positions marked with the current epoch are queued for re-evaluation;
    // lz_full asks for all of them.  Each iteration end raises lz_seq and
    // records the moved variable (lz_var, -1 after a weight update); the
    // marking kernel handles every sequence number once (lz_done).
    int lz_on;
    int lz_full;
    int lz_count;              // queued positions
    unsigned lz_epoch;
    long long lz_seq, lz_done;
    int lz_var;
    unsigned lz_ticket;
};

// Work tiles of the best-shift pass.  A tile covers var_list[begin, end).
enum TileKind : int {
    T_BIN = 0,                // binary flips: a group of lanes per column
    T_NB,                     // short breakpoint lists: one warp per column
    T_NB_CTA,                 // CTA bitonic sort in shared memory
    T_NB_HIST,                // multi-CTA counting sort (long integer columns)
    T_NB_LONG,                // multi-CTA merge sort (lists longer than a CTA sorts)
    T_NUM_KINDS
};

struct Tile {
    int kind;
    int begin;   // first position (var_list index) of the tile
    int end;     // one past the last position
    int aux;     // T_NB_CTA: padded entry count; T_NB_HIST: chunk index
};

// Counting-sort bin of one integer value v of a column: the entries (v, pre)
// carry score deltas that count at v, the entries (v, post) deltas that count
// right of v; every pre entry lowers the violation count by one, every post
// entry raises it by one (Algorithm 1 case table).
struct __align__(8) HBin {
    long long spre;
    long long spost;
    int n1;   // number of pre entries at v
    int n2;   // number of post entries at v
};

struct HistCol {
    int pos;              // position of the column in var_list
    int nchunks;
    long long bin_off;    // offset of the column's bins in the HBin scratch
    int e_mid, e_end;     // virtual entry range: [0, e_mid) integral part, [e_mid, e_end) FP part
    int slot;             // block_best slot of the column
    int pad;
};

// Accumulators of one histogram column (global, reset after use).
struct __align__(16) HistAcc {
    long long beta, alpha;
    int beta_c, alpha_c;
    unsigned int ticket;
    int pad;
};

// Breakpoint entry staged in shared memory (and in the long lists' global
// buffers): key (t in order-preserving form), score delta (|delta| <= 2w <
// 2^31), aux = entry class and count delta.
struct __align__(16) SEntry {
    unsigned long long key;
    int del;
    unsigned aux;
};

// Best candidate of one scan tile of a long list (score, key, count change).
struct __align__(8) LCand {
    long long s;
    unsigned long long key;
    int dc;
    int valid;
};

// A column whose breakpoint list is longer than one CTA sorts (continuous
// variables, integer variables with a wide domain): its entries are generated
// and sorted in runs of kLongRun entries, one chunk of kLongChunk nonzeros per
// CTA, the runs merged pairwise across the grid, and the merged list scanned
// in tiles of kLongTile entries with a carry across tiles.
struct LongCol {
    int pos;              // position of the column in var_list
    int nchunks;          // chunks of kLongChunk nonzeros (= generated runs)
    int runs;             // runs rounded up to a power of two (pads: empty runs)
    int e_mid, e_end;     // virtual entry range: [0, e_mid) integral part, [e_mid, e_end) FP part
    int ntiles;           // scan tiles of the merged list
    int tile0;            // first tile of the column in the per-tile arrays
    int slot;             // block_best slot of the column
    long long base;       // first entry of the column in the entry buffers
};

// Row-wise binary flips (Sec. 3.1, "Memory Considerations", third point: the
// binary columns scored row by row).  The binary positions are dealt round
// robin into blocks of at most kRbCols columns (position q = c * blocks + b
// is column c of block b); each block has two CSR stores of its nonzeros, one
// over the integral rows and one over the others, holding only rows with
// entries in the block (row id, entry offsets, 16-bit local column,
// coefficient).  A cluster of kRbCluster CTAs scores one block: each CTA
// streams a share of the block's rows, reads each row state once for all its
// entries and adds the penalty changes into shared-memory accumulators of the
// block's columns; the cluster then sums the CTAs' accumulators through
// distributed shared memory.
struct RowBin {
    int blocks;                       // column blocks (clusters)
    int pad;
    const int *rows_i, *eptr_i;       // integral rows: row ids, entry offsets (rows + 1 per store, concatenated)
    const unsigned short *col_i;
    const unsigned char *own_i;       // per entry: its row's place in the row's aligned chunk of 32 rows
    const int *val_i;
    const int *rows_f, *eptr_f;       // other rows
    const unsigned short *col_f;
    const unsigned char *own_f;
    const double *val_f;
    const int *split_i, *split_f;     // per block: kRbCluster + 1 row-list boundaries of the CTAs
};

// Row-blocked binary flips (k_eval_bin_blk).  The physical rows are cut into
// blocks of at most 8192 consecutive rows; one CTA copies a block's row states
// into shared memory (24 B a row: r or eps - r, eps + r, both weights) and
// scores the binary entries whose rows lie in that block, for a span of
// binary positions: the row-state lookups become shared-memory loads instead
// of one L2 gather per nonzero.  Per block, the entries on integral rows and
// on the other rows form two streams ordered by position, then row; an entry
// is a 32-bit word (position << 13 | row inside the block) and its int32 /
// double coefficient.  Every work item (block, position span, the span's
// entry ranges of both streams) is split evenly over the CTA's warps, which
// stream their entries 32 at a time and sum each position's terms with a
// segmented warp scan; the blocks' partial sums meet in acc_s / acc_dc
// (device atomics, zero between passes).  A second kernel, one CTA per
// finalize range of kBlkFin positions, applies tabu and aspiration to the
// sums, writes the range's candidate slot and returns the accumulators to
// zero.
struct BlkItem {
    int b;                         // row block
    int q0, q1;                    // position span [q0, q1)
    int eI0, eI1, eF0, eF1;        // its entries in the two streams
    int pad;
};

struct BinBlk {
    int nblk;                      // row blocks
    int rows;                      // rows per block (kBlkRows unless set smaller at create)
    int n_items;                   // work items = CTAs of one launch
    int n_fin;                     // finalize ranges (= CTAs of the finalize kernel = candidate slots)
    const BlkItem *items;
    const unsigned *metaI, *metaF; // position << 13 | row inside the block
    const int *valI;
    const double *valF;
    long long *acc_s;
    int *acc_dc;
};

struct Dev {
    int n, m;
    int tenure;
    int m_norm;              // normalised rows ("=" rows count twice)
    // CSC split, columns in var_list order (pointers indexed by position)
    const int *ci_ptr, *ci_row, *ci_val;
    const int *cf_ptr, *cf_row;
    const double *cf_val;
    // inside each column part the single rows come first, the "=" rows from
    // ci_eq[q] / cf_eq[q] on
    const int *ci_eq, *cf_eq;
    // CSR of the physical rows (set-state only)
    const long long *row_ptr;
    const int *col_idx;
    const double *row_val;
    double *rhs;             // rhs of the first half (the cutoff row's changes during a run)
    double *eps;             // 0 on integral rows
    const unsigned char *row_int;
    const int *nrow_base;    // canonical index of the first normalised half of row i
    // variables
    const unsigned char *vtype;
    const double *lb, *ub, *obj;
    // state
    double *x;
    RowState *rs;
    int *tabu_inc, *tabu_dec;
    Ctl *ctl;
    double *x_best;          // copy of x at the last recorded cutoff solution (null: no cutoff)
    // selective binary re-evaluation (null unless enabled): flip score and
    // violation change of each binary position, epoch marks, queued positions
    long long *lz_s;
    int *lz_dc;
    unsigned *lz_mark;
    int *lz_list;
    // best-shift work
    const int *var_list;     // position -> variable
    const int *vpos;         // variable -> position
    Cand *block_best;
    int n_block_best;
    int pad1;
    HBin *hbins;
    HistAcc *hacc;
    const HistCol *hcols;
    // long lists: entry buffers (ping-pong of the merge), per-column
    // accumulators, per-tile sums and candidates, column table
    SEntry *lbuf0, *lbuf1;
    HistAcc *lacc;
    long long *ltsum;        // per tile: score delta sum
    int *ltsumc;             // per tile: count delta sum
    LCand *lcand;            // per tile: best candidate
    const LongCol *lcols;
    int n_long;
    // rows of the residual computation (set-state only): the integral rows,
    // then the others by decreasing length
    int n_res_int;
    const int *res_rows;
    // row-blocked binary flips only (else null / 0): per binary position 1 when
    // x of its variable is 0 (the flip raises it), kept by every x update
    unsigned char *bup;
    int n_bup;
};



// Optional per-variable outputs of a best-shift pass (device pointers, may be null).
struct VarOut {
    double *xhat;
    long long *s;
    int *dc;
};

struct LaunchPlan {
    int bin_cols;              // binary columns: positions [0, bin_cols)
    int n_bin;                 // CTAs of the persistent binary kernel (0: no binary column)
    int bin_G;                 // lanes per binary column (2, 4 or 8, from the mean column length)
    int nb_q0, nb_cols;        // positions of the short non-binary columns (<= kWarpSortMax entries)
    int nb_grid;               // CTAs of the persistent short-column kernel (0: no such column)
    int nb_G;                  // lanes per short non-binary column (4 or 8, from the mean column length)
    const Tile *tiles_cta;
    int n_cta;
    int cta_smem;              // dynamic shared memory of the CTA-sort kernel
    const Tile *tiles_hist;
    int n_hist_tiles;
    int hist_smem;
    const Tile *tiles_lgen;    // long lists: (column, chunk) of the generation kernel
    int n_lgen;
    const Tile *tiles_lscan;   // (column, tile) of the scan kernels
    int n_lscan;
    int long_rounds;           // pairwise merge rounds (log2 of the most runs)
    long long long_entries;    // entries of all long lists (merge grid)
    int slot_nb, slot_cta;     // first block_best slot of each kernel
    int lazy;                  // binary flips through the kept scores (k_eval_bin_lazy, k_bin_scan)
    int bin_rows;              // binary flips row-wise (k_eval_bin_rows, n_bin = blocks * kRbCluster CTAs)
    RowBin rb;
    int bin_blk;               // binary flips row-blocked (k_eval_bin_blk, bb.n_items CTAs; k_bin_blk_final, n_bin = bb.n_fin)
    BinBlk bb;
    int lazy_mark_blocks;      // CTAs of the marking kernel
    int apply_blocks;          // CTAs of the weight bump
    int apply_move_blocks;     // CTAs of the move apply (longest column / kApplyMoveThreads)
    cudaStream_t side[3];      // side streams of the non-binary evaluation kernels
    cudaEvent_t ev_fork, ev_join[3];
    // optional timing of the kernels of one pass (outside graph capture):
    // pev[2k], pev[2k+1] around evaluation kernel k (bin, nb, cta, hist) on its
    // stream, pev[8], pev[9] around the selection
    int profile;
    cudaEvent_t pev[10];
};

// Kernel launchers (kernels.cu).  All are asynchronous on `st`; `gate` makes a
// kernel return at once when the run's done flag is set (graph replays).
cudaError_t setup_kernel_attributes(const LaunchPlan &p);
int long_gen_smem();                  // dynamic shared memory of the long lists' generation kernel
// Device addresses of the fixed counting-sort scratch (kStaticHistBins bins,
// kStaticHistCols accumulators) on the current device.
cudaError_t static_hist_scratch(HBin **bins, HistAcc **acc);
int bin_grid_size(int ncols, int G);  // persistent grids of the binary (G lanes per column) and
                                      // short-column kernels on the current device
int nb_grid_size(int ncols, int G);
cudaError_t launch_eval_gated(const Dev &d, const LaunchPlan &p, const VarOut &o, int gate, cudaStream_t st);
cudaError_t launch_select_gated(const Dev &d, const LaunchPlan &p, int gate, cudaStream_t st);
cudaError_t launch_apply_gated(const Dev &d, const LaunchPlan &p, int gate, cudaStream_t st);
cudaError_t launch_set_move(const Dev &d, int var, double new_value, cudaStream_t st);
cudaError_t launch_residuals(const Dev &d, const int *w, cudaStream_t st);
cudaError_t launch_finish_set_state(const Dev &d, long long iter, long long best_nviol, int use_best, cudaStream_t st);
cudaError_t launch_begin_run(const Dev &d, long long max_iters, int stop_at_feasible, cudaStream_t st);
cudaError_t launch_set_cutoff(const Dev &d, int on, int row, int integral, double delta, double tol, cudaStream_t st);
cudaError_t launch_lazy_init(const Dev &d, cudaStream_t st);
cudaError_t launch_unpack_w(const Dev &d, int *w_norm, cudaStream_t st);
cudaError_t launch_unpack_r(const Dev &d, double *r_norm, cudaStream_t st);
cudaError_t launch_tabu_convert(int n, const int *src32, long long *dst64, cudaStream_t st);
// c^T x into out[0] (device); partial: device scratch of 128 doubles (kObjBlocks)
cudaError_t launch_objective(const Dev &d, double *out, double *partial, cudaStream_t st);
cudaError_t launch_move_record(const Dev &d, chap_move_record *rec, cudaStream_t st);
// Learned proposal: exact best shift of the short non-binary columns among list[0..k)
// (whole-warp path), folded into *key with their values in xh (see kernels.cu).
cudaError_t launch_subset_nb(const Dev &d, const LaunchPlan &p, const int *list, int k, double *xh,
                             unsigned long long *key, int gate, cudaStream_t st);
cudaError_t launch_apply_records(const Dev &d, const chap_move_record *recs, int k, cudaStream_t st);

// Sizes used by both sides.
constexpr int kEvalThreads = 256;
constexpr int kCtaMaxEntries = 8192;    // largest entry list sorted by one CTA
constexpr int kCtaThreads = 512;
constexpr int kHistMaxDomain = 4096;    // largest integer domain of the multi-CTA counting sort
constexpr int kHistChunk = 16384;       // matrix entries per counting-sort CTA
constexpr int kHistThreads = 512;
constexpr int kRbCols = 8192;          // binary columns of one row-wise block
constexpr int kRbCluster = 8;          // CTAs per block (one thread-block cluster)
constexpr int kRbThreads = 1024;
constexpr int kLongChunk = 1020;       // nonzeros per generating CTA: <= 4 entries each, + 2 bounds
constexpr int kLongRun = 4096;         // entries of one sorted run (power of two)
constexpr int kLongThreads = 512;
constexpr int kLongTile = 2048;        // entries per scan CTA (4 per thread)
constexpr int kStaticHistBins = 1 << 16;  // fixed counting-sort scratch: bins (24 B each, 1.5 MiB)
constexpr int kStaticHistCols = 256;      // and columns
constexpr int kBlkRows = 8192;          // rows of one row block of the row-blocked binary flips (24 B each in shared memory)
constexpr int kBlkRowBits = 13;        // bits of the row inside a block in an entry word (kBlkRows = 2^13)
constexpr int kBlkMaxPos = 1 << (32 - kBlkRowBits);  // binary positions an entry word can name
constexpr int kBlkThreads = 1024;
constexpr int kBlkFin = 1024;           // binary positions of one finalize range (one CTA)
constexpr int kBlkFinThreads = 256;
constexpr int kBlkMaxBlocks = 32;       // the library picks the row-blocked flips up to this many row blocks,
constexpr int kBlkMinCols = 16384;      // from this many binary columns,
constexpr double kBlkMinSeg = 2.0;      // and from this many entries per (block, column) on average
constexpr int kApplyThreads = 256;
constexpr int kApplyMoveThreads = 1024;
constexpr int kLazyMaxRows = 2048;      // longer moved columns re-evaluate every kept binary score
constexpr int kWarpSortMax = 128;       // longest list of an integer short column (one warp sorts it, K <= 4)
constexpr int kWarpListMax = 256;       // ... of a continuous short column (a delta and a marker per half, K <= 8)
constexpr double kBinG2MaxLen = 6.0;    // mean binary column length up to which 2 lanes score a column
constexpr int kBinG2MinCols = 32768;    // (and only with this many binary columns: small instances are latency-bound)
constexpr double kBinG4MaxLen = 16.0;   // ... up to which 4 lanes do
constexpr double kBinG8MaxLen = 1.0e30; // ... up to which 8 lanes do (16 above)
constexpr double kNbG4MaxLen = 16.0;    // mean short non-binary column length up to which 4 lanes score a column (8 above)

}  // namespace chap
