// Internal layout shared by the host code (capi.cu) and the kernels (kernels.cu).
//
// Device layout (all arrays owned by one handle):
//  - Physical rows: one per original row, stored in "<=" orientation: ">=" rows
//    are negated once at create time; an "=" row is stored once as (a, b) and
//    evaluated as its two normalised halves (a, b) and (-a, -b) (Sec. 3.1,
//    "Memory Considerations", second point), which avoids storing its nonzeros
//    twice.
//  - RowState (16 B, one coalesced load per nonzero gather): the residual
//    r = a.x - b of the first half (int64 on integral rows, IEEE double bits on
//    the others) and the integer weights of both halves (w2 = -1 for a single
//    row).  Storing r instead of the activity is the paper's first memory point.
//  - Two CSC matrices: CSC_I holds the nonzeros of integral rows (int32 row,
//    int32 coefficient: 8 B/nnz), CSC_F those of the other rows (int32 row,
//    double coefficient: 12 B/nnz).  A column j owns ci_ptr[j]..ci_ptr[j+1] and
//    cf_ptr[j]..cf_ptr[j+1]; the arithmetic type of a nonzero is known from the
//    matrix it sits in, so no per-row flag is gathered.
//  - CSR (double) of the physical rows, used only to recompute residuals from
//    scratch when a state is set.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace chap {

constexpr int kVarBin = 0, kVarInt = 1, kVarCont = 2;

struct __align__(16) RowState {
    long long r;  // int64 residual or the bits of a double residual
    int w1;       // weight of the first normalised half
    int w2;       // weight of the second half of an "=" row, -1 otherwise
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
};

// Work tiles of the best-shift pass.  A tile covers var_list[begin, end).
enum TileKind : int {
    T_BIN_G4 = 0, T_BIN_G8, T_BIN_G16, T_BIN_G32, T_BIN_CTA,   // binary flips, G lanes per column
    T_NB_K1, T_NB_K2, T_NB_K4, T_NB_K8,                         // warp sort of <= 32K entries
    T_NB_CTA,                                                   // CTA sort in shared memory
    T_NB_HIST                                                   // multi-CTA key histogram (integer keys)
};

struct Tile {
    int kind;
    int begin;
    int end;
    int aux;   // T_NB_CTA: padded entry count; T_NB_HIST: chunk index
};

// Histogram bin of one integer value v of a long integer column (T_NB_HIST).
struct __align__(16) HBin {
    long long sm;  // sum of the score deltas of the entries (v, -1)
    long long sp;  // sum of the score deltas of the entries (v, +1)
    int cm;        // sum of the count deltas of the entries (v, -1)
    int cp;        // sum of the count deltas of the entries (v, +1)
    int np;        // number of entries (v, -1): v is a candidate when > 0
    int pad;
};

struct HistCol {
    int var;
    int nchunks;
    long long bin_off;    // offset of the column's bins in the HBin scratch
    int e_begin, e_mid, e_end;  // virtual entry range: [0, e_mid) integral part, [e_mid, e_end) FP part
    int slot;             // block_best slot of the column
};

// Accumulators of one histogram column (global, reset after use).
struct __align__(16) HistAcc {
    long long beta, alpha;
    int beta_c, alpha_c;
    unsigned int ticket;
    int pad;
};

struct Dev {
    int n, m;
    int tenure;
    int pad0;
    // CSC split
    const int *ci_ptr, *ci_row, *ci_val;
    const int *cf_ptr, *cf_row;
    const double *cf_val;
    // CSR of the physical rows (set-state only)
    const long long *row_ptr;
    const int *col_idx;
    const double *row_val;
    const double *rhs;       // rhs of the first half
    const double *eps;       // 0 on integral rows
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
    // best-shift work
    const int *var_list;
    Cand *block_best;
    int n_block_best;
    int pad1;
    HBin *hbins;
    HistAcc *hacc;
    const HistCol *hcols;
};

// Optional per-variable outputs of a best-shift pass (device pointers, may be null).
struct VarOut {
    double *xhat;
    long long *s;
    int *dc;
};

// Kernel launchers (kernels.cu).  All are asynchronous on `st`.
struct LaunchPlan {
    const Tile *tiles_small;   // device
    int n_small;
    const Tile *tiles_cta;     // device
    int n_cta;
    int cta_smem;              // dynamic shared memory of the CTA-sort kernel
    const Tile *tiles_hist;    // device
    int n_hist_tiles;
    int hist_smem;
    int apply_blocks;
};

cudaError_t launch_eval(const Dev &d, const LaunchPlan &p, const VarOut &o, cudaStream_t st);
cudaError_t launch_select(const Dev &d, cudaStream_t st);
cudaError_t launch_apply(const Dev &d, const LaunchPlan &p, cudaStream_t st);
cudaError_t launch_set_move(const Dev &d, int var, double new_value, cudaStream_t st);
cudaError_t launch_residuals(const Dev &d, cudaStream_t st);
cudaError_t launch_finish_set_state(const Dev &d, long long iter, long long best_nviol, int use_best, cudaStream_t st);
cudaError_t launch_begin_run(const Dev &d, long long max_iters, int stop_at_feasible, cudaStream_t st);
cudaError_t launch_pack_w(const Dev &d, const int *w_norm, cudaStream_t st);
cudaError_t launch_unpack_w(const Dev &d, int *w_norm, cudaStream_t st);
cudaError_t launch_unpack_r(const Dev &d, double *r_norm, cudaStream_t st);
cudaError_t launch_tabu_convert(int n, const int *src32, long long *dst64, cudaStream_t st);
cudaError_t launch_tabu_narrow(int n, const long long *src64, int *dst32, cudaStream_t st);

// Sizes used by both sides.
constexpr int kEvalThreads = 256;
constexpr int kWarpStageCap = 256;     // entries staged per warp (K <= 8)
constexpr int kCtaMaxEntries = 8192;   // largest column list sorted by one CTA
constexpr int kCtaThreads = 512;
constexpr int kHistMaxDomain = 4096;   // largest integer domain of the histogram path
constexpr int kHistChunk = 16384;      // matrix entries per histogram CTA
constexpr int kHistThreads = 512;
constexpr int kApplyThreads = 256;

}  // namespace chap
