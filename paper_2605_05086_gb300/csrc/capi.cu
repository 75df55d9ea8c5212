// Host side of the C ABI declared in include/chap.h: validation, row
// normalisation (Sec. 3.1, "Memory Considerations"), the split CSC store,
// work tiles of the best-shift pass, state handling and the CUDA-graph driver
// of the tabu loop (Sec. 3.1, "Kernel Specialization", last point).
#include "../../include/chap.h"
#include "chap_internal.h"
#include "chap_handle.h"

#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

using namespace chap;


namespace {

const double kLim52 = 4503599627370496.0;

bool is_int_value(double v) { return std::isfinite(v) && std::floor(v) == v; }

chap_status fail(chap_bs *h, chap_status s, const std::string &msg)
{
    if (h) h->err = msg;
    return s;
}

chap_status cuda_fail(chap_bs *h, cudaError_t e, const char *what)
{
    if (h) {
        h->err = std::string(what) + ": " + cudaGetErrorString(e);
        if (e == cudaErrorIllegalAddress || e == cudaErrorLaunchFailure || e == cudaErrorIllegalInstruction ||
            e == cudaErrorMisalignedAddress || e == cudaErrorHardwareStackError)
            h->broken = true;
    }
    return CHAP_E_CUDA;
}

#define CK(h, call, what)                                  \
    do {                                                   \
        cudaError_t _e = (call);                           \
        if (_e != cudaSuccess) return cuda_fail(h, _e, what); \
    } while (0)

template <class T>
T *dalloc(chap_bs *h, size_t count)
{
    void *p = nullptr;
    if (h->fail_allocs_after == 0) return nullptr;   // injected allocation failure (testing)
    if (h->fail_allocs_after > 0) --h->fail_allocs_after;
    if (count == 0) count = 1;
    if (cudaMalloc(&p, count * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    h->allocs.push_back(p);
    return static_cast<T *>(p);
}

template <class T>
cudaError_t h2d(T *dst, const T *src, size_t count, cudaStream_t st)
{
    if (count == 0) return cudaSuccess;
    return cudaMemcpyAsync(dst, src, count * sizeof(T), cudaMemcpyHostToDevice, st);
}

int next_pow2(int v)
{
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

chap_status validate(const chap_problem *p, std::string &msg)
{
    if (!p) { msg = "problem is NULL"; return CHAP_E_INVALID; }
    if (p->n < 0 || p->m < 0 || p->nnz < 0) { msg = "negative size"; return CHAP_E_INVALID; }
    if (p->nnz > (int64_t)INT_MAX - 1) { msg = "more than 2^31-1 nonzeros"; return CHAP_E_UNSUPPORTED; }
    const int n = p->n, m = p->m;
    const int64_t nnz = p->nnz;
    if (!p->row_ptr || !p->col_ptr) { msg = "row_ptr/col_ptr is NULL"; return CHAP_E_INVALID; }
    if (nnz > 0 && (!p->col_idx || !p->row_val || !p->row_idx || !p->col_val)) { msg = "index/value array is NULL"; return CHAP_E_INVALID; }
    if (n > 0 && (!p->lb || !p->ub || !p->vtype)) { msg = "variable array is NULL"; return CHAP_E_INVALID; }
    if (m > 0 && (!p->rhs || !p->sense)) { msg = "row array is NULL"; return CHAP_E_INVALID; }
    if (p->row_ptr[0] != 0 || p->row_ptr[m] != nnz) { msg = "row_ptr does not span [0, nnz]"; return CHAP_E_INVALID; }
    if (p->col_ptr[0] != 0 || p->col_ptr[n] != nnz) { msg = "col_ptr does not span [0, nnz]"; return CHAP_E_INVALID; }
    for (int i = 0; i < m; ++i) {
        if (p->row_ptr[i + 1] < p->row_ptr[i]) { msg = "row_ptr decreases at row " + std::to_string(i); return CHAP_E_INVALID; }
        for (int64_t e = p->row_ptr[i]; e < p->row_ptr[i + 1]; ++e) {
            int j = p->col_idx[e];
            if (j < 0 || j >= n) { msg = "column index out of range in row " + std::to_string(i); return CHAP_E_INVALID; }
            if (e > p->row_ptr[i] && p->col_idx[e - 1] >= j) { msg = "column indices not strictly increasing in row " + std::to_string(i); return CHAP_E_INVALID; }
            double a = p->row_val[e];
            if (!std::isfinite(a) || a == 0.0) { msg = "zero, NaN or infinite coefficient in row " + std::to_string(i); return CHAP_E_INVALID; }
        }
        if (!std::isfinite(p->rhs[i])) { msg = "non-finite rhs in row " + std::to_string(i); return CHAP_E_INVALID; }
        if (p->sense[i] > CHAP_ROW_EQ) { msg = "bad sense in row " + std::to_string(i); return CHAP_E_INVALID; }
    }
    std::vector<int64_t> cur(p->row_ptr, p->row_ptr + m);
    for (int j = 0; j < n; ++j) {
        if (p->col_ptr[j + 1] < p->col_ptr[j]) { msg = "col_ptr decreases at column " + std::to_string(j); return CHAP_E_INVALID; }
        for (int64_t e = p->col_ptr[j]; e < p->col_ptr[j + 1]; ++e) {
            int i = p->row_idx[e];
            if (i < 0 || i >= m) { msg = "row index out of range in column " + std::to_string(j); return CHAP_E_INVALID; }
            if (e > p->col_ptr[j] && p->row_idx[e - 1] >= i) { msg = "row indices not strictly increasing in column " + std::to_string(j); return CHAP_E_INVALID; }
            int64_t c = cur[i];
            if (c >= p->row_ptr[i + 1] || p->col_idx[c] != j || p->row_val[c] != p->col_val[e]) {
                msg = "CSC is not the transpose of CSR at column " + std::to_string(j); return CHAP_E_INVALID;
            }
            cur[i] = c + 1;
        }
    }
    for (int i = 0; i < m; ++i)
        if (cur[i] != p->row_ptr[i + 1]) { msg = "CSC is not the transpose of CSR at row " + std::to_string(i); return CHAP_E_INVALID; }
    for (int j = 0; j < n; ++j) {
        double l = p->lb[j], u = p->ub[j];
        if (std::isnan(l) || std::isnan(u) || l > u || l == INFINITY || u == -INFINITY) { msg = "bad bounds of variable " + std::to_string(j); return CHAP_E_INVALID; }
        int t = p->vtype[j];
        if (t > CHAP_VAR_CONT) { msg = "bad type of variable " + std::to_string(j); return CHAP_E_INVALID; }
        if (t == CHAP_VAR_BIN && !((l == 0.0 || l == 1.0) && (u == 0.0 || u == 1.0))) { msg = "binary bounds not in {0,1} for variable " + std::to_string(j); return CHAP_E_INVALID; }
        if (t == CHAP_VAR_INT && ((std::isfinite(l) && !is_int_value(l)) || (std::isfinite(u) && !is_int_value(u)))) { msg = "fractional integer bound of variable " + std::to_string(j); return CHAP_E_INVALID; }
        if (p->obj && !std::isfinite(p->obj[j])) { msg = "non-finite objective of variable " + std::to_string(j); return CHAP_E_INVALID; }
    }
    return CHAP_OK;
}

void free_all(chap_bs *h)
{
    learn_free(h);
    if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
    for (void *p : h->allocs) cudaFree(p);
    h->allocs.clear();
    if (h->h_ctl) { cudaFreeHost(h->h_ctl); h->h_ctl = nullptr; }
    if (h->cap_st) { cudaStreamDestroy(h->cap_st); h->cap_st = nullptr; }
    for (int k = 0; k < 3; ++k) {
        if (h->plan.side[k]) { cudaStreamDestroy(h->plan.side[k]); h->plan.side[k] = nullptr; }
        if (h->plan.ev_join[k]) { cudaEventDestroy(h->plan.ev_join[k]); h->plan.ev_join[k] = nullptr; }
    }
    if (h->plan.ev_fork) { cudaEventDestroy(h->plan.ev_fork); h->plan.ev_fork = nullptr; }
    for (int k = 0; k < 10; ++k)
        if (h->plan.pev[k]) { cudaEventDestroy(h->plan.pev[k]); h->plan.pev[k] = nullptr; }
}

chap_status read_ctl(chap_bs *h)
{
    CK(h, cudaMemcpyAsync(h->h_ctl, h->dev.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->st), "read control block");
    CK(h, cudaStreamSynchronize(h->st), "synchronise");
    return CHAP_OK;
}

chap_status check_x(chap_bs *h, const double *x)
{
    for (int j = 0; j < h->n; ++j) {
        double v = x[j];
        if (!(v >= h->lb[j] && v <= h->ub[j])) return fail(h, CHAP_E_INVALID, "x out of bounds at variable " + std::to_string(j));
        if (h->vtype[j] != CHAP_VAR_CONT && !is_int_value(v)) return fail(h, CHAP_E_INVALID, "fractional value of integer variable " + std::to_string(j));
    }
    return CHAP_OK;
}

// Load x (host array) and normalised weights (host array, NULL = 1), recompute
// residuals.  x and w go to the device as they are (x canonicalised there);
// the row states are built on the device from the uploaded weights.
chap_status load_state(chap_bs *h, const double *x, const int *w, const int *tabu_inc, const int *tabu_dec,
                       long long iter, long long best_nviol, int use_best)
{
    if (h->broken) return fail(h, CHAP_E_STATE, "handle unusable after a CUDA fault");
    chap_status s = check_x(h, x);
    if (s != CHAP_OK) return s;
    if (w)
        for (int i = 0; i < h->m; ++i) {
            const int k = h->nrow_base[i];
            if (w[k] < 1 || (h->row_eq[i] && w[k + 1] < 1)) return fail(h, CHAP_E_INVALID, "weights must be >= 1");
        }
    Dev &d = h->dev;
    CK(h, h2d(d.x, x, h->n, h->st), "copy x");
    if (w) CK(h, h2d(h->t_w, w, h->m_norm, h->st), "copy weights");
    if (tabu_inc) {
        CK(h, h2d(d.tabu_inc, tabu_inc, h->n, h->st), "copy tabu");
        CK(h, h2d(d.tabu_dec, tabu_dec, h->n, h->st), "copy tabu");
    } else {
        CK(h, cudaMemsetAsync(d.tabu_inc, 0, sizeof(int) * (size_t)std::max(h->n, 1), h->st), "reset tabu");
        CK(h, cudaMemsetAsync(d.tabu_dec, 0, sizeof(int) * (size_t)std::max(h->n, 1), h->st), "reset tabu");
    }
    CK(h, cudaMemsetAsync(&d.ctl->nviol, 0, sizeof(long long), h->st), "reset nviol");
    CK(h, launch_residuals(d, w ? h->t_w : nullptr, h->st), "residual kernel");
    CK(h, launch_finish_set_state(d, iter, best_nviol, use_best, h->st), "finish set_state");
    // the caller may reuse (or free) its host arrays on return: wait for the copies
    CK(h, cudaStreamSynchronize(h->st), "synchronise");
    return CHAP_OK;
}

}  // namespace

namespace chap {
// Validation of a problem, shared with the batched path.
chap_status validate_problem(const chap_problem *p, std::string &msg) { return validate(p, msg); }

cudaError_t bs_pass(chap_bs *h, const VarOut &o)
{
    cudaError_t e = launch_eval_gated(h->dev, h->plan, o, 0, h->st);
    if (e == cudaSuccess) e = launch_select_gated(h->dev, h->plan, 0, h->st);
    return e;
}

cudaError_t bs_apply_selected(chap_bs *h) { return launch_apply_gated(h->dev, h->plan, 0, h->st); }

chap_status whole_instance_ok(chap_bs *h)
{
    if (h->shard_count > 1)
        return fail(h, CHAP_E_STATE,
                    "column-sharded handle: its pass covers a share of the columns; exchange the shards' move "
                    "records (chap_bs_move_record) and apply the winner with chap_bs_apply_records");
    return CHAP_OK;
}

chap_status own_scratch_ok(chap_bs *h)
{
    if (h->no_hist_scratch && h->info.n_hist_cols > 0)
        return fail(h, CHAP_E_STATE,
                    "handle created with static_scratch_only: its passes run through "
                    "chap_bs_best_shift_static_scratch");
    return CHAP_OK;
}
}  // namespace chap

extern "C" {

void chap_options_default(chap_options *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->feas_tol = 1e-9;
    o->tenure = 10;
    o->graph_iters = 64;
    o->max_iters = 1000;
    o->stop_at_feasible = 1;
}

const char *chap_status_str(chap_status s)
{
    switch (s) {
    case CHAP_OK: return "ok";
    case CHAP_E_INVALID: return "invalid argument";
    case CHAP_E_OOM: return "out of memory";
    case CHAP_E_CUDA: return "CUDA error";
    case CHAP_E_TIMEOUT: return "device wait timed out";
    case CHAP_E_STATE: return "invalid state";
    case CHAP_E_UNSUPPORTED: return "unsupported";
    default: return "unknown status";
    }
}

const char *chap_last_error(const chap_bs *h) { return h ? h->err.c_str() : "NULL handle"; }

chap_status chap_bs_destroy(chap_bs *h)
{
    if (!h) return CHAP_OK;
    cudaStreamSynchronize(h->st);
    free_all(h);
    delete h;
    return CHAP_OK;
}

chap_status chap_bs_create(const chap_problem *p, const chap_options *opts, void *stream, chap_bs **out)
{
    if (!out) return CHAP_E_INVALID;
    *out = nullptr;
    chap_bs *h = new (std::nothrow) chap_bs();
    if (!h) return CHAP_E_OOM;
    std::string msg;
    chap_status vs = validate(p, msg);
    if (vs != CHAP_OK) {
        // report the message through a throw-away handle-less path
        std::fprintf(stderr, "chap_bs_create: %s\n", msg.c_str());
        delete h;
        return vs;
    }
    if (opts) h->opt = *opts; else chap_options_default(&h->opt);
    if (const char *f = std::getenv("CHAP_FAIL_ALLOC_AFTER")) h->fail_allocs_after = std::atol(f);
    if (!(h->opt.feas_tol >= 0.0) || h->opt.tenure < 0 || h->opt.graph_iters < 1 ||
        (h->opt.lazy_binary != 0 && h->opt.lazy_binary != 1) ||
        (h->opt.static_scratch_only != 0 && h->opt.static_scratch_only != 1) ||
        h->opt.bin_kernel < 0 || h->opt.bin_kernel > 3 ||
        h->opt.bin_block_rows < 0 || h->opt.bin_block_rows > kBlkRows ||
        h->opt.shard_count < 0 || (h->opt.shard_count > 1 && (h->opt.shard_rank < 0 ||
                                                              h->opt.shard_rank >= h->opt.shard_count))) {
        delete h;
        return CHAP_E_INVALID;
    }
    h->shard_count = std::max(1, (int)h->opt.shard_count);
    h->shard_rank = h->shard_count > 1 ? (int)h->opt.shard_rank : 0;
    h->st = static_cast<cudaStream_t>(stream);
    const int n = p->n, m = p->m;
    h->n = n;
    h->m = m;
    h->lb.assign(p->lb, p->lb + n);
    h->ub.assign(p->ub, p->ub + n);
    h->obj.assign(n, 0.0);
    if (p->obj) h->obj.assign(p->obj, p->obj + n);
    h->vtype.assign(p->vtype, p->vtype + n);

    // ---- row normalisation and integrality
    std::vector<double> sign(m), rhs(m), eps(m);
    std::vector<uint8_t> rint(m);
    h->row_eq.assign(m, 0);
    h->nrow_base.assign(m, 0);
    int mn = 0;
    int64_t nnz_int = 0, m_fp = 0;
    for (int i = 0; i < m; ++i) {
        sign[i] = p->sense[i] == CHAP_ROW_GE ? -1.0 : 1.0;
        h->row_eq[i] = p->sense[i] == CHAP_ROW_EQ;
        h->nrow_base[i] = mn;
        mn += h->row_eq[i] ? 2 : 1;
        double b = p->rhs[i];
        bool integral = is_int_value(b) && std::fabs(b) <= kLim52;
        double mag = std::fabs(b);
        for (int64_t e = p->row_ptr[i]; e < p->row_ptr[i + 1] && integral; ++e) {
            double a = p->row_val[e];
            int j = p->col_idx[e];
            if (!is_int_value(a) || std::fabs(a) > 2147483647.0) integral = false;
            else if (p->vtype[j] == CHAP_VAR_CONT) integral = false;
            else if (!std::isfinite(p->lb[j]) || !std::isfinite(p->ub[j])) integral = false;
            else {
                mag += std::fabs(a) * std::max(std::fabs(p->lb[j]), std::fabs(p->ub[j]));
                if (!(mag <= kLim52)) integral = false;
            }
        }
        rint[i] = integral ? 1 : 0;
        h->row_int.push_back(rint[i]);
        h->row_le.push_back(p->sense[i] == CHAP_ROW_LE);
        rhs[i] = sign[i] * b;
        eps[i] = integral ? 0.0 : h->opt.feas_tol * std::max(1.0, std::fabs(b));
        if (integral) nnz_int += p->row_ptr[i + 1] - p->row_ptr[i];
        else ++m_fp;
    }
    h->m_norm = mn;

    // rows of the residual kernel: the integral ones in index order, then the
    // others by decreasing length (32 rows of like length per CTA)
    std::vector<int> res_rows;
    res_rows.reserve(m);
    for (int i = 0; i < m; ++i)
        if (rint[i]) res_rows.push_back(i);
    const int n_res_int = (int)res_rows.size();
    for (int i = 0; i < m; ++i)
        if (!rint[i]) res_rows.push_back(i);
    std::stable_sort(res_rows.begin() + n_res_int, res_rows.end(), [&](int a, int b) {
        return p->row_ptr[a + 1] - p->row_ptr[a] > p->row_ptr[b + 1] - p->row_ptr[b];
    });

    std::vector<double> row_val(p->nnz);
    for (int i = 0; i < m; ++i)
        for (int64_t e = p->row_ptr[i]; e < p->row_ptr[i + 1]; ++e) row_val[e] = sign[i] * p->row_val[e];

    // ---- classify variables
    //  binary: streamed by T_BIN tiles; other columns by breakpoint entries (one
    //  per normalised half plus the bounds): one warp per column (T_NB,
    //  <= kWarpSortMax), then multi-CTA counting sort (integer, domain <=
    //  kHistMaxDomain) or CTA bitonic (<= kCtaMaxEntries).
    std::vector<std::vector<int>> kind_vars(T_NUM_KINDS);
    std::vector<int> fixed_vars;
    std::vector<int> cta_n;  // padded entry count of each CTA-sorted column, in kind order
    std::vector<int> nb_cap; // breakpoint entries of each T_NB column, in kind order
    int n_bin = 0, n_int = 0, n_cont = 0;
    int max_col = 0;
    int64_t nb_bytes_vars = 0;
    for (int j = 0; j < n; ++j) {
        const int len = (int)(p->col_ptr[j + 1] - p->col_ptr[j]);
        max_col = std::max(max_col, len);
        if (h->lb[j] == h->ub[j]) { fixed_vars.push_back(j); continue; }
        const int t = h->vtype[j];
        if (t == CHAP_VAR_BIN) { ++n_bin; kind_vars[T_BIN].push_back(j); continue; }
        (t == CHAP_VAR_INT ? n_int : n_cont)++;
        nb_bytes_vars += 16;
        const bool fin = std::isfinite(h->lb[j]) && std::isfinite(h->ub[j]);
        const double dom = fin ? h->ub[j] - h->lb[j] + 1 : INFINITY;
        // sort entries: one per normalised half (a continuous variable's half
        // may add a second, the marker of its tight point) and the bounds
        const int per_half = t == CHAP_VAR_CONT ? 2 : 1;
        int64_t E = (std::isfinite(h->lb[j]) ? 1 : 0) + (std::isfinite(h->ub[j]) ? 1 : 0);
        for (int64_t e = p->col_ptr[j]; e < p->col_ptr[j + 1]; ++e) E += (h->row_eq[p->row_idx[e]] ? 2 : 1) * per_half;
        int k;
        if (E <= (t == CHAP_VAR_CONT ? kWarpListMax : kWarpSortMax)) k = T_NB;
        else if (t == CHAP_VAR_INT && dom <= kHistMaxDomain) k = T_NB_HIST;
        else if (E <= kCtaMaxEntries) k = T_NB_CTA;
        else k = T_NB_LONG;
        if (k == T_NB_CTA) cta_n.push_back(std::max(next_pow2((int)E), kCtaThreads));
        if (k == T_NB) nb_cap.push_back((int)E);
        kind_vars[k].push_back(j);
    }
    {
        // binary columns (four to a warp): order them by length
        std::vector<int> &bv = kind_vars[T_BIN];
        std::stable_sort(bv.begin(), bv.end(), [&](int x, int y) {
            return p->col_ptr[x + 1] - p->col_ptr[x] < p->col_ptr[y + 1] - p->col_ptr[y];
        });
    }
    {
        // short columns (four to a warp): order them by type, then entry count,
        // so that the columns of one warp have similar lengths and row mixes
        std::vector<int> ord(nb_cap.size());
        for (size_t q = 0; q < ord.size(); ++q) ord[q] = (int)q;
        std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
            const int tx = h->vtype[kind_vars[T_NB][x]], ty = h->vtype[kind_vars[T_NB][y]];
            return tx != ty ? tx < ty : nb_cap[x] < nb_cap[y];
        });
        std::vector<int> vs(ord.size()), cs(ord.size());
        for (size_t q = 0; q < ord.size(); ++q) { vs[q] = kind_vars[T_NB][ord[q]]; cs[q] = nb_cap[ord[q]]; }
        kind_vars[T_NB].swap(vs);
        nb_cap.swap(cs);
    }
    const int n_fixed = (int)fixed_vars.size();
    // column shard (Sec. 3.1's pass split by columns over several GPUs): this
    // handle evaluates every world-th column of each class (round robin over
    // the class order, so every shard gets a like mix of lengths); the others
    // stay in the store for the apply and sit, unevaluated, after the fixed
    // variables
    std::vector<int> other_vars;
    if (h->shard_count > 1) {
        auto keep = [&](std::vector<int> &v, std::vector<int> *aux) {
            std::vector<int> kept, kept_aux;
            for (size_t q = 0; q < v.size(); ++q) {
                if ((int)(q % (size_t)h->shard_count) == h->shard_rank) {
                    kept.push_back(v[q]);
                    if (aux) kept_aux.push_back((*aux)[q]);
                } else {
                    other_vars.push_back(v[q]);
                }
            }
            v.swap(kept);
            if (aux) aux->swap(kept_aux);
        };
        for (int k = 0; k < T_NUM_KINDS; ++k)
            keep(kind_vars[k], k == T_NB ? &nb_cap : (k == T_NB_CTA ? &cta_n : nullptr));
    }
    std::vector<int> var_list;
    var_list.reserve(n);
    std::vector<int> kind_base(T_NUM_KINDS + 1, 0);
    for (int k = 0; k < T_NUM_KINDS; ++k) {
        kind_base[k] = (int)var_list.size();
        var_list.insert(var_list.end(), kind_vars[k].begin(), kind_vars[k].end());
    }
    kind_base[T_NUM_KINDS] = (int)var_list.size();
    var_list.insert(var_list.end(), fixed_vars.begin(), fixed_vars.end());
    var_list.insert(var_list.end(), other_vars.begin(), other_vars.end());
    std::vector<int> vpos(n);
    for (int q = 0; q < n; ++q) vpos[var_list[q]] = q;

    // ---- split CSC in var_list order (integral rows: int32 coefficients; others: double)
    //      inside each part the rows of one normalised half come first and the
    //      "=" rows (two halves) after them, from ci_eq[q] / cf_eq[q] on
    std::vector<int> ci_ptr(n + 1, 0), cf_ptr(n + 1, 0), ci_eq(n, 0), cf_eq(n, 0);
    std::vector<int> ci_row, ci_val, cf_row;
    std::vector<double> cf_val;
    ci_row.reserve(nnz_int);
    ci_val.reserve(nnz_int);
    cf_row.reserve(p->nnz - nnz_int);
    cf_val.reserve(p->nnz - nnz_int);
    for (int q = 0; q < n; ++q) {
        const int j = var_list[q];
        for (int eq = 0; eq < 2; ++eq) {
            if (eq) {
                ci_eq[q] = (int)ci_row.size();
                cf_eq[q] = (int)cf_row.size();
            }
            for (int64_t e = p->col_ptr[j]; e < p->col_ptr[j + 1]; ++e) {
                const int i = p->row_idx[e];
                if ((h->row_eq[i] != 0) != (eq != 0)) continue;
                const double a = sign[i] * p->col_val[e];
                if (rint[i]) { ci_row.push_back(i); ci_val.push_back((int)a); }
                else { cf_row.push_back(i); cf_val.push_back(a); }
            }
        }
        ci_ptr[q + 1] = (int)ci_row.size();
        cf_ptr[q + 1] = (int)cf_row.size();
    }

    // ---- work tiles
    std::vector<Tile> tiles_cta, tiles_hist;
    std::vector<HistCol> hcols;
    int max_cta_n = 0, max_hist_d = 0;
    int64_t hist_bins = 0;
    for (int k = T_NB; k < T_NUM_KINDS; ++k) {
        const int base = kind_base[k], cnt = kind_base[k + 1] - base;
        if (cnt == 0) continue;
        if (k == T_NB || k == T_NB_LONG) {
            continue;  // one warp per column, no tiles; long lists: tiled below
        } else if (k == T_NB_CTA) {
            for (int b = 0; b < cnt; ++b) {
                max_cta_n = std::max(max_cta_n, cta_n[b]);
                tiles_cta.push_back(Tile{k, base + b, base + b + 1, cta_n[b]});
            }
        } else {
            for (int b = 0; b < cnt; ++b) {
                const int q = base + b, j = var_list[q];
                HistCol hc{};
                hc.pos = q;
                const int D = (int)(h->ub[j] - h->lb[j]) + 1;
                max_hist_d = std::max(max_hist_d, D);
                hc.bin_off = hist_bins;
                hist_bins += D;
                hc.e_mid = ci_ptr[q + 1] - ci_ptr[q];
                hc.e_end = hc.e_mid + (cf_ptr[q + 1] - cf_ptr[q]);
                hc.nchunks = std::max(1, (hc.e_end + kHistChunk - 1) / kHistChunk);
                const int hidx = (int)hcols.size();
                for (int c = 0; c < hc.nchunks; ++c) tiles_hist.push_back(Tile{k, hidx, hidx + 1, c});
                hcols.push_back(hc);
            }
        }
    }
    // long lists: runs of kLongRun sorted entries per chunk of kLongChunk
    // nonzeros, padded to a power of two runs per column
    std::vector<LongCol> lcols;
    std::vector<Tile> tiles_lgen, tiles_lscan;
    long long long_entries = 0;
    int long_rounds = 0, long_tiles = 0;
    for (int q = kind_base[T_NB_LONG]; q < kind_base[T_NB_LONG + 1]; ++q) {
        LongCol lc{};
        lc.pos = q;
        lc.e_mid = ci_ptr[q + 1] - ci_ptr[q];
        lc.e_end = lc.e_mid + (cf_ptr[q + 1] - cf_ptr[q]);
        lc.nchunks = std::max(1, (lc.e_end + kLongChunk - 1) / kLongChunk);
        int runs = 1, rounds = 0;
        while (runs < lc.nchunks) { runs <<= 1; ++rounds; }
        lc.runs = runs;
        long_rounds = std::max(long_rounds, rounds);
        lc.ntiles = (int)((long long)runs * kLongRun / kLongTile);
        lc.tile0 = long_tiles;
        long_tiles += lc.ntiles;
        lc.base = long_entries;
        long_entries += (long long)runs * kLongRun;
        const int li = (int)lcols.size();
        for (int c = 0; c < runs; ++c) tiles_lgen.push_back(Tile{T_NB_LONG, li, li + 1, c});
        for (int t2 = 0; t2 < lc.ntiles; ++t2) tiles_lscan.push_back(Tile{T_NB_LONG, li, li + 1, t2});
        lcols.push_back(lc);
    }
    const int nb_cols = kind_base[T_NB + 1] - kind_base[T_NB];
    // lanes per short non-binary column: 4 when the columns are short on average
    int nb_G = 8;
    if (nb_cols > 0) {
        const double mean = (double)((ci_ptr[kind_base[T_NB + 1]] - ci_ptr[kind_base[T_NB]]) +
                                     (cf_ptr[kind_base[T_NB + 1]] - cf_ptr[kind_base[T_NB]])) / nb_cols;
        nb_G = mean <= kNbG4MaxLen ? 4 : 8;
    }
    const int n_tn = nb_cols > 0 ? nb_grid_size(nb_cols, nb_G) : 0;
    const int bin_cols = kind_base[T_BIN + 1] - kind_base[T_BIN];
    // lanes per binary column: enough for one or two rounds of a mean-length column
    int bin_G = 8;
    if (bin_cols > 0) {
        const double mean = (double)((ci_ptr[kind_base[T_BIN + 1]] - ci_ptr[kind_base[T_BIN]]) +
                                     (cf_ptr[kind_base[T_BIN + 1]] - cf_ptr[kind_base[T_BIN]])) / bin_cols;
        bin_G = (mean <= kBinG2MaxLen && bin_cols >= kBinG2MinCols) ? 2
                : mean <= kBinG4MaxLen ? 4 : (mean <= kBinG8MaxLen ? 8 : 16);
    }
    // row-wise binary flips (k_eval_bin_rows) on request (option bin_kernel:
    // 0 automatic = column-wise, which measured faster on every workload here;
    // 1 column-wise; 2 row-wise); the kept scores of lazy_binary stay column-wise
    const bool lazy_bin = h->opt.lazy_binary != 0 && bin_cols > 0;
    const bool bin_rows = bin_cols > 0 && !lazy_bin && h->opt.bin_kernel == 2;
    const int rb_blocks = bin_rows ? (bin_cols + kRbCols - 1) / kRbCols : 0;
    std::vector<int> rb_rows[2], rb_eptr[2], rb_split[2], rb_vi;
    std::vector<unsigned short> rb_col[2];
    std::vector<unsigned char> rb_own[2];
    std::vector<double> rb_vf;
    int64_t rb_bytes = 0;
    if (bin_rows) {
        // per block and store (0: integral rows, 1: others): the rows with
        // entries in the block, in order, and their entries
        struct Part { std::vector<int> rows, eptr; std::vector<unsigned short> col; std::vector<int> vi; std::vector<double> vf; int last = -1; };
        std::vector<Part> parts(2 * (size_t)rb_blocks);
        for (int i = 0; i < m; ++i) {
            const int t = rint[i] ? 0 : 1;
            for (int64_t e = p->row_ptr[i]; e < p->row_ptr[i + 1]; ++e) {
                const int q = vpos[p->col_idx[e]];
                if (q >= bin_cols) continue;
                const int b = q % rb_blocks;
                Part &pt = parts[2 * (size_t)b + t];
                if (pt.last != i) { pt.last = i; pt.rows.push_back(i); pt.eptr.push_back((int)pt.col.size()); }
                pt.col.push_back((unsigned short)(q / rb_blocks));
                if (t == 0) pt.vi.push_back((int)row_val[e]); else pt.vf.push_back(row_val[e]);
            }
        }
        for (int t = 0; t < 2; ++t) {
            rb_eptr[t].push_back(0);
            for (int b = 0; b < rb_blocks; ++b) {
                Part &pt = parts[2 * (size_t)b + t];
                const int r0 = (int)rb_rows[t].size(), e0 = (int)rb_col[t].size();
                const int nrow = (int)pt.rows.size(), nent = (int)pt.col.size();
                rb_rows[t].insert(rb_rows[t].end(), pt.rows.begin(), pt.rows.end());
                for (int k = 1; k < nrow; ++k) rb_eptr[t].push_back(e0 + pt.eptr[k]);
                if (nrow) rb_eptr[t].push_back(e0 + nent);
                rb_col[t].insert(rb_col[t].end(), pt.col.begin(), pt.col.end());
                if (t == 0) rb_vi.insert(rb_vi.end(), pt.vi.begin(), pt.vi.end());
                else rb_vf.insert(rb_vf.end(), pt.vf.begin(), pt.vf.end());
                // the CTAs of the block's cluster split its rows by entries
                for (int r = 0; r <= kRbCluster; ++r) {
                    const int64_t want = (int64_t)nent * r / kRbCluster;
                    int k = 0;
                    while (k < nrow && (int64_t)pt.eptr[k] < want) ++k;
                    rb_split[t].push_back(r == kRbCluster ? r0 + nrow : r0 + k);
                }
                // each entry's row place inside the 32-row chunk it is processed in
                // (chunks aligned at the start of every CTA's share)
                rb_own[t].resize(rb_col[t].size());
                for (int r = 0; r < kRbCluster; ++r) {
                    const int s0 = rb_split[t][rb_split[t].size() - (kRbCluster + 1) + r];
                    const int s1 = rb_split[t][rb_split[t].size() - (kRbCluster + 1) + r + 1];
                    for (int k = s0; k < s1; ++k)
                        for (int e = rb_eptr[t][k]; e < rb_eptr[t][k + 1]; ++e)
                            rb_own[t][e] = (unsigned char)((k - s0) & 31);
                }
                rb_bytes += (int64_t)nent * (3 + (t == 0 ? 4 : 8)) + (int64_t)nrow * (8 + (t == 0 ? 16 : 32));
                std::vector<int>().swap(pt.rows);
                std::vector<int>().swap(pt.eptr);
                std::vector<unsigned short>().swap(pt.col);
                std::vector<int>().swap(pt.vi);
                std::vector<double>().swap(pt.vf);
            }
        }
        rb_bytes += (int64_t)bin_cols * (4 + 8 + 8);
    }
    // row-blocked binary flips (k_eval_bin_blk): option bin_kernel 3, or the
    // library's choice (0) when the rows form few blocks, there are many binary
    // columns and a column meets a block in enough entries on average (kept
    // scores and the row-wise option keep their kernels)
    const int blk_rows = h->opt.bin_block_rows > 0 ? (int)h->opt.bin_block_rows : kBlkRows;
    const int nblk = m > 0 ? (m + blk_rows - 1) / blk_rows : 0;
    const int64_t nnz_bin = (int64_t)(ci_ptr[bin_cols] - ci_ptr[0]) + (cf_ptr[bin_cols] - cf_ptr[0]);
    bool bin_blk = false;
    if (bin_cols > 0 && !lazy_bin && !bin_rows && nblk > 0) {
        if (h->opt.bin_kernel == 3) {
            if (bin_cols >= kBlkMaxPos) {
                delete h;
                std::fprintf(stderr, "chap_bs_create: row-blocked binary flips name at most %d binary positions\n",
                             kBlkMaxPos - 1);
                return CHAP_E_UNSUPPORTED;
            }
            bin_blk = true;
        } else if (h->opt.bin_kernel == 0) {
            bin_blk = nblk <= kBlkMaxBlocks && bin_cols >= kBlkMinCols && bin_cols < kBlkMaxPos &&
                      (double)nnz_bin / ((double)nblk * bin_cols) >= kBlkMinSeg;
        }
    }
    const int blk_nfin = bin_blk ? (bin_cols + kBlkFin - 1) / kBlkFin : 0;
    std::vector<unsigned> blk_metaI, blk_metaF;
    std::vector<int> blk_valI;
    std::vector<double> blk_valF;
    std::vector<BlkItem> blk_items;
    int64_t blk_bytes = 0;
    if (bin_blk) {
        // per block the entries of each stream ordered by position, then row:
        // count, offsets (cI / cF: first entry of position q in block b), fill
        std::vector<int> cI((size_t)nblk * (bin_cols + 1), 0), cF((size_t)nblk * (bin_cols + 1), 0);
        for (int q = 0; q < bin_cols; ++q) {
            for (int e = ci_ptr[q]; e < ci_ptr[q + 1]; ++e) ++cI[(size_t)(ci_row[e] / blk_rows) * (bin_cols + 1) + q];
            for (int e = cf_ptr[q]; e < cf_ptr[q + 1]; ++e) ++cF[(size_t)(cf_row[e] / blk_rows) * (bin_cols + 1) + q];
        }
        int tI = 0, tF = 0;
        for (int b = 0; b < nblk; ++b)
            for (int q = 0; q <= bin_cols; ++q) {
                const size_t k = (size_t)b * (bin_cols + 1) + q;
                const int a = cI[k], c = cF[k];
                cI[k] = tI;
                cF[k] = tF;
                tI += a;
                tF += c;
            }
        blk_metaI.resize(tI);
        blk_valI.resize(tI);
        blk_metaF.resize(tF);
        blk_valF.resize(tF);
        {
            std::vector<int> fI(cI), fF(cF);
            for (int q = 0; q < bin_cols; ++q) {
                for (int e = ci_ptr[q]; e < ci_ptr[q + 1]; ++e) {
                    const int b = ci_row[e] / blk_rows;
                    const int k = fI[(size_t)b * (bin_cols + 1) + q]++;
                    blk_metaI[k] = ((unsigned)q << kBlkRowBits) | (unsigned)(ci_row[e] - b * blk_rows);
                    blk_valI[k] = ci_val[e];
                }
                for (int e = cf_ptr[q]; e < cf_ptr[q + 1]; ++e) {
                    const int b = cf_row[e] / blk_rows;
                    const int k = fF[(size_t)b * (bin_cols + 1) + q]++;
                    blk_metaF[k] = ((unsigned)q << kBlkRowBits) | (unsigned)(cf_row[e] - b * blk_rows);
                    blk_valF[k] = cf_val[e];
                }
            }
        }
        // padding: the kernel reads four entries at a time, past a stream's end
        blk_metaI.resize(blk_metaI.size() + 8, 0u);
        blk_valI.resize(blk_valI.size() + 8, 0);
        blk_metaF.resize(blk_metaF.size() + 8, 0u);
        blk_valF.resize(blk_valF.size() + 8, 0.0);
        // work items: every block gets CTAs in proportion to its work (an
        // integral entry 2, another 3, a position 1), at least one, one wave on
        // the device; each block's positions are cut into spans of like work
        int dev = 0, sms = 152;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            sms = 152;
        }
        auto work = [&](int b, int q) {   // work of block b's positions [0, q)
            const size_t k = (size_t)b * (bin_cols + 1);
            return 2LL * (cI[k + q] - cI[k]) + 3LL * (cF[k + q] - cF[k]) + q;
        };
        std::vector<int64_t> bw(nblk);
        int64_t tot = 0;
        for (int b = 0; b < nblk; ++b) { bw[b] = work(b, bin_cols); tot += bw[b]; }
        std::vector<int> ncta(nblk);
        int sum = 0;
        for (int b = 0; b < nblk; ++b) {
            ncta[b] = std::max<int>(1, (int)std::llround((double)sms * (double)bw[b] / (double)tot));
            ncta[b] = std::min(ncta[b], bin_cols);
            sum += ncta[b];
        }
        while (sum > std::max(sms, nblk)) {
            int bmax = 0;
            for (int b = 1; b < nblk; ++b)
                if (ncta[b] > ncta[bmax]) bmax = b;
            if (ncta[bmax] <= 1) break;
            --ncta[bmax];
            --sum;
        }
        for (int b = 0; b < nblk; ++b) {
            const size_t k = (size_t)b * (bin_cols + 1);
            int qa = 0;
            for (int part = 1; part <= ncta[b]; ++part) {
                int qb = bin_cols;
                if (part < ncta[b]) {
                    // first position at which the work reaches part / ncta of the block's
                    const int64_t want = bw[b] * part / ncta[b];
                    int lo = qa, hi = bin_cols;
                    while (lo < hi) {
                        const int mid = (lo + hi) / 2;
                        if (work(b, mid) >= want) hi = mid; else lo = mid + 1;
                    }
                    qb = lo;
                }
                if (qb > qa) blk_items.push_back(BlkItem{b, qa, qb, cI[k + qa], cI[k + qb], cF[k + qa], cF[k + qb], 0});
                qa = std::max(qa, qb);
            }
        }
        // algorithmic bytes of one launch: every entry once (word +
        // coefficient), every row state and its integrality flag once, per
        // position its variable, direction, tabu stamps and the accumulators
        // read and cleared
        blk_bytes = 8LL * tI + 12LL * tF + 33LL * m + (int64_t)bin_cols * (4 + 1 + 8 + 24);
    }
    const int n_tb = bin_blk ? blk_nfin
                   : bin_rows ? rb_blocks * kRbCluster : (bin_cols > 0 ? bin_grid_size(bin_cols, bin_G) : 0);
    const int n_tc = (int)tiles_cta.size();
    const int slot_hist = n_tb + n_tn + n_tc;
    for (size_t q = 0; q < hcols.size(); ++q) hcols[q].slot = slot_hist + (int)q;
    const int slot_long = slot_hist + (int)hcols.size();
    for (size_t q = 0; q < lcols.size(); ++q) lcols[q].slot = slot_long + (int)q;
    const int n_bb = slot_long + (int)lcols.size();

    // ---- device allocation
    Dev &d = h->dev;
    d.n = n;
    d.m = m;
    d.tenure = h->opt.tenure;
    // the nonzero arrays are padded by 8 elements: kernels read aligned groups of 8
    ci_row.resize(ci_row.size() + 8, 0); ci_val.resize(ci_val.size() + 8, 0);
    cf_row.resize(cf_row.size() + 8, 0); cf_val.resize(cf_val.size() + 8, 0.0);
    int *ci_ptr_d = dalloc<int>(h, n + 1), *ci_row_d = dalloc<int>(h, ci_row.size()), *ci_val_d = dalloc<int>(h, ci_val.size());
    int *cf_ptr_d = dalloc<int>(h, n + 1), *cf_row_d = dalloc<int>(h, cf_row.size());
    int *ci_eq_d = dalloc<int>(h, n), *cf_eq_d = dalloc<int>(h, n);
    double *cf_val_d = dalloc<double>(h, cf_val.size());
    long long *row_ptr_d = dalloc<long long>(h, m + 1);
    int *col_idx_d = dalloc<int>(h, p->nnz);
    double *row_val_d = dalloc<double>(h, p->nnz), *rhs_d = dalloc<double>(h, m), *eps_d = dalloc<double>(h, m);
    unsigned char *rint_d = dalloc<unsigned char>(h, m);
    int *nrb_d = dalloc<int>(h, m);
    int *resr_d = dalloc<int>(h, m);
    unsigned char *vt_d = dalloc<unsigned char>(h, n);
    double *lb_d = dalloc<double>(h, n), *ub_d = dalloc<double>(h, n), *obj_d = dalloc<double>(h, n);
    d.x = dalloc<double>(h, n);
    d.x_best = dalloc<double>(h, n);
    const bool lazy = h->opt.lazy_binary != 0 && bin_cols > 0;
    if (lazy) {
        d.lz_s = dalloc<long long>(h, bin_cols);
        d.lz_dc = dalloc<int>(h, bin_cols);
        d.lz_mark = dalloc<unsigned>(h, bin_cols);
        d.lz_list = dalloc<int>(h, bin_cols);
    }
    d.rs = dalloc<RowState>(h, m);
    d.tabu_inc = dalloc<int>(h, n);
    d.tabu_dec = dalloc<int>(h, n);
    d.ctl = dalloc<Ctl>(h, 1);
    int *vl_d = dalloc<int>(h, var_list.size());
    int *vpos_d = dalloc<int>(h, n);
    d.block_best = dalloc<Cand>(h, n_bb);
    d.n_block_best = n_bb;
    Tile *tc_d = dalloc<Tile>(h, tiles_cta.size());
    Tile *th_d = dalloc<Tile>(h, tiles_hist.size());
    HistCol *hc_d = dalloc<HistCol>(h, hcols.size());
    // the counting-sort scratch (none for a handle whose passes use the
    // library's fixed scratch)
    h->no_hist_scratch = h->opt.static_scratch_only != 0;
    d.hbins = dalloc<HBin>(h, h->no_hist_scratch ? 0 : hist_bins);
    h->hist_bins = hist_bins;
    d.hacc = dalloc<HistAcc>(h, h->no_hist_scratch ? 0 : hcols.size());
    const bool has_long = !lcols.empty();
    if (has_long) {
        d.lbuf0 = dalloc<SEntry>(h, (size_t)long_entries);
        d.lbuf1 = dalloc<SEntry>(h, (size_t)long_entries);
        d.lacc = dalloc<HistAcc>(h, lcols.size());
        d.ltsum = dalloc<long long>(h, long_tiles);
        d.ltsumc = dalloc<int>(h, long_tiles);
        d.lcand = dalloc<LCand>(h, long_tiles);
    }
    int *rbr_d[2] = {nullptr, nullptr}, *rbe_d[2] = {nullptr, nullptr}, *rbs_d[2] = {nullptr, nullptr};
    unsigned short *rbc_d[2] = {nullptr, nullptr};
    unsigned char *rbo_d[2] = {nullptr, nullptr};
    int *rbvi_d = nullptr;
    double *rbvf_d = nullptr;
    if (bin_rows) {
        for (int t = 0; t < 2; ++t) {
            rbr_d[t] = dalloc<int>(h, rb_rows[t].size());
            rbe_d[t] = dalloc<int>(h, rb_eptr[t].size());
            rbs_d[t] = dalloc<int>(h, rb_split[t].size());
            rbc_d[t] = dalloc<unsigned short>(h, rb_col[t].size());
            rbo_d[t] = dalloc<unsigned char>(h, rb_own[t].size());
        }
        rbvi_d = dalloc<int>(h, rb_vi.size());
        rbvf_d = dalloc<double>(h, rb_vf.size());
    }
    BinBlk bbd{};
    if (bin_blk) {
        d.bup = dalloc<unsigned char>(h, bin_cols);
        d.n_bup = bin_cols;
        bbd.nblk = nblk;
        bbd.rows = blk_rows;
        bbd.n_items = (int)blk_items.size();
        bbd.n_fin = blk_nfin;
        bbd.items = dalloc<BlkItem>(h, blk_items.size());
        bbd.metaI = dalloc<unsigned>(h, blk_metaI.size());
        bbd.metaF = dalloc<unsigned>(h, blk_metaF.size());
        bbd.valI = dalloc<int>(h, blk_valI.size());
        bbd.valF = dalloc<double>(h, blk_valF.size());
        bbd.acc_s = dalloc<long long>(h, bin_cols);
        bbd.acc_dc = dalloc<int>(h, bin_cols);
    }
    const bool blk_ok = !bin_blk || (d.bup && bbd.items && bbd.metaI && bbd.metaF && bbd.valI && bbd.valF &&
                                     bbd.acc_s && bbd.acc_dc);
    LongCol *lc_d = dalloc<LongCol>(h, lcols.size());
    Tile *tlg_d = dalloc<Tile>(h, tiles_lgen.size()), *tls_d = dalloc<Tile>(h, tiles_lscan.size());
    d.n_long = (int)lcols.size();
    h->t_rec = dalloc<chap_move_record>(h, kMaxRecords);
    h->t_obj = dalloc<double>(h, 1 + 128);
    h->t_xhat = dalloc<double>(h, n);
    h->t_s = dalloc<long long>(h, n);
    h->t_dc = dalloc<int>(h, n);
    h->t_w = dalloc<int>(h, mn);
    h->t_r = dalloc<double>(h, mn);
    h->t_tabu = dalloc<long long>(h, n);
    bool ok = ci_ptr_d && ci_row_d && ci_val_d && cf_ptr_d && cf_row_d && cf_val_d && ci_eq_d && cf_eq_d && row_ptr_d && col_idx_d &&
              row_val_d && rhs_d && eps_d && rint_d && nrb_d && resr_d && vt_d && lb_d && ub_d && obj_d && d.x && d.x_best && d.rs &&
              d.tabu_inc && d.tabu_dec && d.ctl && vl_d && vpos_d && d.block_best && tc_d && th_d && hc_d &&
              d.hbins && d.hacc && h->t_rec && h->t_obj && h->t_xhat && h->t_s && h->t_dc && h->t_w && h->t_r && h->t_tabu &&
              (!lazy || (d.lz_s && d.lz_dc && d.lz_mark && d.lz_list)) && lc_d && tlg_d && tls_d &&
              (!has_long || (d.lbuf0 && d.lbuf1 && d.lacc && d.ltsum && d.ltsumc && d.lcand)) &&
              (!bin_rows || (rbr_d[0] && rbr_d[1] && rbe_d[0] && rbe_d[1] && rbs_d[0] && rbs_d[1] && rbc_d[0] &&
                             rbc_d[1] && rbo_d[0] && rbo_d[1] && rbvi_d && rbvf_d));
    ok = ok && blk_ok;
    if (ok && cudaMallocHost(&h->h_ctl, sizeof(Ctl)) != cudaSuccess) { cudaGetLastError(); h->h_ctl = nullptr; ok = false; }
    if (ok && cudaStreamCreateWithFlags(&h->cap_st, cudaStreamNonBlocking) != cudaSuccess) { cudaGetLastError(); ok = false; }
    for (int k = 0; k < 3 && ok; ++k)
        if (cudaStreamCreateWithFlags(&h->plan.side[k], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->plan.ev_join[k], cudaEventDisableTiming) != cudaSuccess) { cudaGetLastError(); ok = false; }
    if (ok && cudaEventCreateWithFlags(&h->plan.ev_fork, cudaEventDisableTiming) != cudaSuccess) { cudaGetLastError(); ok = false; }
    for (int k = 0; k < 10 && ok; ++k)
        if (cudaEventCreate(&h->plan.pev[k]) != cudaSuccess) { cudaGetLastError(); ok = false; }
    if (!ok) {
        free_all(h);
        delete h;
        return CHAP_E_OOM;
    }
    d.ci_ptr = ci_ptr_d; d.ci_row = ci_row_d; d.ci_val = ci_val_d;
    d.cf_ptr = cf_ptr_d; d.cf_row = cf_row_d; d.cf_val = cf_val_d;
    d.ci_eq = ci_eq_d; d.cf_eq = cf_eq_d;
    d.row_ptr = row_ptr_d; d.col_idx = col_idx_d; d.row_val = row_val_d;
    d.rhs = rhs_d; d.eps = eps_d; d.row_int = rint_d; d.nrow_base = nrb_d;
    d.res_rows = resr_d; d.n_res_int = n_res_int; d.m_norm = mn;
    d.vtype = vt_d; d.lb = lb_d; d.ub = ub_d; d.obj = obj_d;
    d.var_list = vl_d;
    d.vpos = vpos_d;
    d.hcols = hc_d;
    d.lcols = lc_d;
    cudaStream_t st = h->st;
    std::vector<long long> rp(p->row_ptr, p->row_ptr + m + 1);
    cudaError_t e = cudaSuccess;
#define UP(dst, src, cnt) if (e == cudaSuccess) e = h2d(dst, src, cnt, st)
    UP(ci_ptr_d, ci_ptr.data(), n + 1); UP(ci_row_d, ci_row.data(), ci_row.size()); UP(ci_val_d, ci_val.data(), ci_val.size());
    UP(cf_ptr_d, cf_ptr.data(), n + 1); UP(cf_row_d, cf_row.data(), cf_row.size()); UP(cf_val_d, cf_val.data(), cf_val.size());
    UP(ci_eq_d, ci_eq.data(), n); UP(cf_eq_d, cf_eq.data(), n);
    UP(row_ptr_d, rp.data(), m + 1); UP(col_idx_d, p->col_idx, p->nnz); UP(row_val_d, row_val.data(), p->nnz);
    UP(rhs_d, rhs.data(), m); UP(eps_d, eps.data(), m); UP(rint_d, rint.data(), m); UP(nrb_d, h->nrow_base.data(), m); UP(resr_d, res_rows.data(), m);
    UP(vt_d, p->vtype, n); UP(lb_d, p->lb, n); UP(ub_d, p->ub, n); UP(obj_d, h->obj.data(), n);
    UP(vl_d, var_list.data(), var_list.size()); UP(vpos_d, vpos.data(), n);
    UP(tc_d, tiles_cta.data(), tiles_cta.size());
    UP(th_d, tiles_hist.data(), tiles_hist.size()); UP(hc_d, hcols.data(), hcols.size());
    UP(lc_d, lcols.data(), lcols.size());
    for (int t = 0; t < 2 && bin_rows; ++t) {
        UP(rbr_d[t], rb_rows[t].data(), rb_rows[t].size()); UP(rbe_d[t], rb_eptr[t].data(), rb_eptr[t].size());
        UP(rbs_d[t], rb_split[t].data(), rb_split[t].size()); UP(rbc_d[t], rb_col[t].data(), rb_col[t].size());
        UP(rbo_d[t], rb_own[t].data(), rb_own[t].size());
    }
    if (bin_rows) { UP(rbvi_d, rb_vi.data(), rb_vi.size()); UP(rbvf_d, rb_vf.data(), rb_vf.size()); }
    UP(tlg_d, tiles_lgen.data(), tiles_lgen.size()); UP(tls_d, tiles_lscan.data(), tiles_lscan.size());
    if (bin_blk) {
        UP(const_cast<BlkItem *>(bbd.items), blk_items.data(), blk_items.size());
        UP(const_cast<unsigned *>(bbd.metaI), blk_metaI.data(), blk_metaI.size());
        UP(const_cast<unsigned *>(bbd.metaF), blk_metaF.data(), blk_metaF.size());
        UP(const_cast<int *>(bbd.valI), blk_valI.data(), blk_valI.size());
        UP(const_cast<double *>(bbd.valF), blk_valF.data(), blk_valF.size());
        if (e == cudaSuccess) e = cudaMemsetAsync(bbd.acc_s, 0, sizeof(long long) * (size_t)bin_cols, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(bbd.acc_dc, 0, sizeof(int) * (size_t)bin_cols, st);
    }
#undef UP
    if (e == cudaSuccess && has_long) e = cudaMemsetAsync(d.lacc, 0, sizeof(HistAcc) * lcols.size(), st);
    if (e == cudaSuccess && hist_bins > 0 && !h->no_hist_scratch)
        e = cudaMemsetAsync(d.hbins, 0, sizeof(HBin) * hist_bins, st);
    if (e == cudaSuccess && !hcols.empty() && !h->no_hist_scratch)
        e = cudaMemsetAsync(d.hacc, 0, sizeof(HistAcc) * hcols.size(), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.ctl, 0, sizeof(Ctl), st);
    if (e == cudaSuccess && lazy) e = cudaMemsetAsync(d.lz_mark, 0, sizeof(unsigned) * bin_cols, st);
    if (e == cudaSuccess && lazy) e = launch_lazy_init(d, st);
    LaunchPlan &pl = h->plan;
    pl.lazy = lazy ? 1 : 0;
    pl.lazy_mark_blocks = 64;
    pl.bin_cols = bin_cols; pl.n_bin = n_tb; pl.bin_G = bin_G;
    pl.bin_rows = bin_rows ? 1 : 0;
    pl.bin_blk = bin_blk ? 1 : 0;
    pl.bb = bbd;
    pl.rb = RowBin{rb_blocks, 0, rbr_d[0], rbe_d[0], rbc_d[0], rbo_d[0], rbvi_d, rbr_d[1], rbe_d[1], rbc_d[1],
                   rbo_d[1], rbvf_d, rbs_d[0], rbs_d[1]};
    pl.nb_q0 = kind_base[T_NB]; pl.nb_cols = nb_cols; pl.nb_grid = n_tn; pl.nb_G = nb_G;
    pl.tiles_cta = tc_d; pl.n_cta = n_tc; pl.cta_smem = max_cta_n * 20;
    pl.tiles_hist = th_d; pl.n_hist_tiles = (int)tiles_hist.size(); pl.hist_smem = max_hist_d * (int)sizeof(HBin);
    pl.slot_nb = n_tb; pl.slot_cta = n_tb + n_tn;
    pl.tiles_lgen = tlg_d; pl.n_lgen = (int)tiles_lgen.size();
    pl.tiles_lscan = tls_d; pl.n_lscan = (int)tiles_lscan.size();
    pl.long_rounds = long_rounds; pl.long_entries = long_entries;
    if (e == cudaSuccess) e = setup_kernel_attributes(pl);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        std::fprintf(stderr, "chap_bs_create: %s\n", cudaGetErrorString(e));
        free_all(h);
        delete h;
        return CHAP_E_CUDA;
    }
    pl.apply_blocks = (int)std::min<int64_t>(304, std::max<int64_t>(1, ((int64_t)m + kApplyThreads - 1) / kApplyThreads));
    pl.apply_move_blocks = (int)std::min<int64_t>(152, std::max<int64_t>(1, ((int64_t)max_col + kApplyMoveThreads - 1) / kApplyMoveThreads));

    chap_info &in = h->info;
    in.n = n; in.m = m; in.m_norm = mn;
    in.n_bin = n_bin; in.n_int = n_int; in.n_cont = n_cont; in.n_fixed = n_fixed;
    in.nnz = p->nnz; in.nnz_int_rows = nnz_int; in.nnz_fp_rows = p->nnz - nnz_int;
    in.eval_blocks = (bin_blk ? (int)blk_items.size() : n_tb) + n_tn + n_tc + (int)tiles_hist.size() + (int)tiles_lscan.size();
    in.n_hist_cols = (int)hcols.size();
    in.n_long_cols = (int)lcols.size();
    in.n_cta_cols = n_tc;
    // evaluation kernels (they also select the move), a selection kernel only
    // when none runs, the move apply and the weight bump
    in.launches_per_step = (n_tb > 0) + (bin_blk ? 1 : 0) + (n_tn > 0) + (n_tc > 0) + (!tiles_hist.empty()) + (n_bb == 0) + 2 +
                           (lazy ? 2 : 0) +   // kept binary scores: the scan and the marking kernel
                           (has_long ? 3 + long_rounds : 0);   // long lists: generation, merges, tile sums, scan
    // algorithmic bytes of one pass: every nonzero once (row + coefficient),
    // every row state and tolerance once, every active variable's state once.
    int64_t n_act = kind_base[T_NUM_KINDS];   // evaluated columns
    in.bytes_per_pass = 8 * nnz_int + 12 * (p->nnz - nnz_int) + 16LL * (m - m_fp) + 32LL * m_fp +
                        n_act * (8 /*x*/ + 8 /*column pointers*/ + 8 /*tabu*/ + 1 /*type*/) + nb_bytes_vars;
    // algorithmic bytes of one launch of the binary and short-column kernels:
    // their nonzeros (row + coefficient), the state of every row they touch
    // once, and per column its position entry, x, four part offsets and, for
    // the short columns, the bounds, the type and the two tabu stamps
    {
        auto kernel_bytes = [&](int q0, int q1, int64_t per_col) {
            std::vector<char> touched(m, 0);
            int64_t b = 8LL * (ci_ptr[q1] - ci_ptr[q0]) + 12LL * (cf_ptr[q1] - cf_ptr[q0]);
            for (int e = ci_ptr[q0]; e < ci_ptr[q1]; ++e) touched[ci_row[e]] = 1;
            for (int e = cf_ptr[q0]; e < cf_ptr[q1]; ++e) touched[cf_row[e]] = 1;
            for (int i = 0; i < m; ++i)
                if (touched[i]) b += rint[i] ? 16 : 32;
            return b + per_col * (q1 - q0);
        };
        in.grid_bin = bin_blk ? (int)blk_items.size() : n_tb;
        in.bin_row_blocks = bin_blk ? nblk : 0;
        in.bin_lanes = bin_G;
        in.grid_nb = n_tn;
        in.nb_lanes = nb_G;
        in.bytes_bin = !bin_cols ? 0 : bin_blk ? blk_bytes : bin_rows ? rb_bytes
                                                        : kernel_bytes(kind_base[T_BIN], kind_base[T_BIN + 1], 4 + 8 + 16);
        in.bin_rows = bin_rows ? 1 : 0;
        in.bytes_nb = nb_cols ? kernel_bytes(kind_base[T_NB], kind_base[T_NB + 1], 4 + 8 + 16 + 1 + 8 + 16) : 0;
        const int ncta = kind_base[T_NB_CTA + 1] - kind_base[T_NB_CTA];
        const int nhist = kind_base[T_NB_HIST + 1] - kind_base[T_NB_HIST];
        in.bytes_cta = ncta ? kernel_bytes(kind_base[T_NB_CTA], kind_base[T_NB_CTA + 1], 4 + 8 + 16 + 1 + 8 + 16) : 0;
        in.bytes_hist = nhist ? kernel_bytes(kind_base[T_NB_HIST], kind_base[T_NB_HIST + 1], 4 + 8 + 16 + 1 + 8 + 16) : 0;
    }

    std::vector<double> x0(n);
    for (int j = 0; j < n; ++j) x0[j] = std::min(std::max(0.0, h->lb[j]), h->ub[j]);
    chap_status s = load_state(h, x0.data(), nullptr, nullptr, nullptr, 0, 0, 0);
    if (s != CHAP_OK) {
        std::fprintf(stderr, "chap_bs_create: %s\n", h->err.c_str());
        free_all(h);
        delete h;
        return s;
    }
    *out = h;
    return CHAP_OK;
}

chap_status chap_bs_info(const chap_bs *h, chap_info *info)
{
    if (!h || !info) return CHAP_E_INVALID;
    *info = h->info;
    return CHAP_OK;
}

chap_status chap_bs_profile(chap_bs *h, int32_t enable)
{
    if (!h) return CHAP_E_INVALID;
    h->plan.profile = enable != 0;
    h->prof_valid = false;
    return CHAP_OK;
}

chap_status chap_bs_kernel_ms(chap_bs *h, float *ms)
{
    if (!h || !ms) return CHAP_E_INVALID;
    if (h->broken) return fail(h, CHAP_E_STATE, "handle unusable after a CUDA fault");
    if (!h->prof_valid) return fail(h, CHAP_E_STATE, "no profiled pass since chap_bs_profile(h, 1)");
    CK(h, cudaStreamSynchronize(h->st), "synchronise");
    const bool launched[5] = {h->plan.n_bin > 0, h->plan.nb_grid > 0, h->plan.n_cta > 0 || h->plan.n_lgen > 0,
                              h->plan.n_hist_tiles > 0, true};
    for (int k = 0; k < 5; ++k) {
        ms[k] = 0.0f;
        if (launched[k]) CK(h, cudaEventElapsedTime(&ms[k], h->plan.pev[2 * k], h->plan.pev[2 * k + 1]), "kernel timing");
    }
    return CHAP_OK;
}

chap_status chap_bs_set_state(chap_bs *h, const double *x, const int32_t *w, int32_t mem)
{
    if (!h) return CHAP_E_INVALID;
    if (mem != CHAP_MEM_HOST && mem != CHAP_MEM_DEVICE) return fail(h, CHAP_E_INVALID, "bad mem kind");
    if (mem == CHAP_MEM_HOST && x) return load_state(h, x, w, nullptr, nullptr, 0, 0, 0);
    // device arrays are checked on the host, so they are read back first
    std::vector<double> xh(h->n);
    std::vector<int> wh;
    if (x) CK(h, cudaMemcpy(xh.data(), x, sizeof(double) * h->n, cudaMemcpyDeviceToHost), "read x");
    else
        for (int j = 0; j < h->n; ++j) xh[j] = std::min(std::max(0.0, h->lb[j]), h->ub[j]);
    const int *wp = w;
    if (w && mem == CHAP_MEM_DEVICE) {
        wh.resize(h->m_norm);
        CK(h, cudaMemcpy(wh.data(), w, sizeof(int) * h->m_norm, cudaMemcpyDeviceToHost), "read w");
        wp = wh.data();
    }
    return load_state(h, xh.data(), wp, nullptr, nullptr, 0, 0, 0);
}

chap_status chap_bs_set_checkpoint(chap_bs *h, const double *x, const int32_t *w, const int64_t *tabu_inc,
                                   const int64_t *tabu_dec, int64_t iter, int64_t best_nviol)
{
    if (!h || !x || !w || !tabu_inc || !tabu_dec) return h ? fail(h, CHAP_E_INVALID, "NULL checkpoint array") : CHAP_E_INVALID;
    if (iter < 0 || iter > INT_MAX / 2) return fail(h, CHAP_E_INVALID, "iteration out of range");
    std::vector<int> ti(h->n), td(h->n);
    for (int j = 0; j < h->n; ++j) {
        if (tabu_inc[j] < 0 || tabu_inc[j] > INT_MAX || tabu_dec[j] < 0 || tabu_dec[j] > INT_MAX)
            return fail(h, CHAP_E_INVALID, "tabu stamp out of range");
        ti[j] = (int)tabu_inc[j];
        td[j] = (int)tabu_dec[j];
    }
    return load_state(h, x, w, ti.data(), td.data(), iter, best_nviol, 1);
}

chap_status chap_bs_get_state(chap_bs *h, double *x, int32_t *w, int64_t *tabu_inc, int64_t *tabu_dec,
                              int64_t *scalars, int32_t mem)
{
    if (!h) return CHAP_E_INVALID;
    if (mem != CHAP_MEM_HOST && mem != CHAP_MEM_DEVICE) return fail(h, CHAP_E_INVALID, "bad mem kind");
    cudaMemcpyKind k = mem == CHAP_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    Dev &d = h->dev;
    if (x && h->n) CK(h, cudaMemcpyAsync(x, d.x, sizeof(double) * h->n, k, h->st), "copy x");
    if (w && h->m) {
        CK(h, launch_unpack_w(d, h->t_w, h->st), "unpack w");
        CK(h, cudaMemcpyAsync(w, h->t_w, sizeof(int) * h->m_norm, k, h->st), "copy w");
    }
    if (tabu_inc && h->n) {
        CK(h, launch_tabu_convert(h->n, d.tabu_inc, h->t_tabu, h->st), "widen tabu");
        CK(h, cudaMemcpyAsync(tabu_inc, h->t_tabu, sizeof(long long) * h->n, k, h->st), "copy tabu");
    }
    if (tabu_dec && h->n) {
        if (tabu_inc) CK(h, cudaStreamSynchronize(h->st), "synchronise");
        CK(h, launch_tabu_convert(h->n, d.tabu_dec, h->t_tabu, h->st), "widen tabu");
        CK(h, cudaMemcpyAsync(tabu_dec, h->t_tabu, sizeof(long long) * h->n, k, h->st), "copy tabu");
    }
    if (scalars || mem == CHAP_MEM_HOST) {
        chap_status s = read_ctl(h);
        if (s != CHAP_OK) return s;
        if (scalars) {
            scalars[0] = h->h_ctl->iter;
            scalars[1] = h->h_ctl->nviol;
            scalars[2] = h->h_ctl->best_nviol;
            scalars[3] = h->h_ctl->feasible_iter;
            scalars[4] = h->h_ctl->moves;
            scalars[5] = h->h_ctl->bumps;
        }
    }
    return CHAP_OK;
}

chap_status chap_bs_residuals(chap_bs *h, double *r, int32_t mem)
{
    if (!h || !r) return h ? fail(h, CHAP_E_INVALID, "NULL output") : CHAP_E_INVALID;
    if (mem != CHAP_MEM_HOST && mem != CHAP_MEM_DEVICE) return fail(h, CHAP_E_INVALID, "bad mem kind");
    if (h->m == 0) return CHAP_OK;
    CK(h, launch_unpack_r(h->dev, h->t_r, h->st), "unpack residuals");
    CK(h, cudaMemcpyAsync(r, h->t_r, sizeof(double) * h->m_norm,
                          mem == CHAP_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, h->st), "copy residuals");
    if (mem == CHAP_MEM_HOST) CK(h, cudaStreamSynchronize(h->st), "synchronise");
    return CHAP_OK;
}

chap_status chap_bs_best_shift(chap_bs *h, double *xhat, int64_t *score_half, int32_t *dnviol, chap_move *best,
                               int32_t mem)
{
    if (!h) return CHAP_E_INVALID;
    if (h->broken) return fail(h, CHAP_E_STATE, "handle unusable after a CUDA fault");
    if (mem != CHAP_MEM_HOST && mem != CHAP_MEM_DEVICE) return fail(h, CHAP_E_INVALID, "bad mem kind");
    if (own_scratch_ok(h) != CHAP_OK) return CHAP_E_STATE;
    VarOut o{nullptr, nullptr, nullptr};
    bool host = mem == CHAP_MEM_HOST;
    if (xhat) o.xhat = host ? h->t_xhat : xhat;
    if (score_half) o.s = host ? h->t_s : reinterpret_cast<long long *>(score_half);
    if (dnviol) o.dc = host ? h->t_dc : dnviol;
    CK(h, launch_eval_gated(h->dev, h->plan, o, 0, h->st), "best-shift kernels");
    CK(h, launch_select_gated(h->dev, h->plan, 0, h->st), "selection kernel");
    if (h->plan.profile) h->prof_valid = true;
    if (host && h->n) {
        if (xhat) CK(h, cudaMemcpyAsync(xhat, h->t_xhat, sizeof(double) * h->n, cudaMemcpyDeviceToHost, h->st), "copy xhat");
        if (score_half) CK(h, cudaMemcpyAsync(score_half, h->t_s, sizeof(long long) * h->n, cudaMemcpyDeviceToHost, h->st), "copy scores");
        if (dnviol) CK(h, cudaMemcpyAsync(dnviol, h->t_dc, sizeof(int) * h->n, cudaMemcpyDeviceToHost, h->st), "copy dnviol");
    }
    if (best || host) {
        chap_status s = read_ctl(h);
        if (s != CHAP_OK) return s;
        if (best) {
            const Ctl &c = *h->h_ctl;
            best->var = c.mv_var;
            best->dnviol = c.mv_dc;
            best->score_half = c.mv_s;
            best->old_value = c.mv_old;
            best->new_value = c.mv_new;
        }
    }
    return CHAP_OK;
}

chap_status chap_bs_best_shift_static_scratch(chap_bs *h, double *xhat, int64_t *score_half, int32_t *dnviol,
                                              chap_move *best, int32_t mem)
{
    if (!h) return CHAP_E_INVALID;
    if (h->broken) return fail(h, CHAP_E_STATE, "handle unusable after a CUDA fault");
    if (mem != CHAP_MEM_HOST && mem != CHAP_MEM_DEVICE) return fail(h, CHAP_E_INVALID, "bad mem kind");
    if (h->hist_bins > kStaticHistBins || h->info.n_hist_cols > kStaticHistCols)
        return fail(h, CHAP_E_UNSUPPORTED,
                    "counting-sort columns need " + std::to_string(h->hist_bins) + " bins and " +
                        std::to_string(h->info.n_hist_cols) + " accumulators; the static scratch holds " +
                        std::to_string(kStaticHistBins) + " and " + std::to_string(kStaticHistCols));
    Dev d = h->dev;
    CK(h, static_hist_scratch(&d.hbins, &d.hacc), "static scratch address");
    VarOut o{nullptr, nullptr, nullptr};
    bool host = mem == CHAP_MEM_HOST;
    if (xhat) o.xhat = host ? h->t_xhat : xhat;
    if (score_half) o.s = host ? h->t_s : reinterpret_cast<long long *>(score_half);
    if (dnviol) o.dc = host ? h->t_dc : dnviol;
    CK(h, launch_eval_gated(d, h->plan, o, 0, h->st), "best-shift kernels");
    CK(h, launch_select_gated(d, h->plan, 0, h->st), "selection kernel");
    if (h->plan.profile) h->prof_valid = true;
    if (host && h->n) {
        if (xhat) CK(h, cudaMemcpyAsync(xhat, h->t_xhat, sizeof(double) * h->n, cudaMemcpyDeviceToHost, h->st), "copy xhat");
        if (score_half) CK(h, cudaMemcpyAsync(score_half, h->t_s, sizeof(long long) * h->n, cudaMemcpyDeviceToHost, h->st), "copy scores");
        if (dnviol) CK(h, cudaMemcpyAsync(dnviol, h->t_dc, sizeof(int) * h->n, cudaMemcpyDeviceToHost, h->st), "copy dnviol");
    }
    if (best || host) {
        chap_status s = read_ctl(h);
        if (s != CHAP_OK) return s;
        if (best) {
            const Ctl &c = *h->h_ctl;
            best->var = c.mv_var;
            best->dnviol = c.mv_dc;
            best->score_half = c.mv_s;
            best->old_value = c.mv_old;
            best->new_value = c.mv_new;
        }
    }
    return CHAP_OK;
}

chap_status chap_bs_apply(chap_bs *h, int32_t var, double new_value)
{
    if (!h) return CHAP_E_INVALID;
    if (h->broken) return fail(h, CHAP_E_STATE, "handle unusable after a CUDA fault");
    if (var < -1 || var >= h->n) return fail(h, CHAP_E_INVALID, "variable index out of range");
    if (var >= 0) {
        if (!(new_value >= h->lb[var] && new_value <= h->ub[var])) return fail(h, CHAP_E_INVALID, "value outside the bounds");
        if (h->vtype[var] != CHAP_VAR_CONT && !is_int_value(new_value)) return fail(h, CHAP_E_INVALID, "fractional value of an integer variable");
        if (h->lb[var] == h->ub[var]) return fail(h, CHAP_E_INVALID, "fixed variable");
    }
    CK(h, launch_set_move(h->dev, var, new_value + 0.0, h->st), "set move");
    CK(h, launch_apply_gated(h->dev, h->plan, 0, h->st), "apply kernel");
    return CHAP_OK;
}

chap_status chap_bs_move_record(chap_bs *h, chap_move_record *rec, int32_t mem)
{
    if (!h || !rec) return h ? fail(h, CHAP_E_INVALID, "NULL record") : CHAP_E_INVALID;
    if (h->broken) return fail(h, CHAP_E_STATE, "handle unusable after a CUDA fault");
    if (mem != CHAP_MEM_HOST && mem != CHAP_MEM_DEVICE) return fail(h, CHAP_E_INVALID, "bad mem kind");
    if (mem == CHAP_MEM_DEVICE) {
        CK(h, launch_move_record(h->dev, rec, h->st), "move record");
        return CHAP_OK;
    }
    CK(h, launch_move_record(h->dev, h->t_rec, h->st), "move record");
    CK(h, cudaMemcpyAsync(rec, h->t_rec, sizeof(chap_move_record), cudaMemcpyDeviceToHost, h->st), "copy record");
    CK(h, cudaStreamSynchronize(h->st), "synchronise");
    return CHAP_OK;
}

chap_status chap_bs_apply_records(chap_bs *h, const chap_move_record *recs, int32_t k, int32_t mem)
{
    if (!h || !recs) return h ? fail(h, CHAP_E_INVALID, "NULL records") : CHAP_E_INVALID;
    if (h->broken) return fail(h, CHAP_E_STATE, "handle unusable after a CUDA fault");
    if (mem != CHAP_MEM_HOST && mem != CHAP_MEM_DEVICE) return fail(h, CHAP_E_INVALID, "bad mem kind");
    if (k < 1 || k > kMaxRecords) return fail(h, CHAP_E_INVALID, "record count out of range [1, 1024]");
    const chap_move_record *src = recs;
    if (mem == CHAP_MEM_HOST) {
        for (int q = 0; q < k; ++q) {
            const chap_move_record &r = recs[q];
            if (r.score_half > 0 && (r.var < 0 || r.var >= h->n))
                return fail(h, CHAP_E_INVALID, "record names a variable out of range");
        }
        CK(h, cudaMemcpyAsync(h->t_rec, recs, sizeof(chap_move_record) * k, cudaMemcpyHostToDevice, h->st),
           "copy records");
        src = h->t_rec;
    }
    CK(h, launch_apply_records(h->dev, src, k, h->st), "select record");
    CK(h, launch_apply_gated(h->dev, h->plan, 0, h->st), "apply kernel");
    return CHAP_OK;
}

chap_status chap_bs_step(chap_bs *h, chap_move *out)
{
    if (!h) return CHAP_E_INVALID;
    if (h->broken) return fail(h, CHAP_E_STATE, "handle unusable after a CUDA fault");
    if (own_scratch_ok(h) != CHAP_OK || whole_instance_ok(h) != CHAP_OK) return CHAP_E_STATE;
    VarOut o{nullptr, nullptr, nullptr};
    CK(h, launch_eval_gated(h->dev, h->plan, o, 0, h->st), "best-shift kernels");
    CK(h, launch_select_gated(h->dev, h->plan, 0, h->st), "selection kernel");
    if (h->plan.profile) h->prof_valid = true;
    CK(h, launch_apply_gated(h->dev, h->plan, 0, h->st), "apply kernel");
    if (out) {
        chap_status s = read_ctl(h);
        if (s != CHAP_OK) return s;
        const Ctl &c = *h->h_ctl;
        out->var = c.mv_var;
        out->dnviol = c.mv_dc;
        out->score_half = c.mv_s;
        out->old_value = c.mv_old;
        out->new_value = c.mv_new;
    }
    return CHAP_OK;
}

chap_status chap_bs_set_cutoff(chap_bs *h, int32_t row, double delta)
{
    if (!h) return CHAP_E_INVALID;
    if (h->broken) return fail(h, CHAP_E_STATE, "handle unusable after a CUDA fault");
    if (row < -1 || row >= h->m) return fail(h, CHAP_E_INVALID, "cutoff row out of range");
    int integral = 0;
    if (row >= 0) {
        if (!h->row_le[row]) return fail(h, CHAP_E_INVALID, "the cutoff row must be a \"<=\" row");
        integral = h->row_int[row];
        if (!(delta > 0.0) || !std::isfinite(delta)) return fail(h, CHAP_E_INVALID, "delta must be positive");
        if (integral && (!is_int_value(delta) || delta >= 2147483648.0))
            return fail(h, CHAP_E_INVALID, "delta on an integral cutoff row must be an integer in [1, 2^31)");
    }
    CK(h, launch_set_cutoff(h->dev, row >= 0, row, integral, row >= 0 ? delta : 0.0, h->opt.feas_tol, h->st),
       "set cutoff");
    return CHAP_OK;
}

chap_status chap_bs_get_cutoff(chap_bs *h, chap_cutoff_info *info, double *x_best, int32_t mem)
{
    if (!h) return CHAP_E_INVALID;
    if (h->broken) return fail(h, CHAP_E_STATE, "handle unusable after a CUDA fault");
    if (mem != CHAP_MEM_HOST && mem != CHAP_MEM_DEVICE) return fail(h, CHAP_E_INVALID, "bad mem kind");
    if (x_best && h->n)
        CK(h, cudaMemcpyAsync(x_best, h->dev.x_best, sizeof(double) * h->n,
                              mem == CHAP_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, h->st),
           "copy best solution");
    chap_status s = read_ctl(h);
    if (s != CHAP_OK) return s;
    if (info) {
        const Ctl &c = *h->h_ctl;
        info->solutions = c.cut_on ? c.cut_count : 0;
        info->best_iter = c.cut_on ? c.cut_iter : -1;
        info->best_objective = c.cut_on ? c.cut_obj : std::nan("");
        info->rhs = c.cut_on ? c.cut_rhs : std::nan("");
        info->row = c.cut_on ? c.cut_row : -1;
        info->reserved = 0;
    }
    return CHAP_OK;
}

chap_status chap_tabu_run(chap_bs *h, const chap_options *opts, chap_tabu_result *res)
{
    if (!h || !res) return h ? fail(h, CHAP_E_INVALID, "NULL result") : CHAP_E_INVALID;
    if (h->broken) return fail(h, CHAP_E_STATE, "handle unusable after a CUDA fault");
    if (own_scratch_ok(h) != CHAP_OK || whole_instance_ok(h) != CHAP_OK) return CHAP_E_STATE;
    chap_options o = opts ? *opts : h->opt;
    if (o.graph_iters < 1 || o.max_iters < 0) return fail(h, CHAP_E_INVALID, "bad run options");
    if (o.tenure != h->opt.tenure) return fail(h, CHAP_E_INVALID, "tenure is fixed at create time");
    auto t0 = std::chrono::steady_clock::now();
    chap_status s = read_ctl(h);
    if (s != CHAP_OK) return s;
    const long long iter0 = h->h_ctl->iter;
    const long long moves0 = h->h_ctl->moves;
    if (iter0 + o.max_iters + h->opt.tenure + 1 >= (long long)INT_MAX)
        return fail(h, CHAP_E_UNSUPPORTED, "iteration counter would exceed the 32-bit tabu stamps");
    Dev &d = h->dev;
    CK(h, launch_begin_run(d, o.max_iters, o.stop_at_feasible, h->st), "begin run");
    if (!h->gexec || h->g_iters != o.graph_iters) {
        if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
        cudaGraph_t g = nullptr;
        CK(h, cudaStreamBeginCapture(h->cap_st, cudaStreamCaptureModeThreadLocal), "begin capture");
        VarOut none{nullptr, nullptr, nullptr};
        cudaError_t e = cudaSuccess;
        for (int k = 0; k < o.graph_iters && e == cudaSuccess; ++k) {
            e = launch_eval_gated(d, h->plan, none, 1, h->cap_st);
            if (e == cudaSuccess) e = launch_select_gated(d, h->plan, 1, h->cap_st);
            if (e == cudaSuccess) e = launch_apply_gated(d, h->plan, 1, h->cap_st);
        }
        cudaError_t e2 = cudaStreamEndCapture(h->cap_st, &g);
        if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_fail(h, e, "capture"); }
        if (e2 != cudaSuccess) return cuda_fail(h, e2, "end capture");
        cudaError_t e3 = cudaGraphInstantiate(&h->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e3 != cudaSuccess) { h->gexec = nullptr; return cuda_fail(h, e3, "instantiate graph"); }
        h->g_iters = o.graph_iters;
    }
    long long max_replays = o.max_iters / o.graph_iters + 2;
    for (long long r = 0; r < max_replays; ++r) {
        CK(h, cudaGraphLaunch(h->gexec, h->st), "graph launch");
        s = read_ctl(h);
        if (s != CHAP_OK) return s;
        if (h->h_ctl->done) break;
    }
    auto t1 = std::chrono::steady_clock::now();
    const Ctl c = *h->h_ctl;
    res->iters = c.iter - iter0;
    res->moves = c.moves - moves0;
    res->feasible_iter = c.feasible_iter;
    res->final_nviol = c.nviol;
    res->best_nviol = c.best_nviol;
    res->seconds = std::chrono::duration<double>(t1 - t0).count();
    res->time_to_feasible_s = c.feasible_iter >= 0 ? (double)(c.t_feas_ns - c.t_start_ns) * 1e-9 : -1.0;
    // c^T x reduced on the device; only the value crosses to the host
    double obj = 0.0;
    if (h->n) {
        CK(h, launch_objective(d, h->t_obj, h->t_obj + 1, h->st), "objective");
        CK(h, cudaMemcpyAsync(&obj, h->t_obj, sizeof(double), cudaMemcpyDeviceToHost, h->st), "copy objective");
        CK(h, cudaStreamSynchronize(h->st), "synchronise");
    }
    res->objective = obj;
    return CHAP_OK;
}

}  // extern "C"
