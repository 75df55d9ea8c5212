// Batched tabu chains (growth path: many independent chains over several
// instances in one set of launches; Sec. 3.1, "Parallel Tabu Search
// Instances").  Every chain runs the plain exact iteration of the single-handle
// path -- best flip of every variable, best admissible move (larger score,
// then lower variable), incremental residual update or weight bump -- on
// all-binary instances whose rows are integral (int64 residuals, exact).
//
// Layout: the instances' columns are concatenated (each instance's columns
// ordered by length, rows as int32 local indices, single rows before "=" rows
// in every column); each chain owns its x (u8), tabu stamps and 16-byte row
// states.  One iteration of all chains is three launches:
//   k_batch_eval   persistent grid over (chain, 32-column tile) items; G lanes
//                  per column; a positive admissible flip is folded into the
//                  chain's best move with one 64-bit atomicMax on
//                  (score << 22 | ~var): larger score first, then lower var;
//   k_batch_apply  one CTA per chain: flips the chosen variable and updates its
//                  column's residuals, or flags a weight bump; finishes the
//                  chain's iteration (counters, best, feasibility, done flag);
//   k_batch_bump   chains flagged for a bump add 1 to the weight of every
//                  violated normalised row.
// The three are captured for K iterations into one CUDA graph and replayed.
// The autotuner times each (G, CTAs per SM) schedule on the batch itself.
#include "../../include/chap.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

namespace chap {
chap_status validate_problem(const chap_problem *p, std::string &msg);
}

namespace {

#define FULLMASK 0xffffffffu

constexpr int kTile = 32;            // columns of one work item
constexpr int kBThreads = 256;       // threads of the evaluation CTAs
constexpr int kApplyT = 256;         // threads of one chain's apply CTA
constexpr int kBumpBlocks = 8;       // bump CTAs per chain
constexpr int kVarBits = 22;         // variables per instance < 2^22
constexpr long long kScoreLimit = 1LL << 41;

struct __align__(16) BRow {
    long long r;  // residual of the first half (a.x - b, "<=" orientation)
    int w1, w2;   // weights of the halves (w2 = -1 for a single row)
};

struct __align__(16) BCtl {
    long long iter, nviol, best_nviol, feasible_iter, moves, bumps, max_iter;
    unsigned long long t_start_ns, t_feas_ns;
    unsigned long long best_key;     // best move of the current iteration (0: none)
    int done, bump, stop_at_feasible, pad;
};

struct BDev {
    int n_chains;
    int pad;
    long long total_items;
    // instances
    const int *inst_n, *inst_m, *inst_col0;
    // columns (concatenated, position order inside each instance)
    const int *cptr, *ceq, *crow, *cval;
    const int *var_of;   // position -> variable of the instance
    const int *pos_of;   // instance col0 + variable -> position
    // chains
    const int *ch_inst, *ch_tenure;
    const long long *ch_xoff, *ch_roff, *ch_item0;  // item0: first work item (prefix, n_chains + 1)
    unsigned char *x;
    int *tinc, *tdec;
    BRow *rs;
    BCtl *ctl;
    unsigned int *n_done;
};

__device__ __forceinline__ unsigned long long bglobal_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Penalty change of a half in half-weight units (Sec. 3.1, Scoring Functions):
// becomes violated -2, becomes satisfied +2, stays violated +1 when the
// residual falls and -1 when it grows.
__device__ __forceinline__ int bflip_f(bool v0, bool v1, bool dec)
{
    return 2 * ((int)v0 - (int)v1) + ((v0 && v1) ? (dec ? 1 : -1) : 0);
}

template <int G, bool EQ>
__device__ __forceinline__ void bpart(const BDev &d, const BRow *rs, int e0, int n, int nmax, int sub, bool up,
                                      long long &s, int &dc)
{
    for (int base = 0; base < nmax; base += G) {
        const int v = base + sub;
        const bool ok = v < n;
        const int row = ok ? __ldg(d.crow + e0 + v) : 0;
        const int av = ok ? __ldg(d.cval + e0 + v) : 0;
        const int4 st = ok ? __ldg(reinterpret_cast<const int4 *>(rs + row)) : make_int4(0, 0, 0, 0);
        const long long r = (long long)(((unsigned long long)(unsigned)st.y << 32) | (unsigned)st.x);
        const int ad = up ? av : -av;
        const long long r1 = r + ad;
        const bool v0 = r > 0, v1 = r1 > 0;
        s += (long long)bflip_f(v0, v1, ad < 0) * st.z;
        dc += (int)v1 - (int)v0;
        if (EQ) {
            const bool u0 = r < 0, u1 = r1 < 0;
            s += (long long)bflip_f(u0, u1, ad > 0) * st.w;
            dc += (int)u1 - (int)u0;
        }
    }
}

template <int G>
__device__ __forceinline__ int gmax(int v)
{
#pragma unroll
    for (int o = 16; o >= G; o >>= 1) v = max(v, __shfl_xor_sync(FULLMASK, v, o));
    return v;
}

template <int G>
__global__ void __launch_bounds__(kBThreads) k_batch_eval(BDev d)
{
    constexpr int CPW = 32 / G;   // columns per warp step
    const int lane = threadIdx.x & 31;
    const int g = lane / G, sub = lane & (G - 1);
    const long long nwarps = (long long)gridDim.x * (kBThreads / 32);
    for (long long it = (long long)blockIdx.x * (kBThreads / 32) + (threadIdx.x >> 5); it < d.total_items; it += nwarps) {
        // chain of the item: last c with ch_item0[c] <= it
        int lo = 0, hi = d.n_chains - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(d.ch_item0 + mid) <= it) lo = mid; else hi = mid - 1;
        }
        const int c = lo;
        BCtl *ctl = d.ctl + c;
        if (*(volatile int *)&ctl->done) continue;
        const int k = __ldg(d.ch_inst + c);
        const int n = __ldg(d.inst_n + k), col0 = __ldg(d.inst_col0 + k);
        const long long xoff = __ldg(d.ch_xoff + c);
        const BRow *rs = d.rs + __ldg(d.ch_roff + c);
        const long long iter = ctl->iter, nviol = ctl->nviol, bestnv = ctl->best_nviol;
        const int tile0 = (int)(it - __ldg(d.ch_item0 + c)) * kTile;
        for (int step = 0; step < kTile; step += CPW) {
            const int q = tile0 + step + g;   // position inside the instance
            const bool live = q < n;
            if (!__any_sync(FULLMASK, live)) break;
            const int gq = col0 + (live ? q : 0);
            const int e0 = __ldg(d.cptr + gq), em = __ldg(d.ceq + gq);
            const int e1 = live ? __ldg(d.cptr + gq + 1) : e0;
            const int ns = live ? em - e0 : 0, ne = live ? e1 - em : 0;
            const int j = __ldg(d.var_of + gq);
            const bool up = live && d.x[xoff + j] == 0;
            long long s = 0;
            int dc = 0;
            bpart<G, false>(d, rs, e0, ns, gmax<G>(ns), sub, up, s, dc);
            bpart<G, true>(d, rs, em, ne, gmax<G>(ne), sub, up, s, dc);
#pragma unroll
            for (int o = G >> 1; o > 0; o >>= 1) {
                s += __shfl_xor_sync(FULLMASK, s, o);
                dc += __shfl_xor_sync(FULLMASK, dc, o);
            }
            if (sub == 0 && live && s > 0) {
                const int stamp = up ? d.tinc[xoff + j] : d.tdec[xoff + j];
                if (iter >= (long long)stamp || nviol + (long long)dc < bestnv) {
                    const unsigned long long key =
                        ((unsigned long long)s << kVarBits) | (unsigned long long)((1 << kVarBits) - 1 - j);
                    if (key > *(volatile unsigned long long *)&ctl->best_key) atomicMax(&ctl->best_key, key);
                }
            }
        }
    }
}

__global__ void __launch_bounds__(kApplyT) k_batch_apply(BDev d)
{
    const int c = blockIdx.x;
    BCtl *ctl = d.ctl + c;
    __shared__ long long red[kApplyT / 32];
    if (ctl->done) {         // uniform for the CTA: only this kernel writes done
        if (threadIdx.x == 0) ctl->bump = 0;
        return;
    }
    const unsigned long long key = ctl->best_key;
    const int k = d.ch_inst[c];
    const long long xoff = d.ch_xoff[c];
    BRow *rs = d.rs + d.ch_roff[c];
    long long local = 0;
    int var = -1;
    bool up = false;
    if (key != 0ull) {
        var = (1 << kVarBits) - 1 - (int)(key & ((1ull << kVarBits) - 1));
        up = d.x[xoff + var] == 0;
        const int ad = up ? 1 : -1;
        const int gq = d.inst_col0[k] + d.pos_of[d.inst_col0[k] + var];
        const int e0 = d.cptr[gq], em = d.ceq[gq], e1 = d.cptr[gq + 1];
        for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
            BRow *p = rs + d.crow[e];
            const long long r0 = p->r;
            const long long r1 = r0 + (long long)d.cval[e] * ad;
            p->r = r1;
            local += (long long)(r1 > 0) - (long long)(r0 > 0);
            if (e >= em) local += (long long)(r1 < 0) - (long long)(r0 < 0);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(FULLMASK, local, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = local;
    __syncthreads();
    if (threadIdx.x != 0) return;
    long long t = 0;
    for (int w = 0; w < kApplyT / 32; ++w) t += red[w];
    const long long nv = ctl->nviol + t;
    const long long it = ctl->iter;
    ctl->nviol = nv;
    if (var >= 0) {
        d.x[xoff + var] = up ? 1 : 0;
        const int stamp = (int)(it + 1 + d.ch_tenure[c]);
        if (up) d.tdec[xoff + var] = stamp;
        else d.tinc[xoff + var] = stamp;
        ctl->moves += 1;
        ctl->bump = 0;
    } else {
        ctl->bumps += 1;
        ctl->bump = 1;
    }
    ctl->best_key = 0ull;
    ctl->iter = it + 1;
    if (nv < ctl->best_nviol) ctl->best_nviol = nv;
    if (nv == 0 && ctl->feasible_iter < 0) {
        ctl->feasible_iter = it + 1;
        ctl->t_feas_ns = bglobal_ns();
    }
    if ((ctl->stop_at_feasible && nv == 0) || it + 1 >= ctl->max_iter) {
        ctl->done = 1;
        atomicAdd(d.n_done, 1u);
    }
}

__global__ void k_batch_bump(BDev d)
{
    const int c = blockIdx.y;
    BCtl *ctl = d.ctl + c;
    if (!ctl->bump) return;
    const int m = d.inst_m[d.ch_inst[c]];
    BRow *rs = d.rs + d.ch_roff[c];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const BRow s = rs[i];
        if (s.r > 0) rs[i].w1 = s.w1 + 1;
        if (s.w2 >= 0 && s.r < 0) rs[i].w2 = s.w2 + 1;
    }
}

__global__ void k_batch_clear_bump(BDev d)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < d.n_chains) d.ctl[c].bump = 0;
}

__global__ void k_batch_begin(BDev d, long long max_iters, int stop_at_feasible)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d.n_chains) return;
    BCtl *ctl = d.ctl + c;
    ctl->max_iter = ctl->iter + max_iters;
    ctl->stop_at_feasible = stop_at_feasible;
    ctl->t_start_ns = bglobal_ns();
    if (ctl->nviol == 0) { ctl->feasible_iter = ctl->iter; ctl->t_feas_ns = ctl->t_start_ns; }
    else { ctl->feasible_iter = -1; ctl->t_feas_ns = 0; }
    ctl->bump = 0;
    ctl->best_key = 0ull;
    ctl->done = (max_iters <= 0 || (stop_at_feasible && ctl->nviol == 0)) ? 1 : 0;
    if (ctl->done) atomicAdd(d.n_done, 1u);
}

}  // namespace

// ------------------------------------------------------------------ host

struct chap_batch {
    cudaStream_t st = nullptr;
    int n_probs = 0, n_chains = 0;
    std::vector<void *> allocs;
    BDev dev{};
    // per chain, host
    std::vector<int> ch_inst, ch_tenure;
    std::vector<int> inst_n, inst_m;
    std::vector<long long> ch_xoff, ch_roff;
    std::vector<BRow> rs0;                 // initial row states of every chain (x = 0, unit weights)
    std::vector<BCtl> ctl0;
    std::vector<std::vector<double>> obj;
    long long total_x = 0, total_rows = 0;
    int max_col = 0;
    // schedule
    int G = 8, ctas_per_sm = 4, sms = 152;
    cudaGraphExec_t gexec = nullptr;
    int g_iters = 0, g_G = 0, g_ctas = 0;
    unsigned int *h_done = nullptr;  // pinned
    std::string err;
};

namespace {

chap_status bfail(chap_batch *b, chap_status s, const std::string &msg)
{
    if (b) b->err = msg;
    return s;
}

#define BCK(b, expr, what)                                                                   \
    do {                                                                                     \
        cudaError_t e_ = (expr);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            cudaGetLastError();                                                              \
            return bfail(b, CHAP_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e_)); \
        }                                                                                    \
    } while (0)

template <class T>
T *balloc(chap_batch *b, size_t count)
{
    void *p = nullptr;
    if (cudaMalloc(&p, sizeof(T) * std::max<size_t>(count, 1)) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    b->allocs.push_back(p);
    return static_cast<T *>(p);
}

void bfree(chap_batch *b)
{
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    for (void *p : b->allocs) cudaFree(p);
    b->allocs.clear();
    if (b->h_done) cudaFreeHost(b->h_done);
    b->h_done = nullptr;
}

cudaError_t launch_eval(const chap_batch *b, int G, int ctas, cudaStream_t st)
{
    const long long want = (b->dev.total_items + kBThreads / 32 - 1) / (kBThreads / 32);
    const int grid = (int)std::max<long long>(1, std::min<long long>((long long)b->sms * ctas, want));
    switch (G) {
    case 2: k_batch_eval<2><<<grid, kBThreads, 0, st>>>(b->dev); break;
    case 4: k_batch_eval<4><<<grid, kBThreads, 0, st>>>(b->dev); break;
    case 16: k_batch_eval<16><<<grid, kBThreads, 0, st>>>(b->dev); break;
    default: k_batch_eval<8><<<grid, kBThreads, 0, st>>>(b->dev); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_iteration(const chap_batch *b, int G, int ctas, cudaStream_t st)
{
    cudaError_t e = launch_eval(b, G, ctas, st);
    if (e != cudaSuccess) return e;
    k_batch_apply<<<b->n_chains, kApplyT, 0, st>>>(b->dev);
    k_batch_bump<<<dim3(kBumpBlocks, b->n_chains), 256, 0, st>>>(b->dev);
    return cudaGetLastError();
}

chap_status upload_state(chap_batch *b)
{
    BCK(b, cudaMemsetAsync(b->dev.x, 0, std::max<long long>(b->total_x, 1), b->st), "reset x");
    BCK(b, cudaMemsetAsync(b->dev.tinc, 0, sizeof(int) * std::max<long long>(b->total_x, 1), b->st), "reset tabu");
    BCK(b, cudaMemsetAsync(b->dev.tdec, 0, sizeof(int) * std::max<long long>(b->total_x, 1), b->st), "reset tabu");
    BCK(b, cudaMemcpyAsync(b->dev.rs, b->rs0.data(), sizeof(BRow) * b->rs0.size(), cudaMemcpyHostToDevice, b->st),
        "upload row states");
    BCK(b, cudaMemcpyAsync(b->dev.ctl, b->ctl0.data(), sizeof(BCtl) * b->ctl0.size(), cudaMemcpyHostToDevice, b->st),
        "upload control");
    BCK(b, cudaStreamSynchronize(b->st), "synchronise");
    return CHAP_OK;
}

}  // namespace

extern "C" {

chap_status chap_batch_create(const chap_problem *probs, int32_t n_probs, const int32_t *chain_prob,
                              const int32_t *chain_tenure, int32_t n_chains, void *stream, chap_batch **out)
{
    if (!out) return CHAP_E_INVALID;
    *out = nullptr;
    if (!probs || n_probs < 1 || !chain_prob || !chain_tenure || n_chains < 1) return CHAP_E_INVALID;
    chap_batch *b = new (std::nothrow) chap_batch();
    if (!b) return CHAP_E_OOM;
    b->st = static_cast<cudaStream_t>(stream);
    b->n_probs = n_probs;
    b->n_chains = n_chains;
    // ---- validate and normalise every instance (all binary, integral rows)
    std::vector<int> cptr{0}, ceq, crow, cval, var_of, pos_of, inst_col0;
    std::vector<std::vector<BRow>> rows0(n_probs);
    b->obj.resize(n_probs);
    int col_total = 0;
    for (int k = 0; k < n_probs; ++k) {
        const chap_problem *p = probs + k;
        std::string msg;
        chap_status s = chap::validate_problem(p, msg);
        if (s != CHAP_OK) {
            *out = nullptr;
            delete b;
            std::fprintf(stderr, "chap_batch_create: instance %d: %s\n", k, msg.c_str());
            return s;
        }
        if (p->n >= (1 << kVarBits)) { delete b; return CHAP_E_UNSUPPORTED; }
        const int n = p->n, m = p->m;
        std::vector<int> sign(m, 1), eq(m, 0);
        for (int j = 0; j < n; ++j)
            if (p->vtype[j] != CHAP_VAR_BIN) {
                std::fprintf(stderr, "chap_batch_create: instance %d: variable %d is not binary\n", k, j);
                delete b;
                return CHAP_E_UNSUPPORTED;
            }
        for (int i = 0; i < m; ++i) {
            if (p->sense[i] == CHAP_ROW_GE) sign[i] = -1;
            eq[i] = p->sense[i] == CHAP_ROW_EQ;
            if (!(std::floor(p->rhs[i]) == p->rhs[i] && std::fabs(p->rhs[i]) < 4.0e15)) {
                std::fprintf(stderr, "chap_batch_create: instance %d: row %d is not integral\n", k, i);
                delete b;
                return CHAP_E_UNSUPPORTED;
            }
            for (int64_t e = p->row_ptr[i]; e < p->row_ptr[i + 1]; ++e)
                if (!(std::floor(p->row_val[e]) == p->row_val[e] && std::fabs(p->row_val[e]) < 2147483647.0)) {
                    std::fprintf(stderr, "chap_batch_create: instance %d: row %d is not integral\n", k, i);
                    delete b;
                    return CHAP_E_UNSUPPORTED;
                }
        }
        // row states at x = 0: r = -b (orientation applied), unit weights
        rows0[k].resize(m);
        for (int i = 0; i < m; ++i) rows0[k][i] = BRow{-(long long)(sign[i] * p->rhs[i]), 1, eq[i] ? 1 : -1};
        // columns ordered by length; nonzeros single rows first, "=" rows after
        std::vector<int> ord(n);
        for (int j = 0; j < n; ++j) ord[j] = j;
        std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
            return p->col_ptr[x + 1] - p->col_ptr[x] < p->col_ptr[y + 1] - p->col_ptr[y];
        });
        inst_col0.push_back(col_total);
        pos_of.resize(col_total + n);
        for (int q = 0; q < n; ++q) {
            const int j = ord[q];
            var_of.push_back(j);
            pos_of[col_total + j] = q;
            b->max_col = std::max(b->max_col, (int)(p->col_ptr[j + 1] - p->col_ptr[j]));
            for (int pass = 0; pass < 2; ++pass) {
                if (pass == 1) ceq.push_back((int)crow.size());
                for (int64_t e = p->col_ptr[j]; e < p->col_ptr[j + 1]; ++e) {
                    const int i = p->row_idx[e];
                    if (eq[i] != pass) continue;
                    crow.push_back(i);
                    cval.push_back((int)(sign[i] * p->col_val[e]));
                }
            }
            cptr.push_back((int)crow.size());
        }
        col_total += n;
        b->inst_n.push_back(n);
        b->inst_m.push_back(m);
        b->obj[k].assign(p->obj, p->obj + n);
    }
    // ---- chains
    std::vector<long long> item0{0};
    long long xo = 0, ro = 0;
    for (int c = 0; c < n_chains; ++c) {
        const int k = chain_prob[c];
        if (k < 0 || k >= n_probs || chain_tenure[c] < 0) { delete b; return CHAP_E_INVALID; }
        b->ch_inst.push_back(k);
        b->ch_tenure.push_back(chain_tenure[c]);
        b->ch_xoff.push_back(xo);
        b->ch_roff.push_back(ro);
        xo += b->inst_n[k];
        ro += b->inst_m[k];
        item0.push_back(item0.back() + (b->inst_n[k] + kTile - 1) / kTile);
        b->rs0.insert(b->rs0.end(), rows0[k].begin(), rows0[k].end());
        long long nv = 0;
        for (const BRow &r : rows0[k]) nv += (r.r > 0) + (r.w2 >= 0 && r.r < 0);
        BCtl cz{};
        cz.nviol = nv;
        cz.best_nviol = nv;
        cz.feasible_iter = nv == 0 ? 0 : -1;
        b->ctl0.push_back(cz);
    }
    b->total_x = xo;
    b->total_rows = ro;
    // ---- device
    BDev &d = b->dev;
    d.n_chains = n_chains;
    d.total_items = item0.back();
    int *in_d = balloc<int>(b, n_probs), *im_d = balloc<int>(b, n_probs), *ic_d = balloc<int>(b, n_probs);
    int *cptr_d = balloc<int>(b, cptr.size()), *ceq_d = balloc<int>(b, ceq.size());
    int *crow_d = balloc<int>(b, crow.size()), *cval_d = balloc<int>(b, cval.size());
    int *vo_d = balloc<int>(b, var_of.size()), *po_d = balloc<int>(b, pos_of.size());
    int *chi_d = balloc<int>(b, n_chains), *cht_d = balloc<int>(b, n_chains);
    long long *chx_d = balloc<long long>(b, n_chains), *chr_d = balloc<long long>(b, n_chains);
    long long *chi0_d = balloc<long long>(b, item0.size());
    d.x = balloc<unsigned char>(b, xo);
    d.tinc = balloc<int>(b, xo);
    d.tdec = balloc<int>(b, xo);
    d.rs = balloc<BRow>(b, ro);
    d.ctl = balloc<BCtl>(b, n_chains);
    d.n_done = balloc<unsigned int>(b, 1);
    const bool ok = in_d && im_d && ic_d && cptr_d && ceq_d && crow_d && cval_d && vo_d && po_d && chi_d && cht_d &&
                    chx_d && chr_d && chi0_d && d.x && d.tinc && d.tdec && d.rs && d.ctl && d.n_done &&
                    cudaMallocHost(&b->h_done, sizeof(unsigned int)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        bfree(b);
        delete b;
        return CHAP_E_OOM;
    }
    cudaError_t e = cudaSuccess;
#define BUP(dst, v) if (e == cudaSuccess && !(v).empty()) e = cudaMemcpyAsync(dst, (v).data(), sizeof((v)[0]) * (v).size(), cudaMemcpyHostToDevice, b->st)
    BUP(in_d, b->inst_n); BUP(im_d, b->inst_m); BUP(ic_d, inst_col0);
    BUP(cptr_d, cptr); BUP(ceq_d, ceq); BUP(crow_d, crow); BUP(cval_d, cval); BUP(vo_d, var_of); BUP(po_d, pos_of);
    BUP(chi_d, b->ch_inst); BUP(cht_d, b->ch_tenure); BUP(chx_d, b->ch_xoff); BUP(chr_d, b->ch_roff); BUP(chi0_d, item0);
#undef BUP
    if (e == cudaSuccess) e = cudaMemsetAsync(d.n_done, 0, sizeof(unsigned int), b->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
    if (e != cudaSuccess) {
        std::fprintf(stderr, "chap_batch_create: %s\n", cudaGetErrorString(e));
        cudaGetLastError();
        bfree(b);
        delete b;
        return CHAP_E_CUDA;
    }
    d.inst_n = in_d; d.inst_m = im_d; d.inst_col0 = ic_d;
    d.cptr = cptr_d; d.ceq = ceq_d; d.crow = crow_d; d.cval = cval_d; d.var_of = vo_d; d.pos_of = po_d;
    d.ch_inst = chi_d; d.ch_tenure = cht_d; d.ch_xoff = chx_d; d.ch_roff = chr_d; d.ch_item0 = chi0_d;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        b->sms = 152;
    }
    chap_status s = upload_state(b);
    if (s != CHAP_OK) {
        std::fprintf(stderr, "chap_batch_create: %s\n", b->err.c_str());
        bfree(b);
        delete b;
        return s;
    }
    *out = b;
    return CHAP_OK;
}

chap_status chap_batch_destroy(chap_batch *b)
{
    if (!b) return CHAP_OK;
    bfree(b);
    delete b;
    return CHAP_OK;
}

chap_status chap_batch_reset(chap_batch *b)
{
    if (!b) return CHAP_E_INVALID;
    return upload_state(b);
}

chap_status chap_batch_run(chap_batch *b, int64_t max_iters, int32_t stop_at_feasible, int32_t graph_iters,
                           chap_chain_result *res, double *seconds)
{
    if (!b || max_iters < 0 || graph_iters < 1) return CHAP_E_INVALID;
    // scores must fit the packed move key: |s| <= 2 * max weight * column length
    std::vector<BCtl> h(b->n_chains);
    BCK(b, cudaMemcpyAsync(h.data(), b->dev.ctl, sizeof(BCtl) * b->n_chains, cudaMemcpyDeviceToHost, b->st), "read control");
    BCK(b, cudaStreamSynchronize(b->st), "synchronise");
    long long it_max = 0;
    for (const BCtl &c : h) it_max = std::max(it_max, c.iter);
    if ((double)(it_max + max_iters + 2) * 2.0 * (double)std::max(1, b->max_col) >= (double)kScoreLimit)
        return bfail(b, CHAP_E_UNSUPPORTED, "weights could outgrow the packed move key for this many iterations");
    const auto t0 = std::chrono::steady_clock::now();
    BCK(b, cudaMemsetAsync(b->dev.n_done, 0, sizeof(unsigned int), b->st), "reset done count");
    k_batch_begin<<<(b->n_chains + 255) / 256, 256, 0, b->st>>>(b->dev, max_iters, stop_at_feasible);
    BCK(b, cudaGetLastError(), "begin run");
    if (!b->gexec || b->g_iters != graph_iters || b->g_G != b->G || b->g_ctas != b->ctas_per_sm) {
        if (b->gexec) cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
        cudaStream_t cs;
        BCK(b, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "capture stream");
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        for (int k = 0; k < graph_iters && e == cudaSuccess; ++k) e = launch_iteration(b, b->G, b->ctas_per_sm, cs);
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->gexec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cs);
        BCK(b, e, "graph capture");
        b->g_iters = graph_iters;
        b->g_G = b->G;
        b->g_ctas = b->ctas_per_sm;
    }
    // a chain that stops early idles through the rest of its graph replay (its
    // kernels return at once); replay until every chain is done
    for (;;) {
        BCK(b, cudaGraphLaunch(b->gexec, b->st), "graph launch");
        BCK(b, cudaMemcpyAsync(b->h_done, b->dev.n_done, sizeof(unsigned int), cudaMemcpyDeviceToHost, b->st), "read done");
        BCK(b, cudaStreamSynchronize(b->st), "synchronise");
        if (*b->h_done >= (unsigned)b->n_chains) break;
    }
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (seconds) *seconds = secs;
    if (res) {
        BCK(b, cudaMemcpyAsync(h.data(), b->dev.ctl, sizeof(BCtl) * b->n_chains, cudaMemcpyDeviceToHost, b->st), "read control");
        BCK(b, cudaStreamSynchronize(b->st), "synchronise");
        for (int c = 0; c < b->n_chains; ++c) {
            res[c].iters = h[c].iter;
            res[c].moves = h[c].moves;
            res[c].feasible_iter = h[c].feasible_iter;
            res[c].final_nviol = h[c].nviol;
            res[c].best_nviol = h[c].best_nviol;
            res[c].time_to_feasible_s = h[c].feasible_iter >= 0 ? (h[c].t_feas_ns - h[c].t_start_ns) * 1e-9 : -1.0;
        }
    }
    return CHAP_OK;
}

chap_status chap_batch_autotune(chap_batch *b, int32_t iters, int32_t *chosen)
{
    if (!b || iters < 1) return CHAP_E_INVALID;
    // time every schedule for `iters` iterations from the initial state, keep the fastest
    const int Gs[4] = {2, 4, 8, 16};
    const int Cs[3] = {2, 4, 8};
    cudaEvent_t a, z;
    BCK(b, cudaEventCreate(&a), "event");
    BCK(b, cudaEventCreate(&z), "event");
    float best_ms = 1e30f;
    int bg = b->G, bc = b->ctas_per_sm;
    for (int gi = 0; gi < 4; ++gi)
        for (int ci = 0; ci < 3; ++ci) {
            chap_status s = upload_state(b);
            if (s != CHAP_OK) { cudaEventDestroy(a); cudaEventDestroy(z); return s; }
            k_batch_begin<<<(b->n_chains + 255) / 256, 256, 0, b->st>>>(b->dev, iters + 1, 0);
            cudaError_t e = launch_iteration(b, Gs[gi], Cs[ci], b->st);  // warm-up
            if (e == cudaSuccess) e = cudaEventRecord(a, b->st);
            for (int k = 0; k < iters && e == cudaSuccess; ++k) e = launch_iteration(b, Gs[gi], Cs[ci], b->st);
            if (e == cudaSuccess) e = cudaEventRecord(z, b->st);
            if (e == cudaSuccess) e = cudaEventSynchronize(z);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, z);
            if (e != cudaSuccess) {
                cudaEventDestroy(a);
                cudaEventDestroy(z);
                BCK(b, e, "autotune run");
            }
            if (ms < best_ms) { best_ms = ms; bg = Gs[gi]; bc = Cs[ci]; }
        }
    cudaEventDestroy(a);
    cudaEventDestroy(z);
    b->G = bg;
    b->ctas_per_sm = bc;
    if (chosen) { chosen[0] = bg; chosen[1] = bc; }
    return upload_state(b);
}

chap_status chap_batch_set_schedule(chap_batch *b, int32_t lanes_per_column, int32_t ctas_per_sm)
{
    if (!b || !(lanes_per_column == 2 || lanes_per_column == 4 || lanes_per_column == 8 || lanes_per_column == 16) ||
        ctas_per_sm < 1 ||
        ctas_per_sm > 32)
        return CHAP_E_INVALID;
    b->G = lanes_per_column;
    b->ctas_per_sm = ctas_per_sm;
    return CHAP_OK;
}

chap_status chap_batch_get_x(chap_batch *b, int32_t chain, double *x)
{
    if (!b || chain < 0 || chain >= b->n_chains || !x) return CHAP_E_INVALID;
    const int n = b->inst_n[b->ch_inst[chain]];
    std::vector<unsigned char> t(n);
    BCK(b, cudaMemcpyAsync(t.data(), b->dev.x + b->ch_xoff[chain], n, cudaMemcpyDeviceToHost, b->st), "read x");
    BCK(b, cudaStreamSynchronize(b->st), "synchronise");
    for (int j = 0; j < n; ++j) x[j] = t[j];
    return CHAP_OK;
}

const char *chap_batch_last_error(const chap_batch *b) { return b ? b->err.c_str() : ""; }

}  // extern "C"
