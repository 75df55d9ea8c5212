// Batched tabu chains (growth path: many independent chains over several
// instances in one set of launches; Sec. 3.1, "Parallel Tabu Search
// Instances").  Every chain runs the plain exact iteration of the single-handle
// path -- best flip of every variable, best admissible move (larger score,
// then lower variable), incremental residual update or weight bump -- on
// all-binary instances whose rows are integral (int64 residuals, exact).
//
// Layout: the instances' columns are concatenated (each instance's columns
// ordered by length, rows as int32 local indices, single rows before "=" rows
// in every column); each chain owns its incumbent x as a bitset (one bit per
// binary variable, 32-bit words; Sec. 3.1, "Memory Considerations", fourth
// point: the bitsets are kept in L2 with a persisting access-policy window),
// its tabu stamps and 16-byte row states.  One iteration of all chains has
// three phases:
//   eval   (chain, 32-column tile) items over the whole grid; G lanes per
//          column; a positive admissible flip is folded into the chain's best
//          move with one 64-bit atomicMax on (score << 22 | ~var): larger
//          score first, then lower variable;
//   apply  per chain: flips the chosen variable and updates its column's
//          residuals, or flags a weight bump; finishes the chain's iteration
//          (counters, best, feasibility, done flag);
//   bump   chains flagged for a bump add 1 to the weight of every violated
//          normalised row.
// Two schedules run them: three launches per iteration captured K times into
// one CUDA graph, or one persistent cooperative launch per K iterations whose
// phases are separated by software grid barriers (each wait bounded by a
// time limit; a wait that runs out stops the launch and the run returns
// CHAP_E_TIMEOUT).  The autotuner times the (G, CTAs per SM) schedules on the
// batch itself.
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

// Software grid barrier of the persistent schedule (sense by generation).
struct __align__(16) GridBar {
    unsigned int count;
    unsigned int gen;
    int error;      // set when a wait ran out: every CTA leaves the launch
    int pad;
};

struct BDev {
    int n_chains;
    int pad;
    long long total_items;
    long long total_rows;
    // instances
    const int *inst_n, *inst_m, *inst_col0;
    // columns (concatenated, position order inside each instance)
    const int *cptr, *ceq, *crow, *cval;
    const int *var_of;   // position -> variable of the instance
    const int *pos_of;   // instance col0 + variable -> position
    // chains
    const int *ch_inst, *ch_tenure;
    const long long *ch_xoff, *ch_roff, *ch_item0;  // xoff in bitset words; item0: first work item (prefix)
    unsigned int *x;     // incumbent bitsets
    int *tinc, *tdec;    // tabu stamps (indexed by chain variable offset)
    const long long *ch_voff;
    BRow *rs;
    BCtl *ctl;
    unsigned int *n_done;
    GridBar *bar;
};

// Loads of chain state.  Inside one launch of the three-launch schedule the
// state a phase reads does not change, so it may take the read-only path
// (ld.global.nc).  The persistent launch changes it between its phases, so
// it uses ordinary (coherent) loads: the grid barrier's release and acquire
// fences make the writes of the previous phase visible to them, which the
// read-only path does not promise.
template <bool P, class T>
__device__ __forceinline__ T ld_state(const T *p)
{
    if (P) return *p;
    return __ldg(p);
}

template <bool P>
__device__ __forceinline__ bool x_bit(const BDev &d, long long xoff, int j)
{
    return (ld_state<P>(d.x + xoff + (j >> 5)) >> (j & 31)) & 1u;
}

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

template <int G, bool EQ, bool P>
__device__ __forceinline__ void bpart(const BDev &d, const BRow *rs, int e0, int n, int nmax, int sub, bool up,
                                      long long &s, int &dc)
{
    for (int base = 0; base < nmax; base += G) {
        const int v = base + sub;
        const bool ok = v < n;
        const int row = ok ? __ldg(d.crow + e0 + v) : 0;
        const int av = ok ? __ldg(d.cval + e0 + v) : 0;
        const int4 *rp = reinterpret_cast<const int4 *>(rs + row);
        const int4 st = ok ? ld_state<P>(rp) : make_int4(0, 0, 0, 0);
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

// Evaluation of the work items of one iteration by the calling warps (all
// lanes); P: inside the persistent launch (state loads through L2).
template <int G, bool P>
__device__ __forceinline__ void eval_items(const BDev &d, long long first, long long stride)
{
    constexpr int CPW = 32 / G;   // columns per warp step
    const int lane = threadIdx.x & 31;
    const int g = lane / G, sub = lane & (G - 1);
    for (long long it = first; it < d.total_items; it += stride) {
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
        const long long xoff = __ldg(d.ch_xoff + c), voff = __ldg(d.ch_voff + c);
        const BRow *rs = d.rs + __ldg(d.ch_roff + c);
        const long long iter = ld_state<P>(&ctl->iter), nviol = ld_state<P>(&ctl->nviol);
        const long long bestnv = ld_state<P>(&ctl->best_nviol);
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
            const bool up = live && !x_bit<P>(d, xoff, j);
            long long s = 0;
            int dc = 0;
            bpart<G, false, P>(d, rs, e0, ns, gmax<G>(ns), sub, up, s, dc);
            bpart<G, true, P>(d, rs, em, ne, gmax<G>(ne), sub, up, s, dc);
#pragma unroll
            for (int o = G >> 1; o > 0; o >>= 1) {
                s += __shfl_xor_sync(FULLMASK, s, o);
                dc += __shfl_xor_sync(FULLMASK, dc, o);
            }
            if (sub == 0 && live && s > 0) {
                const int stamp = ld_state<P>(up ? d.tinc + voff + j : d.tdec + voff + j);
                if (iter >= (long long)stamp || nviol + (long long)dc < bestnv) {
                    const unsigned long long key =
                        ((unsigned long long)s << kVarBits) | (unsigned long long)((1 << kVarBits) - 1 - j);
                    if (key > *(volatile unsigned long long *)&ctl->best_key) atomicMax(&ctl->best_key, key);
                }
            }
        }
    }
}

template <int G>
__global__ void __launch_bounds__(kBThreads) k_batch_eval(BDev d)
{
    eval_items<G, false>(d, (long long)blockIdx.x * (kBThreads / 32) + (threadIdx.x >> 5),
                         (long long)gridDim.x * (kBThreads / 32));
}

// Apply of chain c's move (or its bump flag) by all threads of the calling
// CTA, and the end of its iteration; red: shared scratch of blockDim / 32.
template <bool P>
__device__ void apply_chain(const BDev &d, int c, long long *red)
{
    BCtl *ctl = d.ctl + c;
    if (*(volatile int *)&ctl->done) {   // uniform for the CTA: only this phase writes done
        __syncthreads();
        if (threadIdx.x == 0) ctl->bump = 0;
        return;
    }
    // the best move key was built with atomics (in L2)
    const unsigned long long key = __ldcg(&ctl->best_key);
    const int k = d.ch_inst[c];
    const long long xoff = d.ch_xoff[c], voff = d.ch_voff[c];
    BRow *rs = d.rs + d.ch_roff[c];
    long long local = 0;
    int var = -1;
    bool up = false;
    if (key != 0ull) {
        var = (1 << kVarBits) - 1 - (int)(key & ((1ull << kVarBits) - 1));
        up = !x_bit<P>(d, xoff, var);
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
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        const long long nv = ctl->nviol + t;
        const long long it = ctl->iter;
        ctl->nviol = nv;
        if (var >= 0) {
            atomicXor(d.x + xoff + (var >> 5), 1u << (var & 31));
            const int stamp = (int)(it + 1 + d.ch_tenure[c]);
            if (up) d.tdec[voff + var] = stamp;
            else d.tinc[voff + var] = stamp;
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
    __syncthreads();
}

__global__ void __launch_bounds__(kApplyT) k_batch_apply(BDev d)
{
    __shared__ long long red[kApplyT / 32];
    apply_chain<false>(d, blockIdx.x, red);
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

// Grid barrier of the persistent launch: the last CTA to arrive releases the
// others; a CTA whose wait runs past limit_ns (globaltimer), or that sees
// another CTA's error, returns false and the launch ends.
__device__ bool grid_sync(GridBar *b, unsigned long long limit_ns)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        bool ok = true;
        const unsigned int g = *(volatile unsigned int *)&b->gen;
        __threadfence();
        if (atomicAdd(&b->count, 1u) == gridDim.x - 1) {
            b->count = 0;
            __threadfence();
            atomicAdd(&b->gen, 1u);
        } else {
            const unsigned long long t0 = bglobal_ns();
            while (*(volatile unsigned int *)&b->gen == g) {
                if (*(volatile int *)&b->error) { ok = false; break; }
                if (bglobal_ns() - t0 > limit_ns) {
                    atomicExch(&b->error, 1);
                    ok = false;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok && !*(volatile int *)&b->error;
    }
    __syncthreads();
    return s_ok != 0;
}

// Persistent schedule: `iters` iterations of every chain in one cooperative
// launch (all CTAs resident), phases separated by grid barriers.
template <int G>
__global__ void __launch_bounds__(kBThreads) k_batch_persistent(BDev d, int iters, unsigned long long limit_ns)
{
    __shared__ long long red[kBThreads / 32];
    const long long warps = (long long)gridDim.x * (kBThreads / 32);
    const long long wid = (long long)blockIdx.x * (kBThreads / 32) + (threadIdx.x >> 5);
    for (int k = 0; k < iters; ++k) {
        // every CTA reads the count from L2 after the same barrier: uniform
        if (atomicOr(d.n_done, 0u) >= (unsigned)d.n_chains) return;
        eval_items<G, true>(d, wid, warps);
        if (!grid_sync(d.bar, limit_ns)) return;
        for (int c = blockIdx.x; c < d.n_chains; c += gridDim.x) apply_chain<true>(d, c, red);
        if (!grid_sync(d.bar, limit_ns)) return;
        // weight bumps: the rows of every chain flagged for one, over the whole grid
        for (int c = 0; c < d.n_chains; ++c) {
            if (!ld_state<true>(&d.ctl[c].bump)) continue;   // set in the apply phase, before the barrier
            const int m = __ldg(d.inst_m + __ldg(d.ch_inst + c));
            BRow *rs = d.rs + __ldg(d.ch_roff + c);
            for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
                BRow *p = rs + i;
                const int4 v = *reinterpret_cast<const int4 *>(p);
                const long long r = (long long)(((unsigned long long)(unsigned)v.y << 32) | (unsigned)v.x);
                if (r > 0) p->w1 = v.z + 1;
                if (v.w >= 0 && r < 0) p->w2 = v.w + 1;
            }
        }
        if (!grid_sync(d.bar, limit_ns)) return;
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
    std::vector<long long> ch_xoff, ch_roff, ch_voff;   // bitset words / rows / variables
    std::vector<BRow> rs0;                 // initial row states of every chain (x = 0, unit weights)
    std::vector<BCtl> ctl0;
    std::vector<std::vector<double>> obj;
    long long total_x = 0, total_rows = 0, total_words = 0;
    int max_col = 0;
    // schedule
    int G = 8, ctas_per_sm = 4, sms = 152;
    int persistent = 1;                       // one cooperative launch per graph segment
    unsigned long long bar_limit_ns = 2000000000ull;   // bound of one grid-barrier wait
    bool broken = false;                      // a barrier wait ran out: state invalid until reset
    size_t l2_prev = 0;                       // persisting-L2 limit before this batch raised it
    bool l2_set = false;
    size_t max_window = 0;                    // largest access-policy window of the device (0: none)
    cudaGraphExec_t gexec = nullptr;
    int g_iters = 0, g_G = 0, g_ctas = 0, g_persistent = -1;
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
    if (b->l2_set) {
        cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, b->l2_prev);
        cudaGetLastError();
        b->l2_set = false;
    }
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    for (void *p : b->allocs) cudaFree(p);
    b->allocs.clear();
    if (b->h_done) cudaFreeHost(b->h_done);
    b->h_done = nullptr;
}

// Launch attributes: the incumbent bitsets as a persisting L2 window (and,
// for the persistent schedule, a cooperative launch: every CTA resident).
int launch_attrs(const chap_batch *b, bool cooperative, cudaLaunchAttribute *at)
{
    int n = 0;
    if (b->max_window > 0) {
        at[n].id = cudaLaunchAttributeAccessPolicyWindow;
        at[n].val.accessPolicyWindow.base_ptr = b->dev.x;
        at[n].val.accessPolicyWindow.num_bytes =
            std::min((size_t)std::max<long long>(b->total_words, 1) * sizeof(unsigned int), b->max_window);
        at[n].val.accessPolicyWindow.hitRatio = 1.0f;
        at[n].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
        at[n].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
        ++n;
    }
    if (cooperative) {
        at[n].id = cudaLaunchAttributeCooperative;
        at[n].val.cooperative = 1;
        ++n;
    }
    return n;
}

template <class K, class... A>
cudaError_t launch_ex(const chap_batch *b, K kern, int grid, int threads, bool cooperative, cudaStream_t st, A... args)
{
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute at[2];
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = launch_attrs(b, cooperative, at);
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

cudaError_t launch_eval(const chap_batch *b, int G, int ctas, cudaStream_t st)
{
    const long long want = (b->dev.total_items + kBThreads / 32 - 1) / (kBThreads / 32);
    const int grid = (int)std::max<long long>(1, std::min<long long>((long long)b->sms * ctas, want));
    switch (G) {
    case 2: return launch_ex(b, k_batch_eval<2>, grid, kBThreads, false, st, b->dev);
    case 4: return launch_ex(b, k_batch_eval<4>, grid, kBThreads, false, st, b->dev);
    case 16: return launch_ex(b, k_batch_eval<16>, grid, kBThreads, false, st, b->dev);
    default: return launch_ex(b, k_batch_eval<8>, grid, kBThreads, false, st, b->dev);
    }
}

// CTAs of the persistent launch: ctas per SM, capped by what is resident.
int persistent_grid(const chap_batch *b, int G, int ctas)
{
    const void *fn = G == 2 ? (const void *)k_batch_persistent<2> : G == 4 ? (const void *)k_batch_persistent<4>
                     : G == 16 ? (const void *)k_batch_persistent<16> : (const void *)k_batch_persistent<8>;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBThreads, 0) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    return b->sms * std::min(per_sm, ctas);
}

cudaError_t launch_persistent(const chap_batch *b, int G, int ctas, int iters, cudaStream_t st)
{
    const int grid = persistent_grid(b, G, ctas);
    const unsigned long long lim = b->bar_limit_ns;
    switch (G) {
    case 2: return launch_ex(b, k_batch_persistent<2>, grid, kBThreads, true, st, b->dev, iters, lim);
    case 4: return launch_ex(b, k_batch_persistent<4>, grid, kBThreads, true, st, b->dev, iters, lim);
    case 16: return launch_ex(b, k_batch_persistent<16>, grid, kBThreads, true, st, b->dev, iters, lim);
    default: return launch_ex(b, k_batch_persistent<8>, grid, kBThreads, true, st, b->dev, iters, lim);
    }
}

cudaError_t launch_iteration(const chap_batch *b, int G, int ctas, cudaStream_t st)
{
    cudaError_t e = launch_eval(b, G, ctas, st);
    if (e != cudaSuccess) return e;
    k_batch_apply<<<b->n_chains, kApplyT, 0, st>>>(b->dev);
    k_batch_bump<<<dim3(kBumpBlocks, b->n_chains), 256, 0, st>>>(b->dev);
    return cudaGetLastError();
}

// `iters` iterations of every chain in the batch's schedule.
cudaError_t launch_iterations(const chap_batch *b, int G, int ctas, int persistent, int iters, cudaStream_t st)
{
    if (persistent) return launch_persistent(b, G, ctas, iters, st);
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < iters && e == cudaSuccess; ++k) e = launch_iteration(b, G, ctas, st);
    return e;
}

chap_status upload_state(chap_batch *b)
{
    BCK(b, cudaMemsetAsync(b->dev.n_done, 0, sizeof(unsigned int), b->st), "reset done count");
    BCK(b, cudaMemsetAsync(b->dev.x, 0, sizeof(unsigned int) * std::max<long long>(b->total_words, 1), b->st),
        "reset x");
    BCK(b, cudaMemsetAsync(b->dev.bar, 0, sizeof(GridBar), b->st), "reset barrier");
    BCK(b, cudaMemsetAsync(b->dev.tinc, 0, sizeof(int) * std::max<long long>(b->total_x, 1), b->st), "reset tabu");
    BCK(b, cudaMemsetAsync(b->dev.tdec, 0, sizeof(int) * std::max<long long>(b->total_x, 1), b->st), "reset tabu");
    BCK(b, cudaMemcpyAsync(b->dev.rs, b->rs0.data(), sizeof(BRow) * b->rs0.size(), cudaMemcpyHostToDevice, b->st),
        "upload row states");
    BCK(b, cudaMemcpyAsync(b->dev.ctl, b->ctl0.data(), sizeof(BCtl) * b->ctl0.size(), cudaMemcpyHostToDevice, b->st),
        "upload control");
    BCK(b, cudaStreamSynchronize(b->st), "synchronise");
    b->broken = false;
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
    long long xo = 0, ro = 0, wo = 0;
    for (int c = 0; c < n_chains; ++c) {
        const int k = chain_prob[c];
        if (k < 0 || k >= n_probs || chain_tenure[c] < 0) { delete b; return CHAP_E_INVALID; }
        b->ch_inst.push_back(k);
        b->ch_tenure.push_back(chain_tenure[c]);
        b->ch_xoff.push_back(wo);
        b->ch_voff.push_back(xo);
        b->ch_roff.push_back(ro);
        xo += b->inst_n[k];
        wo += (b->inst_n[k] + 31) / 32;
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
    b->total_words = wo;
    b->total_rows = ro;
    // ---- device
    BDev &d = b->dev;
    d.n_chains = n_chains;
    d.total_items = item0.back();
    d.total_rows = ro;
    int *in_d = balloc<int>(b, n_probs), *im_d = balloc<int>(b, n_probs), *ic_d = balloc<int>(b, n_probs);
    int *cptr_d = balloc<int>(b, cptr.size()), *ceq_d = balloc<int>(b, ceq.size());
    int *crow_d = balloc<int>(b, crow.size()), *cval_d = balloc<int>(b, cval.size());
    int *vo_d = balloc<int>(b, var_of.size()), *po_d = balloc<int>(b, pos_of.size());
    int *chi_d = balloc<int>(b, n_chains), *cht_d = balloc<int>(b, n_chains);
    long long *chx_d = balloc<long long>(b, n_chains), *chr_d = balloc<long long>(b, n_chains);
    long long *chv_d = balloc<long long>(b, n_chains);
    long long *chi0_d = balloc<long long>(b, item0.size());
    d.x = balloc<unsigned int>(b, wo);
    d.bar = balloc<GridBar>(b, 1);
    d.tinc = balloc<int>(b, xo);
    d.tdec = balloc<int>(b, xo);
    d.rs = balloc<BRow>(b, ro);
    d.ctl = balloc<BCtl>(b, n_chains);
    d.n_done = balloc<unsigned int>(b, 1);
    const bool ok = in_d && im_d && ic_d && cptr_d && ceq_d && crow_d && cval_d && vo_d && po_d && chi_d && cht_d &&
                    chx_d && chr_d && chv_d && chi0_d && d.x && d.bar && d.tinc && d.tdec && d.rs && d.ctl &&
                    d.n_done &&
                    cudaMallocHost(&b->h_done, 2 * sizeof(unsigned int)) == cudaSuccess;
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
    BUP(chv_d, b->ch_voff);
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
    d.ch_voff = chv_d;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        b->sms = 152;
    }
    // persisting L2 set-aside for the incumbent bitsets (restored at destroy)
    {
        int win = 0;
        if (cudaDeviceGetAttribute(&win, cudaDevAttrMaxAccessPolicyWindowSize, dev) == cudaSuccess && win > 0)
            b->max_window = (size_t)win;
        int max_persist = 0;
        const size_t want = (size_t)std::max<long long>(wo, 1) * sizeof(unsigned int);
        if (cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, dev) == cudaSuccess &&
            max_persist > 0 && cudaDeviceGetLimit(&b->l2_prev, cudaLimitPersistingL2CacheSize) == cudaSuccess &&
            b->l2_prev < want) {
            if (cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, std::min(want, (size_t)max_persist)) == cudaSuccess)
                b->l2_set = true;
        }
        cudaGetLastError();
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
    if (b->broken) return bfail(b, CHAP_E_STATE, "a grid-barrier wait ran out: chap_batch_reset first");
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
    if (!b->gexec || b->g_iters != graph_iters || b->g_G != b->G || b->g_ctas != b->ctas_per_sm ||
        b->g_persistent != b->persistent) {
        if (b->gexec) cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
        cudaStream_t cs;
        BCK(b, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "capture stream");
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) e = launch_iterations(b, b->G, b->ctas_per_sm, b->persistent, graph_iters, cs);
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->gexec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cs);
        BCK(b, e, "graph capture");
        b->g_iters = graph_iters;
        b->g_G = b->G;
        b->g_ctas = b->ctas_per_sm;
        b->g_persistent = b->persistent;
    }
    // a chain that stops early idles through the rest of its graph replay (its
    // kernels return at once); replay until every chain is done
    for (;;) {
        BCK(b, cudaGraphLaunch(b->gexec, b->st), "graph launch");
        BCK(b, cudaMemcpyAsync(b->h_done, b->dev.n_done, sizeof(unsigned int), cudaMemcpyDeviceToHost, b->st), "read done");
        BCK(b, cudaMemcpyAsync(b->h_done + 1, &b->dev.bar->error, sizeof(int), cudaMemcpyDeviceToHost, b->st),
            "read barrier");
        BCK(b, cudaStreamSynchronize(b->st), "synchronise");
        if (b->h_done[1] != 0) {
            b->broken = true;
            return bfail(b, CHAP_E_TIMEOUT, "a grid-barrier wait of the persistent launch ran out");
        }
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

chap_status chap_batch_autotune_mode(chap_batch *b, int32_t iters, int32_t mode, int32_t *chosen)
{
    if (!b || iters < 1 || mode < -1 || mode > 1) return CHAP_E_INVALID;
    // time every schedule for `iters` iterations from the initial state, keep the fastest
    const int Gs[4] = {2, 4, 8, 16};
    const int Cs[3] = {2, 4, 8};
    cudaEvent_t a, z;
    BCK(b, cudaEventCreate(&a), "event");
    BCK(b, cudaEventCreate(&z), "event");
    float best_ms = 1e30f;
    int bg = b->G, bc = b->ctas_per_sm, bp = b->persistent;
    for (int pm = 0; pm < 2; ++pm)
    for (int gi = 0; gi < 4 && (mode < 0 || mode == pm); ++gi)
        for (int ci = 0; ci < 3; ++ci) {
            chap_status s = upload_state(b);
            if (s != CHAP_OK) { cudaEventDestroy(a); cudaEventDestroy(z); return s; }
            k_batch_begin<<<(b->n_chains + 255) / 256, 256, 0, b->st>>>(b->dev, iters + 1, 0);
            cudaError_t e = launch_iterations(b, Gs[gi], Cs[ci], pm, 1, b->st);  // warm-up
            if (e == cudaSuccess) e = cudaEventRecord(a, b->st);
            if (e == cudaSuccess) e = launch_iterations(b, Gs[gi], Cs[ci], pm, iters, b->st);
            if (e == cudaSuccess) e = cudaEventRecord(z, b->st);
            if (e == cudaSuccess) e = cudaEventSynchronize(z);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, z);
            if (e != cudaSuccess) {
                cudaEventDestroy(a);
                cudaEventDestroy(z);
                BCK(b, e, "autotune run");
            }
            int err = 0;
            if (e == cudaSuccess) e = cudaMemcpy(&err, &b->dev.bar->error, sizeof(int), cudaMemcpyDeviceToHost);
            if (e == cudaSuccess && err) {
                cudaEventDestroy(a);
                cudaEventDestroy(z);
                upload_state(b);
                return bfail(b, CHAP_E_TIMEOUT, "a grid-barrier wait ran out while timing the schedules");
            }
            if (ms < best_ms) { best_ms = ms; bg = Gs[gi]; bc = Cs[ci]; bp = pm; }
        }
    cudaEventDestroy(a);
    cudaEventDestroy(z);
    b->G = bg;
    b->ctas_per_sm = bc;
    b->persistent = bp;
    if (chosen) { chosen[0] = bg; chosen[1] = bc; chosen[2] = bp; }
    return upload_state(b);
}

chap_status chap_batch_autotune(chap_batch *b, int32_t iters, int32_t *chosen)
{
    return chap_batch_autotune_mode(b, iters, -1, chosen);
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
    std::vector<unsigned int> t((n + 31) / 32);
    if (!t.empty())
        BCK(b, cudaMemcpyAsync(t.data(), b->dev.x + b->ch_xoff[chain], sizeof(unsigned int) * t.size(),
                               cudaMemcpyDeviceToHost, b->st), "read x");
    BCK(b, cudaStreamSynchronize(b->st), "synchronise");
    for (int j = 0; j < n; ++j) x[j] = (t[j >> 5] >> (j & 31)) & 1u;
    return CHAP_OK;
}

chap_status chap_batch_set_persistent(chap_batch *b, int32_t on, int64_t barrier_limit_ns)
{
    if (!b || (on != 0 && on != 1) || barrier_limit_ns < 0) return CHAP_E_INVALID;
    b->persistent = on;
    if (barrier_limit_ns > 0) b->bar_limit_ns = (unsigned long long)barrier_limit_ns;
    if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
    return CHAP_OK;
}

const char *chap_batch_last_error(const chap_batch *b) { return b ? b->err.c_str() : ""; }

}  // extern "C"
