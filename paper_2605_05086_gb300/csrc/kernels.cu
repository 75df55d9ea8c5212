// Kernels of the best-shift tabu search (sm_103a).
//
// One tabu iteration = best-shift pass (eval kernels) -> selection -> apply.
//
//  * Binary columns: the only move is the flip (Sec. 3.1, "Best Shift Moves");
//    its score is a segmented sum of penalties over the column.  G lanes work
//    on one column (G = 4..32 by column length, or a whole CTA for very long
//    columns); nonzeros are read coalesced inside the column and the row
//    residual + weights are gathered with one 16-byte load.
//  * Other columns: Algorithm 1 (sort -> scan -> argmax).  Breakpoint entries
//    (t, marker, score delta, count delta) are generated from each nonzero,
//    entries below l are folded into the base beta, entries above u are
//    dropped, and the rest are
//      - sorted by a warp-level bitonic network held in registers (up to 32K
//        entries, K per lane), or
//      - sorted in shared memory by one CTA (up to kCtaMaxEntries), or
//      - bucketed by key (an integer counting sort) across many CTAs for long
//        integer columns with small domains;
//    then prefix-scanned, and reduced to the best admissible entry.
//  * Each CTA reduces its columns to one candidate; the selection kernel
//    reduces the CTA candidates (largest score, then lowest variable).
//  * Apply walks the chosen column and updates the residuals incrementally
//    (Sec. 3.1, "Memory Considerations", first point); when no positive move
//    exists it adds 1 to the weight of every violated normalised row.
//
// All arithmetic that decides a score is exact: integral rows use int64
// residuals, non-integral rows IEEE double with explicit round-to-nearest
// intrinsics (no fused multiply-add), and scores are int64 half-weight counts.
#include "chap_internal.h"

#include <climits>
#include <cstdint>

namespace chap {

#define FULLMASK 0xffffffffu

constexpr unsigned long long kPadKey = 0xffffffffffffffffull;
constexpr int kNoVar = INT_MAX;

// ---------------------------------------------------------------- helpers

// Order-preserving map of a double to an unsigned 64-bit key.
__device__ __forceinline__ unsigned long long ord_key(double t)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(t);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ double key_to_double(unsigned long long k)
{
    unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)b);
}

__device__ __forceinline__ long long floor_div(long long a, long long b)
{
    long long q = a / b, r = a % b;
    if (r != 0 && ((r < 0) != (b < 0))) --q;
    return q;
}

__device__ __forceinline__ long long ceil_div(long long a, long long b)
{
    long long q = a / b, r = a % b;
    if (r != 0 && ((r < 0) == (b < 0))) ++q;
    return q;
}

__device__ __forceinline__ RowState load_row(const Dev &d, int i)
{
    int4 v = __ldg(reinterpret_cast<const int4 *>(d.rs) + i);
    RowState s;
    s.r = (long long)(((unsigned long long)(unsigned)v.y << 32) | (unsigned)v.x);
    s.w1 = v.z;
    s.w2 = v.w;
    return s;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Global candidate order: larger score, then lower variable index.
__device__ __forceinline__ bool cand_better(long long s1, int v1, long long s2, int v2)
{
    return s1 > s2 || (s1 == s2 && v1 < v2);
}

__device__ __forceinline__ void warp_reduce_cand(long long &s, int &var, int &dc, double &xh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        long long s2 = __shfl_xor_sync(FULLMASK, s, o);
        int v2 = __shfl_xor_sync(FULLMASK, var, o);
        int d2 = __shfl_xor_sync(FULLMASK, dc, o);
        double x2 = __shfl_xor_sync(FULLMASK, xh, o);
        if (cand_better(s2, v2, s, var)) { s = s2; var = v2; dc = d2; xh = x2; }
    }
}

// Reduce one candidate per thread to thread 0 of the block; returns it there.
__device__ Cand block_reduce_cand(Cand c)
{
    __shared__ Cand red[32];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    warp_reduce_cand(c.s, c.var, c.dc, c.xhat);
    if (lane == 0) red[warp] = c;
    __syncthreads();
    int nw = (blockDim.x + 31) >> 5;
    if (warp == 0) {
        Cand r = lane < nw ? red[lane] : Cand{0, kNoVar, 0, 0.0};
        warp_reduce_cand(r.s, r.var, r.dc, r.xhat);
        c = r;
    }
    __syncthreads();
    return c;
}

// Per-variable candidate order (Eq. best_move ties): larger score, then
// smaller |t - xbar|, then smaller t.
struct VCand {
    long long s;
    double t;
    int dc;
    int valid;
};

__device__ __forceinline__ bool vc_better(const VCand &a, const VCand &b, double xb)
{
    if (!a.valid) return false;
    if (!b.valid) return true;
    if (a.s != b.s) return a.s > b.s;
    double da = fabs(a.t - xb), db = fabs(b.t - xb);
    if (da != db) return da < db;
    return a.t < b.t;
}

__device__ __forceinline__ void warp_reduce_vc(VCand &c, double xb)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        VCand p;
        p.s = __shfl_xor_sync(FULLMASK, c.s, o);
        p.t = __shfl_xor_sync(FULLMASK, c.t, o);
        p.dc = __shfl_xor_sync(FULLMASK, c.dc, o);
        p.valid = __shfl_xor_sync(FULLMASK, c.valid, o);
        if (vc_better(p, c, xb)) c = p;
    }
}

__device__ VCand block_reduce_vc(VCand c, double xb)
{
    __shared__ VCand red[32];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    warp_reduce_vc(c, xb);
    if (lane == 0) red[warp] = c;
    __syncthreads();
    int nw = (blockDim.x + 31) >> 5;
    if (warp == 0) {
        VCand r = lane < nw ? red[lane] : VCand{0, 0.0, 0, 0};
        warp_reduce_vc(r, xb);
        c = r;
    }
    __syncthreads();
    return c;
}

// Admissibility under tabu and aspiration.
__device__ __forceinline__ bool admissible(bool increase, int j, int dc, const Dev &d, long long iter,
                                           long long nviol, long long bestnv)
{
    int stamp = increase ? d.tabu_inc[j] : d.tabu_dec[j];
    bool tabu = iter < (long long)stamp;
    return !tabu || (nviol + (long long)dc < bestnv);
}

// Column result -> optional per-variable outputs and the caller's running best.
__device__ __forceinline__ void finish_column(const Dev &d, const VarOut &o, int j, double xb, const VCand &b,
                                              Cand &best)
{
    bool mv = b.valid && b.s > 0;
    if (o.xhat) o.xhat[j] = mv ? b.t : xb;
    if (o.s) o.s[j] = mv ? b.s : 0;
    if (o.dc) o.dc[j] = mv ? b.dc : 0;
    if (mv && cand_better(b.s, j, best.s, best.var)) best = Cand{b.s, j, b.dc, b.t};
}

// ------------------------------------------------------- binary flip scoring

// Penalty of a flip on one normalised half with integer residual r and signed
// coefficient change ad = a * (new - old) (Sec. 3.1, Scoring Functions).
__device__ __forceinline__ void flip_int(long long r, long long ad, long long w, long long &s, int &dc)
{
    long long r1 = r + ad;
    bool v0 = r > 0, v1 = r1 > 0;
    if (!v0 && v1) s -= 2 * w;
    else if (v0 && !v1) s += 2 * w;
    else if (v0 && v1) s += (ad < 0) ? w : -w;
    dc += (int)v1 - (int)v0;
}

__device__ __forceinline__ void flip_fp(double r, double ad, double eps, long long w, long long &s, int &dc)
{
    double r1 = __dadd_rn(r, ad);
    bool v0 = r > eps, v1 = r1 > eps;
    if (!v0 && v1) s -= 2 * w;
    else if (v0 && !v1) s += 2 * w;
    else if (v0 && v1) s += (ad < 0.0) ? w : -w;
    dc += (int)v1 - (int)v0;
}

// Partial flip score of column j over the lanes sub, sub+G, ...
__device__ __forceinline__ void bin_col_partial(const Dev &d, int j, bool up, int sub, int G, long long &s, int &dc)
{
    int e0 = __ldg(d.ci_ptr + j), e1 = __ldg(d.ci_ptr + j + 1);
    for (int e = e0 + sub; e < e1; e += G) {
        int i = __ldg(d.ci_row + e);
        long long a = __ldg(d.ci_val + e);
        RowState st = load_row(d, i);
        long long ad = up ? a : -a;
        flip_int(st.r, ad, st.w1, s, dc);
        if (st.w2 >= 0) flip_int(-st.r, -ad, st.w2, s, dc);
    }
    int f0 = __ldg(d.cf_ptr + j), f1 = __ldg(d.cf_ptr + j + 1);
    for (int e = f0 + sub; e < f1; e += G) {
        int i = __ldg(d.cf_row + e);
        double a = __ldg(d.cf_val + e);
        RowState st = load_row(d, i);
        double eps = __ldg(d.eps + i);
        double r = __longlong_as_double(st.r);
        double ad = up ? a : -a;
        flip_fp(r, ad, eps, st.w1, s, dc);
        if (st.w2 >= 0) flip_fp(-r, -ad, eps, st.w2, s, dc);
    }
}

template <int G>
__device__ void eval_bin_tile(const Dev &d, const Tile &tl, const VarOut &o, long long iter, long long nviol,
                              long long bestnv, Cand &best)
{
    const int groups = kEvalThreads / G;
    int g = threadIdx.x / G, sub = threadIdx.x % G;
    int count = tl.end - tl.begin;
    int rounds = (count + groups - 1) / groups;
    for (int rd = 0; rd < rounds; ++rd) {
        int q = rd * groups + g;
        bool active = q < count;
        int j = active ? __ldg(d.var_list + tl.begin + q) : 0;
        long long s = 0;
        int dc = 0;
        double xb = 0.0;
        bool up = true;
        if (active) {
            xb = d.x[j];
            up = xb == 0.0;
            bin_col_partial(d, j, up, sub, G, s, dc);
        }
#pragma unroll
        for (int off = G / 2; off > 0; off >>= 1) {
            s += __shfl_xor_sync(FULLMASK, s, off, G);
            dc += __shfl_xor_sync(FULLMASK, dc, off, G);
        }
        if (active && sub == 0) {
            VCand b{s, up ? 1.0 : 0.0, dc, 0};
            b.valid = admissible(up, j, dc, d, iter, nviol, bestnv) ? 1 : 0;
            finish_column(d, o, j, xb, b, best);
        }
    }
}

__device__ void eval_bin_cta(const Dev &d, const Tile &tl, const VarOut &o, long long iter, long long nviol,
                             long long bestnv, Cand &best)
{
    int j = __ldg(d.var_list + tl.begin);
    double xb = d.x[j];
    bool up = xb == 0.0;
    long long s = 0;
    int dc = 0;
    bin_col_partial(d, j, up, threadIdx.x, blockDim.x, s, dc);
    __shared__ long long rs_[32];
    __shared__ int rc_[32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        s += __shfl_xor_sync(FULLMASK, s, off);
        dc += __shfl_xor_sync(FULLMASK, dc, off);
    }
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { rs_[warp] = s; rc_[warp] = dc; }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long ts = 0;
        int tc = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { ts += rs_[w]; tc += rc_[w]; }
        VCand b{ts, up ? 1.0 : 0.0, tc, 0};
        b.valid = admissible(up, j, tc, d, iter, nviol, bestnv) ? 1 : 0;
        finish_column(d, o, j, xb, b, best);
    }
    __syncthreads();
}

// ---------------------------------------------- breakpoint generation (Alg. 1)

// Scalars of Algorithm 1: beta (score as x -> -inf), alpha (adjustment right of
// xbar) and their count-lane twins, all in half-weight / row units.
struct Acc {
    long long beta, alpha;
    int beta_c, alpha_c;
};

// Entries produced by one normalised half of a nonzero.
//  type 1: (t, -1, +D, count -1)            rows with a < 0 (need x >= t)
//  type 2: (t, -1, 0, 0), (t, +1, D, +1)    rows with a > 0 (need x <= t)
struct Half {
    double t;
    long long D;
    int type;
};

__device__ __forceinline__ int half_count(const Half &h) { return h.type; }

// Case table of Algorithm 1 in half units: the row's state at xbar (violated,
// satisfied, tight) decides beta/alpha and the entries; entries left of l are
// folded into beta, entries right of u are dropped.
__device__ __forceinline__ void half_case(bool viol, bool tight, bool apos, double t, long long w, double l,
                                          double u, Acc &acc, Half &h)
{
    h.type = 0;
    if (tight) {
        if (apos) { acc.alpha -= 2 * w; acc.alpha_c += 1; }
        else { acc.beta -= 2 * w; acc.alpha += 2 * w; acc.beta_c += 1; acc.alpha_c -= 1; }
        return;
    }
    long long D;
    int type;
    if (!apos) {
        if (viol) { acc.beta -= w; acc.alpha += 2 * w; D = w; }
        else { acc.beta -= 2 * w; acc.beta_c += 1; D = 2 * w; }
        type = 1;
    } else {
        if (viol) { acc.beta += 2 * w; acc.alpha -= 2 * w; acc.beta_c -= 1; D = -w; }
        else { D = -2 * w; }
        type = 2;
    }
    if (t < l) {
        acc.beta += D;
        acc.beta_c += (type == 1) ? -1 : 1;
        return;
    }
    if (t > u) return;
    h.t = t;
    h.D = D;
    h.type = type;
}

// Integral row, integer variable: exact integer breakpoint offset.
__device__ __forceinline__ void int_half(long long r, long long a, long long w, double xb, double l, double u,
                                         Acc &acc, Half &h)
{
    bool viol = r > 0;
    long long dd = (a > 0) ? floor_div(-r, a) : ceil_div(-r, a);
    bool tight = !viol && dd == 0;
    double t = __dadd_rn(xb, (double)dd);
    half_case(viol, tight, a > 0, t, w, l, u, acc, h);
}

// Non-integral row.  Continuous variable: t = xbar - r / a (the row becomes
// tight); integer variable: the last integer at which the row is satisfied
// within eps, xbar + floor((eps - r) / a) for a > 0 (ceil for a < 0).
__device__ __forceinline__ void fp_half(double r, double a, double eps, long long w, double xb, bool isint,
                                        double l, double u, Acc &acc, Half &h)
{
    bool viol = r > eps;
    double t;
    bool tight;
    if (isint) {
        double q = __ddiv_rn(__dsub_rn(eps, r), a);
        double dd = (a > 0.0) ? floor(q) : ceil(q);
        t = __dadd_rn(xb, dd);
        tight = !viol && dd == 0.0;
    } else {
        double q = __ddiv_rn(r, a);
        t = __dsub_rn(xb, q);
        tight = !viol && (fabs(r) <= eps || t == xb);
    }
    t = __dadd_rn(t, 0.0);
    half_case(viol, tight, a > 0.0, t, w, l, u, acc, h);
}

// Both halves of one nonzero of column j.  v < nI indexes the integral part
// (ci_*), otherwise v - nI the non-integral part (cf_*).
__device__ __forceinline__ void gen_entry(const Dev &d, int ci0, int cf0, int nI, int v, double xb, bool isint,
                                          double l, double u, Acc &acc, Half &h1, Half &h2)
{
    h1.type = 0;
    h2.type = 0;
    if (v < nI) {
        int e = ci0 + v;
        int i = __ldg(d.ci_row + e);
        long long a = __ldg(d.ci_val + e);
        RowState st = load_row(d, i);
        int_half(st.r, a, st.w1, xb, l, u, acc, h1);
        if (st.w2 >= 0) int_half(-st.r, -a, st.w2, xb, l, u, acc, h2);
    } else {
        int e = cf0 + (v - nI);
        int i = __ldg(d.cf_row + e);
        double a = __ldg(d.cf_val + e);
        RowState st = load_row(d, i);
        double eps = __ldg(d.eps + i);
        double r = __longlong_as_double(st.r);
        fp_half(r, a, eps, st.w1, xb, isint, l, u, acc, h1);
        if (st.w2 >= 0) fp_half(-r, -a, eps, st.w2, xb, isint, l, u, acc, h2);
    }
}

// aux word of a sort entry: bit 31 = marker (+1), bits 0..1 = count delta + 1.
__device__ __forceinline__ unsigned make_aux(int plus, int dc) { return ((unsigned)plus << 31) | (unsigned)(dc + 1); }
__device__ __forceinline__ int aux_dc(unsigned a) { return (int)(a & 3u) - 1; }
__device__ __forceinline__ unsigned aux_plus(unsigned a) { return a >> 31; }

__device__ __forceinline__ void put_half(const Half &h, int pos, unsigned long long *k, long long *dl, unsigned *ax)
{
    if (h.type == 1) {
        k[pos] = ord_key(h.t); dl[pos] = h.D; ax[pos] = make_aux(0, -1);
    } else if (h.type == 2) {
        unsigned long long kk = ord_key(h.t);
        k[pos] = kk; dl[pos] = 0; ax[pos] = make_aux(0, 0);
        k[pos + 1] = kk; dl[pos + 1] = h.D; ax[pos + 1] = make_aux(1, 1);
    }
}

__device__ __forceinline__ void warp_allreduce_acc(Acc &a)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a.beta += __shfl_xor_sync(FULLMASK, a.beta, o);
        a.alpha += __shfl_xor_sync(FULLMASK, a.alpha, o);
        a.beta_c += __shfl_xor_sync(FULLMASK, a.beta_c, o);
        a.alpha_c += __shfl_xor_sync(FULLMASK, a.alpha_c, o);
    }
}

// Lexicographic (t, marker) order of sort entries.
__device__ __forceinline__ bool entry_less(unsigned long long k1, unsigned a1, unsigned long long k2, unsigned a2)
{
    return k1 < k2 || (k1 == k2 && aux_plus(a1) < aux_plus(a2));
}

// ------------------------------------------- warp sort / scan / argmax (K/lane)

template <int K>
__device__ __forceinline__ void warp_bitonic(unsigned long long (&key)[K], long long (&del)[K], unsigned (&aux)[K],
                                             int lane)
{
    constexpr int N = 32 * K;
#pragma unroll
    for (int size = 2; size <= N; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride < K) {
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    if ((k & stride) == 0) {
                        const int k2 = k | stride;
                        int i = lane * K + k;
                        bool asc = (i & size) == 0;
                        bool gt = entry_less(key[k2], aux[k2], key[k], aux[k]);
                        if (gt == asc) {
                            unsigned long long tk = key[k]; key[k] = key[k2]; key[k2] = tk;
                            long long td = del[k]; del[k] = del[k2]; del[k2] = td;
                            unsigned ta = aux[k]; aux[k] = aux[k2]; aux[k2] = ta;
                        }
                    }
                }
            } else {
                const int ls = stride / K;
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    unsigned long long pk = __shfl_xor_sync(FULLMASK, key[k], ls);
                    long long pd = __shfl_xor_sync(FULLMASK, del[k], ls);
                    unsigned pa = __shfl_xor_sync(FULLMASK, aux[k], ls);
                    int i = lane * K + k;
                    bool lower = (i & stride) == 0;
                    bool asc = (i & size) == 0;
                    bool take = (lower == asc) ? entry_less(pk, pa, key[k], aux[k])
                                               : entry_less(key[k], aux[k], pk, pa);
                    if (take) { key[k] = pk; del[k] = pd; aux[k] = pa; }
                }
            }
        }
    }
}

// Algorithm 1 for one column by one warp; the staged entries of this warp live
// in skey/sdel/saux (capacity 32 * K).
template <int K>
__device__ void nb_warp_column(const Dev &d, const VarOut &o, int j, int lane, unsigned long long *skey,
                               long long *sdel, unsigned *saux, long long iter, long long nviol, long long bestnv,
                               Cand &best)
{
    const double xb = d.x[j];
    const bool isint = __ldg(d.vtype + j) == kVarInt;
    const double l = __ldg(d.lb + j), u = __ldg(d.ub + j);
    const int ci0 = __ldg(d.ci_ptr + j), nI = __ldg(d.ci_ptr + j + 1) - ci0;
    const int cf0 = __ldg(d.cf_ptr + j), nF = __ldg(d.cf_ptr + j + 1) - cf0;
    Acc acc{0, 0, 0, 0};
    const bool fl = isfinite(l), fu = isfinite(u);
    int cnt = (fl ? 1 : 0) + (fu ? 1 : 0);
    if (lane == 0) {
        if (fl) { skey[0] = ord_key(__dadd_rn(l, 0.0)); sdel[0] = 0; saux[0] = make_aux(0, 0); }
        if (fu) { int p = fl ? 1 : 0; skey[p] = ord_key(__dadd_rn(u, 0.0)); sdel[p] = 0; saux[p] = make_aux(0, 0); }
    }
    const int total = nI + nF;
    for (int base = 0; base < total; base += 32) {
        int v = base + lane;
        Half h1, h2;
        h1.type = 0;
        h2.type = 0;
        if (v < total) gen_entry(d, ci0, cf0, nI, v, xb, isint, l, u, acc, h1, h2);
        int c = half_count(h1) + half_count(h2);
        int incl = c;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            int t = __shfl_up_sync(FULLMASK, incl, off);
            if (lane >= off) incl += t;
        }
        int pos = cnt + incl - c;
        put_half(h1, pos, skey, sdel, saux);
        put_half(h2, pos + half_count(h1), skey, sdel, saux);
        cnt += __shfl_sync(FULLMASK, incl, 31);
    }
    __syncwarp();
    warp_allreduce_acc(acc);
    unsigned long long key[K];
    long long del[K];
    unsigned aux[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        int idx = lane * K + k;
        if (idx < cnt) { key[k] = skey[idx]; del[k] = sdel[idx]; aux[k] = saux[idx]; }
        else { key[k] = kPadKey; del[k] = 0; aux[k] = make_aux(1, 0); }
    }
    __syncwarp();
    warp_bitonic<K>(key, del, aux, lane);
    // inclusive scan of the score and count deltas along the sorted entries
    long long P[K];
    int Pc[K];
    long long run = 0;
    int runc = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) { run += del[k]; runc += aux_dc(aux[k]); P[k] = run; Pc[k] = runc; }
    long long tot = run;
    int totc = runc;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        long long a = __shfl_up_sync(FULLMASK, tot, off);
        int b = __shfl_up_sync(FULLMASK, totc, off);
        if (lane >= off) { tot += a; totc += b; }
    }
    long long ex = tot - run;
    int exc = totc - runc;
    unsigned long long nk = __shfl_down_sync(FULLMASK, key[0], 1);
    unsigned na = __shfl_down_sync(FULLMASK, aux[0], 1);
    if (lane == 31) { nk = kPadKey; na = make_aux(1, 0); }
    VCand vb{0, 0.0, 0, 0};
#pragma unroll
    for (int k = 0; k < K; ++k) {
        unsigned long long kk = key[k];
        unsigned long long nxk = (k + 1 < K) ? key[(k + 1) % K] : nk;
        unsigned nxa = (k + 1 < K) ? aux[(k + 1) % K] : na;
        bool cand = kk != kPadKey && aux_plus(aux[k]) == 0 && (nxk != kk || aux_plus(nxa) != 0);
        if (!cand) continue;
        double t = key_to_double(kk);
        if (t == xb) continue;
        bool right = t > xb;
        long long sg = acc.beta + ex + P[k] + (right ? acc.alpha : 0);
        int dcv = acc.beta_c + exc + Pc[k] + (right ? acc.alpha_c : 0);
        if (!admissible(right, j, dcv, d, iter, nviol, bestnv)) continue;
        VCand c{sg, t, dcv, 1};
        if (vc_better(c, vb, xb)) vb = c;
    }
    warp_reduce_vc(vb, xb);
    if (lane == 0) finish_column(d, o, j, xb, vb, best);
    __syncwarp();
}

template <int K>
__device__ void eval_nb_tile(const Dev &d, const Tile &tl, const VarOut &o, long long iter, long long nviol,
                             long long bestnv, Cand &best, unsigned long long *skey, long long *sdel,
                             unsigned *saux)
{
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = tl.begin + warp; q < tl.end; q += kEvalThreads / 32) {
        int j = __ldg(d.var_list + q);
        nb_warp_column<K>(d, o, j, lane, skey, sdel, saux, iter, nviol, bestnv, best);
    }
}

// ------------------------------------------------------------ eval kernels

__device__ __forceinline__ bool gated_done(const Dev &d, int gate)
{
    return gate && *(volatile int *)&d.ctl->done;
}

__global__ void __launch_bounds__(kEvalThreads) k_eval_small(Dev d, const Tile *tiles, VarOut o, int gate)
{
    if (gated_done(d, gate)) return;
    __shared__ unsigned long long skey[kEvalThreads / 32][kWarpStageCap];
    __shared__ long long sdel[kEvalThreads / 32][kWarpStageCap];
    __shared__ unsigned saux[kEvalThreads / 32][kWarpStageCap];
    const Tile tl = tiles[blockIdx.x];
    const long long iter = d.ctl->iter, nviol = d.ctl->nviol, bestnv = d.ctl->best_nviol;
    Cand best{0, kNoVar, 0, 0.0};
    int warp = threadIdx.x >> 5;
    switch (tl.kind) {
    case T_BIN_G4: eval_bin_tile<4>(d, tl, o, iter, nviol, bestnv, best); break;
    case T_BIN_G8: eval_bin_tile<8>(d, tl, o, iter, nviol, bestnv, best); break;
    case T_BIN_G16: eval_bin_tile<16>(d, tl, o, iter, nviol, bestnv, best); break;
    case T_BIN_G32: eval_bin_tile<32>(d, tl, o, iter, nviol, bestnv, best); break;
    case T_BIN_CTA: eval_bin_cta(d, tl, o, iter, nviol, bestnv, best); break;
    case T_NB_K1: eval_nb_tile<1>(d, tl, o, iter, nviol, bestnv, best, skey[warp], sdel[warp], saux[warp]); break;
    case T_NB_K2: eval_nb_tile<2>(d, tl, o, iter, nviol, bestnv, best, skey[warp], sdel[warp], saux[warp]); break;
    case T_NB_K4: eval_nb_tile<4>(d, tl, o, iter, nviol, bestnv, best, skey[warp], sdel[warp], saux[warp]); break;
    case T_NB_K8: eval_nb_tile<8>(d, tl, o, iter, nviol, bestnv, best, skey[warp], sdel[warp], saux[warp]); break;
    default: break;
    }
    Cand b = block_reduce_cand(best);
    if (threadIdx.x == 0) d.block_best[blockIdx.x] = b;
}

// One column per CTA, entries sorted in shared memory (bitonic, N = tile.aux).
__global__ void __launch_bounds__(kCtaThreads) k_eval_cta(Dev d, const Tile *tiles, VarOut o, int slot_base, int gate)
{
    if (gated_done(d, gate)) return;
    extern __shared__ __align__(16) unsigned char smem[];
    const Tile tl = tiles[blockIdx.x];
    const int N = tl.aux;
    unsigned long long *skey = reinterpret_cast<unsigned long long *>(smem);
    long long *sdel = reinterpret_cast<long long *>(skey + N);
    unsigned *saux = reinterpret_cast<unsigned *>(sdel + N);
    __shared__ int s_cnt;
    __shared__ long long s_beta, s_alpha;
    __shared__ int s_bc, s_ac;
    const long long iter = d.ctl->iter, nviol = d.ctl->nviol, bestnv = d.ctl->best_nviol;
    const int j = __ldg(d.var_list + tl.begin);
    const double xb = d.x[j];
    const bool isint = __ldg(d.vtype + j) == kVarInt;
    const double l = __ldg(d.lb + j), u = __ldg(d.ub + j);
    const int ci0 = __ldg(d.ci_ptr + j), nI = __ldg(d.ci_ptr + j + 1) - ci0;
    const int cf0 = __ldg(d.cf_ptr + j), nF = __ldg(d.cf_ptr + j + 1) - cf0;
    const bool fl = isfinite(l), fu = isfinite(u);
    if (threadIdx.x == 0) {
        s_cnt = (fl ? 1 : 0) + (fu ? 1 : 0);
        s_beta = 0; s_alpha = 0; s_bc = 0; s_ac = 0;
        if (fl) { skey[0] = ord_key(__dadd_rn(l, 0.0)); sdel[0] = 0; saux[0] = make_aux(0, 0); }
        if (fu) { int p = fl ? 1 : 0; skey[p] = ord_key(__dadd_rn(u, 0.0)); sdel[p] = 0; saux[p] = make_aux(0, 0); }
    }
    __syncthreads();
    Acc acc{0, 0, 0, 0};
    const int total = nI + nF;
    for (int v = threadIdx.x; v < total; v += blockDim.x) {
        Half h1, h2;
        gen_entry(d, ci0, cf0, nI, v, xb, isint, l, u, acc, h1, h2);
        int c = half_count(h1) + half_count(h2);
        if (c) {
            int pos = atomicAdd(&s_cnt, c);
            put_half(h1, pos, skey, sdel, saux);
            put_half(h2, pos + half_count(h1), skey, sdel, saux);
        }
    }
    warp_allreduce_acc(acc);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(reinterpret_cast<unsigned long long *>(&s_beta), (unsigned long long)acc.beta);
        atomicAdd(reinterpret_cast<unsigned long long *>(&s_alpha), (unsigned long long)acc.alpha);
        atomicAdd(&s_bc, acc.beta_c);
        atomicAdd(&s_ac, acc.alpha_c);
    }
    __syncthreads();
    const int cnt = s_cnt;
    for (int i = cnt + threadIdx.x; i < N; i += blockDim.x) { skey[i] = kPadKey; sdel[i] = 0; saux[i] = make_aux(1, 0); }
    __syncthreads();
    // bitonic sort of N entries in shared memory
    for (int size = 2; size <= N; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int p = threadIdx.x; p < (N >> 1); p += blockDim.x) {
                int i = 2 * stride * (p / stride) + (p % stride);
                int k2 = i + stride;
                bool asc = (i & size) == 0;
                unsigned long long ka = skey[i], kb = skey[k2];
                unsigned aa = saux[i], ab = saux[k2];
                bool gt = entry_less(kb, ab, ka, aa);
                if (gt == asc) {
                    skey[i] = kb; skey[k2] = ka;
                    saux[i] = ab; saux[k2] = aa;
                    long long t = sdel[i]; sdel[i] = sdel[k2]; sdel[k2] = t;
                }
            }
            __syncthreads();
        }
    }
    // block scan: each thread owns N / blockDim consecutive entries
    const int per = N / blockDim.x;
    const int b0 = threadIdx.x * per;
    long long run = 0;
    int runc = 0;
    for (int q = 0; q < per; ++q) { run += sdel[b0 + q]; runc += aux_dc(saux[b0 + q]); }
    __shared__ long long wsum[32];
    __shared__ int wsumc[32];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long tot = run;
    int totc = runc;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        long long a = __shfl_up_sync(FULLMASK, tot, off);
        int b = __shfl_up_sync(FULLMASK, totc, off);
        if (lane >= off) { tot += a; totc += b; }
    }
    if (lane == 31) { wsum[warp] = tot; wsumc[warp] = totc; }
    __syncthreads();
    if (warp == 0) {
        int nw = blockDim.x >> 5;
        long long v = lane < nw ? wsum[lane] : 0;
        int vc = lane < nw ? wsumc[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            long long a = __shfl_up_sync(FULLMASK, v, off);
            int b = __shfl_up_sync(FULLMASK, vc, off);
            if (lane >= off) { v += a; vc += b; }
        }
        if (lane < nw) { wsum[lane] = v; wsumc[lane] = vc; }
    }
    __syncthreads();
    long long ex = (tot - run) + (warp > 0 ? wsum[warp - 1] : 0);
    int exc = (totc - runc) + (warp > 0 ? wsumc[warp - 1] : 0);
    const long long beta = s_beta, alpha = s_alpha;
    const int bc = s_bc, ac = s_ac;
    VCand vb{0, 0.0, 0, 0};
    long long P = ex;
    int Pc = exc;
    for (int q = 0; q < per; ++q) {
        int i = b0 + q;
        unsigned long long kk = skey[i];
        unsigned a = saux[i];
        P += sdel[i];
        Pc += aux_dc(a);
        if (kk == kPadKey || aux_plus(a) != 0) continue;
        bool last = (i + 1 >= N) || skey[i + 1] != kk || aux_plus(saux[i + 1]) != 0;
        if (!last) continue;
        double t = key_to_double(kk);
        if (t == xb) continue;
        bool right = t > xb;
        long long sg = beta + P + (right ? alpha : 0);
        int dcv = bc + Pc + (right ? ac : 0);
        if (!admissible(right, j, dcv, d, iter, nviol, bestnv)) continue;
        VCand c{sg, t, dcv, 1};
        if (vc_better(c, vb, xb)) vb = c;
    }
    vb = block_reduce_vc(vb, xb);
    if (threadIdx.x == 0) {
        Cand best{0, kNoVar, 0, 0.0};
        finish_column(d, o, j, xb, vb, best);
        d.block_best[slot_base + blockIdx.x] = best;
    }
}

// Long integer column with a small domain: every CTA bins one chunk of the
// column's nonzeros by breakpoint value (a counting sort on the key (t,
// marker)); the last CTA of the column scans the bins and takes the argmax.
__global__ void __launch_bounds__(kHistThreads) k_eval_hist(Dev d, const Tile *tiles, VarOut o, int gate)
{
    if (gated_done(d, gate)) return;
    extern __shared__ __align__(16) unsigned char smem[];
    HBin *sb = reinterpret_cast<HBin *>(smem);
    const Tile tl = tiles[blockIdx.x];
    const HistCol hc = d.hcols[tl.begin];
    const int chunk = tl.aux;
    const int j = hc.var;
    const double xb = d.x[j];
    const double l = __ldg(d.lb + j), u = __ldg(d.ub + j);
    const int D = (int)(u - l) + 1;
    const int ci0 = __ldg(d.ci_ptr + j), nI = __ldg(d.ci_ptr + j + 1) - ci0;
    const int cf0 = __ldg(d.cf_ptr + j);
    const int total = hc.e_end;
    for (int b = threadIdx.x; b < D; b += blockDim.x) sb[b] = HBin{0, 0, 0, 0, 0, 0};
    __syncthreads();
    const int v0 = chunk * kHistChunk;
    const int v1 = min(total, v0 + kHistChunk);
    Acc acc{0, 0, 0, 0};
    for (int v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
        Half h[2];
        gen_entry(d, ci0, cf0, nI, v, xb, true, l, u, acc, h[0], h[1]);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            if (h[q].type == 0) continue;
            int b = (int)(h[q].t - l);
            HBin *p = sb + b;
            atomicAdd(&p->np, 1);
            if (h[q].type == 1) {
                atomicAdd(reinterpret_cast<unsigned long long *>(&p->sm), (unsigned long long)h[q].D);
                atomicAdd(&p->cm, -1);
            } else {
                atomicAdd(reinterpret_cast<unsigned long long *>(&p->sp), (unsigned long long)h[q].D);
                atomicAdd(&p->cp, 1);
            }
        }
    }
    if (chunk == 0 && threadIdx.x == 0) {
        atomicAdd(&sb[0].np, 1);      // bound entry (l, -1, 0)
        atomicAdd(&sb[D - 1].np, 1);  // bound entry (u, -1, 0)
    }
    warp_allreduce_acc(acc);
    HistAcc *ha = d.hacc + tl.begin;
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(reinterpret_cast<unsigned long long *>(&ha->beta), (unsigned long long)acc.beta);
        atomicAdd(reinterpret_cast<unsigned long long *>(&ha->alpha), (unsigned long long)acc.alpha);
        atomicAdd(&ha->beta_c, acc.beta_c);
        atomicAdd(&ha->alpha_c, acc.alpha_c);
    }
    __syncthreads();
    HBin *gb = d.hbins + hc.bin_off;
    for (int b = threadIdx.x; b < D; b += blockDim.x) {
        HBin s = sb[b];
        if (s.np | s.cm | s.cp) {
            if (s.sm) atomicAdd(reinterpret_cast<unsigned long long *>(&gb[b].sm), (unsigned long long)s.sm);
            if (s.sp) atomicAdd(reinterpret_cast<unsigned long long *>(&gb[b].sp), (unsigned long long)s.sp);
            if (s.cm) atomicAdd(&gb[b].cm, s.cm);
            if (s.cp) atomicAdd(&gb[b].cp, s.cp);
            if (s.np) atomicAdd(&gb[b].np, s.np);
        }
    }
    __threadfence();
    __syncthreads();
    __shared__ int s_last;
    if (threadIdx.x == 0) s_last = (atomicAdd(&ha->ticket, 1u) == (unsigned)(hc.nchunks - 1));
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // last CTA of the column: scan the bins in value order
    const long long beta = __ldcg(&ha->beta), alpha = __ldcg(&ha->alpha);
    const int bc = __ldcg(&ha->beta_c), ac = __ldcg(&ha->alpha_c);
    const long long iter = d.ctl->iter, nviol = d.ctl->nviol, bestnv = d.ctl->best_nviol;
    const int per = (D + blockDim.x - 1) / blockDim.x;
    const int b0 = threadIdx.x * per;
    long long run = 0;
    int runc = 0;
    for (int q = 0; q < per; ++q) {
        int b = b0 + q;
        if (b >= D) break;
        run += __ldcg(&gb[b].sm) + __ldcg(&gb[b].sp);
        runc += __ldcg(&gb[b].cm) + __ldcg(&gb[b].cp);
    }
    __shared__ long long wsum[32];
    __shared__ int wsumc[32];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long tot = run;
    int totc = runc;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        long long a = __shfl_up_sync(FULLMASK, tot, off);
        int b = __shfl_up_sync(FULLMASK, totc, off);
        if (lane >= off) { tot += a; totc += b; }
    }
    if (lane == 31) { wsum[warp] = tot; wsumc[warp] = totc; }
    __syncthreads();
    if (warp == 0) {
        int nw = blockDim.x >> 5;
        long long v = lane < nw ? wsum[lane] : 0;
        int vc = lane < nw ? wsumc[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            long long a = __shfl_up_sync(FULLMASK, v, off);
            int b = __shfl_up_sync(FULLMASK, vc, off);
            if (lane >= off) { v += a; vc += b; }
        }
        if (lane < nw) { wsum[lane] = v; wsumc[lane] = vc; }
    }
    __syncthreads();
    long long P = (tot - run) + (warp > 0 ? wsum[warp - 1] : 0);
    int Pc = (totc - runc) + (warp > 0 ? wsumc[warp - 1] : 0);
    VCand vb{0, 0.0, 0, 0};
    for (int q = 0; q < per; ++q) {
        int b = b0 + q;
        if (b >= D) break;
        HBin s;
        s.sm = __ldcg(&gb[b].sm); s.sp = __ldcg(&gb[b].sp);
        s.cm = __ldcg(&gb[b].cm); s.cp = __ldcg(&gb[b].cp); s.np = __ldcg(&gb[b].np);
        long long sig_part = P + s.sm;
        int dc_part = Pc + s.cm;
        P += s.sm + s.sp;
        Pc += s.cm + s.cp;
        if (s.np == 0) continue;
        double t = l + (double)b;
        if (t == xb) continue;
        bool right = t > xb;
        long long sg = beta + sig_part + (right ? alpha : 0);
        int dcv = bc + dc_part + (right ? ac : 0);
        if (!admissible(right, j, dcv, d, iter, nviol, bestnv)) continue;
        VCand c{sg, t, dcv, 1};
        if (vc_better(c, vb, xb)) vb = c;
    }
    vb = block_reduce_vc(vb, xb);
    // reset the column's scratch for the next pass
    for (int b = threadIdx.x; b < D; b += blockDim.x) gb[b] = HBin{0, 0, 0, 0, 0, 0};
    if (threadIdx.x == 0) {
        Cand best{0, kNoVar, 0, 0.0};
        finish_column(d, o, j, xb, vb, best);
        d.block_best[hc.slot] = best;
        *ha = HistAcc{0, 0, 0, 0, 0u, 0};
    }
}

// Fixed variables and the default of every per-variable output.
__global__ void k_fill_outputs(Dev d, VarOut o)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d.n; j += gridDim.x * blockDim.x) {
        if (o.xhat) o.xhat[j] = d.x[j];
        if (o.s) o.s[j] = 0;
        if (o.dc) o.dc[j] = 0;
    }
}

// ------------------------------------------------------------- selection

__global__ void __launch_bounds__(1024) k_select(Dev d, int gate)
{
    if (gated_done(d, gate)) return;
    Cand best{0, kNoVar, 0, 0.0};
    for (int b = threadIdx.x; b < d.n_block_best; b += blockDim.x) {
        Cand c = d.block_best[b];
        if (c.s > 0 && cand_better(c.s, c.var, best.s, best.var)) best = c;
    }
    best = block_reduce_cand(best);
    if (threadIdx.x == 0) {
        Ctl *c = d.ctl;
        if (best.s > 0 && best.var != kNoVar) {
            c->mv_var = best.var;
            c->mv_s = best.s;
            c->mv_dc = best.dc;
            c->mv_new = best.xhat;
            c->mv_old = d.x[best.var];
        } else {
            c->mv_var = -1;
            c->mv_s = 0;
            c->mv_dc = 0;
            c->mv_new = 0.0;
            c->mv_old = 0.0;
        }
    }
}

__global__ void k_set_move(Dev d, int var, double nv)
{
    Ctl *c = d.ctl;
    c->mv_var = var;
    c->mv_s = 0;
    c->mv_dc = 0;
    c->mv_new = var >= 0 ? nv : 0.0;
    c->mv_old = var >= 0 ? d.x[var] : 0.0;
}

// ------------------------------------------------------------------- apply

__global__ void __launch_bounds__(kApplyThreads) k_apply(Dev d, int gate)
{
    if (gated_done(d, gate)) return;
    Ctl *c = d.ctl;
    const int var = c->mv_var;
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int gstride = gridDim.x * blockDim.x;
    long long local = 0;
    if (var >= 0) {
        const double dl = __dsub_rn(c->mv_new, c->mv_old);
        const long long di = (long long)dl;
        int e0 = d.ci_ptr[var], e1 = d.ci_ptr[var + 1];
        for (int e = e0 + gtid; e < e1; e += gstride) {
            int i = d.ci_row[e];
            long long a = d.ci_val[e];
            RowState *p = d.rs + i;
            long long r0 = p->r;
            long long r1 = r0 + a * di;
            p->r = r1;
            local += (long long)(r1 > 0) - (long long)(r0 > 0);
            if (p->w2 >= 0) local += (long long)(-r1 > 0) - (long long)(-r0 > 0);
        }
        int f0 = d.cf_ptr[var], f1 = d.cf_ptr[var + 1];
        for (int e = f0 + gtid; e < f1; e += gstride) {
            int i = d.cf_row[e];
            double a = d.cf_val[e];
            RowState *p = d.rs + i;
            double eps = d.eps[i];
            double r0 = __longlong_as_double(p->r);
            double r1 = __dadd_rn(r0, __dmul_rn(a, dl));
            p->r = __double_as_longlong(r1);
            local += (long long)(r1 > eps) - (long long)(r0 > eps);
            if (p->w2 >= 0) local += (long long)(-r1 > eps) - (long long)(-r0 > eps);
        }
    } else {
        for (int i = gtid; i < d.m; i += gstride) {
            RowState *p = d.rs + i;
            RowState s = *p;
            bool v1, v2;
            if (d.row_int[i]) { v1 = s.r > 0; v2 = -s.r > 0; }
            else {
                double r = __longlong_as_double(s.r);
                double eps = d.eps[i];
                v1 = r > eps;
                v2 = -r > eps;
            }
            if (v1) p->w1 = s.w1 + 1;
            if (s.w2 >= 0 && v2) p->w2 = s.w2 + 1;
        }
    }
    // block reduce of the violation-count change
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) local += __shfl_xor_sync(FULLMASK, local, off);
    __shared__ long long red[kApplyThreads / 32];
    __shared__ int s_last;
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = local;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int w = 0; w < kApplyThreads / 32; ++w) t += red[w];
        if (t) atomicAdd(reinterpret_cast<unsigned long long *>(&c->nviol_delta), (unsigned long long)t);
        __threadfence();
        s_last = (atomicAdd(&c->apply_ticket, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last || threadIdx.x != 0) return;
    __threadfence();
    // last CTA: finish the iteration
    long long nv = c->nviol + (long long)__ldcg(reinterpret_cast<const long long *>(&c->nviol_delta));
    c->nviol = nv;
    c->nviol_delta = 0;
    c->apply_ticket = 0;
    const long long it = c->iter;
    if (var >= 0) {
        d.x[var] = c->mv_new;
        int stamp = (int)(it + 1 + d.tenure);
        if (c->mv_new > c->mv_old) d.tabu_dec[var] = stamp;
        else d.tabu_inc[var] = stamp;
        c->moves += 1;
    } else {
        c->bumps += 1;
    }
    c->iter = it + 1;
    if (nv < c->best_nviol) c->best_nviol = nv;
    if (nv == 0 && c->feasible_iter < 0) {
        c->feasible_iter = it + 1;
        c->t_feas_ns = global_ns();
    }
    if ((c->stop_at_feasible && nv == 0) || it + 1 >= c->max_iter) c->done = 1;
}

// --------------------------------------------------------- state handling

// r = (sum of a x in CSR order) - b per physical row; exact int64 on integral rows.
__global__ void k_residuals(Dev d)
{
    long long local = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.m; i += gridDim.x * blockDim.x) {
        long long p0 = d.row_ptr[i], p1 = d.row_ptr[i + 1];
        RowState *p = d.rs + i;
        if (d.row_int[i]) {
            long long y = 0;
            for (long long e = p0; e < p1; ++e) y += (long long)d.row_val[e] * (long long)d.x[d.col_idx[e]];
            long long r = y - (long long)d.rhs[i];
            p->r = r;
            local += (r > 0) + (p->w2 >= 0 && -r > 0);
        } else {
            double y = 0.0;
            for (long long e = p0; e < p1; ++e) y = __dadd_rn(y, __dmul_rn(d.row_val[e], d.x[d.col_idx[e]]));
            double r = __dsub_rn(y, d.rhs[i]);
            p->r = __double_as_longlong(r);
            double eps = d.eps[i];
            local += (r > eps) + (p->w2 >= 0 && -r > eps);
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) local += __shfl_xor_sync(FULLMASK, local, off);
    if ((threadIdx.x & 31) == 0 && local)
        atomicAdd(reinterpret_cast<unsigned long long *>(&d.ctl->nviol), (unsigned long long)local);
}

__global__ void k_finish_set_state(Dev d, long long iter, long long best_nviol, int use_best)
{
    Ctl *c = d.ctl;
    c->iter = iter;
    c->best_nviol = use_best ? best_nviol : c->nviol;
    c->feasible_iter = c->nviol == 0 ? iter : -1;
    c->done = 0;
    c->max_iter = LLONG_MAX;
    c->moves = 0;
    c->bumps = 0;
    c->nviol_delta = 0;
    c->apply_ticket = 0;
    c->select_ticket = 0;
    c->error = 0;
}

__global__ void k_begin_run(Dev d, long long max_iters, int stop_at_feasible)
{
    Ctl *c = d.ctl;
    c->max_iter = c->iter + max_iters;
    c->stop_at_feasible = stop_at_feasible;
    c->t_start_ns = global_ns();
    if (c->nviol == 0) { c->feasible_iter = c->iter; c->t_feas_ns = c->t_start_ns; }
    else { c->feasible_iter = -1; c->t_feas_ns = 0; }
    c->done = ((stop_at_feasible && c->nviol == 0) || max_iters <= 0) ? 1 : 0;
}

__global__ void k_pack_w(Dev d, const int *w)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.m; i += gridDim.x * blockDim.x) {
        int k = d.nrow_base[i];
        d.rs[i].w1 = w[k];
        if (d.rs[i].w2 >= 0) d.rs[i].w2 = w[k + 1];
    }
}

__global__ void k_unpack_w(Dev d, int *w)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.m; i += gridDim.x * blockDim.x) {
        int k = d.nrow_base[i];
        RowState s = d.rs[i];
        w[k] = s.w1;
        if (s.w2 >= 0) w[k + 1] = s.w2;
    }
}

__global__ void k_unpack_r(Dev d, double *r)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.m; i += gridDim.x * blockDim.x) {
        int k = d.nrow_base[i];
        RowState s = d.rs[i];
        double v = d.row_int[i] ? (double)s.r : __longlong_as_double(s.r);
        r[k] = v;
        if (s.w2 >= 0) r[k + 1] = -v;
    }
}

__global__ void k_widen(int n, const int *a, long long *b)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) b[j] = a[j];
}

__global__ void k_narrow(int n, const long long *a, int *b)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) b[j] = (int)a[j];
}

// ---------------------------------------------------------------- launchers

static int grid_for(long long n, int threads, int cap = 152 * 8)
{
    long long g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

cudaError_t setup_kernel_attributes(int cta_smem, int hist_smem)
{
    cudaError_t e = cudaSuccess;
    if (cta_smem > 0)
        e = cudaFuncSetAttribute(k_eval_cta, cudaFuncAttributeMaxDynamicSharedMemorySize, cta_smem);
    if (e == cudaSuccess && hist_smem > 0)
        e = cudaFuncSetAttribute(k_eval_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, hist_smem);
    return e;
}

cudaError_t launch_eval_gated(const Dev &d, const LaunchPlan &p, const VarOut &o, int gate, cudaStream_t st)
{
    if (o.xhat || o.s || o.dc) k_fill_outputs<<<grid_for(d.n, 256), 256, 0, st>>>(d, o);
    if (p.n_small) k_eval_small<<<p.n_small, kEvalThreads, 0, st>>>(d, p.tiles_small, o, gate);
    if (p.n_cta) k_eval_cta<<<p.n_cta, kCtaThreads, p.cta_smem, st>>>(d, p.tiles_cta, o, p.n_small, gate);
    if (p.n_hist_tiles) k_eval_hist<<<p.n_hist_tiles, kHistThreads, p.hist_smem, st>>>(d, p.tiles_hist, o, gate);
    return cudaGetLastError();
}

cudaError_t launch_eval(const Dev &d, const LaunchPlan &p, const VarOut &o, cudaStream_t st)
{
    return launch_eval_gated(d, p, o, 0, st);
}

cudaError_t launch_select_gated(const Dev &d, int gate, cudaStream_t st)
{
    k_select<<<1, 1024, 0, st>>>(d, gate);
    return cudaGetLastError();
}

cudaError_t launch_select(const Dev &d, cudaStream_t st) { return launch_select_gated(d, 0, st); }

cudaError_t launch_apply_gated(const Dev &d, const LaunchPlan &p, int gate, cudaStream_t st)
{
    k_apply<<<p.apply_blocks, kApplyThreads, 0, st>>>(d, gate);
    return cudaGetLastError();
}

cudaError_t launch_apply(const Dev &d, const LaunchPlan &p, cudaStream_t st) { return launch_apply_gated(d, p, 0, st); }

cudaError_t launch_set_move(const Dev &d, int var, double nv, cudaStream_t st)
{
    k_set_move<<<1, 1, 0, st>>>(d, var, nv);
    return cudaGetLastError();
}

cudaError_t launch_residuals(const Dev &d, cudaStream_t st)
{
    k_residuals<<<grid_for(d.m, 128, 152 * 16), 128, 0, st>>>(d);
    return cudaGetLastError();
}

cudaError_t launch_finish_set_state(const Dev &d, long long iter, long long best_nviol, int use_best, cudaStream_t st)
{
    k_finish_set_state<<<1, 1, 0, st>>>(d, iter, best_nviol, use_best);
    return cudaGetLastError();
}

cudaError_t launch_begin_run(const Dev &d, long long max_iters, int stop_at_feasible, cudaStream_t st)
{
    k_begin_run<<<1, 1, 0, st>>>(d, max_iters, stop_at_feasible);
    return cudaGetLastError();
}

cudaError_t launch_pack_w(const Dev &d, const int *w, cudaStream_t st)
{
    k_pack_w<<<grid_for(d.m, 256), 256, 0, st>>>(d, w);
    return cudaGetLastError();
}

cudaError_t launch_unpack_w(const Dev &d, int *w, cudaStream_t st)
{
    k_unpack_w<<<grid_for(d.m, 256), 256, 0, st>>>(d, w);
    return cudaGetLastError();
}

cudaError_t launch_unpack_r(const Dev &d, double *r, cudaStream_t st)
{
    k_unpack_r<<<grid_for(d.m, 256), 256, 0, st>>>(d, r);
    return cudaGetLastError();
}

cudaError_t launch_tabu_convert(int n, const int *a, long long *b, cudaStream_t st)
{
    k_widen<<<grid_for(n, 256), 256, 0, st>>>(n, a, b);
    return cudaGetLastError();
}

cudaError_t launch_tabu_narrow(int n, const long long *a, int *b, cudaStream_t st)
{
    k_narrow<<<grid_for(n, 256), 256, 0, st>>>(n, a, b);
    return cudaGetLastError();
}

}  // namespace chap
