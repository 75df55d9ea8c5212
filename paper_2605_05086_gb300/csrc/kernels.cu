// Kernels of the best-shift tabu search (sm_103a).
//
// One tabu iteration = best-shift pass (evaluation kernels) -> selection -> apply.
//
//  * Binary columns (k_eval_bin): the only move is the flip (Sec. 3.1, "Best
//    Shift Moves"); its score is the sum of the penalty changes over the
//    column.  A group of G lanes (2 .. 16 by mean column length) scores one
//    column: coalesced reads of the column's nonzeros, one row-state gather per
//    nonzero, branch-free penalty changes in registers.
//  * Other columns: Algorithm 1 (sort -> scan -> argmax).  Each normalised half
//    of a nonzero gives at most one entry (`half_case`, the case table of
//    Algorithm 1): an a<0 half a "pre" entry (its delta counts at t), an a>0
//    half a "post" entry (t is a candidate and its delta counts right of t: the
//    two entries of Algorithm 1 merged); entries left of l fold into beta,
//    entries right of u are dropped.  Short columns (k_eval_nb, at most 128
//    entries) place every half by products first and compute exact breakpoints
//    only for the undecided ones, 32 at a time; their lists are sorted by
//    group bitonic networks in registers.  Longer columns are bitonic-sorted in
//    shared memory by one CTA (k_eval_cta, up to 8192 entries) or
//    counting-sorted across many CTAs (k_eval_hist, long integer columns).
//  * Every CTA reduces its columns to one candidate; the CTA that writes the
//    last candidate slot reduces them all into the move (finish_pass: largest
//    score, then lowest variable; k_select only when no evaluation CTA runs).
//  * k_apply_move walks the chosen column and updates the residuals
//    incrementally (Sec. 3.1, "Memory Considerations", first point); when no
//    positive move exists k_apply_bump adds 1 to the weight of every violated
//    normalised row.  The CTA that ends the iteration (finish_iteration) also
//    tightens the objective cutoff row when the iteration ends feasible
//    (Sec. 3.2) and copies x to the best solution.
//  * Optional kept binary scores (k_eval_bin_lazy, k_bin_scan, k_lazy_mark):
//    the flips of the binaries in the moved column's rows are re-evaluated,
//    tabu and aspiration are applied to the kept values of all of them.
//
// Exactness: integral rows use int64 residuals and integer arithmetic only;
// non-integral rows keep r, eps - r and eps + r (double, explicit
// round-to-nearest, no contraction), and every comparison of doubles is done on
// order-preserving integer keys.  Scores are int64 half-weight counts.
#include "chap_internal.h"

#include <cooperative_groups.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <mutex>
#include <type_traits>

namespace chap {

#define FULLMASK 0xffffffffu

constexpr unsigned long long kSign = 0x8000000000000000ull;
constexpr unsigned long long kPadKey = ~0ull;
constexpr int kNoVar = INT_MAX;
constexpr long long kDdMax = 1LL << 60;

// ---------------------------------------------------------------- helpers

// Order-preserving maps of doubles and int64 to unsigned 64-bit keys.
__device__ __forceinline__ unsigned long long dkey(double t)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(t);
    return (b & kSign) ? ~b : (b | kSign);
}

__device__ __forceinline__ double dkey_val(unsigned long long k)
{
    unsigned long long b = (k & kSign) ? (k & ~kSign) : ~k;
    return __longlong_as_double((long long)b);
}

__device__ __forceinline__ unsigned long long ikey(long long t) { return (unsigned long long)t ^ kSign; }
__device__ __forceinline__ long long ikey_val(unsigned long long k) { return (long long)(k ^ kSign); }

// Sign of a double that is never -0.0 here (margins are eps -+ r rounded to nearest).
__device__ __forceinline__ bool dneg(double v) { return __double_as_longlong(v) < 0; }
__device__ __forceinline__ bool dgt(double a, double b) { return dkey(a) > dkey(b); }
// -v by flipping the sign bit in an integer register: written as PTX so that
// the compiler cannot turn it into an FP64 negation (GB300's FP64 pipe is
// narrow, and these flips run once per nonzero).
__device__ __forceinline__ double dflip(double v)
{
    long long b;
    asm("xor.b64 %0, %1, 0x8000000000000000;" : "=l"(b) : "l"(__double_as_longlong(v)));
    return __longlong_as_double(b);
}

// Conversions between doubles and integers run on GB300's narrow FP64 pipe;
// the per-column setup below uses these integer-only forms instead.
__device__ __forceinline__ bool dfinite(double v) { return ((__double_as_longlong(v) >> 52) & 0x7ff) != 0x7ff; }

// Exact int64 value of an integral double with |v| < 2^63.
__device__ __forceinline__ long long dbl_int(double v)
{
    const long long b = __double_as_longlong(v);
    const int ex = (int)((b >> 52) & 0x7ff);
    if (ex == 0) return 0;  // +-0 (an integral double is never subnormal)
    const long long mant = (b & 0xfffffffffffffLL) | (1LL << 52);
    const int sh = ex - 1075;  // |v| = mant * 2^sh
    const long long m = sh >= 0 ? (mant << sh) : (sh <= -53 ? 0 : (mant >> -sh));
    return b < 0 ? -m : m;
}

// Float value of an integer with |v| < 2^22: add v to the bits of 1.5 * 2^23
// and subtract that constant again (both exact; integer and FP32 pipes).
__device__ __forceinline__ float small_int_f(long long v) { return __int_as_float(0x4B400000 + (int)v) - 12582912.0f; }

// Single-precision estimate of a double from its bits (mantissa truncated,
// relative error < 2^-23); ok is cleared when |v| is outside the normal float
// range (zero is exact).
__device__ __forceinline__ float approx_f(double v, bool &ok)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    const int e = (int)((b >> 52) & 0x7ff) - 1023;
    if (e > 127) { ok = false; return __int_as_float(sign | 0x7f7fffffu); }
    if (e < -126) {
        if ((b << 1) != 0ull) ok = false;
        return __int_as_float(sign);
    }
    return __int_as_float(sign | ((unsigned)(e + 127) << 23) | (unsigned)((b >> 29) & 0x7fffffu));
}

// floor(n / d) for d != 0: single precision estimate and exact integer correction
// when the operands are small, int64 division otherwise.
__device__ __forceinline__ long long floor_div(long long n, long long d)
{
    if (d < 0) { n = -n; d = -d; }
    if (n > -(1LL << 22) && n < (1LL << 22) && d < (1LL << 22)) {
        int ni = (int)n, di = (int)d;
        int q = __float2int_rd(__fdividef((float)ni, (float)di));
        int r = ni - q * di;
        while (r < 0) { --q; r += di; }
        while (r >= di) { ++q; r -= di; }
        return q;
    }
    long long q = n / d, r = n % d;
    if (r < 0) --q;
    return q;
}

__device__ __forceinline__ long long ceil_div(long long n, long long d) { return -floor_div(-n, d); }

__device__ __forceinline__ long long clamp_dd(long long v)
{
    return v > kDdMax ? kDdMax : (v < -kDdMax ? -kDdMax : v);
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int4 ld_row16(const RowState *p) { return __ldg(reinterpret_cast<const int4 *>(p)); }

// The whole 32-byte row state in one 256-bit load: one L1 wavefront per lane
// instead of one for each 16-byte half (the per-nonzero gathers of the
// evaluation kernels are bound by these wavefronts).  Row states are 32-byte
// aligned and not written while an evaluation kernel runs.
__device__ __forceinline__ void ld_row32(const RowState *p, int4 &s0, int4 &s1)
{
    unsigned long long a, b, c, e;
    asm("ld.global.nc.v4.u64 {%0, %1, %2, %3}, [%4];" : "=l"(a), "=l"(b), "=l"(c), "=l"(e) : "l"(p));
    s0 = make_int4((int)(unsigned)a, (int)(unsigned)(a >> 32), (int)(unsigned)b, (int)(unsigned)(b >> 32));
    s1 = make_int4((int)(unsigned)c, (int)(unsigned)(c >> 32), (int)(unsigned)e, (int)(unsigned)(e >> 32));
}

__device__ __forceinline__ long long row_r(const int4 &v)
{
    return (long long)(((unsigned long long)(unsigned)v.y << 32) | (unsigned)v.x);
}

__device__ __forceinline__ double i4_double_lo(const int4 &v)
{
    return __longlong_as_double((long long)(((unsigned long long)(unsigned)v.y << 32) | (unsigned)v.x));
}

__device__ __forceinline__ double i4_double_hi(const int4 &v)
{
    return __longlong_as_double((long long)(((unsigned long long)(unsigned)v.w << 32) | (unsigned)v.z));
}

// Global candidate order: larger score, then lower variable index.
__device__ __forceinline__ bool cand_better(long long s1, int v1, long long s2, int v2)
{
    return s1 > s2 || (s1 == s2 && v1 < v2);
}

__device__ __forceinline__ void warp_reduce_cand(Cand &c)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        long long s2 = __shfl_xor_sync(FULLMASK, c.s, o);
        int v2 = __shfl_xor_sync(FULLMASK, c.var, o);
        int d2 = __shfl_xor_sync(FULLMASK, c.dc, o);
        double x2 = __shfl_xor_sync(FULLMASK, c.xhat, o);
        if (cand_better(s2, v2, c.s, c.var)) { c.s = s2; c.var = v2; c.dc = d2; c.xhat = x2; }
    }
}

// Reduce one candidate per thread to thread 0 of the block.
__device__ Cand block_reduce_cand(Cand c)
{
    __shared__ Cand red[32];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    warp_reduce_cand(c);
    if (lane == 0) red[warp] = c;
    __syncthreads();
    int nw = (blockDim.x + 31) >> 5;
    if (warp == 0) {
        Cand r = lane < nw ? red[lane] : Cand{0, kNoVar, 0, 0.0};
        warp_reduce_cand(r);
        c = r;
    }
    __syncthreads();
    return c;
}

// Column being evaluated: keys of xbar and of the bounds, single-precision
// estimates for the pre-filters, entry ranges.
struct ColCtx {
    int j;
    bool isint;
    bool fok;              // the single-precision estimates below are usable
    bool inc_free, dec_free;  // increasing / decreasing x_j is not tabu at this iteration
    double xb;
    long long xbi;
    unsigned long long kxb, kl, ku;
    long long lo, hi;      // integer: l - xbar, u - xbar (+-2^62 for infinite bounds)
    float lof, hif;        // integer: the same as floats (+-inf unless |.| < 2^22)
    float dlf, duf, xaf;   // continuous: estimates of xbar - l, xbar - u (+-inf for infinite bounds), |xbar|
    int ci0, nI, cf0, nF;
};

__device__ __forceinline__ ColCtx make_col(const Dev &d, int q, long long iter)
{
    ColCtx c;
    c.j = __ldg(d.var_list + q);
    const int j = c.j;
    c.inc_free = iter >= (long long)d.tabu_inc[j];
    c.dec_free = iter >= (long long)d.tabu_dec[j];
    c.isint = __ldg(d.vtype + j) != kVarCont;
    c.xb = d.x[j];
    const double l = __ldg(d.lb + j), u = __ldg(d.ub + j);
    const bool fl = dfinite(l), fu = dfinite(u);
    c.fok = true;
    if (c.isint) {
        c.xbi = dbl_int(c.xb);
        c.kxb = ikey(c.xbi);
        const long long li = fl ? dbl_int(l) : LLONG_MIN, ui = fu ? dbl_int(u) : LLONG_MAX;
        c.kl = ikey(li);
        c.ku = ikey(ui);
        c.lo = fl ? li - c.xbi : -(1LL << 62);
        c.hi = fu ? ui - c.xbi : (1LL << 62);
        c.lof = c.lo > -(1LL << 22) ? small_int_f(c.lo) : -INFINITY;
        c.hif = c.hi < (1LL << 22) ? small_int_f(c.hi) : INFINITY;
        c.dlf = c.duf = c.xaf = 0.0f;
    } else {
        c.xbi = 0;
        c.kxb = dkey(c.xb);
        c.kl = fl ? dkey(l) : dkey(-1.7976931348623157e308);
        c.ku = fu ? dkey(u) : dkey(1.7976931348623157e308);
        c.lo = c.hi = 0;
        c.lof = c.hif = 0.0f;
        c.dlf = fl ? approx_f(__dsub_rn(c.xb, l), c.fok) : INFINITY;
        c.duf = fu ? approx_f(__dsub_rn(c.xb, u), c.fok) : -INFINITY;
        c.xaf = fabsf(approx_f(c.xb, c.fok));
    }
    c.ci0 = __ldg(d.ci_ptr + q);
    c.nI = __ldg(d.ci_ptr + q + 1) - c.ci0;
    c.cf0 = __ldg(d.cf_ptr + q);
    c.nF = __ldg(d.cf_ptr + q + 1) - c.cf0;
    return c;
}

__device__ __forceinline__ double key_value(const ColCtx &c, unsigned long long k)
{
    return c.isint ? (double)ikey_val(k) : dkey_val(k);
}

// Per-variable candidate; order (Eq. best_move ties): larger score, then smaller
// |t - xbar|, then smaller t.  Distances are only computed on score ties.
struct VCand {
    long long s;
    unsigned long long key;
    int dc;
    int valid;
};

__device__ __forceinline__ bool vc_better(const VCand &a, const VCand &b, const ColCtx &c)
{
    if (!a.valid) return false;
    if (!b.valid) return true;
    if (a.s != b.s) return a.s > b.s;
    if (c.isint) {
        long long ta = ikey_val(a.key), tb = ikey_val(b.key);
        unsigned long long da = (unsigned long long)(ta > c.xbi ? ta - c.xbi : c.xbi - ta);
        unsigned long long db = (unsigned long long)(tb > c.xbi ? tb - c.xbi : c.xbi - tb);
        if (da != db) return da < db;
    } else {
        double da = fabs(__dsub_rn(dkey_val(a.key), c.xb)), db = fabs(__dsub_rn(dkey_val(b.key), c.xb));
        if (da != db) return dkey(da) < dkey(db);
    }
    return a.key < b.key;
}

__device__ __forceinline__ void warp_reduce_vc(VCand &v, const ColCtx &c)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        VCand p;
        p.s = __shfl_xor_sync(FULLMASK, v.s, o);
        p.key = __shfl_xor_sync(FULLMASK, v.key, o);
        p.dc = __shfl_xor_sync(FULLMASK, v.dc, o);
        p.valid = __shfl_xor_sync(FULLMASK, v.valid, o);
        if (vc_better(p, v, c)) v = p;
    }
}

__device__ VCand block_reduce_vc(VCand v, const ColCtx &c)
{
    __shared__ VCand red[32];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    warp_reduce_vc(v, c);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    int nw = (blockDim.x + 31) >> 5;
    if (warp == 0) {
        VCand r = lane < nw ? red[lane] : VCand{0, 0ull, 0, 0};
        warp_reduce_vc(r, c);
        v = r;
    }
    __syncthreads();
    return v;
}

// Admissibility under tabu and aspiration.
__device__ __forceinline__ bool admissible(bool increase, int j, int dc, const Dev &d, long long iter,
                                           long long nviol, long long bestnv)
{
    int stamp = increase ? d.tabu_inc[j] : d.tabu_dec[j];
    return iter >= (long long)stamp || (nviol + (long long)dc < bestnv);
}

// A candidate of column c at key k with score sg and count change dcv:
// admissible when its direction is not tabu, or by aspiration.
__device__ __forceinline__ void consider(VCand &vb, const ColCtx &c, unsigned long long k, long long sg, int dcv,
                                         long long nviol, long long bestnv)
{
    if (k == c.kxb) return;
    const bool inc = k > c.kxb;
    if (!((inc ? c.inc_free : c.dec_free) || nviol + (long long)dcv < bestnv)) return;
    const VCand n{sg, k, dcv, 1};
    if (vc_better(n, vb, c)) vb = n;
}

// Column result -> optional per-variable outputs and the caller's running best.
__device__ __forceinline__ void finish_column(const Dev &d, const VarOut &o, const ColCtx &c, const VCand &b,
                                              Cand &best)
{
    bool mv = b.valid && b.s > 0;
    double xh = mv ? key_value(c, b.key) : c.xb;
    if (o.xhat) o.xhat[c.j] = xh;
    if (o.s) o.s[c.j] = mv ? b.s : 0;
    if (o.dc) o.dc[c.j] = mv ? b.dc : 0;
    if (mv && cand_better(b.s, c.j, best.s, best.var)) best = Cand{b.s, c.j, b.dc, xh};
}

__device__ __forceinline__ bool gated_done(const Dev &d, int gate)
{
    return gate && *(volatile int *)&d.ctl->done;
}

// Selection of the pass (Sec. 3.1: the best admissible move over all
// variables), folded into the evaluation kernels: after writing its candidate
// slot every CTA takes a ticket, and the CTA that writes the last slot reduces
// all of them (larger score, then lower variable) into the move record.  All
// threads of the CTA call it; the ticket is reset for the next pass.
__device__ void finish_pass(const Dev &d)
{
    __shared__ int s_sel;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_sel = atomicAdd(&d.ctl->select_ticket, 1u) == (unsigned)(d.n_block_best - 1);
    }
    __syncthreads();
    if (!s_sel) return;
    __threadfence();
    Cand best{0, kNoVar, 0, 0.0};
    for (int b = threadIdx.x; b < d.n_block_best; b += blockDim.x) {
        const Cand *p = d.block_best + b;
        const long long cs = __ldcg(&p->s);
        const int cv = __ldcg(&p->var);
        if (cs > 0 && cand_better(cs, cv, best.s, best.var)) best = Cand{cs, cv, __ldcg(&p->dc), __ldcg(&p->xhat)};
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
        c->select_ticket = 0u;
        c->pass_best = 0;
    }
}

// ------------------------------------------------------- binary flip scoring
//
// The only move of a binary variable is the flip (Sec. 3.1, "Best Shift
// Moves"); its score is the sum over the column of the penalty changes of the
// normalised halves.  A group of G lanes scores one column (32 / G columns
// per warp, persistent grid, columns ordered by length; G = 2 .. 16 from the
// mean column length): the lanes read the column's nonzeros coalesced, gather
// the row states and add the penalty changes branch-free in registers; a
// shuffle reduction closes the column.

constexpr int kEvalWarps = kEvalThreads / 32;

// Penalty change of a half in weight units for violated-before v0,
// violated-after v1 and the sign of the residual change (Sec. 3.1, Scoring
// Functions): becomes violated -2, becomes satisfied +2, stays violated +1
// when the residual falls and -1 when it grows (half-weight units).
__device__ __forceinline__ int flip_f(bool v0, bool v1, bool dec)
{
    return 2 * ((int)v0 - (int)v1) + ((v0 && v1) ? (dec ? 1 : -1) : 0);
}

// Largest value of v over the groups of G lanes of the warp.
template <int G>
__device__ __forceinline__ int groups_max(int v)
{
#pragma unroll
    for (int o2 = 16; o2 >= G; o2 >>= 1) v = max(v, __shfl_xor_sync(FULLMASK, v, o2));
    return v;
}


// Flip score terms of one nonzero of an integral row (int64 residual r; a rise
// of x_j changes r by a; the second half of an "=" row has residual -r and
// change -a) and of a non-integral row (below).
template <bool EQ>
__device__ __forceinline__ void flip_int(const int4 &st, int av, bool up, long long &s, int &dc)
{
    const long long r = row_r(st);
    const int ad = up ? av : -av;
    const long long r1 = r + ad;
    const bool v0 = r > 0, v1 = r1 > 0;
    s += (long long)flip_f(v0, v1, ad < 0) * st.z;
    dc += (int)v1 - (int)v0;
    if (EQ) {
        const bool u0 = r < 0, u1 = r1 < 0;
        s += (long long)flip_f(u0, u1, ad > 0) * st.w;
        dc += (int)u1 - (int)u0;
    }
}

// Non-integral row: violated <=> m < 0 with m = eps - r of the half; violated
// after the move <=> change > m.
template <bool EQ>
__device__ __forceinline__ void flip_fp(const int4 &s0, const int4 &s1, double av, bool up, long long &s, int &dc)
{
    const double ad = up ? av : dflip(av);
    const bool neg = dneg(ad);
    const double m1 = i4_double_lo(s1);
    const bool v0 = dneg(m1), v1 = dgt(ad, m1);
    s += (long long)flip_f(v0, v1, neg) * s0.z;
    dc += (int)v1 - (int)v0;
    if (EQ) {
        const double m2 = i4_double_hi(s1);
        const bool u0 = dneg(m2), u1 = dgt(dflip(ad), m2);
        s += (long long)flip_f(u0, u1, !neg) * s0.w;
        dc += (int)u1 - (int)u0;
    }
}

// Flip scores of one part of a column (FP: non-integral rows; EQ: "=" rows,
// both halves), one nonzero per lane and round.  The row index and
// coefficient of the next round are loaded while the current round's row
// state is gathered, so a round waits for one memory latency, not two.
template <int G, bool FP, bool EQ>
__device__ __forceinline__ void bin_part(const Dev &d, int e0, int n, int nmax, int sub, bool up, long long &s, int &dc)
{
    using Val = typename std::conditional<FP, double, int>::type;
    const int *rowp = (FP ? d.cf_row : d.ci_row) + e0;
    const Val *valp = reinterpret_cast<const Val *>(FP ? (const void *)d.cf_val : (const void *)d.ci_val) + e0;
    bool ok = sub < n;
    int row = ok ? __ldg(rowp + sub) : 0;
    Val av = ok ? __ldg(valp + sub) : Val(0);
    const int4 z4 = make_int4(0, 0, 0, 0);
    for (int base = 0; base < nmax; base += G) {
        int4 s0, s1 = z4;
        if (!FP) {
            s0 = ok ? ld_row16(d.rs + row) : z4;
        } else {
            s0 = z4;
            if (ok) ld_row32(d.rs + row, s0, s1);
        }
        const int vn = base + G + sub;
        const bool okn = vn < n;
        const int rown = okn ? __ldg(rowp + vn) : 0;
        const Val avn = okn ? __ldg(valp + vn) : Val(0);
        if (!FP) flip_int<EQ>(s0, (int)av, up, s, dc);
        else flip_fp<EQ>(s0, s1, (double)av, up, s, dc);
        ok = okn;
        row = rown;
        av = avn;
    }
}

// Flip score s and violation change dc of the binary column at position q
// (all G lanes of its group take part; every lane returns the column sums),
// with the column's variable j and the flip direction up (0 -> 1).
template <int G>
__device__ __forceinline__ void bin_column(const Dev &d, int q, bool live, int sub, int &j, bool &up, long long &s,
                                           int &dc)
{
    const int qq = live ? q : 0;
    const int ci0 = __ldg(d.ci_ptr + qq), cf0 = __ldg(d.cf_ptr + qq);
    const int cim = __ldg(d.ci_eq + qq), cfm = __ldg(d.cf_eq + qq);
    const int ci1 = live ? __ldg(d.ci_ptr + qq + 1) : ci0, cf1 = live ? __ldg(d.cf_ptr + qq + 1) : cf0;
    j = __ldg(d.var_list + qq);
    up = __double_as_longlong(d.x[j]) == 0;
    const int nIs = live ? cim - ci0 : 0, nIe = ci1 - (live ? cim : ci1);
    const int nFs = live ? cfm - cf0 : 0, nFe = cf1 - (live ? cfm : cf1);
    s = 0;
    dc = 0;
    bin_part<G, false, false>(d, ci0, nIs, groups_max<G>(nIs), sub, up, s, dc);
    bin_part<G, false, true>(d, cim, nIe, groups_max<G>(nIe), sub, up, s, dc);
    bin_part<G, true, false>(d, cf0, nFs, groups_max<G>(nFs), sub, up, s, dc);
    bin_part<G, true, true>(d, cfm, nFe, groups_max<G>(nFe), sub, up, s, dc);
#pragma unroll
    for (int o2 = G >> 1; o2 > 0; o2 >>= 1) {
        s += __shfl_xor_sync(FULLMASK, s, o2);
        dc += __shfl_xor_sync(FULLMASK, dc, o2);
    }
}

template <int G>
__global__ void __launch_bounds__(kEvalThreads) k_eval_bin(Dev d, int ncols, VarOut o, int gate)
{
    if (gated_done(d, gate)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int CPW = 32 / G;   // columns per warp
    const int g = lane / G, sub = lane & (G - 1);
    const long long iter = d.ctl->iter, nviol = d.ctl->nviol, bestnv = d.ctl->best_nviol;
    Cand best{0, kNoVar, 0, 0.0};
    const int nquad = (ncols + CPW - 1) / CPW;
    for (int qd = blockIdx.x * kEvalWarps + warp; qd < nquad; qd += gridDim.x * kEvalWarps) {
        const int q = qd * CPW + g;
        const bool live = q < ncols;
        int j, dc;
        bool up;
        long long s;
        bin_column<G>(d, q, live, sub, j, up, s, dc);
        if (sub == 0 && live) {
            bool mv = s > 0;
            if (mv) {
                const int stamp = up ? d.tabu_inc[j] : d.tabu_dec[j];
                mv = iter >= (long long)stamp || nviol + (long long)dc < bestnv;
            }
            const double xh = up ? 1.0 : 0.0;
            if (o.xhat) o.xhat[j] = mv ? xh : d.x[j];
            if (o.s) o.s[j] = mv ? s : 0;
            if (o.dc) o.dc[j] = mv ? dc : 0;
            if (mv && cand_better(s, j, best.s, best.var)) best = Cand{s, j, dc, xh};
        }
    }
    const Cand b = block_reduce_cand(best);
    if (threadIdx.x == 0) {
        d.block_best[blockIdx.x] = b;
        if (b.s > 0) atomicMax(&d.ctl->pass_best, b.s);
    }
    finish_pass(d);
}

// ------------------------------------------------ row-wise binary flips
//
// k_eval_bin_rows: one thread-block cluster per block of binary columns (see
// RowBin).  Every warp takes 32 rows of its CTA's share at a time: each lane
// loads one row (id, entry range, row state) and the rows' entries are then
// scored 32 at a time in order, each lane finding the row of its entry by a
// binary search over the lanes' entry prefix and reading that row's state
// from the lane that holds it (no per-entry gather).  The flip's penalty
// change (the same terms as the column kernel) goes into the CTA's
// shared-memory accumulators of the block's columns; after a cluster barrier
// every CTA sums its share of the columns over the cluster's CTAs (distributed
// shared memory), applies tabu and aspiration and reduces to its candidate.

template <bool FP>
__device__ __forceinline__ void rb_rows_chunk(const Dev &d, const int *rows, const int *eptr,
                                              const unsigned short *cols, const unsigned char *own, const void *vals,
                                              int k0, int k1, const unsigned *xb, int4 *wrow, long long *sacc,
                                              int *cacc)
{
    const int lane = threadIdx.x & 31;
    const int k = k0 + lane;
    const bool ok = k < k1;
    // this chunk's entries: from the first row's start to the last row's end
    const int ebase = __ldg(eptr + k0);
    const int eend = __ldg(eptr + min(k0 + 32, k1));
    if (ok) {
        const int4 *p = reinterpret_cast<const int4 *>(d.rs + __ldg(rows + k));
        wrow[2 * lane] = __ldg(p);
        if (FP) wrow[2 * lane + 1] = __ldg(p + 1);
    }
    __syncwarp();
    for (int e = ebase + lane; e < eend; e += 32) {
        const int c = __ldg(cols + e);
        const int o = __ldg(own + e);   // lane (row) of the entry inside the chunk
        const int4 r0 = wrow[2 * o];
        const bool up = ((xb[c >> 5] >> (c & 31)) & 1u) == 0;
        long long sc = 0;
        int dc = 0;
        if (!FP) {
            const int a = __ldg(reinterpret_cast<const int *>(vals) + e);
            if (r0.w >= 0) flip_int<true>(r0, a, up, sc, dc);
            else flip_int<false>(r0, a, up, sc, dc);
        } else {
            const int4 r1 = wrow[2 * o + 1];
            const double a = __ldg(reinterpret_cast<const double *>(vals) + e);
            if (r0.w >= 0) flip_fp<true>(r0, r1, a, up, sc, dc);
            else flip_fp<false>(r0, r1, a, up, sc, dc);
        }
        if (sc) atomicAdd(reinterpret_cast<unsigned long long *>(sacc + c), (unsigned long long)sc);
        if (dc) atomicAdd(cacc + c, dc);
    }
    __syncwarp();
}

// shared memory of k_eval_bin_rows: column accumulators (score, count), the x
// bits and every warp's 32 row states
constexpr int kRbSmem = kRbCols * (int)(sizeof(long long) + sizeof(int)) + kRbCols / 8 +
                        (kRbThreads / 32) * 64 * (int)sizeof(int4);

__global__ void __launch_bounds__(kRbThreads) k_eval_bin_rows(Dev d, RowBin rb, int bin_cols, VarOut o, int gate)
{
    if (gated_done(d, gate)) return;   // the same for every CTA of the grid
    extern __shared__ __align__(16) unsigned char rb_smem[];
    long long *sacc = reinterpret_cast<long long *>(rb_smem);
    int *cacc = reinterpret_cast<int *>(sacc + kRbCols);
    unsigned *xb = reinterpret_cast<unsigned *>(cacc + kRbCols);
    int4 *wrows = reinterpret_cast<int4 *>(xb + kRbCols / 32);
    __shared__ int s_next[2];
    cooperative_groups::cluster_group cluster = cooperative_groups::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int B = rb.blocks, b = blockIdx.x / kRbCluster;
    const int ncols = (bin_cols - b + B - 1) / B;   // column c of block b is position c * B + b
    for (int c = threadIdx.x; c < ncols; c += blockDim.x) {
        sacc[c] = 0;
        cacc[c] = 0;
    }
    if (threadIdx.x < 2) s_next[threadIdx.x] = 0;
    for (int c0 = warp * 32; c0 < ncols; c0 += nwarps * 32) {
        const int c = c0 + lane;
        bool bit = false;
        if (c < ncols) bit = __double_as_longlong(d.x[__ldg(d.var_list + c * B + b)]) != 0;
        const unsigned w = __ballot_sync(FULLMASK, bit);
        if (lane == 0) xb[c0 >> 5] = w;
    }
    __syncthreads();
    // chunks of 32 rows taken dynamically by the warps (row lengths vary)
    int4 *wrow = wrows + warp * 64;
    {
        const int r0 = __ldg(rb.split_i + b * (kRbCluster + 1) + rank), r1 = __ldg(rb.split_i + b * (kRbCluster + 1) + rank + 1);
        for (;;) {
            int ch = 0;
            if (lane == 0) ch = atomicAdd(&s_next[0], 1);
            const int k0 = r0 + 32 * __shfl_sync(FULLMASK, ch, 0);
            if (k0 >= r1) break;
            rb_rows_chunk<false>(d, rb.rows_i, rb.eptr_i, rb.col_i, rb.own_i, rb.val_i, k0, r1, xb, wrow, sacc, cacc);
        }
    }
    {
        const int r0 = __ldg(rb.split_f + b * (kRbCluster + 1) + rank), r1 = __ldg(rb.split_f + b * (kRbCluster + 1) + rank + 1);
        for (;;) {
            int ch = 0;
            if (lane == 0) ch = atomicAdd(&s_next[1], 1);
            const int k0 = r0 + 32 * __shfl_sync(FULLMASK, ch, 0);
            if (k0 >= r1) break;
            rb_rows_chunk<true>(d, rb.rows_f, rb.eptr_f, rb.col_f, rb.own_f, rb.val_f, k0, r1, xb, wrow, sacc, cacc);
        }
    }
    cluster.sync();   // every CTA's accumulators are complete
    const long long iter = d.ctl->iter, nviol = d.ctl->nviol, bestnv = d.ctl->best_nviol;
    const int per = (ncols + kRbCluster - 1) / kRbCluster;
    const int c0 = rank * per, c1 = min(ncols, c0 + per);
    Cand best{0, kNoVar, 0, 0.0};
    for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
        long long s = 0;
        int dc = 0;
#pragma unroll
        for (int k = 0; k < kRbCluster; ++k) {
            s += cluster.map_shared_rank(sacc, k)[c];
            dc += cluster.map_shared_rank(cacc, k)[c];
        }
        const int j = __ldg(d.var_list + c * B + b);
        const bool up = ((xb[c >> 5] >> (c & 31)) & 1u) == 0;
        bool mv = s > 0;
        if (mv) {
            const int stamp = up ? d.tabu_inc[j] : d.tabu_dec[j];
            mv = iter >= (long long)stamp || nviol + (long long)dc < bestnv;
        }
        const double xh = up ? 1.0 : 0.0;
        if (o.xhat) o.xhat[j] = mv ? xh : d.x[j];
        if (o.s) o.s[j] = mv ? s : 0;
        if (o.dc) o.dc[j] = mv ? dc : 0;
        if (mv && cand_better(s, j, best.s, best.var)) best = Cand{s, j, dc, xh};
    }
    const Cand bb = block_reduce_cand(best);
    if (threadIdx.x == 0) {
        d.block_best[blockIdx.x] = bb;
        if (bb.s > 0) atomicMax(&d.ctl->pass_best, bb.s);
    }
    cluster.sync();   // the other CTAs are done reading this CTA's accumulators
    finish_pass(d);
}

// ------------------------------------------------ row-blocked binary flips
//
// The layout is described with BinBlk (chap_internal.h).  k_eval_bin_blk: one
// CTA per work item (row block, position span); the block's row states are
// copied into shared memory once, then each warp streams its share of the
// span's entries of both streams, four consecutive entries per lane (16-byte
// loads of the entry words and coefficients; shared-memory row states; the
// penalty changes of both halves, the second only on an "=" row, w2 >= 0).
// A lane sums its entries by position; the runs that lie inside the lane are
// added to their positions' accumulators at once, and one segmented warp scan
// joins the runs that cross lanes.  k_bin_blk_final: one CTA per finalize
// range applies tabu and aspiration to the positions' sums (as k_eval_bin
// does), writes the range's candidate slot and returns the accumulators to
// zero.

constexpr int kBlkWarps = kBlkThreads / 32;
static_assert(kBlkRows == 1 << kBlkRowBits, "an entry word holds the row inside a block");

__host__ __device__ constexpr int blk_smem(int rows) { return rows * (2 * (int)sizeof(long long) + (int)sizeof(int2)); }

// Flip terms of one entry of an integral row: residual r, weights w (w.y < 0
// on a single row), change ad of the residual.
__device__ __forceinline__ void blk_int(long long r, int2 w, int ad, long long &s, int &dc)
{
    const long long r1 = r + ad;
    const bool v0 = r > 0, v1 = r1 > 0;
    s += (long long)flip_f(v0, v1, ad < 0) * w.x;
    dc += (int)v1 - (int)v0;
    if (w.y >= 0) {
        const bool u0 = r < 0, u1 = r1 < 0;
        s += (long long)flip_f(u0, u1, ad > 0) * w.y;
        dc += (int)u1 - (int)u0;
    }
}

// Flip terms of one entry of a non-integral row: margins m1 = eps - r and
// (read only on an "=" row) m2 = eps + r, change ad of the residual.
__device__ __forceinline__ void blk_fp(double m1, const long long *m2p, int2 w, double ad, long long &s, int &dc)
{
    const bool neg = dneg(ad);
    const bool v0 = dneg(m1), v1 = dgt(ad, m1);
    s += (long long)flip_f(v0, v1, neg) * w.x;
    dc += (int)v1 - (int)v0;
    if (w.y >= 0) {
        const double m2 = __longlong_as_double(*m2p);
        const bool u0 = dneg(m2), u1 = dgt(dflip(ad), m2);
        s += (long long)flip_f(u0, u1, !neg) * w.y;
        dc += (int)u1 - (int)u0;
    }
}

__device__ __forceinline__ void blk_add(const BinBlk &bb, int q, long long s, int dc)
{
    if (s) atomicAdd(reinterpret_cast<unsigned long long *>(bb.acc_s + q), (unsigned long long)s);
    if (dc) atomicAdd(bb.acc_dc + q, dc);
}

// Terms of one entry: word mw, coefficient av (position q; no entry: q < 0).
template <bool FP, typename Val>
__device__ __forceinline__ void blk_entry(const Dev &d, const long long *sA, const long long *sB, const int2 *sW,
                                          unsigned mw, Val av, int q, long long &s, int &dc)
{
    s = 0;
    dc = 0;
    if (q < 0) return;
    const int l = (int)(mw & ((1u << kBlkRowBits) - 1u));
    const bool up = __ldg(d.bup + q) != 0;
    const int2 w = sW[l];
    if (!FP) blk_int(sA[l], w, up ? (int)av : -(int)av, s, dc);
    else blk_fp(__longlong_as_double(sA[l]), sB + l, w, up ? (double)av : dflip((double)av), s, dc);
}

// One warp's entries [a, b) of one stream (FP: the non-integral rows), in
// rounds of 128: lane k holds entries base + 4k .. base + 4k + 3 (base a
// multiple of 4; the arrays are padded past their end).  Positions ascend
// along the entries; entries outside [a, b) take the key -1 before a and
// INT_MAX after b and add nothing.
template <bool FP>
__device__ __forceinline__ void blk_stream(const Dev &d, const BinBlk &bb, const long long *sA, const long long *sB,
                                           const int2 *sW, int a, int b, int lane)
{
    using Val = typename std::conditional<FP, double, int>::type;
    const unsigned *metap = FP ? bb.metaF : bb.metaI;
    const Val *valp = reinterpret_cast<const Val *>(FP ? (const void *)bb.valF : (const void *)bb.valI);
    // the next round's words and coefficients are loaded before this round's
    // terms are computed
    unsigned nw[4];
    Val nv[4];
    auto load = [&](int e) {
#pragma unroll
        for (int k = 0; k < 4; ++k) { nw[k] = 0u; nv[k] = Val(1); }
        if (e + 3 >= a && e < b) {
            const uint4 m4 = __ldg(reinterpret_cast<const uint4 *>(metap + e));
            nw[0] = m4.x; nw[1] = m4.y; nw[2] = m4.z; nw[3] = m4.w;
            if (FP) {
                const double2 v0 = __ldg(reinterpret_cast<const double2 *>(valp + e));
                const double2 v1 = __ldg(reinterpret_cast<const double2 *>(valp + e + 2));
                nv[0] = (Val)v0.x; nv[1] = (Val)v0.y; nv[2] = (Val)v1.x; nv[3] = (Val)v1.y;
            } else {
                const int4 v = __ldg(reinterpret_cast<const int4 *>(valp + e));
                nv[0] = (Val)v.x; nv[1] = (Val)v.y; nv[2] = (Val)v.z; nv[3] = (Val)v.w;
            }
        }
    };
    load((a & ~3) + 4 * lane);
    for (int base = a & ~3; base < b; base += 128) {
        const int e = base + 4 * lane;
        unsigned mw[4];
        Val av[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) { mw[k] = nw[k]; av[k] = nv[k]; }
        load(e + 128);
        int key[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) key[k] = e + k < a ? -1 : (e + k >= b ? INT_MAX : (int)(mw[k] >> kBlkRowBits));
        // the lane's runs: the first (key[0]) and the last (key[3]) may
        // continue in the neighbouring lanes, the ones between are complete
        long long sa = 0, sz = 0;
        int da = 0, dz = 0;
        int cur = key[0];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            long long s;
            int dc;
            blk_entry<FP>(d, sA, sB, sW, mw[k], av[k], (key[k] >= 0 && key[k] != INT_MAX) ? key[k] : -1, s, dc);
            if (key[k] != cur) {
                // the run of cur ends here: the first run is kept, a middle one is added
                if (cur != key[0] && cur >= 0 && cur != INT_MAX) blk_add(bb, cur, sz, dz);
                else if (cur == key[0]) { sa = sz; da = dz; }
                sz = 0;
                dz = 0;
                cur = key[k];
            }
            sz += s;
            dz += dc;
        }
        const bool uni = key[0] == key[3];
        if (uni) { sa = 0; da = 0; }   // one run: all of it is in sz
        // segmented scan of the last runs: a lane continues its left
        // neighbour's last run when it is one run of the same key
        const int prev3 = __shfl_up_sync(FULLMASK, key[3], 1), next0 = __shfl_down_sync(FULLMASK, key[0], 1);
        long long v = sz;
        int vd = dz;
        int f = (lane == 0 || !uni || prev3 != key[0]) ? 1 : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long ts = __shfl_up_sync(FULLMASK, v, o);
            const int td = __shfl_up_sync(FULLMASK, vd, o), tf = __shfl_up_sync(FULLMASK, f, o);
            if (lane >= o) {
                if (!f) { v += ts; vd += td; }
                f |= tf;
            }
        }
        // a lane of several runs closes its first run with the left
        // neighbour's open sum (when that one continues into it)
        const long long lv = __shfl_up_sync(FULLMASK, v, 1);
        const int lvd = __shfl_up_sync(FULLMASK, vd, 1);
        if (!uni && key[0] >= 0 && key[0] != INT_MAX) {
            const bool join = lane > 0 && prev3 == key[0];
            blk_add(bb, key[0], sa + (join ? lv : 0), da + (join ? lvd : 0));
        }
        // the last run is added by the lane where it ends
        if ((lane == 31 || next0 != key[3]) && key[3] >= 0 && key[3] != INT_MAX) blk_add(bb, key[3], v, vd);
    }
}

__global__ void __launch_bounds__(kBlkThreads, 1) k_eval_bin_blk(Dev d, BinBlk bb, int gate)
{
    if (gated_done(d, gate)) return;
    extern __shared__ __align__(16) unsigned char blk_smem_raw[];
    long long *sA = reinterpret_cast<long long *>(blk_smem_raw);   // r (integral row) or eps - r
    long long *sB = sA + bb.rows;                                   // eps + r (other rows)
    int2 *sW = reinterpret_cast<int2 *>(sB + bb.rows);              // w1, w2
    const BlkItem it = bb.items[blockIdx.x];
    const int r0 = it.b * bb.rows, nr = min(bb.rows, d.m - r0);
    // kBlkRows / kBlkThreads rows per thread, their loads issued together
#pragma unroll
    for (int k = 0; k < kBlkRows / kBlkThreads; ++k) {
        const int l = k * kBlkThreads + (int)threadIdx.x;
        if (l < nr) {
            int4 s0, s1;
            ld_row32(d.rs + r0 + l, s0, s1);
            const bool integ = __ldg(d.row_int + r0 + l) != 0;
            sA[l] = integ ? row_r(s0) : row_r(s1);
            sB[l] = (long long)(((unsigned long long)(unsigned)s1.w << 32) | (unsigned)s1.z);
            sW[l] = make_int2(s0.z, s0.w);
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // the warps' shares of each stream, cut at multiples of 4 entries
    auto cut = [&](int e0, int e1, int k) {
        if (k <= 0) return e0;
        if (k >= kBlkWarps) return e1;
        const int c = (int)(e0 + (long long)(e1 - e0) * k / kBlkWarps) & ~3;
        return max(e0, c);
    };
    blk_stream<false>(d, bb, sA, sB, sW, cut(it.eI0, it.eI1, warp), cut(it.eI0, it.eI1, warp + 1), lane);
    blk_stream<true>(d, bb, sA, sB, sW, cut(it.eF0, it.eF1, warp), cut(it.eF0, it.eF1, warp + 1), lane);
}

__global__ void __launch_bounds__(kBlkFinThreads) k_bin_blk_final(Dev d, BinBlk bb, int ncols, VarOut o, int gate)
{
    if (gated_done(d, gate)) return;
    const long long iter = d.ctl->iter, nviol = d.ctl->nviol, bestnv = d.ctl->best_nviol;
    Cand best{0, kNoVar, 0, 0.0};
    for (int q = blockIdx.x * kBlkFin + threadIdx.x; q < min(ncols, (blockIdx.x + 1) * kBlkFin); q += blockDim.x) {
        const long long s = bb.acc_s[q];
        const int dc = bb.acc_dc[q];
        bb.acc_s[q] = 0;
        bb.acc_dc[q] = 0;
        const int j = __ldg(d.var_list + q);
        const bool up = d.bup[q] != 0;
        bool mv = s > 0;
        if (mv) {
            const int stamp = up ? d.tabu_inc[j] : d.tabu_dec[j];
            mv = iter >= (long long)stamp || nviol + (long long)dc < bestnv;
        }
        const double xh = up ? 1.0 : 0.0;
        if (o.xhat) o.xhat[j] = mv ? xh : d.x[j];
        if (o.s) o.s[j] = mv ? s : 0;
        if (o.dc) o.dc[j] = mv ? dc : 0;
        if (mv && cand_better(s, j, best.s, best.var)) best = Cand{s, j, dc, xh};
    }
    const Cand cb = block_reduce_cand(best);
    if (threadIdx.x == 0) {
        d.block_best[blockIdx.x] = cb;
        if (cb.s > 0) atomicMax(&d.ctl->pass_best, cb.s);
    }
    finish_pass(d);
}

// Flip direction of every binary position from x (after a new state).
__global__ void k_bup_init(Dev d)
{
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < d.n_bup; q += gridDim.x * blockDim.x)
        d.bup[q] = __double_as_longlong(d.x[__ldg(d.var_list + q)]) == 0 ? 1 : 0;
}

// Selective re-evaluation of the binary flips.  k_eval_bin_lazy recomputes the
// kept score and violation change of the queued positions (all of them when
// lz_full); k_bin_scan applies tabu and aspiration to the kept values of every
// binary position, writes the per-CTA candidates of the binary slots and
// consumes the queue; k_lazy_mark queues the binary positions of every row
// of the moved column after each iteration.
template <int G>
__global__ void __launch_bounds__(kEvalThreads) k_eval_bin_lazy(Dev d, int ncols, int gate)
{
    if (gated_done(d, gate)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int CPW = 32 / G;
    const int g = lane / G, sub = lane & (G - 1);
    const bool full = d.ctl->lz_full != 0;
    const int items = full ? ncols : min(d.ctl->lz_count, ncols);
    const int nquad = (items + CPW - 1) / CPW;
    for (int qd = blockIdx.x * kEvalWarps + warp; qd < nquad; qd += gridDim.x * kEvalWarps) {
        const int it = qd * CPW + g;
        const bool live = it < items;
        const int q = live ? (full ? it : d.lz_list[it]) : 0;
        int j, dc;
        bool up;
        long long s;
        bin_column<G>(d, q, live, sub, j, up, s, dc);
        if (sub == 0 && live) {
            d.lz_s[q] = s;
            d.lz_dc[q] = dc;
        }
    }
}

__global__ void __launch_bounds__(kEvalThreads) k_bin_scan(Dev d, int ncols, VarOut o, int gate)
{
    if (gated_done(d, gate)) return;
    Ctl *c = d.ctl;
    const long long iter = c->iter, nviol = c->nviol, bestnv = c->best_nviol;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        // the queue was consumed by k_eval_bin_lazy
        c->lz_count = 0;
        c->lz_full = 0;
        c->lz_epoch += 1u;
    }
    Cand best{0, kNoVar, 0, 0.0};
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < ncols; q += gridDim.x * blockDim.x) {
        const int j = __ldg(d.var_list + q);
        const bool up = __double_as_longlong(d.x[j]) == 0;
        const long long s = d.lz_s[q];
        const int dc = d.lz_dc[q];
        bool mv = s > 0;
        if (mv) {
            const int stamp = up ? d.tabu_inc[j] : d.tabu_dec[j];
            mv = iter >= (long long)stamp || nviol + (long long)dc < bestnv;
        }
        const double xh = up ? 1.0 : 0.0;
        if (o.xhat) o.xhat[j] = mv ? xh : d.x[j];
        if (o.s) o.s[j] = mv ? s : 0;
        if (o.dc) o.dc[j] = mv ? dc : 0;
        if (mv && cand_better(s, j, best.s, best.var)) best = Cand{s, j, dc, xh};
    }
    const Cand b = block_reduce_cand(best);
    if (threadIdx.x == 0) {
        d.block_best[blockIdx.x] = b;
        if (b.s > 0) atomicMax(&d.ctl->pass_best, b.s);
    }
    finish_pass(d);
}

// Runs after every apply (not gated by the done flag: the last iteration of
// a run must be marked as well); acts once per iteration end (lz_seq).  The
// entries of all rows of the moved column are spread over the whole grid
// (row offsets in shared memory, a binary search per entry), so a long row
// does not serialise on one warp.
__global__ void __launch_bounds__(kEvalThreads) k_lazy_mark(Dev d, int nbin)
{
    Ctl *c = d.ctl;
    const long long seq = c->lz_seq;
    if (!c->lz_on || seq == c->lz_done) return;
    const int var = c->lz_var;
    const unsigned epoch = c->lz_epoch;
    const int lane = threadIdx.x & 31;
    __shared__ long long s_off[kLazyMaxRows + 1];   // prefix of the row lengths
    __shared__ long long s_start[kLazyMaxRows];     // CSR offset of each row
    int nrows = 0;
    if (var >= 0 && !c->lz_full) {
        const int qv = d.vpos[var];
        const int e0 = d.ci_ptr[qv], f0 = d.cf_ptr[qv];
        const int nI = d.ci_ptr[qv + 1] - e0, nF = d.cf_ptr[qv + 1] - f0;
        if (nI + nF > kLazyMaxRows) {
            // a long column touches most rows: re-evaluate everything instead
            if (blockIdx.x == 0 && threadIdx.x == 0) c->lz_full = 1;
        } else {
            nrows = nI + nF;
            for (int k = threadIdx.x; k < nrows; k += blockDim.x) {
                const int i = k < nI ? d.ci_row[e0 + k] : d.cf_row[f0 + (k - nI)];
                const long long p0 = d.row_ptr[i];
                s_start[k] = p0;
                s_off[k + 1] = d.row_ptr[i + 1] - p0;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && nrows > 0) {
        s_off[0] = 0;
        for (int k = 1; k <= nrows; ++k) s_off[k] += s_off[k - 1];
    }
    __syncthreads();
    const long long total = nrows > 0 ? s_off[nrows] : 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < total; base += stride) {
        const long long g = base + lane;
        bool fresh = false;
        int q = 0;
        if (g < total) {
            int lo = 0, hi = nrows;   // the row k with s_off[k] <= g < s_off[k + 1]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (s_off[mid] <= g) lo = mid;
                else hi = mid;
            }
            q = d.vpos[d.col_idx[s_start[lo] + (g - s_off[lo])]];
            fresh = q < nbin && atomicExch(d.lz_mark + q, epoch) != epoch;
        }
        const unsigned bal = __ballot_sync(FULLMASK, fresh);
        if (bal) {
            int b0 = 0;
            if (lane == __ffs(bal) - 1) b0 = atomicAdd(&c->lz_count, __popc(bal));
            b0 = __shfl_sync(FULLMASK, b0, __ffs(bal) - 1);
            if (fresh) d.lz_list[b0 + __popc(bal & ((1u << lane) - 1u))] = q;
        }
    }
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&c->lz_ticket, 1u) == gridDim.x - 1;
        if (s_last) {
            c->lz_ticket = 0;
            c->lz_done = seq;
        }
    }
}

// ---------------------------------------------- breakpoint generation (Alg. 1)

// Scalars of Algorithm 1 in half-weight units: beta (score as x -> -inf),
// alpha (added right of xbar) and their violation-count twins.
struct Acc {
    long long beta, alpha;
    int beta_c, alpha_c;
};

// Entry of one normalised half: type 1 "pre" (a < 0: delta D counts from t on,
// violation count -1), type 2 "post" (a > 0: t is a candidate, D counts right of
// t, violation count +1), type 0 none.  On a continuous variable the delta
// entry sits where the row's status changes (the boundary of its satisfied set
// within eps) and is not a candidate itself (nocand); the candidate is the
// point where the row becomes tight, a separate marker entry (mark, mkey) with
// no delta.
struct Half {
    unsigned long long key;
    long long D;
    int type;
    int nocand;
    int mark;
    unsigned long long mkey;
};

// Case table of Algorithm 1 for one normalised half (half-weight units).  The
// entry lands left of l (side -1: folded into beta), right of u (side +1:
// dropped) or at key (side 0, compared with the bound keys here).
__device__ __forceinline__ void half_case(bool viol, bool tight, bool apos, int side, unsigned long long key,
                                          long long w, unsigned long long kl, unsigned long long ku, Acc &acc, Half &h)
{
    h.type = 0;
    h.nocand = 0;
    h.mark = 0;
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
    if (side == 0) side = key < kl ? -1 : (key > ku ? 1 : 0);
    if (side < 0) {
        acc.beta += D;
        acc.beta_c += (type == 1) ? -1 : 1;
        return;
    }
    if (side > 0) return;
    h.key = key;
    h.D = D;
    h.type = type;
}

// Integral row (integer variable).  The breakpoint xbar + floor(-r/a) (a > 0)
// or xbar + ceil(-r/a) (a < 0) is compared with the bounds by exact int64
// products first (|lo a|, |hi a| <= 2^53 on integral rows); the division runs
// only for breakpoints inside [l, u].
__device__ __forceinline__ void int_half(long long r, long long a, long long w, const ColCtx &c, Acc &acc, Half &h)
{
    const bool viol = r > 0;
    const bool apos = a > 0;
    int side;
    if (apos) side = (r > -c.lo * a) ? -1 : ((-r >= (c.hi + 1) * a) ? 1 : 0);
    else side = (-r >= (c.lo - 1) * a) ? -1 : ((-r < c.hi * a) ? 1 : 0);
    if (side != 0) {
        half_case(viol, false, apos, side, 0ull, w, c.kl, c.ku, acc, h);
        return;
    }
    const long long dd = apos ? floor_div(-r, a) : ceil_div(-r, a);
    half_case(viol, !viol && dd == 0, apos, 0, ikey(c.xbi + dd), w, c.kl, c.ku, acc, h);
}

// |x| with a relative error bound e and an absolute floor, for the certain
// comparisons below: x < y is certain when x + slack(x) < y - slack(y).
__device__ __forceinline__ float slack(float x) { return fabsf(x) * 1.0e-5f + 1.0e-30f; }

// Integer variable on a non-integral row with margin m = eps - r: the
// breakpoint is xbar + floor(m / a) (a > 0) or xbar + ceil(m / a) (a < 0).
// Returns the side (-1 left of l, +1 right of u) when single-precision
// products decide it, else 0.
__device__ __forceinline__ int int_fp_side(double m, double a, bool apos, const ColCtx &c)
{
    bool ok = true;
    const float mf = approx_f(m, ok), af = approx_f(a, ok);
    if (!ok) return 0;
    if (apos) {
        const float P = c.lof * af;              // t < l  <=>  m < lo a
        if (mf + slack(mf) < P - slack(P)) return -1;
        const float Q = (c.hif + 1.0f) * af;     // t > u  <=>  m >= (hi + 1) a
        if (mf - slack(mf) > Q + slack(Q)) return 1;
    } else {
        const float P = (c.lof - 1.0f) * af;     // t < l  <=>  m >= (lo - 1) a
        if (mf - slack(mf) > P + slack(P)) return -1;
        const float Q = c.hif * af;              // t > u  <=>  m < hi a
        if (mf + slack(mf) < Q - slack(Q)) return 1;
    }
    return 0;
}

// Continuous variable: side of xbar - q / a (left of l <=> q/a > xbar - l,
// right of u <=> q/a < xbar - u) for q = r (the tight point) or q = -m (the
// boundary), decided from single-precision products with a margin that also
// covers the rounding of the point itself; else 0.
__device__ __forceinline__ int cont_side1(float qf, float af, bool apos, const ColCtx &c)
{
    const float tol = c.xaf * fabsf(af) * 1.0e-10f;
    const float P = c.dlf * af, Q = c.duf * af;
    if (apos) {
        if (qf - slack(qf) - tol > P + slack(P)) return -1;
        if (qf + slack(qf) + tol < Q - slack(Q)) return 1;
    } else {
        if (qf + slack(qf) + tol < P - slack(P)) return -1;
        if (qf - slack(qf) - tol > Q + slack(Q)) return 1;
    }
    return 0;
}

// Both points of a continuous half (tight point t = xbar - r/a and boundary
// tb = xbar + m/a) certainly left of l (-1) or right of u (+1); else 0.
__device__ __forceinline__ int cont_fp_side(double r, double m, double a, bool apos, const ColCtx &c)
{
    bool ok = c.fok;
    const float rf = approx_f(r, ok), mf = approx_f(m, ok), af = approx_f(a, ok);
    if (!ok) return 0;
    const int s1 = cont_side1(rf, af, apos, c);
    return s1 != 0 && cont_side1(-mf, af, apos, c) == s1 ? s1 : 0;
}

__device__ __forceinline__ unsigned long long cont_key(double t)
{
    const unsigned long long k = dkey(t);
    return k == dkey(-0.0) ? dkey(0.0) : k;
}

// Continuous variable, one normalised half with residual r, coefficient a and
// margin m = eps - r (Algorithm 1 with the tolerance of the definition): the
// row is satisfied at x iff a (x - xbar) <= m, i.e. up to (a > 0) or from
// (a < 0) the boundary tb = xbar + m / a, so the delta of the case table sits
// at tb (not a candidate itself).  The candidate of the row is its tight point
// t = xbar - r / a, a marker entry, unless |r| <= eps (near0): such a row is
// already tight and its point is xbar.
__device__ __forceinline__ void cont_exact(double r, double a, double m, bool viol, bool near0, long long w,
                                           const ColCtx &c, Acc &acc, Half &h)
{
    const bool apos = !dneg(a);
    half_case(viol, false, apos, 0, cont_key(__dadd_rn(c.xb, __ddiv_rn(m, a))), w, c.kl, c.ku, acc, h);
    h.nocand = 1;
    if (!near0) {
        const unsigned long long k = cont_key(__dsub_rn(c.xb, __ddiv_rn(r, a)));
        if (k != c.kxb && k >= c.kl && k <= c.ku) {
            h.mark = 1;
            h.mkey = k;
        }
    }
}

// Non-integral row, one half with residual r, coefficient a and margins
// m = eps - r (own), mo = eps + r (other half).  Integer variable: the last
// integer at which the row is satisfied within eps.  Continuous variable:
// cont_exact.  The double divisions run only when the side test cannot place
// the half's points outside [l, u].
__device__ __forceinline__ void fp_half(double r, double a, double m, double mo, long long w, const ColCtx &c,
                                        Acc &acc, Half &h)
{
    const bool viol = dneg(m);
    const bool apos = !dneg(a);
    if (c.isint) {
        const int side = int_fp_side(m, a, apos, c);
        if (side != 0) {
            half_case(viol, false, apos, side, 0ull, w, c.kl, c.ku, acc, h);
            return;
        }
        const double q = __ddiv_rn(m, a);
        const long long dd = clamp_dd(apos ? __double2ll_rd(q) : __double2ll_ru(q));
        half_case(viol, !viol && dd == 0, apos, 0, ikey(c.xbi + dd), w, c.kl, c.ku, acc, h);
    } else {
        const bool near0 = !viol && !dneg(mo);  // |r| <= eps
        const int side = cont_fp_side(r, m, a, apos, c);
        if (side != 0) {
            half_case(viol, false, apos, side, 0ull, w, c.kl, c.ku, acc, h);
            return;
        }
        cont_exact(r, a, m, viol, near0, w, c, acc, h);
    }
}

// Both halves of the v-th nonzero of the column (integral part first).
__device__ __forceinline__ void gen_entry(const Dev &d, const ColCtx &c, int v, Acc &acc, Half &h1, Half &h2)
{
    h1.type = 0; h1.mark = 0;
    h2.type = 0; h2.mark = 0;
    if (v < c.nI) {
        const int e = c.ci0 + v;
        const int i = __ldg(d.ci_row + e);
        const long long a = __ldg(d.ci_val + e);
        const int4 st = ld_row16(d.rs + i);
        const long long r = row_r(st);
        int_half(r, a, st.z, c, acc, h1);
        if (st.w >= 0) int_half(-r, -a, st.w, c, acc, h2);
    } else {
        const int e = c.cf0 + (v - c.nI);
        const int i = __ldg(d.cf_row + e);
        const double a = __ldg(d.cf_val + e);
        const int4 *p = reinterpret_cast<const int4 *>(d.rs + i);
        const int4 s0 = __ldg(p), s1 = __ldg(p + 1);
        const double r = i4_double_lo(s0), m1 = i4_double_lo(s1), m2 = i4_double_hi(s1);
        fp_half(r, a, m1, m2, s0.z, c, acc, h1);
        if (s0.w >= 0) fp_half(dflip(r), dflip(a), m2, m1, s0.w, c, acc, h2);
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

// aux word of a sort entry: bits 31..30 = class, bits 0..1 = count delta + 1.
// Classes in their order at equal t: 0 pre entry that is no candidate (the
// boundary delta of a continuous half), 1 pre entry (also bounds and the
// tight-point markers, delta 0), 2 post entry, 3 post entry that is no
// candidate.  Bit 31 is the post marker of Algorithm 1's (t, marker) order.
constexpr int kClsPreDelta = 0, kClsPre = 1, kClsPost = 2, kClsPostDelta = 3;
__device__ __forceinline__ unsigned make_aux(int cls, int dc) { return ((unsigned)cls << 30) | (unsigned)(dc + 1); }
__device__ __forceinline__ int aux_dc(unsigned a) { return (int)(a & 3u) - 1; }
__device__ __forceinline__ unsigned aux_post(unsigned a) { return a >> 31; }
__device__ __forceinline__ unsigned aux_cls(unsigned a) { return a >> 30; }

// Sort entry of a half's delta and of its marker.
__device__ __forceinline__ unsigned half_aux(const Half &h)
{
    return h.type == 1 ? make_aux(h.nocand ? kClsPreDelta : kClsPre, -1) : make_aux(h.nocand ? kClsPostDelta : kClsPost, 1);
}
__device__ __forceinline__ unsigned marker_aux() { return make_aux(kClsPre, 0); }

// Number of sort entries of a half (delta and marker).
__device__ __forceinline__ int half_entries(const Half &h) { return (h.type != 0) + h.mark; }

__device__ __forceinline__ void put_half(const Half &h, int pos, unsigned long long *k, long long *dl, unsigned *ax)
{
    if (h.type != 0) {
        k[pos] = h.key;
        dl[pos] = h.D;
        ax[pos] = half_aux(h);
        ++pos;
    }
    if (h.mark) {
        k[pos] = h.mkey;
        dl[pos] = 0;
        ax[pos] = marker_aux();
    }
}

// Lexicographic (t, class) order: pre entries before post entries at equal t.
__device__ __forceinline__ bool entry_less(unsigned long long k1, unsigned a1, unsigned long long k2, unsigned a2)
{
    return k1 < k2 || (k1 == k2 && aux_cls(a1) < aux_cls(a2));
}

// Candidate test of a sorted entry given its neighbours (Algorithm 1, phase 4):
// the last class-1 entry of an equal-t run (every pre delta at t counted), or
// the first post entry of a run without class-1 entries (no post delta at t
// counted).  Boundary deltas are never candidates.
__device__ __forceinline__ bool is_candidate(unsigned long long k, unsigned a, unsigned long long kprev, unsigned aprev,
                                             bool has_prev, unsigned long long knext, unsigned anext)
{
    if (k == kPadKey) return false;
    const unsigned c = aux_cls(a);
    if (c == kClsPre) return knext != k || aux_cls(anext) != kClsPre;
    if (c == kClsPost) return !has_prev || kprev != k || aux_cls(aprev) == kClsPreDelta;
    return false;
}

// ------------------------------------------------- short non-binary columns
//
// Columns with at most kWarpSortMax breakpoint entries (bounds included).  A
// group of G lanes evaluates one column (G = 8, or 4 when the columns are short
// on average), so one warp holds 32 / G columns at a time; a persistent grid
// takes the warps' column groups in a strided order.
//  1. Classification.  The lanes of a group read the column's nonzeros
//     coalesced (integral-row part, then the non-integral part), two per lane
//     in flight, and gather their row states.  Every half is first placed by
//     single-precision products with error margins (no division): a half
//     whose breakpoint is certainly left of l or right of u only changes the
//     scalars beta / alpha of Algorithm 1.  Integral and non-integral rows
//     share this test (on an integral row m = -r exactly), so the lanes do not
//     diverge by row type.
//  2. The undecided halves (a few percent) go to a per-warp queue with their
//     operands; whenever 32 are queued all lanes compute 32 exact breakpoints
//     at once (FP64 divisions are slow on this part, so they are never issued
//     for a single lane), and the entries inside [l, u] are appended to the
//     column's list in shared memory.
//  3. Each group sorts its list (bitonic over G lanes, 1, 2 or 4 entries per
//     lane), prefix-scans it with shuffles and reduces it to the column's best
//     admissible candidate.  A column whose list outgrows 4 G entries is
//     evaluated again by the whole warp with a list of kWarpSortMax entries.

constexpr int kNbWarps = kEvalWarps;
constexpr int kQCap = 160;                  // queued halves per warp (more: the whole-warp path)
using SEnt = SEntry;

// Shape of the group path for G lanes per column: 32 / G columns per warp,
// 4 G list entries per column, together the whole-warp list.
template <int G>
struct NbGeom {
    static constexpr int kCols = 32 / G;
    static constexpr int kStage = 4 * G;
    static_assert(kCols * kStage == kWarpSortMax, "the whole-warp path reuses the group lists");
};


// Undecided half (operands already negated for the second half of an "=" row):
//  integral row:      x = r, a (int64);
//  non-integral row:  x = eps - r (integer variable) or r (continuous), a (double bits),
//                     y = eps - r (continuous);
// meta = group | row kind << 3 | violated << 4 | near 0 (|r| <= eps) << 5.
struct __align__(16) QItem {
    long long x, a, y;
    int w, meta;
};

template <int G>
struct __align__(16) NbWarp {
    SEnt stage[kWarpSortMax];               // the groups' lists, or (with q) the whole-warp list
    QItem q[kQCap];                         // queued halves; free again when the whole-warp path runs
    ColCtx ctx[32 / G];
    long long beta[32 / G], alpha[32 / G];
    int beta_c[32 / G], alpha_c[32 / G], cnt[32 / G];
};
// The whole-warp path lays its list over stage and q (kWarpListMax entries).
static_assert(sizeof(SEnt) * kWarpSortMax + sizeof(QItem) * kQCap >= sizeof(SEnt) * kWarpListMax,
              "the whole-warp list fits over the stage and the queue");
// dynamic shared memory of k_eval_nb<G>
template <int G>
constexpr int nb_smem() { return kNbWarps * (int)sizeof(NbWarp<G>); }

// Scalars of a decided half as multiples of its weight, branch-free: the case
// table of Algorithm 1 (as in half_case) for index
// T*8 + P*4 + V*2 + L (T tight, P a > 0, V violated, L left of l; a half right
// of u has L = 0), packed as mb + 2 (3 bits), ma / 2 + 1, bc + 1, ac + 1
// (2 bits each), where beta += mb w, alpha += ma w, beta_c += bc,
// alpha_c += ac.  Index 1 adds nothing (used for inactive or queued halves).
constexpr unsigned long long kTabB = 0x492000702450ull;
constexpr unsigned kTabA = 0xaa05a5u, kTabBC = 0x55aa4916u, kTabAC = 0xaa005555u;

__device__ __forceinline__ void acc_decided(int idx, int w, Acc &acc)
{
    const int mb = (int)((kTabB >> (3 * idx)) & 7ull) - 2;
    const int ma = 2 * ((int)((kTabA >> (2 * idx)) & 3u) - 1);
    acc.beta += (long long)mb * w;
    acc.alpha += (long long)ma * w;
    acc.beta_c += (int)((kTabBC >> (2 * idx)) & 3u) - 1;
    acc.alpha_c += (int)((kTabAC >> (2 * idx)) & 3u) - 1;
}

// Side of the points z / a for z in [zlo, zhi] from single-precision products
// (against the thresholds L, U of the column, a > 0 after normalisation), with
// relative margins covering the float estimates and an absolute term tol: sets
// left / right only when certain for both ends.
__device__ __forceinline__ void side_test(float zlo, float zhi, float a, float L, float U, float tol, bool &left,
                                          bool &right)
{
    const float P = L * a, Q = U * a;
    left = zhi + (fabsf(zhi) * 1.0e-5f + tol + 1.0e-30f) < P - (fabsf(P) * 1.0e-5f + 1.0e-30f);
    right = zlo - (fabsf(zlo) * 1.0e-5f + tol + 1.0e-30f) > Q + (fabsf(Q) * 1.0e-5f + 1.0e-30f);
}

// Exact breakpoint of one queued half (Algorithm 1 case table, as int_half /
// fp_half after an undecided side test).
__device__ __forceinline__ void exact_item(const QItem &it, const ColCtx &ci, Acc &acc, Half &h)
{
    const bool viol = ((it.meta >> 4) & 1) != 0;
    bool apos, tight;
    unsigned long long key;
    if (((it.meta >> 3) & 1) == 0) {
        const long long r = it.x, a = it.a;
        apos = a > 0;
        const long long dd = apos ? floor_div(-r, a) : ceil_div(-r, a);
        tight = !viol && dd == 0;
        key = ikey(ci.xbi + dd);
    } else {
        const double a = __longlong_as_double(it.a);
        apos = !dneg(a);
        if (ci.isint) {
            const double q = __ddiv_rn(__longlong_as_double(it.x), a);
            const long long dd = clamp_dd(apos ? __double2ll_rd(q) : __double2ll_ru(q));
            tight = !viol && dd == 0;
            key = ikey(ci.xbi + dd);
        } else {
            cont_exact(__longlong_as_double(it.x), a, __longlong_as_double(it.y), viol, ((it.meta >> 5) & 1) != 0, it.w,
                       ci, acc, h);
            return;
        }
    }
    half_case(viol, tight, apos, 0, key, it.w, ci.kl, ci.ku, acc, h);
}

// Exact pass over n <= 32 queued halves starting at queue position head, one per lane.
template <int G>
__device__ __noinline__ void flush_queue(NbWarp<G> &W, int head, int n, int lane)
{
    if (lane < n) {
        const QItem it = W.q[head + lane];
        const int g = it.meta & 7;
        Acc acc{0, 0, 0, 0};
        Half h;
        h.type = 0;
        h.mark = 0;
        exact_item(it, W.ctx[g], acc, h);
        if (acc.beta) atomicAdd(reinterpret_cast<unsigned long long *>(&W.beta[g]), (unsigned long long)acc.beta);
        if (acc.alpha) atomicAdd(reinterpret_cast<unsigned long long *>(&W.alpha[g]), (unsigned long long)acc.alpha);
        if (acc.beta_c) atomicAdd(&W.beta_c[g], acc.beta_c);
        if (acc.alpha_c) atomicAdd(&W.alpha_c[g], acc.alpha_c);
        const int ne = half_entries(h);
        if (ne) {
            int pos = atomicAdd(&W.cnt[g], ne);
            SEnt *st = W.stage + g * NbGeom<G>::kStage;
            if (h.type != 0) {
                if (pos < NbGeom<G>::kStage) st[pos] = SEnt{h.key, (int)h.D, half_aux(h)};
                ++pos;
            }
            if (h.mark && pos < NbGeom<G>::kStage) st[pos] = SEnt{h.mkey, 0, marker_aux()};
        }
    }
    __syncwarp();
}

// Candidate evaluation of one sorted entry (prefix sums P / Pc inclusive).
__device__ __forceinline__ void eval_entry(VCand &vb, const ColCtx &c, const Acc &a, unsigned long long kk,
                                           long long del, unsigned aux, long long P, int Pc, unsigned long long kprev,
                                           unsigned aprev, bool has_prev, unsigned long long knext, unsigned anext,
                                           long long nviol, long long bestnv)
{
    if (!is_candidate(kk, aux, kprev, aprev, has_prev, knext, anext)) return;
    const bool post = aux_post(aux) != 0;
    const long long Pi = P - (post ? del : 0);
    const int Pci = Pc - (post ? aux_dc(aux) : 0);
    const bool right = kk > c.kxb;
    consider(vb, c, kk, a.beta + Pi + (right ? a.alpha : 0), a.beta_c + Pci + (right ? a.alpha_c : 0), nviol, bestnv);
}

__device__ __forceinline__ void load_entry(const SEnt *p, unsigned long long &key, long long &del, unsigned &aux)
{
    const int4 raw = *reinterpret_cast<const int4 *>(p);
    key = ((unsigned long long)(unsigned)raw.y << 32) | (unsigned)raw.x;
    del = raw.z;
    aux = (unsigned)raw.w;
}

// Bitonic sort of G * K entries held K per lane by aligned groups of G lanes
// (entry index sub * K + k, sub = lane % G).
template <int K, int G>
__device__ __forceinline__ void group_bitonic(unsigned long long (&key)[K], long long (&del)[K], unsigned (&aux)[K],
                                              int sub)
{
    constexpr int N = G * K;
#pragma unroll
    for (int size = 2; size <= N; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride < K) {
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    if ((k & stride) == 0) {
                        const int k2 = k | stride;
                        const int i = sub * K + k;
                        const bool asc = (i & size) == 0;
                        if (entry_less(key[k2], aux[k2], key[k], aux[k]) == asc) {
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
                    const unsigned long long pk = __shfl_xor_sync(FULLMASK, key[k], ls);
                    const long long pd = __shfl_xor_sync(FULLMASK, del[k], ls);
                    const unsigned pa = __shfl_xor_sync(FULLMASK, aux[k], ls);
                    const int i = sub * K + k;
                    const bool lower = (i & stride) == 0;
                    const bool asc = (i & size) == 0;
                    const bool take = (lower == asc) ? entry_less(pk, pa, key[k], aux[k])
                                                     : entry_less(key[k], aux[k], pk, pa);
                    if (take) { key[k] = pk; del[k] = pd; aux[k] = pa; }
                }
            }
        }
    }
}

// Sort, scan and argmax of each group's list (cnt <= G * K entries at list),
// K entries per lane; every lane returns the best candidate of its group.
template <int K, int G>
__device__ __forceinline__ VCand group_sort_scan(const ColCtx &c, const Acc &a, const SEnt *list, int cnt,
                                                 long long nviol, long long bestnv)
{
    const int sub = (threadIdx.x & 31) & (G - 1);
    unsigned long long key[K];
    long long del[K];
    unsigned aux[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int idx = sub * K + k;
        if (idx < cnt) load_entry(list + idx, key[k], del[k], aux[k]);
        else { key[k] = kPadKey; del[k] = 0; aux[k] = make_aux(kClsPost, 0); }
    }
    group_bitonic<K, G>(key, del, aux, sub);
    long long P[K];
    int Pc[K];
    long long run = 0;
    int runc = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) { run += del[k]; runc += aux_dc(aux[k]); P[k] = run; Pc[k] = runc; }
    long long tot = run;
    int totc = runc;
#pragma unroll
    for (int off = 1; off < G; off <<= 1) {
        const long long x = __shfl_up_sync(FULLMASK, tot, off, G);
        const int y = __shfl_up_sync(FULLMASK, totc, off, G);
        if (sub >= off) { tot += x; totc += y; }
    }
    const long long ex = tot - run;
    const int exc = totc - runc;
    unsigned long long nk = __shfl_down_sync(FULLMASK, key[0], 1, G);
    unsigned na = __shfl_down_sync(FULLMASK, aux[0], 1, G);
    const unsigned long long pk = __shfl_up_sync(FULLMASK, key[K - 1], 1, G);
    const unsigned pa = __shfl_up_sync(FULLMASK, aux[K - 1], 1, G);
    if (sub == G - 1) { nk = kPadKey; na = make_aux(kClsPost, 0); }
    VCand vb{0, 0ull, 0, 0};
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const unsigned long long knext = (k + 1 < K) ? key[(k + 1) % K] : nk;
        const unsigned anext = (k + 1 < K) ? aux[(k + 1) % K] : na;
        const unsigned long long kprev = (k > 0) ? key[(k + K - 1) % K] : pk;
        const unsigned aprev = (k > 0) ? aux[(k + K - 1) % K] : pa;
        eval_entry(vb, c, a, key[k], del[k], aux[k], ex + P[k], exc + Pc[k], kprev, aprev, k > 0 || sub > 0, knext,
                   anext, nviol, bestnv);
    }
#pragma unroll
    for (int o = G >> 1; o > 0; o >>= 1) {
        VCand p;
        p.s = __shfl_xor_sync(FULLMASK, vb.s, o);
        p.key = __shfl_xor_sync(FULLMASK, vb.key, o);
        p.dc = __shfl_xor_sync(FULLMASK, vb.dc, o);
        p.valid = __shfl_xor_sync(FULLMASK, vb.valid, o);
        if (vc_better(p, vb, c)) vb = p;
    }
    return vb;
}

// Whole-warp evaluation of one column with up to kWarpListMax list entries
// (columns whose list outgrew the group path; stage holds that many).  Exact
// breakpoints inline.
__device__ __noinline__ void column_warp(const Dev &d, const VarOut &o, int q, SEnt *stage, long long iter,
                                         long long nviol, long long bestnv, Cand &best)
{
    const int lane = threadIdx.x & 31;
    const ColCtx c = make_col(d, q, iter);
    const int nv = c.nI + c.nF;
    int cnt;
    {
        const bool fl = dfinite(__ldg(d.lb + c.j)), fu = dfinite(__ldg(d.ub + c.j));
        if (lane == 0) {
            if (fl) stage[0] = SEnt{c.kl, 0, make_aux(kClsPre, 0)};
            if (fu) stage[fl ? 1 : 0] = SEnt{c.ku, 0, make_aux(kClsPre, 0)};
        }
        cnt = (int)fl + (int)fu;
    }
    Acc acc{0, 0, 0, 0};
    for (int v = lane; v - lane < nv; v += 32) {
        Half h1, h2;
        h1.type = 0; h1.mark = 0;
        h2.type = 0; h2.mark = 0;
        if (v < nv) gen_entry(d, c, v, acc, h1, h2);
#pragma unroll
        for (int hh = 0; hh < 4; ++hh) {
            const Half &h = (hh & 1) ? h2 : h1;
            const bool has = hh < 2 ? h.type != 0 : h.mark != 0;
            const unsigned bal = __ballot_sync(FULLMASK, has);
            if (has)
                stage[cnt + __popc(bal & ((1u << lane) - 1u))] =
                    hh < 2 ? SEnt{h.key, (int)h.D, half_aux(h)} : SEnt{h.mkey, 0, marker_aux()};
            cnt += __popc(bal);
        }
    }
    warp_allreduce_acc(acc);
    __syncwarp();
    VCand vb;
    if (cnt <= 32) vb = group_sort_scan<1, 32>(c, acc, stage, cnt, nviol, bestnv);
    else if (cnt <= 64) vb = group_sort_scan<2, 32>(c, acc, stage, cnt, nviol, bestnv);
    else if (cnt <= 128) vb = group_sort_scan<4, 32>(c, acc, stage, cnt, nviol, bestnv);
    else vb = group_sort_scan<8, 32>(c, acc, stage, cnt, nviol, bestnv);
    if (lane == 0) finish_column(d, o, c, vb, best);
    __syncwarp();
}

// Classification context of a lane's column (thresholds of the side tests).
struct NbLane {
    long long ilo, ihi;          // integer variable: l - xbar, u - xbar
    float Lp, Ln, Up, Un, tolf;  // float thresholds for a > 0 / a < 0, rounding margin of t
    bool fok, isint;
    int g, lane;
};

struct NbQueue {
    int qn;      // queued halves
    bool ovf;    // the warp's halves did not fit: its columns take the whole-warp path
};

// Append the lanes' undecided halves to the warp's queue (exact breakpoints
// after the classification, 32 at a time); when they do not fit, the warp's
// columns are evaluated again on the whole-warp path instead.
template <int G>
__device__ __forceinline__ void enqueue(NbWarp<G> &W, NbQueue &Q, bool pend, const QItem &it, int lane)
{
    const unsigned bal = __ballot_sync(FULLMASK, pend);
    const int n = __popc(bal);
    if (Q.qn + n > kQCap) {
        Q.ovf = Q.ovf || n > 0;
        return;
    }
    if (pend) W.q[Q.qn + __popc(bal & ((1u << lane) - 1u))] = it;
    Q.qn += n;
}

// One half of an integral row (integer variable, exact int64 r and a).  Exact
// side test with z = -r, aa = a (a > 0) or z = r, aa = -a: t < l <=>
// z <= L' aa - [a > 0] and t > u <=> z > H' aa - [a > 0], where L' = lo,
// H' = hi + 1 (a > 0) or L' = lo - 1, H' = hi (a < 0); |lo a|, |hi a| <= 2^53
// on integral rows.
template <int G>
__device__ __forceinline__ void nb_int_half(long long r, int a, int w, bool act, const NbLane &L, NbWarp<G> &W,
                                            NbQueue &Q, Acc &acc)
{
    const bool V = r > 0, P = a > 0;
    const long long z = P ? -r : r;
    const long long aa = P ? a : -a;
    const long long Lz = (P ? L.ilo : L.ilo - 1) * aa - (long long)P;
    const long long Rz = (P ? L.ihi + 1 : L.ihi) * aa - (long long)P;
    const bool left = z <= Lz, right = z > Rz;
    const bool dec = act && (left || right);
    acc_decided(dec ? (((int)P << 2) | ((int)V << 1) | (int)left) : 1, w, acc);
    enqueue(W, Q, act && !dec, QItem{r, (long long)a, 0, w, L.g | ((int)V << 4)}, L.lane);
}

// Both loops below load the next round's row index and coefficient while the
// current round's row state is gathered (one memory latency per round).
template <int G, bool EQ>
__device__ __forceinline__ void nb_int_part(const Dev &d, int e0, int n, int nmax, int sub, const NbLane &L,
                                            NbWarp<G> &W, NbQueue &Q, Acc &acc)
{
    const int *rowp = d.ci_row + e0, *valp = d.ci_val + e0;
    bool ok = sub < n;
    int row = ok ? __ldg(rowp + sub) : 0;
    int av = ok ? __ldg(valp + sub) : 1;
    for (int base = 0; base < nmax; base += G) {
        const int4 st = ok ? ld_row16(d.rs + row) : make_int4(0, 0, 0, 0);
        const int vn = base + G + sub;
        const bool okn = vn < n;
        const int rown = okn ? __ldg(rowp + vn) : 0;
        const int avn = okn ? __ldg(valp + vn) : 1;
        const long long r = row_r(st);
        nb_int_half(r, av, st.z, ok, L, W, Q, acc);
        if (EQ) nb_int_half(-r, -av, st.w, ok, L, W, Q, acc);
        ok = okn;
        row = rown;
        av = avn;
    }
}

// One half of a non-integral row: residual r, coefficient a, margins m = eps - r
// of the half and mo of the other half.  Integer variable: its breakpoint
// xbar + m / a is placed (z = m); continuous: both the tight point xbar - r / a
// and the boundary xbar + m / a must lie on one side (z from -r to m).  The
// points are placed by float products with margins.
template <int G>
__device__ __forceinline__ void nb_fp_half(double r, double a, double m, double mo, int w, bool act,
                                           const NbLane &L, NbWarp<G> &W, NbQueue &Q, Acc &acc)
{
    const bool V = dneg(m), P = !dneg(a);
    const bool near0 = !L.isint && !V && !dneg(mo);
    // normalised (a > 0) offsets of the points: zb the boundary (the integer
    // variable's breakpoint), zt the continuous variable's tight point; zt <= zb
    // for a > 0 and zb <= zt for a < 0 since eps >= 0
    const double zb = P ? m : dflip(m), zt = P ? dflip(r) : r;
    const double zlo = (L.isint || !P) ? zb : zt, zhi = (L.isint || P) ? zb : zt;
    bool fin = L.fok;
    const float zl = approx_f(zlo, fin), zh = approx_f(zhi, fin), af = approx_f(P ? a : dflip(a), fin);
    bool left = false, right = false;
    if (fin) side_test(zl, zh, af, P ? L.Lp : L.Ln, P ? L.Up : L.Un, L.tolf * af, left, right);
    const bool dec = act && (left || right);
    acc_decided(dec ? (((int)P << 2) | ((int)V << 1) | (int)left) : 1, w, acc);
    enqueue(W, Q, act && !dec,
            QItem{__double_as_longlong(L.isint ? m : r), __double_as_longlong(a), __double_as_longlong(m), w,
                  L.g | 8 | ((int)V << 4) | ((int)near0 << 5)},
            L.lane);
}

template <int G, bool EQ>
__device__ __forceinline__ void nb_fp_part(const Dev &d, int e0, int n, int nmax, int sub, const NbLane &L,
                                           NbWarp<G> &W, NbQueue &Q, Acc &acc)
{
    const int *rowp = d.cf_row + e0;
    const double *valp = d.cf_val + e0;
    bool ok = sub < n;
    int row = ok ? __ldg(rowp + sub) : 0;
    double a = ok ? __ldg(valp + sub) : 1.0;
    for (int base = 0; base < nmax; base += G) {
        const int4 *p = reinterpret_cast<const int4 *>(d.rs + row);
        const int4 s0 = ok ? __ldg(p) : make_int4(0, 0, 0, 0);
        const int4 s1 = ok ? __ldg(p + 1) : make_int4(0, 0, 0, 0);
        const int vn = base + G + sub;
        const bool okn = vn < n;
        const int rown = okn ? __ldg(rowp + vn) : 0;
        const double an = okn ? __ldg(valp + vn) : 1.0;
        const double r = i4_double_lo(s0), m1 = i4_double_lo(s1), m2 = i4_double_hi(s1);
        nb_fp_half(r, a, m1, m2, s0.z, ok, L, W, Q, acc);
        if (EQ) nb_fp_half(dflip(r), dflip(a), m2, m1, s0.w, ok, L, W, Q, acc);
        ok = okn;
        row = rown;
        a = an;
    }
}

template <int G>
__global__ void __launch_bounds__(kEvalThreads, 3) k_eval_nb(Dev d, int q0, int ncols, VarOut o, int slot0, int gate)
{
    if (gated_done(d, gate)) return;
    extern __shared__ __align__(16) unsigned char nb_smem[];
    constexpr int CPW = NbGeom<G>::kCols, STG = NbGeom<G>::kStage;
    NbWarp<G> *warps = reinterpret_cast<NbWarp<G> *>(nb_smem);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane / G, sub = lane & (G - 1);
    NbWarp<G> &W = warps[warp];
    const long long iter = d.ctl->iter, nviol = d.ctl->nviol, bestnv = d.ctl->best_nviol;
    Cand best{0, kNoVar, 0, 0.0};
    const int nquad = (ncols + CPW - 1) / CPW;
    for (int qd = blockIdx.x * kNbWarps + warp; qd < nquad; qd += gridDim.x * kNbWarps) {
        const int cq = qd * CPW + g;
        const bool live = cq < ncols;
        int nI, nv, ci0, cf0;
        float Lp, Ln, Up, Un, tolf;
        long long ilo, ihi;
        bool fok, isint;
        {
            const ColCtx c = make_col(d, q0 + (live ? cq : 0), iter);
            nI = live ? c.nI : 0;
            nv = live ? c.nI + c.nF : 0;
            ci0 = c.ci0;
            cf0 = c.cf0;
            isint = c.isint;
            fok = c.fok;
            // thresholds of the side test (z / a against L, U with a > 0):
            // integer variable (z = eps - r): t < l <=> z/a < lo (a > 0) or
            // z/a <= lo - 1 (a < 0); t > u <=> z/a >= hi + 1 (a > 0) or z/a > hi
            // (a < 0).  Continuous (z = -r): t < l <=> z/a < l - xbar,
            // t > u <=> z/a > u - xbar, with a margin for the rounding of t.
            ilo = c.lo;
            ihi = c.hi;
            Lp = isint ? c.lof : -c.dlf;
            Ln = isint ? c.lof - 1.0f : -c.dlf;
            Up = isint ? c.hif + 1.0f : -c.duf;
            Un = isint ? c.hif : -c.duf;
            tolf = c.xaf * 1.0e-10f;
            if (sub == 0) {
                W.ctx[g] = c;
                W.beta[g] = 0; W.alpha[g] = 0; W.beta_c[g] = 0; W.alpha_c[g] = 0;
                int n = 0;
                if (live) {
                    if (dfinite(__ldg(d.lb + c.j))) W.stage[g * STG + n++] = SEnt{c.kl, 0, make_aux(kClsPre, 0)};
                    if (dfinite(__ldg(d.ub + c.j))) W.stage[g * STG + n++] = SEnt{c.ku, 0, make_aux(kClsPre, 0)};
                }
                W.cnt[g] = n;
            }
        }
        __syncwarp();
        NbQueue Q{0, false};
        Acc acc{0, 0, 0, 0};
        const NbLane L{ilo, ihi, Lp, Ln, Up, Un, tolf, fok, isint, g, lane};
        const int cim = live ? __ldg(d.ci_eq + q0 + cq) : ci0, cfm = live ? __ldg(d.cf_eq + q0 + cq) : cf0;
        const int nIs = cim - ci0, nIe = nI - nIs, nFs = cfm - cf0, nFe = (nv - nI) - nFs;
        nb_int_part<G, false>(d, ci0, nIs, groups_max<G>(nIs), sub, L, W, Q, acc);
        nb_int_part<G, true>(d, cim, nIe, groups_max<G>(nIe), sub, L, W, Q, acc);
        nb_fp_part<G, false>(d, cf0, nFs, groups_max<G>(nFs), sub, L, W, Q, acc);
        nb_fp_part<G, true>(d, cfm, nFe, groups_max<G>(nFe), sub, L, W, Q, acc);
        __syncwarp();
        if (!Q.ovf)
            for (int h0 = 0; h0 < Q.qn; h0 += 32) flush_queue(W, h0, min(32, Q.qn - h0), lane);
        // group sums of the scalars
#pragma unroll
        for (int o2 = G >> 1; o2 > 0; o2 >>= 1) {
            acc.beta += __shfl_xor_sync(FULLMASK, acc.beta, o2);
            acc.alpha += __shfl_xor_sync(FULLMASK, acc.alpha, o2);
            acc.beta_c += __shfl_xor_sync(FULLMASK, acc.beta_c, o2);
            acc.alpha_c += __shfl_xor_sync(FULLMASK, acc.alpha_c, o2);
        }
        acc.beta += W.beta[g];
        acc.alpha += W.alpha[g];
        acc.beta_c += W.beta_c[g];
        acc.alpha_c += W.alpha_c[g];
        const int cnt = W.cnt[g];
        const bool over = cnt > STG || Q.ovf;
        // Bound: no candidate of the column scores above beta + (its positive
        // deltas) + max(alpha, 0).  A column whose bound is not positive, or
        // is below an admissible score already found in this pass, cannot
        // give the move, so its list is not sorted (exact; only when no
        // per-variable output is asked for).
        bool prune = false;
        if (!(o.xhat || o.s || o.dc)) {
            const long long found = *reinterpret_cast<volatile const long long *>(&d.ctl->pass_best);
            long long pos = 0;
            if (!over)
                for (int e = sub; e < cnt; e += G) {
                    const long long D = W.stage[g * STG + e].del;
                    pos += D > 0 ? D : 0;
                }
#pragma unroll
            for (int o2 = G >> 1; o2 > 0; o2 >>= 1) pos += __shfl_xor_sync(FULLMASK, pos, o2);
            const long long bound = acc.beta + pos + (acc.alpha > 0 ? acc.alpha : 0);
            prune = !over && (bound <= 0 || bound < found);
        }
        int cmax = (over || prune) ? 0 : cnt;
#pragma unroll
        for (int o2 = 16; o2 >= G; o2 >>= 1) cmax = max(cmax, __shfl_xor_sync(FULLMASK, cmax, o2));
        {
            const ColCtx &c = W.ctx[g];
            const SEnt *list = W.stage + g * STG;
            VCand vb{0, 0ull, 0, 0};
            const int cn = (over || prune) ? 0 : cnt;
            if (cmax == 0) {
                // every column of the warp pruned, overflowing or without entries
            } else if (cmax <= G) {
                vb = group_sort_scan<1, G>(c, acc, list, cn, nviol, bestnv);
            } else if (cmax <= 2 * G) {
                vb = group_sort_scan<2, G>(c, acc, list, cn, nviol, bestnv);
            } else {
                vb = group_sort_scan<4, G>(c, acc, list, cn, nviol, bestnv);
            }
            if (sub == 0 && live && !over) {
                finish_column(d, o, c, vb, best);
                if (best.s > 0) atomicMax(&d.ctl->pass_best, best.s);
            }
        }
        __syncwarp();
        unsigned ovf = __ballot_sync(FULLMASK, sub == 0 && live && over);
        while (ovf) {
            const int gg = (__ffs(ovf) - 1) / G;
            ovf &= ovf - 1;
            column_warp(d, o, q0 + qd * CPW + gg, W.stage, iter, nviol, bestnv, best);
        }
    }
    const Cand bb = block_reduce_cand(best);
    if (threadIdx.x == 0) d.block_best[slot0 + blockIdx.x] = bb;
    finish_pass(d);
}

// ------------------------------------------------- CTA bitonic sort (smem)

__device__ __forceinline__ void block_scan2(long long &v, int &vc, long long *wsum, int *wsumc)
{
    // exclusive block scan of (v, vc); returns the exclusive prefix in (v, vc)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long tot = v;
    int totc = vc;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        long long a = __shfl_up_sync(FULLMASK, tot, off);
        int b = __shfl_up_sync(FULLMASK, totc, off);
        if (lane >= off) { tot += a; totc += b; }
    }
    if (lane == 31) { wsum[warp] = tot; wsumc[warp] = totc; }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        long long x = lane < nw ? wsum[lane] : 0;
        int xc = lane < nw ? wsumc[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            long long a = __shfl_up_sync(FULLMASK, x, off);
            int b = __shfl_up_sync(FULLMASK, xc, off);
            if (lane >= off) { x += a; xc += b; }
        }
        if (lane < nw) { wsum[lane] = x; wsumc[lane] = xc; }
    }
    __syncthreads();
    long long ex = (tot - v) + (warp > 0 ? wsum[warp - 1] : 0);
    int exc = (totc - vc) + (warp > 0 ? wsumc[warp - 1] : 0);
    v = ex;
    vc = exc;
    __syncthreads();
}

// Bitonic sort of N (a power of two) entries in shared memory by (t, class),
// all threads of the CTA; ends with a barrier.
__device__ void cta_bitonic(unsigned long long *skey, long long *sdel, unsigned *saux, int N)
{
    for (int size = 2; size <= N; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int p = threadIdx.x; p < (N >> 1); p += blockDim.x) {
                const int i = 2 * stride * (p / stride) + (p % stride);
                const int k2 = i + stride;
                const bool asc = (i & size) == 0;
                unsigned long long ka = skey[i], kb = skey[k2];
                unsigned aa = saux[i], ab = saux[k2];
                if (entry_less(kb, ab, ka, aa) == asc) {
                    skey[i] = kb; skey[k2] = ka;
                    saux[i] = ab; saux[k2] = aa;
                    long long t = sdel[i]; sdel[i] = sdel[k2]; sdel[k2] = t;
                }
            }
            __syncthreads();
        }
    }
}

// One column per CTA, entries sorted in shared memory (bitonic, N = tile.aux).
__global__ void __launch_bounds__(kCtaThreads) k_eval_cta(Dev d, const Tile *tiles, VarOut o, int slot0, int gate)
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
    __shared__ long long wsum[32];
    __shared__ int wsumc[32];
    const long long iter = d.ctl->iter, nviol = d.ctl->nviol, bestnv = d.ctl->best_nviol;
    const ColCtx c = make_col(d, tl.begin, iter);
    const double l = __ldg(d.lb + c.j), u = __ldg(d.ub + c.j);
    const bool fl = dfinite(l), fu = dfinite(u);
    if (threadIdx.x == 0) {
        s_cnt = (fl ? 1 : 0) + (fu ? 1 : 0);
        s_beta = 0; s_alpha = 0; s_bc = 0; s_ac = 0;
        if (fl) { skey[0] = c.kl; sdel[0] = 0; saux[0] = make_aux(kClsPre, 0); }
        if (fu) { int p = fl ? 1 : 0; skey[p] = c.ku; sdel[p] = 0; saux[p] = make_aux(kClsPre, 0); }
    }
    __syncthreads();
    Acc acc{0, 0, 0, 0};
    const int total = c.nI + c.nF;
    for (int v = threadIdx.x; v < total; v += blockDim.x) {
        Half h1, h2;
        gen_entry(d, c, v, acc, h1, h2);
        const int n1 = half_entries(h1), n2 = half_entries(h2);
        if (n1 + n2) {
            int pos = atomicAdd(&s_cnt, n1 + n2);
            if (n1) put_half(h1, pos, skey, sdel, saux);
            if (n2) put_half(h2, pos + n1, skey, sdel, saux);
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
    for (int i = cnt + threadIdx.x; i < N; i += blockDim.x) { skey[i] = kPadKey; sdel[i] = 0; saux[i] = make_aux(kClsPost, 0); }
    __syncthreads();
    cta_bitonic(skey, sdel, saux, N);
    const int per = N / blockDim.x;
    const int b0 = threadIdx.x * per;
    long long run = 0;
    int runc = 0;
    for (int q = 0; q < per; ++q) { run += sdel[b0 + q]; runc += aux_dc(saux[b0 + q]); }
    long long P = run;
    int Pc = runc;
    block_scan2(P, Pc, wsum, wsumc);
    const long long beta = s_beta, alpha = s_alpha;
    const int bc = s_bc, ac = s_ac;
    VCand vb{0, 0ull, 0, 0};
    for (int q = 0; q < per; ++q) {
        const int i = b0 + q;
        const unsigned long long kk = skey[i];
        const unsigned a = saux[i];
        P += sdel[i];
        Pc += aux_dc(a);
        const unsigned long long knext = i + 1 < N ? skey[i + 1] : kPadKey;
        const unsigned anext = i + 1 < N ? saux[i + 1] : make_aux(kClsPost, 0);
        const unsigned long long kprev = i > 0 ? skey[i - 1] : 0ull;
        const unsigned aprev = i > 0 ? saux[i - 1] : 0u;
        if (!is_candidate(kk, a, kprev, aprev, i > 0, knext, anext)) continue;
        const bool post = aux_post(a) != 0;
        const long long Pi = P - (post ? sdel[i] : 0);
        const int Pci = Pc - (post ? aux_dc(a) : 0);
        const bool right = kk > c.kxb;
        consider(vb, c, kk, beta + Pi + (right ? alpha : 0), bc + Pci + (right ? ac : 0), nviol, bestnv);
    }
    vb = block_reduce_vc(vb, c);
    if (threadIdx.x == 0) {
        Cand best{0, kNoVar, 0, 0.0};
        finish_column(d, o, c, vb, best);
        d.block_best[slot0 + blockIdx.x] = best;
    }
    finish_pass(d);
}

// ------------------------------- multi-CTA counting sort (long integer columns)

// Every CTA bins one chunk of the column's nonzeros by breakpoint value; the
// last CTA of the column scans the bins in value order and takes the argmax.
__global__ void __launch_bounds__(kHistThreads) k_eval_hist(Dev d, const Tile *tiles, VarOut o, int gate)
{
    if (gated_done(d, gate)) return;
    extern __shared__ __align__(16) unsigned char smem[];
    HBin *sb = reinterpret_cast<HBin *>(smem);
    __shared__ long long wsum[32];
    __shared__ int wsumc[32];
    __shared__ int s_last;
    const Tile tl = tiles[blockIdx.x];
    const HistCol hc = d.hcols[tl.begin];
    const int chunk = tl.aux;
    const ColCtx c = make_col(d, hc.pos, d.ctl->iter);
    const long long lo = ikey_val(c.kl);
    const int D = (int)(ikey_val(c.ku) - lo) + 1;
    for (int b = threadIdx.x; b < D; b += blockDim.x) sb[b] = HBin{0, 0, 0, 0};
    __syncthreads();
    const int v0 = chunk * kHistChunk;
    const int v1 = min(hc.e_end, v0 + kHistChunk);
    Acc acc{0, 0, 0, 0};
    for (int v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
        Half h[2];
        gen_entry(d, c, v, acc, h[0], h[1]);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            if (h[q].type == 0) continue;
            HBin *p = sb + (int)(ikey_val(h[q].key) - lo);
            if (h[q].type == 1) {
                atomicAdd(reinterpret_cast<unsigned long long *>(&p->spre), (unsigned long long)h[q].D);
                atomicAdd(&p->n1, 1);
            } else {
                atomicAdd(reinterpret_cast<unsigned long long *>(&p->spost), (unsigned long long)h[q].D);
                atomicAdd(&p->n2, 1);
            }
        }
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
        const HBin s = sb[b];
        if (s.spre) atomicAdd(reinterpret_cast<unsigned long long *>(&gb[b].spre), (unsigned long long)s.spre);
        if (s.spost) atomicAdd(reinterpret_cast<unsigned long long *>(&gb[b].spost), (unsigned long long)s.spost);
        if (s.n1) atomicAdd(&gb[b].n1, s.n1);
        if (s.n2) atomicAdd(&gb[b].n2, s.n2);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(&ha->ticket, 1u) == (unsigned)(hc.nchunks - 1));
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const long long beta = __ldcg(&ha->beta), alpha = __ldcg(&ha->alpha);
    const int bc = __ldcg(&ha->beta_c), ac = __ldcg(&ha->alpha_c);
    const long long iter = d.ctl->iter, nviol = d.ctl->nviol, bestnv = d.ctl->best_nviol;
    const int per = (D + blockDim.x - 1) / blockDim.x;
    const int b0 = threadIdx.x * per;
    long long run = 0;
    int runc = 0;
    for (int q = 0; q < per; ++q) {
        const int b = b0 + q;
        if (b >= D) break;
        run += __ldcg(&gb[b].spre) + __ldcg(&gb[b].spost);
        runc += __ldcg(&gb[b].n2) - __ldcg(&gb[b].n1);
    }
    long long P = run;
    int Pc = runc;
    block_scan2(P, Pc, wsum, wsumc);
    VCand vb{0, 0ull, 0, 0};
    for (int q = 0; q < per; ++q) {
        const int b = b0 + q;
        if (b >= D) break;
        const long long spre = __ldcg(&gb[b].spre), spost = __ldcg(&gb[b].spost);
        const int n1 = __ldcg(&gb[b].n1), n2 = __ldcg(&gb[b].n2);
        if ((n1 | n2) != 0 || b == 0 || b == D - 1) {
            const unsigned long long k = ikey(lo + b);
            const bool right = k > c.kxb;
            consider(vb, c, k, beta + P + spre + (right ? alpha : 0), bc + Pc - n1 + (right ? ac : 0), nviol, bestnv);
        }
        P += spre + spost;
        Pc += n2 - n1;
    }
    vb = block_reduce_vc(vb, c);
    for (int b = threadIdx.x; b < D; b += blockDim.x) gb[b] = HBin{0, 0, 0, 0};
    if (threadIdx.x == 0) {
        Cand best{0, kNoVar, 0, 0.0};
        finish_column(d, o, c, vb, best);
        d.block_best[hc.slot] = best;
        *ha = HistAcc{0, 0, 0, 0, 0u, 0};
    }
    finish_pass(d);
}

// ------------------------------------ multi-CTA merge sort (long lists)
//
// Lists longer than one CTA sorts (Sec. 3.1, "Kernel Specialization": long
// vectors need grid-wide primitives).  k_long_gen: one CTA per chunk of
// kLongChunk nonzeros generates the chunk's entries (and the bounds in chunk
// 0), sorts them in shared memory and writes a run of kLongRun entries padded
// with pad keys (pad runs fill the column up to a power of two); the
// accumulators beta / alpha go to the column's global accumulator.
// k_long_merge: one pairwise merge round over all columns, one thread per
// output entry placed by a merge-path binary search (stable: the left run
// first on equal (t, class)).  k_long_tilesum / k_long_eval: the merged list is
// scanned in tiles of kLongTile entries; each tile adds the sums of the tiles
// before it (its carry), evaluates its candidates (neighbours read across tile
// edges) and the last tile of the column reduces the tiles' candidates.

__global__ void __launch_bounds__(kLongThreads) k_long_gen(Dev d, const Tile *tiles, int gate)
{
    if (gated_done(d, gate)) return;
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long *skey = reinterpret_cast<unsigned long long *>(smem);
    long long *sdel = reinterpret_cast<long long *>(skey + kLongRun);
    unsigned *saux = reinterpret_cast<unsigned *>(sdel + kLongRun);
    __shared__ int s_cnt;
    const Tile tl = tiles[blockIdx.x];
    const LongCol lc = d.lcols[tl.begin];
    const int chunk = tl.aux;
    const ColCtx c = make_col(d, lc.pos, d.ctl->iter);
    if (threadIdx.x == 0) {
        int n0 = 0;
        if (chunk == 0) {
            if (dfinite(__ldg(d.lb + c.j))) { skey[n0] = c.kl; sdel[n0] = 0; saux[n0] = make_aux(kClsPre, 0); ++n0; }
            if (dfinite(__ldg(d.ub + c.j))) { skey[n0] = c.ku; sdel[n0] = 0; saux[n0] = make_aux(kClsPre, 0); ++n0; }
        }
        s_cnt = n0;
    }
    __syncthreads();
    Acc acc{0, 0, 0, 0};
    if (chunk < lc.nchunks) {
        const int v0 = chunk * kLongChunk, v1 = min(lc.e_end, v0 + kLongChunk);
        for (int v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
            Half h1, h2;
            gen_entry(d, c, v, acc, h1, h2);
            const int n1 = half_entries(h1), n2 = half_entries(h2);
            if (n1 + n2) {
                const int pos = atomicAdd(&s_cnt, n1 + n2);
                if (n1) put_half(h1, pos, skey, sdel, saux);
                if (n2) put_half(h2, pos + n1, skey, sdel, saux);
            }
        }
    }
    warp_allreduce_acc(acc);
    HistAcc *la = d.lacc + tl.begin;
    if ((threadIdx.x & 31) == 0 && (acc.beta | acc.alpha | acc.beta_c | acc.alpha_c)) {
        atomicAdd(reinterpret_cast<unsigned long long *>(&la->beta), (unsigned long long)acc.beta);
        atomicAdd(reinterpret_cast<unsigned long long *>(&la->alpha), (unsigned long long)acc.alpha);
        atomicAdd(&la->beta_c, acc.beta_c);
        atomicAdd(&la->alpha_c, acc.alpha_c);
    }
    __syncthreads();
    const int cnt = s_cnt;
    for (int i = cnt + threadIdx.x; i < kLongRun; i += blockDim.x) {
        skey[i] = kPadKey; sdel[i] = 0; saux[i] = make_aux(kClsPost, 0);
    }
    __syncthreads();
    cta_bitonic(skey, sdel, saux, kLongRun);
    SEntry *out = d.lbuf0 + lc.base + (long long)chunk * kLongRun;
    for (int i = threadIdx.x; i < kLongRun; i += blockDim.x) out[i] = SEntry{skey[i], (int)sdel[i], saux[i]};
}

__device__ __forceinline__ bool sent_less(const SEntry &a, const SEntry &b) { return entry_less(a.key, a.aux, b.key, b.aux); }

// One merge round: runs of `width` entries merged pairwise (columns already
// merged into one run are copied).
__global__ void __launch_bounds__(256) k_long_merge(Dev d, const SEntry *in, SEntry *out, long long width,
                                                    long long total, int gate)
{
    if (gated_done(d, gate)) return;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        int lo = 0, hi = d.n_long - 1;   // the column with base <= e
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (d.lcols[mid].base <= e) lo = mid;
            else hi = mid - 1;
        }
        const LongCol &lc = d.lcols[lo];
        const long long k = e - lc.base;
        if ((long long)lc.runs * kLongRun <= width) {
            out[e] = in[e];
            continue;
        }
        const long long p0 = lc.base + (k / (2 * width)) * 2 * width;
        const long long kk = k % (2 * width);
        const SEntry *A = in + p0, *B = in + p0 + width;
        // smallest i with B[kk - i - 1] < A[i]: the number of A entries among
        // the first kk outputs
        long long a = kk > width ? kk - width : 0, b = kk < width ? kk : width;
        while (a < b) {
            const long long i = (a + b) >> 1;
            const long long j = kk - i - 1;
            if (j < 0 || sent_less(B[j], A[i])) b = i;
            else a = i + 1;
        }
        const long long i = a, j = kk - a;
        out[e] = (i < width && (j >= width || !sent_less(B[j], A[i]))) ? A[i] : B[j];
    }
}

__global__ void __launch_bounds__(kLongThreads) k_long_tilesum(Dev d, const SEntry *buf, const Tile *tiles, int gate)
{
    if (gated_done(d, gate)) return;
    const Tile tl = tiles[blockIdx.x];
    const LongCol lc = d.lcols[tl.begin];
    const SEntry *p = buf + lc.base + (long long)tl.aux * kLongTile;
    long long s = 0;
    int sc = 0;
    for (int i = threadIdx.x; i < kLongTile; i += blockDim.x) {
        s += p[i].del;
        sc += aux_dc(p[i].aux);
    }
    __shared__ long long ws[32];
    __shared__ int wsc[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(FULLMASK, s, o);
        sc += __shfl_xor_sync(FULLMASK, sc, o);
    }
    if ((threadIdx.x & 31) == 0) { ws[threadIdx.x >> 5] = s; wsc[threadIdx.x >> 5] = sc; }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        int tc = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { t += ws[w]; tc += wsc[w]; }
        d.ltsum[lc.tile0 + tl.aux] = t;
        d.ltsumc[lc.tile0 + tl.aux] = tc;
    }
}

__global__ void __launch_bounds__(kLongThreads) k_long_eval(Dev d, const SEntry *buf, const Tile *tiles, VarOut o,
                                                            int gate)
{
    if (gated_done(d, gate)) return;
    __shared__ long long wsum[32];
    __shared__ int wsumc[32];
    __shared__ int s_last;
    const Tile tl = tiles[blockIdx.x];
    const LongCol lc = d.lcols[tl.begin];
    const long long iter = d.ctl->iter, nviol = d.ctl->nviol, bestnv = d.ctl->best_nviol;
    const ColCtx c = make_col(d, lc.pos, iter);
    const long long len = (long long)lc.runs * kLongRun;
    // carry: the sums of the column's earlier tiles (block reduction)
    __shared__ long long s_carry;
    __shared__ int s_carryc;
    {
        long long cs = 0;
        int csc = 0;
        for (int t = threadIdx.x; t < tl.aux; t += blockDim.x) {
            cs += __ldcg(d.ltsum + lc.tile0 + t);
            csc += __ldcg(d.ltsumc + lc.tile0 + t);
        }
#pragma unroll
        for (int o2 = 16; o2 > 0; o2 >>= 1) {
            cs += __shfl_xor_sync(FULLMASK, cs, o2);
            csc += __shfl_xor_sync(FULLMASK, csc, o2);
        }
        if ((threadIdx.x & 31) == 0) { wsum[threadIdx.x >> 5] = cs; wsumc[threadIdx.x >> 5] = csc; }
        __syncthreads();
        if (threadIdx.x == 0) {
            long long t = 0;
            int tc = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { t += wsum[w]; tc += wsumc[w]; }
            s_carry = t;
            s_carryc = tc;
        }
        __syncthreads();
    }
    const long long carry_all = s_carry;
    const int carryc_all = s_carryc;
    const HistAcc *la = d.lacc + tl.begin;
    const long long beta = __ldcg(&la->beta), alpha = __ldcg(&la->alpha);
    const int bc = __ldcg(&la->beta_c), ac = __ldcg(&la->alpha_c);
    constexpr int per = kLongTile / kLongThreads;
    const long long t0 = lc.base + (long long)tl.aux * kLongTile;
    const long long i0 = (long long)tl.aux * kLongTile + threadIdx.x * per;   // index inside the column
    long long run = 0;
    int runc = 0;
    for (int q = 0; q < per; ++q) {
        const SEntry &e = buf[t0 + threadIdx.x * per + q];
        run += e.del;
        runc += aux_dc(e.aux);
    }
    long long P = run;
    int Pc = runc;
    block_scan2(P, Pc, wsum, wsumc);
    P += carry_all;
    Pc += carryc_all;
    VCand vb{0, 0ull, 0, 0};
    for (int q = 0; q < per; ++q) {
        const long long i = i0 + q;
        const SEntry e = buf[lc.base + i];
        P += e.del;
        Pc += aux_dc(e.aux);
        const SEntry nx = i + 1 < len ? buf[lc.base + i + 1] : SEntry{kPadKey, 0, make_aux(kClsPost, 0)};
        const SEntry pv = i > 0 ? buf[lc.base + i - 1] : SEntry{0ull, 0, 0u};
        if (!is_candidate(e.key, e.aux, pv.key, pv.aux, i > 0, nx.key, nx.aux)) continue;
        const bool post = aux_post(e.aux) != 0;
        const long long Pi = P - (post ? e.del : 0);
        const int Pci = Pc - (post ? aux_dc(e.aux) : 0);
        const bool right = e.key > c.kxb;
        consider(vb, c, e.key, beta + Pi + (right ? alpha : 0), bc + Pci + (right ? ac : 0), nviol, bestnv);
    }
    vb = block_reduce_vc(vb, c);
    HistAcc *law = d.lacc + tl.begin;
    if (threadIdx.x == 0) {
        d.lcand[lc.tile0 + tl.aux] = LCand{vb.s, vb.key, vb.dc, vb.valid};
        __threadfence();
        s_last = atomicAdd(&law->ticket, 1u) == (unsigned)(lc.ntiles - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    VCand b{0, 0ull, 0, 0};
    for (int t = threadIdx.x; t < lc.ntiles; t += blockDim.x) {
        const LCand *p = d.lcand + lc.tile0 + t;
        const VCand v{__ldcg(&p->s), __ldcg(&p->key), __ldcg(&p->dc), __ldcg(&p->valid)};
        if (vc_better(v, b, c)) b = v;
    }
    b = block_reduce_vc(b, c);
    if (threadIdx.x == 0) {
        Cand best{0, kNoVar, 0, 0.0};
        finish_column(d, o, c, b, best);
        d.block_best[lc.slot] = best;
        *law = HistAcc{0, 0, 0, 0, 0u, 0};
    }
    finish_pass(d);
}

// Exact evaluation (Algorithm 1 on the whole-warp path) of the short
// non-binary columns among the listed variables, for the learned proposal:
// one warp per listed column; the column's best admissible positive move is
// folded into *key (score << 22 | (2^22 - 1 - var), 64-bit atomicMax: larger
// score, then lower variable) and its value written to xh[var].  Binary
// variables and longer columns in the list are skipped (the flip kernel and
// the exact passes cover them).
__global__ void __launch_bounds__(kEvalThreads) k_subset_eval_nb(Dev d, const int *list, int k, int nb_q0, int nb_cols,
                                                                 double *xh, unsigned long long *key, int gate)
{
    if (gated_done(d, gate)) return;
    __shared__ __align__(16) SEnt stage[kEvalWarps][kWarpListMax];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long iter = d.ctl->iter, nviol = d.ctl->nviol, bestnv = d.ctl->best_nviol;
    for (int idx = blockIdx.x * kEvalWarps + warp; idx < k; idx += gridDim.x * kEvalWarps) {
        const int q = d.vpos[list[idx]];
        if (q < nb_q0 || q >= nb_q0 + nb_cols) continue;   // uniform over the warp
        Cand best{0, kNoVar, 0, 0.0};
        const VarOut none{nullptr, nullptr, nullptr};
        column_warp(d, none, q, stage[warp], iter, nviol, bestnv, best);
        if (lane == 0 && best.s > 0 && best.var != kNoVar) {
            xh[best.var] = best.xhat;
            atomicMax(key, ((unsigned long long)best.s << 22) | (unsigned long long)((1 << 22) - 1 - best.var));
        }
        __syncwarp();
    }
}

// Default of every per-variable output (fixed variables keep it).
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

// The move selected by the last pass as an exchange record.
__global__ void k_move_record(Dev d, chap_move_record *rec)
{
    const Ctl *c = d.ctl;
    chap_move_record r;
    r.score_half = c->mv_var >= 0 ? c->mv_s : 0;
    r.var = c->mv_var;
    r.dnviol = c->mv_dc;
    r.new_value = c->mv_new;
    r.old_value = c->mv_old;
    *rec = r;
}

// The winner of k shards' records (largest score, then lowest variable; no
// positive score: the weight update) becomes the iteration's move.
__global__ void k_apply_records(Dev d, const chap_move_record *recs, int k)
{
    long long bs = 0;
    int bv = kNoVar, bdc = 0;
    double bnew = 0.0;
    for (int q = 0; q < k; ++q) {
        const chap_move_record r = recs[q];
        if (r.score_half > 0 && r.var >= 0 && r.var < d.n && cand_better(r.score_half, r.var, bs, bv)) {
            bs = r.score_half;
            bv = r.var;
            bdc = r.dnviol;
            bnew = r.new_value;
        }
    }
    Ctl *c = d.ctl;
    if (bv != kNoVar) {
        c->mv_var = bv;
        c->mv_s = bs;
        c->mv_dc = bdc;
        c->mv_new = bnew;
        c->mv_old = d.x[bv];
    } else {
        c->mv_var = -1;
        c->mv_s = 0;
        c->mv_dc = 0;
        c->mv_new = 0.0;
        c->mv_old = 0.0;
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

// Objective cutoff (Sec. 3.2): the iteration ended with no violated row, so
// x is feasible and the cutoff row's activity y = r + b is its objective.  It
// becomes the best objective and the row's rhs is tightened to y - delta
// (delta >= 1 and integral on an integral row; on another row at least
// 4 tol max(1, |y|), so that the tightened row is violated beyond its
// tolerance).  Returns the cutoff row's violation count after tightening.
__device__ long long tighten_cutoff(const Dev &d, Ctl *c, long long it)
{
    const int i = c->cut_row;
    RowState *p = d.rs + i;
    const double b = c->cut_rhs;
    double y, bn;
    long long viol;
    if (c->cut_int) {
        const long long yl = p->r + (long long)b;
        const long long bl = yl - (long long)c->cut_delta;
        p->r = yl - bl;
        y = (double)yl;
        bn = (double)bl;
        viol = p->r > 0;
    } else {
        y = __dadd_rn(__longlong_as_double(p->r), b);
        const double tol = c->cut_tol;
        const double dmin = __dmul_rn(__dmul_rn(4.0, tol), fmax(1.0, fabs(y)));
        bn = __dsub_rn(y, fmax(c->cut_delta, dmin));
        const double rn = __dsub_rn(y, bn);
        const double eps = __dmul_rn(tol, fmax(1.0, fabs(bn)));
        p->r = __double_as_longlong(rn);
        p->m1 = __dsub_rn(eps, rn);
        p->m2 = __dadd_rn(eps, rn);
        d.eps[i] = eps;
        viol = dneg(p->m1);
    }
    d.rhs[i] = bn;
    c->cut_rhs = bn;
    c->cut_obj = y;
    c->cut_count += 1;
    c->cut_iter = it;
    return viol;
}

// End of an iteration (one thread): violation count, x and the reverse
// direction's tabu stamp after a move, counters, best count, feasibility, the
// objective cutoff and the run's stop condition (q: the moved variable's
// position).  Returns true when a cutoff
// solution was recorded (the caller's CTA then copies x to x_best).
__device__ bool finish_iteration(const Dev &d, Ctl *c, int var, int q, long long delta)
{
    long long nv = c->nviol + delta;
    c->nviol = nv;
    const long long it = c->iter;
    if (var >= 0) {
        d.x[var] = c->mv_new;
        if (q < d.n_bup) d.bup[q] = __double_as_longlong(c->mv_new) == 0 ? 1 : 0;
        const int stamp = (int)(it + 1 + d.tenure);
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
    bool snap = false;
    if (c->cut_on && nv == 0) {
        // the tightened problem starts a new record of violated rows
        nv = tighten_cutoff(d, c, it + 1);
        c->nviol = nv;
        c->best_nviol = nv;
        snap = true;
    }
    if (c->lz_on) {
        // kept binary scores: the moved column's rows are re-marked; a weight
        // update or a tightened cutoff row changes too many rows to track
        c->lz_var = var;
        if (var < 0 || snap) c->lz_full = 1;
        c->lz_seq += 1;
    }
    if ((c->stop_at_feasible && nv == 0) || it + 1 >= c->max_iter) c->done = 1;
    return snap;
}

// Copy of x into x_best by the threads of one CTA (after a cutoff solution).
__device__ __forceinline__ void snapshot_x(const Dev &d)
{
    for (int j = threadIdx.x; j < d.n; j += blockDim.x) d.x_best[j] = d.x[j];
}

// Apply a move: walk the moved column and update its rows' residuals
// (Sec. 3.1, "Memory Considerations", first point).  The column is split over
// as many CTAs of kApplyMoveThreads as its length needs (one for the usual
// columns); the last of them finishes the iteration.
__global__ void __launch_bounds__(kApplyMoveThreads) k_apply_move(Dev d, int gate)
{
    if (gated_done(d, gate)) return;
    Ctl *c = d.ctl;
    const int var = c->mv_var;
    if (var < 0) return;
    const int q = d.vpos[var];
    const int e0 = d.ci_ptr[q], e1 = d.ci_ptr[q + 1];
    const int f0 = d.cf_ptr[q], f1 = d.cf_ptr[q + 1];
    const int len = (e1 - e0) + (f1 - f0);
    const int nwork = max(1, (len + kApplyMoveThreads - 1) / kApplyMoveThreads);
    if ((int)blockIdx.x >= nwork) return;
    const double dl = __dsub_rn(c->mv_new, c->mv_old);
    const long long di = (long long)dl;
    const int stride = nwork * kApplyMoveThreads;
    long long local = 0;
    for (int v = blockIdx.x * kApplyMoveThreads + threadIdx.x; v < len; v += stride) {
        if (v < e1 - e0) {
            const int e = e0 + v;
            RowState *p = d.rs + d.ci_row[e];
            const long long r0 = p->r;
            const long long r1 = r0 + (long long)d.ci_val[e] * di;
            p->r = r1;
            local += (long long)(r1 > 0) - (long long)(r0 > 0);
            if (p->w2 >= 0) local += (long long)(-r1 > 0) - (long long)(-r0 > 0);
        } else {
            const int e = f0 + (v - (e1 - e0));
            const int i = d.cf_row[e];
            RowState *p = d.rs + i;
            const double eps = d.eps[i];
            const double r1 = __dadd_rn(__longlong_as_double(p->r), __dmul_rn(d.cf_val[e], dl));
            const double m1 = __dsub_rn(eps, r1), m2 = __dadd_rn(eps, r1);
            local += (long long)dneg(m1) - (long long)dneg(p->m1);
            if (p->w2 >= 0) local += (long long)dneg(m2) - (long long)dneg(p->m2);
            p->r = __double_as_longlong(r1);
            p->m1 = m1;
            p->m2 = m2;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) local += __shfl_xor_sync(FULLMASK, local, off);
    __shared__ long long red[kApplyMoveThreads / 32];
    __shared__ int s_snap;
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = local;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int w = 0; w < kApplyMoveThreads / 32; ++w) t += red[w];
        bool last = true;
        if (nwork > 1) {
            if (t) atomicAdd(reinterpret_cast<unsigned long long *>(&c->nviol_delta), (unsigned long long)t);
            __threadfence();
            last = atomicAdd(&c->apply_ticket, 1u) == (unsigned)(nwork - 1);
            if (last) {
                __threadfence();
                t = (long long)__ldcg(reinterpret_cast<const long long *>(&c->nviol_delta));
                c->nviol_delta = 0;
                c->apply_ticket = 0;
            }
        }
        s_snap = last && finish_iteration(d, c, var, q, t);
    }
    __syncthreads();
    if (s_snap) snapshot_x(d);
}

// No admissible positive move: add 1 to the weight of every violated
// normalised row (the weights of Sec. 3.1's scores); the last CTA finishes the
// iteration.
__global__ void __launch_bounds__(kApplyThreads) k_apply_bump(Dev d, int gate)
{
    if (gated_done(d, gate)) return;
    Ctl *c = d.ctl;
    if (c->mv_var >= 0) return;
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int gstride = gridDim.x * blockDim.x;
    for (int i = gtid; i < d.m; i += gstride) {
        RowState *p = d.rs + i;
        const RowState s = *p;
        bool v1, v2;
        if (d.row_int[i]) { v1 = s.r > 0; v2 = -s.r > 0; }
        else { v1 = dneg(s.m1); v2 = dneg(s.m2); }
        if (v1) p->w1 = s.w1 + 1;
        if (s.w2 >= 0 && v2) p->w2 = s.w2 + 1;
    }
    __shared__ int s_snap;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const bool last = atomicAdd(&c->apply_ticket, 1u) == gridDim.x - 1;
        bool snap = false;
        if (last) {
            __threadfence();
            c->apply_ticket = 0;
            snap = finish_iteration(d, c, -1, -1, 0);
        }
        s_snap = snap;
    }
    __syncthreads();
    if (s_snap) snapshot_x(d);
}

// --------------------------------------------------------- state handling

// x_j + 0: a -0 from the caller is stored as +0, like every value the search
// writes itself.
__global__ void k_canon_x(Dev d)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d.n; j += gridDim.x * blockDim.x)
        d.x[j] = __dadd_rn(d.x[j], 0.0);
}

constexpr int kResProd = 15;                      // producer warps of a residual CTA
constexpr int kResThreads = 32 * (kResProd + 1);  // plus the warp that adds
constexpr int kResChunk = 128;                    // entries of each of 32 rows staged per phase
constexpr int kResItems = (kResChunk + kResProd - 1) / kResProd;  // 32-entry pieces per producer lane
constexpr int kResSmem = 2 * kResChunk * 33 * (int)sizeof(double);

// Writes the whole state of physical row i from its sum y (double bits for a
// non-integral row) and returns how many of its normalised halves are
// violated.  Weights: w[k], w[k + 1] of the normalised rows (device), or 1.
__device__ __forceinline__ int put_row_state(const Dev &d, const int *w, int i, long long ybits, bool integral)
{
    const int k = d.nrow_base[i];
    const int kn = i + 1 < d.m ? d.nrow_base[i + 1] : d.m_norm;
    RowState s;
    s.w1 = w ? w[k] : 1;
    s.w2 = kn - k == 2 ? (w ? w[k + 1] : 1) : -1;
    int v;
    if (integral) {
        s.r = ybits - (long long)d.rhs[i];
        s.m1 = 0.0;
        s.m2 = 0.0;
        v = (s.r > 0) + (s.w2 >= 0 && -s.r > 0);
    } else {
        const double r = __dsub_rn(__longlong_as_double(ybits), d.rhs[i]);
        const double eps = d.eps[i];
        s.r = __double_as_longlong(r);
        s.m1 = __dsub_rn(eps, r);
        s.m2 = __dadd_rn(eps, r);
        v = dneg(s.m1) + (s.w2 >= 0 && dneg(s.m2));
    }
    d.rs[i] = s;
    return v;
}

// Residuals at x (Sec. 3.1): r = (sum of a x in CSR order) - b per physical
// row, the margins eps -+ r, the weights, and the count of violated
// normalised rows (set-state only).
//  - The first fp_ctas CTAs take the rows with floating-point data, 32 rows
//    per CTA in decreasing length (res_rows).  Each lane of warp 0 owns one
//    row and adds its products in CSR order, so the residual is the same
//    double as a sequential evaluation, and no lane repeats another lane's
//    adds.  The other kResProd warps form the products of the next phase
//    (kResChunk entries of each row, 32 consecutive entries of one row per
//    warp load, every load of a lane issued before its first gather) into
//    the other half of a shared-memory double buffer.  The add chains of the
//    longest rows set the kernel's duration: a phase is as long as the
//    slower of its kResChunk dependent adds and one round of gathers.
//  - The other CTAs take the integral rows, one warp per row, summing in
//    int64 (exact in any order).
__global__ void __launch_bounds__(kResThreads) k_residuals(Dev d, const int *w, int fp_ctas)
{
    extern __shared__ double res_stage[];  // [2][kResChunk][33]
    __shared__ long long s_p0[32];
    __shared__ int s_len[32];
    __shared__ int s_lmax;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    long long local = 0;
    if ((int)blockIdx.x < fp_ctas) {
        const int n_fp = d.m - d.n_res_int;
        int i = -1;
        if (wib == 0) {
            const int q = blockIdx.x * 32 + lane;
            long long p0 = 0;
            int len = 0;
            if (q < n_fp) {
                i = d.res_rows[d.n_res_int + q];
                p0 = d.row_ptr[i];
                len = (int)(d.row_ptr[i + 1] - p0);
            }
            s_p0[lane] = p0;
            s_len[lane] = len;
            int lmax = len;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) lmax = max(lmax, __shfl_xor_sync(FULLMASK, lmax, off));
            if (lane == 0) s_lmax = lmax;
        }
        __syncthreads();
        const int nch = (s_lmax + kResChunk - 1) / kResChunk;
        const int len = s_len[lane];
        double y = 0.0;
        for (int ph = 0; ph <= nch; ++ph) {
            if (wib > 0 && ph < nch) {
                // pieces it = wib - 1 + kResProd * u of this phase: row it / (kResChunk / 32),
                // entries c0 + 32 (it % (kResChunk / 32)) + lane
                double *t = res_stage + (ph & 1) * (kResChunk * 33);
                const int c0 = ph * kResChunk;
                int col[kResItems];
                double a[kResItems], xv[kResItems];
#pragma unroll
                for (int u = 0; u < kResItems; ++u) {
                    const int it = wib - 1 + kResProd * u;
                    const int rr = it / (kResChunk / 32);
                    const int k = c0 + 32 * (it % (kResChunk / 32)) + lane;
                    col[u] = -1;
                    a[u] = 0.0;
                    if (it < kResChunk && k < s_len[rr]) {
                        const long long e = s_p0[rr] + k;
                        col[u] = __ldg(d.col_idx + e);
                        a[u] = __ldg(d.row_val + e);
                    }
                }
#pragma unroll
                for (int u = 0; u < kResItems; ++u) xv[u] = col[u] >= 0 ? __ldg(d.x + col[u]) : 0.0;
#pragma unroll
                for (int u = 0; u < kResItems; ++u) {
                    const int it = wib - 1 + kResProd * u;
                    if (it < kResChunk) {
                        const int rr = it / (kResChunk / 32);
                        const int kk = 32 * (it % (kResChunk / 32)) + lane;
                        t[kk * 33 + rr] = col[u] >= 0 ? __dmul_rn(a[u], xv[u]) : 0.0;
                    }
                }
            }
            if (wib == 0 && ph > 0) {
                const double *t = res_stage + ((ph - 1) & 1) * (kResChunk * 33);
                const int cnt = min(kResChunk, len - (ph - 1) * kResChunk);
                for (int k = 0; k < cnt; ++k) y = __dadd_rn(y, t[k * 33 + lane]);
            }
            __syncthreads();
        }
        if (wib == 0 && i >= 0) local = put_row_state(d, w, i, __double_as_longlong(y), false);
    } else {
        const int nw = (gridDim.x - fp_ctas) * (kResThreads / 32);
        for (int g = (blockIdx.x - fp_ctas) * (kResThreads / 32) + wib; g < d.n_res_int; g += nw) {
            const int i = d.res_rows[g];
            const long long p0 = d.row_ptr[i], p1 = d.row_ptr[i + 1];
            long long y = 0;
            for (long long e = p0 + lane; e < p1; e += 32) y += (long long)d.row_val[e] * (long long)d.x[d.col_idx[e]];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) y += __shfl_xor_sync(FULLMASK, y, off);
            if (lane == 0) local += put_row_state(d, w, i, y, true);
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) local += __shfl_xor_sync(FULLMASK, local, off);
    if (lane == 0 && local) atomicAdd(reinterpret_cast<unsigned long long *>(&d.ctl->nviol), (unsigned long long)local);
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
    c->pass_best = 0;
    if (c->lz_on) {
        c->lz_full = 1;
        c->lz_count = 0;
        c->lz_done = c->lz_seq;
        c->lz_ticket = 0;
    }
}

__global__ void k_lazy_init(Dev d)
{
    Ctl *c = d.ctl;
    c->lz_on = 1;
    c->lz_full = 1;
    c->lz_count = 0;
    c->lz_epoch = 1u;
    c->lz_seq = 0;
    c->lz_done = 0;
    c->lz_ticket = 0;
}

// Objective cutoff on row `row` (on = 0 switches it off); the rhs is the
// row's current one.
__global__ void k_set_cutoff(Dev d, int on, int row, int integral, double delta, double tol)
{
    Ctl *c = d.ctl;
    c->cut_on = on;
    c->cut_row = on ? row : 0;
    c->cut_int = integral;
    c->cut_rhs = on ? d.rhs[row] : 0.0;
    c->cut_delta = delta;
    c->cut_tol = tol;
    c->cut_obj = __longlong_as_double(0x7ff8000000000000LL);
    c->cut_count = 0;
    c->cut_iter = -1;
}

__global__ void k_begin_run(Dev d, long long max_iters, int stop_at_feasible)
{
    Ctl *c = d.ctl;
    c->max_iter = c->iter + max_iters;
    // a run under the objective cutoff continues past every feasible solution
    if (c->cut_on) stop_at_feasible = 0;
    c->stop_at_feasible = stop_at_feasible;
    c->t_start_ns = global_ns();
    if (c->nviol == 0) { c->feasible_iter = c->iter; c->t_feas_ns = c->t_start_ns; }
    else { c->feasible_iter = -1; c->t_feas_ns = 0; }
    c->done = ((stop_at_feasible && c->nviol == 0) || max_iters <= 0) ? 1 : 0;
}

__global__ void k_unpack_w(Dev d, int *w)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.m; i += gridDim.x * blockDim.x) {
        const int k = d.nrow_base[i];
        const RowState s = d.rs[i];
        w[k] = s.w1;
        if (s.w2 >= 0) w[k + 1] = s.w2;
    }
}

__global__ void k_unpack_r(Dev d, double *r)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.m; i += gridDim.x * blockDim.x) {
        const int k = d.nrow_base[i];
        const RowState s = d.rs[i];
        const double v = d.row_int[i] ? (double)s.r : __longlong_as_double(s.r);
        r[k] = v;
        if (s.w2 >= 0) r[k + 1] = -v;
    }
}

// Objective c^T x of the current assignment: every CTA sums a contiguous chunk
// of the variables (strided per thread, then a fixed tree), and one CTA adds
// the partial sums in CTA order: the same value on every call for the same x.
constexpr int kObjBlocks = 128, kObjThreads = 256;

__device__ __forceinline__ double block_sum_fixed(double s, double *part)
{
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) part[threadIdx.x] = __dadd_rn(part[threadIdx.x], part[threadIdx.x + o]);
        __syncthreads();
    }
    return part[0];
}

__global__ void __launch_bounds__(kObjThreads) k_objective_part(Dev d, double *partial)
{
    __shared__ double part[kObjThreads];
    const int per = (d.n + gridDim.x - 1) / gridDim.x;
    const int j0 = blockIdx.x * per, j1 = min(d.n, j0 + per);
    double s = 0.0;
    for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) s = __dadd_rn(s, __dmul_rn(d.obj[j], d.x[j]));
    const double t = block_sum_fixed(s, part);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kObjThreads) k_objective_final(const double *partial, int np, double *out)
{
    __shared__ double part[kObjThreads];
    double s = 0.0;
    for (int k = threadIdx.x; k < np; k += blockDim.x) s = __dadd_rn(s, partial[k]);
    const double t = block_sum_fixed(s, part);
    if (threadIdx.x == 0) *out = t;
}

__global__ void k_widen(int n, const int *a, long long *b)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) b[j] = a[j];
}

// ---------------------------------------------------------------- launchers

static int grid_for(long long n, int threads, int cap = 152 * 8)
{
    long long g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

static cudaError_t raise_smem_limit(const void *fn, int slot, int bytes);

int bin_grid_size(int ncols, int G)
{
    int per_sm = 0;
    const void *fn = G == 2 ? (const void *)k_eval_bin<2> : G == 4 ? (const void *)k_eval_bin<4>
                     : G == 16 ? (const void *)k_eval_bin<16> : (const void *)k_eval_bin<8>;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kEvalThreads, 0) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        sms = 152;
    }
    const long long cols_per_cta = (long long)kEvalWarps * (32 / G);
    const long long need = ((long long)ncols + cols_per_cta - 1) / cols_per_cta;
    const long long cap = (long long)sms * per_sm;
    return (int)(need < cap ? need : cap);
}

int nb_grid_size(int ncols, int G)
{
    // one resident wave: every SM holds as many CTAs as fit, and no CTA is
    // launched without a column for each of its warps to start with
    int per_sm = 0;
    const void *fn = G == 4 ? (const void *)k_eval_nb<4> : (const void *)k_eval_nb<8>;
    const int smem = G == 4 ? nb_smem<4>() : nb_smem<8>();
    if (raise_smem_limit(fn, G == 4 ? 0 : 1, smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kEvalThreads, smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        sms = 152;
    }
    const long long cols_per_cta = (long long)kNbWarps * (32 / G);
    const long long need = ((long long)ncols + cols_per_cta - 1) / cols_per_cta;
    const long long cap = (long long)sms * per_sm;
    return (int)(need < cap ? need : cap);
}

// Fixed-size scratch of the counting-sort columns for callers that do not
// use the per-handle allocation (chap_bs_best_shift_static_scratch).  Zero at
// module load; k_eval_hist returns every bin and accumulator it touched to
// zero before it finishes, so consecutive passes find it cleared.  Shared by
// every handle of the process: overlapping passes through it race.
static __device__ __align__(256) HBin g_static_bins[kStaticHistBins];
static __device__ __align__(256) HistAcc g_static_acc[kStaticHistCols];

cudaError_t static_hist_scratch(HBin **bins, HistAcc **acc)
{
    // resolved once per device, with that device current; the cache is read
    // and written under a mutex, so first calls from several host threads do
    // not race on it
    constexpr int kMaxDevices = 64;
    static std::mutex s_mu;
    static HBin *s_bins[kMaxDevices] = {};
    static HistAcc *s_acc[kMaxDevices] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(s_mu);
    if (!s_bins[dev] || !s_acc[dev]) {
        void *pb = nullptr, *pa = nullptr;
        e = cudaGetSymbolAddress(&pb, g_static_bins);
        if (e != cudaSuccess) return e;
        e = cudaGetSymbolAddress(&pa, g_static_acc);
        if (e != cudaSuccess) return e;
        s_bins[dev] = static_cast<HBin *>(pb);
        s_acc[dev] = static_cast<HistAcc *>(pa);
    }
    *bins = s_bins[dev];
    *acc = s_acc[dev];
    return cudaSuccess;
}

// The dynamic shared-memory limit is an attribute of the kernel, shared by
// every handle of the process on a device: it is only ever raised (to the
// largest size any handle launches with), under a mutex.
static cudaError_t raise_smem_limit(const void *fn, int slot, int bytes)
{
    constexpr int kMaxDevices = 64, kSlots = 8;
    static std::mutex s_mu;
    static int s_set[kMaxDevices][kSlots] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(s_mu);
    if (bytes <= s_set[dev][slot]) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) s_set[dev][slot] = bytes;
    return e;
}

cudaError_t setup_kernel_attributes(const LaunchPlan &p)
{
    cudaError_t e = cudaSuccess;
    if (p.nb_grid > 0)
        e = p.nb_G == 4 ? raise_smem_limit((const void *)k_eval_nb<4>, 0, nb_smem<4>())
                        : raise_smem_limit((const void *)k_eval_nb<8>, 1, nb_smem<8>());
    if (e == cudaSuccess && p.cta_smem > 0) e = raise_smem_limit((const void *)k_eval_cta, 2, p.cta_smem);
    if (e == cudaSuccess && p.hist_smem > 0) e = raise_smem_limit((const void *)k_eval_hist, 3, p.hist_smem);
    if (e == cudaSuccess && p.n_lgen > 0) e = raise_smem_limit((const void *)k_long_gen, 4, long_gen_smem());
    if (e == cudaSuccess && p.bin_rows) e = raise_smem_limit((const void *)k_eval_bin_rows, 5, kRbSmem);
    if (e == cudaSuccess && p.bin_blk) e = raise_smem_limit((const void *)k_eval_bin_blk, 7, blk_smem(p.bb.rows));
    return e;
}

int long_gen_smem() { return kLongRun * (int)(sizeof(unsigned long long) + sizeof(long long) + sizeof(unsigned)); }

// The long lists' kernels on `st`: generation and run sort, the merge rounds,
// the tile sums and the scan / argmax.
static cudaError_t launch_long(const Dev &d, const LaunchPlan &p, const VarOut &o, int gate, cudaStream_t st)
{
    k_long_gen<<<p.n_lgen, kLongThreads, long_gen_smem(), st>>>(d, p.tiles_lgen, gate);
    const SEntry *in = d.lbuf0;
    SEntry *out = d.lbuf1;
    const int grid = (int)std::min<long long>(152 * 8, (p.long_entries + 255) / 256);
    for (int r = 0; r < p.long_rounds; ++r) {
        k_long_merge<<<grid, 256, 0, st>>>(d, in, out, (long long)kLongRun << r, p.long_entries, gate);
        const SEntry *t = out;
        out = const_cast<SEntry *>(in);
        in = t;
    }
    k_long_tilesum<<<p.n_lscan, kLongThreads, 0, st>>>(d, in, p.tiles_lscan, gate);
    k_long_eval<<<p.n_lscan, kLongThreads, 0, st>>>(d, in, p.tiles_lscan, o, gate);
    return cudaGetLastError();
}

// The row-wise binary kernel: blocks x kRbCluster CTAs in clusters of kRbCluster.
static cudaError_t launch_bin_rows(const Dev &d, const LaunchPlan &p, const VarOut &o, int gate, cudaStream_t st)
{
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = kRbCluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(p.rb.blocks * kRbCluster);
    cfg.blockDim = dim3(kRbThreads);
    cfg.dynamicSmemBytes = kRbSmem;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_eval_bin_rows, d, p.rb, p.bin_cols, o, gate);
}

cudaError_t launch_eval_gated(const Dev &d, const LaunchPlan &p, const VarOut &o, int gate, cudaStream_t st)
{
    // The evaluation kernels are independent: the binary pass (bandwidth bound)
    // runs on `st`, the non-binary classes on side streams, joined before the
    // selection.  The same fork/join shape is recorded by graph capture.
    if (o.xhat || o.s || o.dc) k_fill_outputs<<<grid_for(d.n, 256), 256, 0, st>>>(d, o);
    cudaError_t e = cudaEventRecord(p.ev_fork, st);
    const bool side[3] = {p.nb_grid > 0, p.n_cta > 0 || p.n_lgen > 0, p.n_hist_tiles > 0};
    for (int k = 0; k < 3 && e == cudaSuccess; ++k)
        if (side[k]) e = cudaStreamWaitEvent(p.side[k], p.ev_fork, 0);
    if (e != cudaSuccess) return e;
    const bool prof = p.profile && !gate;
    const cudaStream_t ks[4] = {st, p.side[0], p.side[1], p.side[2]};
#define PROF(k, i) if (prof && e == cudaSuccess) e = cudaEventRecord(p.pev[2 * (k) + (i)], ks[k])
    if (p.n_bin && p.lazy) {
        PROF(0, 0);
        switch (p.bin_G) {
        case 2: k_eval_bin_lazy<2><<<p.n_bin, kEvalThreads, 0, st>>>(d, p.bin_cols, gate); break;
        case 4: k_eval_bin_lazy<4><<<p.n_bin, kEvalThreads, 0, st>>>(d, p.bin_cols, gate); break;
        case 16: k_eval_bin_lazy<16><<<p.n_bin, kEvalThreads, 0, st>>>(d, p.bin_cols, gate); break;
        default: k_eval_bin_lazy<8><<<p.n_bin, kEvalThreads, 0, st>>>(d, p.bin_cols, gate); break;
        }
        k_bin_scan<<<p.n_bin, kEvalThreads, 0, st>>>(d, p.bin_cols, o, gate);
        PROF(0, 1);
    } else if (p.n_bin && p.bin_rows) {
        PROF(0, 0);
        if (e == cudaSuccess) e = launch_bin_rows(d, p, o, gate, st);
        PROF(0, 1);
    } else if (p.n_bin && p.bin_blk) {
        PROF(0, 0);
        k_eval_bin_blk<<<p.bb.n_items, kBlkThreads, blk_smem(p.bb.rows), st>>>(d, p.bb, gate);
        k_bin_blk_final<<<p.bb.n_fin, kBlkFinThreads, 0, st>>>(d, p.bb, p.bin_cols, o, gate);
        PROF(0, 1);
    } else if (p.n_bin) {
        PROF(0, 0);
        switch (p.bin_G) {
        case 2: k_eval_bin<2><<<p.n_bin, kEvalThreads, 0, st>>>(d, p.bin_cols, o, gate); break;
        case 4: k_eval_bin<4><<<p.n_bin, kEvalThreads, 0, st>>>(d, p.bin_cols, o, gate); break;
        case 16: k_eval_bin<16><<<p.n_bin, kEvalThreads, 0, st>>>(d, p.bin_cols, o, gate); break;
        default: k_eval_bin<8><<<p.n_bin, kEvalThreads, 0, st>>>(d, p.bin_cols, o, gate); break;
        }
        PROF(0, 1);
    }
    if (p.nb_grid) {
        PROF(1, 0);
        if (p.nb_G == 4)
            k_eval_nb<4><<<p.nb_grid, kEvalThreads, nb_smem<4>(), p.side[0]>>>(d, p.nb_q0, p.nb_cols, o, p.slot_nb, gate);
        else
            k_eval_nb<8><<<p.nb_grid, kEvalThreads, nb_smem<8>(), p.side[0]>>>(d, p.nb_q0, p.nb_cols, o, p.slot_nb, gate);
        PROF(1, 1);
    }
    if (p.n_cta || p.n_lgen) {
        PROF(2, 0);
        if (p.n_cta) k_eval_cta<<<p.n_cta, kCtaThreads, p.cta_smem, p.side[1]>>>(d, p.tiles_cta, o, p.slot_cta, gate);
        if (p.n_lgen && e == cudaSuccess) e = launch_long(d, p, o, gate, p.side[1]);
        PROF(2, 1);
    }
    if (p.n_hist_tiles) {
        PROF(3, 0);
        k_eval_hist<<<p.n_hist_tiles, kHistThreads, p.hist_smem, p.side[2]>>>(d, p.tiles_hist, o, gate);
        PROF(3, 1);
    }
#undef PROF
    if (e == cudaSuccess) e = cudaGetLastError();
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
        if (!side[k]) continue;
        e = cudaEventRecord(p.ev_join[k], p.side[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, p.ev_join[k], 0);
    }
    return e;
}

cudaError_t launch_select_gated(const Dev &d, const LaunchPlan &p, int gate, cudaStream_t st)
{
    // the evaluation kernels select the move themselves (finish_pass); a
    // kernel is launched only when no evaluation CTA runs
    const bool prof = p.profile && !gate;
    cudaError_t e = prof ? cudaEventRecord(p.pev[8], st) : cudaSuccess;
    if (e != cudaSuccess) return e;
    if (d.n_block_best == 0) {
        k_select<<<1, 1024, 0, st>>>(d, gate);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && prof) e = cudaEventRecord(p.pev[9], st);
    return e;
}

cudaError_t launch_apply_gated(const Dev &d, const LaunchPlan &p, int gate, cudaStream_t st)
{
    k_apply_move<<<p.apply_move_blocks, kApplyMoveThreads, 0, st>>>(d, gate);
    k_apply_bump<<<p.apply_blocks, kApplyThreads, 0, st>>>(d, gate);
    if (p.lazy) k_lazy_mark<<<p.lazy_mark_blocks, kEvalThreads, 0, st>>>(d, p.bin_cols);
    return cudaGetLastError();
}

cudaError_t launch_lazy_init(const Dev &d, cudaStream_t st)
{
    k_lazy_init<<<1, 1, 0, st>>>(d);
    return cudaGetLastError();
}

cudaError_t launch_set_move(const Dev &d, int var, double nv, cudaStream_t st)
{
    k_set_move<<<1, 1, 0, st>>>(d, var, nv);
    return cudaGetLastError();
}

cudaError_t launch_residuals(const Dev &d, const int *w, cudaStream_t st)
{
    k_canon_x<<<grid_for(d.n, 256), 256, 0, st>>>(d);
    if (d.n_bup > 0) k_bup_init<<<grid_for(d.n_bup, 256), 256, 0, st>>>(d);
    const int n_fp = d.m - d.n_res_int;
    const int fp_ctas = (n_fp + 31) / 32;
    const int int_ctas = d.n_res_int > 0 ? std::min((d.n_res_int + kResThreads / 32 - 1) / (kResThreads / 32), 152 * 3) : 0;
    if (fp_ctas + int_ctas == 0) return cudaGetLastError();
    cudaError_t e = raise_smem_limit((const void *)k_residuals, 6, kResSmem);
    if (e != cudaSuccess) return e;
    k_residuals<<<fp_ctas + int_ctas, kResThreads, kResSmem, st>>>(d, w, fp_ctas);
    return cudaGetLastError();
}

cudaError_t launch_finish_set_state(const Dev &d, long long iter, long long best_nviol, int use_best, cudaStream_t st)
{
    k_finish_set_state<<<1, 1, 0, st>>>(d, iter, best_nviol, use_best);
    return cudaGetLastError();
}

cudaError_t launch_set_cutoff(const Dev &d, int on, int row, int integral, double delta, double tol, cudaStream_t st)
{
    k_set_cutoff<<<1, 1, 0, st>>>(d, on, row, integral, delta, tol);
    return cudaGetLastError();
}

cudaError_t launch_begin_run(const Dev &d, long long max_iters, int stop_at_feasible, cudaStream_t st)
{
    k_begin_run<<<1, 1, 0, st>>>(d, max_iters, stop_at_feasible);
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

cudaError_t launch_subset_nb(const Dev &d, const LaunchPlan &p, const int *list, int k, double *xh,
                             unsigned long long *key, int gate, cudaStream_t st)
{
    if (p.nb_cols == 0 || k < 1) return cudaSuccess;
    k_subset_eval_nb<<<grid_for((long long)k * 32, kEvalThreads, 152 * 8), kEvalThreads, 0, st>>>(
        d, list, k, p.nb_q0, p.nb_cols, xh, key, gate);
    return cudaGetLastError();
}

cudaError_t launch_move_record(const Dev &d, chap_move_record *rec, cudaStream_t st)
{
    k_move_record<<<1, 1, 0, st>>>(d, rec);
    return cudaGetLastError();
}

cudaError_t launch_apply_records(const Dev &d, const chap_move_record *recs, int k, cudaStream_t st)
{
    k_apply_records<<<1, 1, 0, st>>>(d, recs, k);
    return cudaGetLastError();
}

cudaError_t launch_objective(const Dev &d, double *out, double *partial, cudaStream_t st)
{
    k_objective_part<<<kObjBlocks, kObjThreads, 0, st>>>(d, partial);
    k_objective_final<<<1, kObjThreads, 0, st>>>(partial, kObjBlocks, out);
    return cudaGetLastError();
}

cudaError_t launch_tabu_convert(int n, const int *a, long long *b, cudaStream_t st)
{
    k_widen<<<grid_for(n, 256), 256, 0, st>>>(n, a, b);
    return cudaGetLastError();
}

}  // namespace chap
