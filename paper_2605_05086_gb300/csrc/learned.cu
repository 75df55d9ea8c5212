// Learned move proposal (growth path, not in the paper): a small network
// 12 -> 64 -> 64 -> 1 (ReLU) predicts each variable's best-shift score from
// per-variable features; the exact best-shift evaluation then runs on the
// top-k predicted variables only, and a full exact pass every E iterations is
// both the fallback move and the judge of the proposal's top-1 misses.  The
// scores that decide moves are always exact.
//
// Kernels: features, refresh of the pass-time features, network forward
// (BF16 parameters and features, FP32 accumulation with explicit FMAs), loss
// gradient over a minibatch (tile of 128 rows per CTA, activations in shared
// memory), Adam, deterministic top-k by three-level radix select + stable
// compaction, exact flip scores of the selected binary columns, and the glue
// that hands the chosen move to the apply kernel of the exact path.
#include "chap_handle.h"

#include <cuda_bf16.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <string>

namespace chap {
namespace {

#define FULLMASK 0xffffffffu

constexpr int kF = 12, kH = 64;
constexpr int kOffW1 = 0, kOffB1 = kF * kH, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH;
constexpr int kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH, kNParams = kOffB3 + 1;  // 5057
constexpr int kGradRows = 128;       // rows of one gradient tile
constexpr int kHPad = kH + 1;        // padded activation rows (no bank conflicts)
constexpr int kTopkPerThread = 4;
constexpr int kTopkBlock = 256 * kTopkPerThread;
constexpr int kVarBits = 22;

// Device state of the learned driver of one handle.
struct __align__(16) LearnCtl {
    unsigned long long key;     // best proposal move: score << 22 | (2^22 - 1 - var), 0 = none
    long long smax;             // max |score| at the last exact pass
    long long passes, misses;   // exact passes and top-1 misses
    long long pass_iter;        // iteration of the last exact pass
    unsigned prefix;            // radix select: digits fixed so far
    int need;                   // elements still to take at the current digit
    unsigned thr;               // k-th largest key
    int total_gt;
};

struct Learn {
    double *xh;                   // value of the best shift of each proposed non-binary column [n]
    float *colviol, *colwv;       // pass-time column features [n]
    long long *s_last;            // exact scores of the last pass [n]
    __nv_bfloat16 *feat;          // [n x 12]
    float *y;                     // predictions [n]
    unsigned *hist;               // 2048 bins
    int *bcnt, *bpre;             // per-block counts / prefixes (2 x nblocks each)
    int *list;                    // selected variables [k]
    LearnCtl *lc;
    int nblocks;
};

__device__ __forceinline__ unsigned long long lglobal_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool done_gate(const Dev &d) { return *(volatile int *)&d.ctl->done != 0; }

__device__ __forceinline__ long long i4_r(const int4 &v)
{
    return (long long)(((unsigned long long)(unsigned)v.y << 32) | (unsigned)v.x);
}

__device__ __forceinline__ bool dbl_neg_bits(long long b) { return b < 0; }

// ---------------------------------------------------------------- features

// Column features recorded at an exact pass: share of violated halves and the
// weighted (w |a|) share, one thread per variable.
__global__ void k_refresh(Dev d, Learn L)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d.n; j += gridDim.x * blockDim.x) {
        const int q = d.vpos[j];
        int halves = 0, viol = 0;
        float wall = 0.0f, wviol = 0.0f;
        for (int e = d.ci_ptr[q]; e < d.ci_ptr[q + 1]; ++e) {
            const RowState s = d.rs[d.ci_row[e]];
            const float a = fabsf((float)d.ci_val[e]);
            halves += 1; wall += s.w1 * a;
            if (s.r > 0) { viol += 1; wviol += s.w1 * a; }
            if (s.w2 >= 0) {
                halves += 1; wall += s.w2 * a;
                if (s.r < 0) { viol += 1; wviol += s.w2 * a; }
            }
        }
        for (int e = d.cf_ptr[q]; e < d.cf_ptr[q + 1]; ++e) {
            const RowState s = d.rs[d.cf_row[e]];
            const float a = fabsf((float)d.cf_val[e]);
            halves += 1; wall += s.w1 * a;
            if (dbl_neg_bits(__double_as_longlong(s.m1))) { viol += 1; wviol += s.w1 * a; }
            if (s.w2 >= 0) {
                halves += 1; wall += s.w2 * a;
                if (dbl_neg_bits(__double_as_longlong(s.m2))) { viol += 1; wviol += s.w2 * a; }
            }
        }
        L.colviol[j] = halves ? (float)viol / (float)halves : 0.0f;
        L.colwv[j] = wall > 0.0f ? wviol / wall : 0.0f;
        const long long sa = L.s_last[j] < 0 ? -L.s_last[j] : L.s_last[j];
        if (sa > 0) atomicMax(reinterpret_cast<unsigned long long *>(&L.lc->smax), (unsigned long long)sa);
    }
}

__global__ void k_refresh_begin(Dev d, Learn L, int gate)
{
    if (gate && done_gate(d)) return;
    L.lc->smax = 0;
    L.lc->pass_iter = d.ctl->iter;
}

// The 12 features of every variable (BF16): x/(u-l), (x-l)/(u-l), (u-x)/(u-l),
// min(tabu age, 64)/64, violated share, violated weighted share, last exact
// score / (1 + max |score|), iterations since the exact pass / 50,
// log2(1 + column length)/16, is_binary, is_integer, c_j / max |c|.
__global__ void k_features(Dev d, Learn L, float cmax, int gate)
{
    if (gate && done_gate(d)) return;
    const long long iter = d.ctl->iter;
    const float smax = (float)L.lc->smax;
    const float since = (float)(iter - L.lc->pass_iter);
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d.n; j += gridDim.x * blockDim.x) {
        const double x = d.x[j], l = d.lb[j], u = d.ub[j];
        const bool fin = isfinite(u - l) && u > l;
        const float w = fin ? (float)(u - l) : 1.0f;
        float f[kF];
        f[0] = fin ? (float)x / w : 0.0f;
        f[1] = fin ? (float)(x - l) / w : 0.0f;
        f[2] = fin ? (float)(u - x) / w : 0.0f;
        const int ti = d.tabu_inc[j], td = d.tabu_dec[j];
        const int st = ti > td ? ti : td;
        long long age = st > 0 ? iter - (long long)(st - 1 - d.tenure) : 64;
        if (age > 64) age = 64;
        f[3] = (float)age / 64.0f;
        f[4] = L.colviol[j];
        f[5] = L.colwv[j];
        f[6] = (float)L.s_last[j] / (1.0f + smax);
        f[7] = since / 50.0f;
        const int q = d.vpos[j];
        const int len = (d.ci_ptr[q + 1] - d.ci_ptr[q]) + (d.cf_ptr[q + 1] - d.cf_ptr[q]);
        f[8] = log2f(1.0f + (float)len) / 16.0f;
        const int vt = d.vtype[j];
        f[9] = vt == kVarBin ? 1.0f : 0.0f;
        f[10] = vt == kVarInt ? 1.0f : 0.0f;
        f[11] = cmax > 0.0f ? (float)d.obj[j] / cmax : 0.0f;
#pragma unroll
        for (int k = 0; k < kF; ++k) L.feat[(long long)j * kF + k] = __float2bfloat16_rn(f[k]);
    }
}

// ----------------------------------------------------------------- network

// Forward pass: one thread per row; parameters broadcast from shared memory
// (16-byte loads of the second layer's weights).
__global__ void __launch_bounds__(256) k_mlp_forward(const __nv_bfloat16 *w, const __nv_bfloat16 *x, long long n,
                                                     float *y, const int *done)
{
    if (done && *(volatile const int *)done) return;
    __shared__ __align__(16) float sw[kNParams + 3];
    for (int i = threadIdx.x; i < kNParams; i += blockDim.x) sw[i] = __bfloat162float(w[i]);
    __syncthreads();
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
        float xi[kF];
#pragma unroll
        for (int f = 0; f < kF; ++f) xi[f] = __bfloat162float(x[r * kF + f]);
        // the second layer in two halves of 32 outputs (the first layer is
        // recomputed for each half: fewer live registers, more warps per SM);
        // every pre-activation sums its terms in increasing i
        float out = sw[kOffB3];
#pragma unroll 1
        for (int h = 0; h < kH; h += 32) {
            float acc[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) acc[j] = sw[kOffB2 + h + j];
#pragma unroll 1
            for (int i = 0; i < kH; ++i) {
                float a = sw[kOffB1 + i];
#pragma unroll
                for (int f = 0; f < kF; ++f) a = __fmaf_rn(xi[f], sw[kOffW1 + f * kH + i], a);
                a = fmaxf(a, 0.0f);
#pragma unroll
                for (int j = 0; j < 32; j += 4) {
                    const float4 w4 = *reinterpret_cast<const float4 *>(&sw[kOffW2 + i * kH + h + j]);
                    acc[j] = __fmaf_rn(a, w4.x, acc[j]);
                    acc[j + 1] = __fmaf_rn(a, w4.y, acc[j + 1]);
                    acc[j + 2] = __fmaf_rn(a, w4.z, acc[j + 2]);
                    acc[j + 3] = __fmaf_rn(a, w4.w, acc[j + 3]);
                }
            }
#pragma unroll
            for (int j = 0; j < 32; ++j) out = __fmaf_rn(fmaxf(acc[j], 0.0f), sw[kOffW3 + h + j], out);
        }
        y[r] = out;
    }
}

// Forward pass with the second layer on the tensor cores: one warp per tile of
// 16 rows; every lane computes, in FP32 on the CUDA cores, exactly the
// first-layer activations its A fragments of mma.m16n8k16 need (rows g and
// g + 8 of the tile, 16 hidden units per 16-wide K chunk), rounds them to BF16,
// and the warp multiplies the 16 x 64 tile by W2 (64 x 64, BF16 from shared
// memory) into FP32 accumulators; the output layer is reduced across the four
// lanes that share a row.  Activations of the first layer are BF16 here
// (FP32 in k_mlp_forward and in training).
__global__ void __launch_bounds__(256) k_mlp_forward_tc(const __nv_bfloat16 *w, const __nv_bfloat16 *x, long long n,
                                                        float *y, const int *done)
{
    if (done && *(volatile const int *)done) return;
    __shared__ float s1[kF * kH + kH];                          // W1, b1
    __shared__ float s2[kH + kH + 1];                           // b2, w3, b3
    __shared__ __align__(16) unsigned short sW2t[kH * (kH + 8)];  // W2 transposed, [n][k], padded rows
    for (int i = threadIdx.x; i < kF * kH + kH; i += blockDim.x) s1[i] = __bfloat162float(w[kOffW1 + i]);
    for (int i = threadIdx.x; i < 2 * kH + 1; i += blockDim.x) s2[i] = __bfloat162float(w[kOffB2 + i]);
    const unsigned short *wraw = reinterpret_cast<const unsigned short *>(w);
    for (int i = threadIdx.x; i < kH * kH; i += blockDim.x) {
        const int k = i / kH, nn = i % kH;                      // W2[k][nn]
        sW2t[nn * (kH + 8) + k] = wraw[kOffW2 + i];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const long long tiles = (n + 15) / 16;
    for (long long tile = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); tile < tiles;
         tile += (long long)gridDim.x * (blockDim.x >> 5)) {
        const long long r0 = tile * 16 + g, r1 = r0 + 8;
        float x0[kF], x1[kF];
#pragma unroll
        for (int f = 0; f < kF; ++f) {
            x0[f] = r0 < n ? __bfloat162float(x[r0 * kF + f]) : 0.0f;
            x1[f] = r1 < n ? __bfloat162float(x[r1 * kF + f]) : 0.0f;
        }
        float acc[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.0f;
#pragma unroll
        for (int kc = 0; kc < 4; ++kc) {
            // A fragment: rows g / g+8, hidden units 16 kc + {2t, 2t+1, 2t+8, 2t+9}
            unsigned a[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = 16 * kc + 2 * t + (q >= 2 ? 8 : 0);
                const float *xr = (q & 1) ? x1 : x0;
                float v[2];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    float s = s1[kF * kH + c + e];
#pragma unroll
                    for (int f = 0; f < kF; ++f) s = __fmaf_rn(xr[f], s1[f * kH + c + e], s);
                    v[e] = fmaxf(s, 0.0f);
                }
                const __nv_bfloat162 pr = __floats2bfloat162_rn(v[0], v[1]);
                a[q] = *reinterpret_cast<const unsigned *>(&pr);
            }
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                // B fragment: k = 16 kc + {2t, 2t+1} and {2t+8, 2t+9}, n = 8 nt + g
                const unsigned short *bp = sW2t + (8 * nt + g) * (kH + 8) + 16 * kc + 2 * t;
                const unsigned b0 = *reinterpret_cast<const unsigned *>(bp);
                const unsigned b1 = *reinterpret_cast<const unsigned *>(bp + 8);
                asm volatile(
                    "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                    "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
                    : "+f"(acc[nt][0]), "+f"(acc[nt][1]), "+f"(acc[nt][2]), "+f"(acc[nt][3])
                    : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
            }
        }
        // output layer: rows g (acc[.][0..1]) and g + 8 (acc[.][2..3]), columns 8 nt + 2t (+1)
        float o0 = 0.0f, o1 = 0.0f;
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int c = 8 * nt + 2 * t;
            o0 = __fmaf_rn(fmaxf(acc[nt][0] + s2[c], 0.0f), s2[kH + c], o0);
            o0 = __fmaf_rn(fmaxf(acc[nt][1] + s2[c + 1], 0.0f), s2[kH + c + 1], o0);
            o1 = __fmaf_rn(fmaxf(acc[nt][2] + s2[c], 0.0f), s2[kH + c], o1);
            o1 = __fmaf_rn(fmaxf(acc[nt][3] + s2[c + 1], 0.0f), s2[kH + c + 1], o1);
        }
        o0 += __shfl_xor_sync(FULLMASK, o0, 1);
        o0 += __shfl_xor_sync(FULLMASK, o0, 2);
        o1 += __shfl_xor_sync(FULLMASK, o1, 1);
        o1 += __shfl_xor_sync(FULLMASK, o1, 2);
        if (t == 0) {
            if (r0 < n) y[r0] = o0 + s2[2 * kH];
            if (r1 < n) y[r1] = o1 + s2[2 * kH];
        }
    }
}

// Gradient of the mean squared error over n rows (scale 2/n), accumulated into
// grad[kNParams] (FP32 atomics, one per parameter and tile), and the sum of
// squared errors into loss[0].  One CTA of kGradRows threads per tile of rows.
__global__ void __launch_bounds__(kGradRows) k_mlp_grad(const __nv_bfloat16 *w, const __nv_bfloat16 *x,
                                                        const float *t, long long n, float scale, float *grad,
                                                        float *loss)
{
    extern __shared__ __align__(16) float gsm[];
    float *sw = gsm;                                  // kNParams (+3 pad)
    float *sx = sw + ((kNParams + 3) & ~3);           // kGradRows x kF
    float *h1 = sx + kGradRows * kF;                  // kGradRows x kHPad (then ga1)
    float *h2 = h1 + kGradRows * kHPad;               // kGradRows x kHPad (then ga2)
    float *gy = h2 + kGradRows * kHPad;               // kGradRows
    const int tid = threadIdx.x;
    for (int i = tid; i < kNParams; i += blockDim.x) sw[i] = __bfloat162float(w[i]);
    const long long r0 = (long long)blockIdx.x * kGradRows;
    const long long left = n - r0;
    const int rows = left < kGradRows ? (int)left : kGradRows;
    for (int i = tid; i < kGradRows * kF; i += blockDim.x) {
        const int r = i / kF;
        sx[i] = r < rows ? __bfloat162float(x[(r0 + r) * kF + (i % kF)]) : 0.0f;
    }
    __syncthreads();
    // forward, one row per thread
    float err = 0.0f;
    if (tid < rows) {
        float *a = h1 + tid * kHPad;
        for (int j = 0; j < kH; ++j) {
            float s = sw[kOffB1 + j];
            for (int f = 0; f < kF; ++f) s = __fmaf_rn(sx[tid * kF + f], sw[kOffW1 + f * kH + j], s);
            a[j] = fmaxf(s, 0.0f);
        }
        float out = sw[kOffB3];
        float *b = h2 + tid * kHPad;
        for (int j = 0; j < kH; ++j) {
            float s = sw[kOffB2 + j];
            for (int i = 0; i < kH; ++i) s = __fmaf_rn(a[i], sw[kOffW2 + i * kH + j], s);
            b[j] = fmaxf(s, 0.0f);
            out = __fmaf_rn(b[j], sw[kOffW3 + j], out);
        }
        err = out - t[r0 + tid];
        gy[tid] = scale * err;
    } else {
        gy[tid] = 0.0f;
        for (int j = 0; j < kH; ++j) { h1[tid * kHPad + j] = 0.0f; h2[tid * kHPad + j] = 0.0f; }
    }
    __syncthreads();
    // output layer
    if (tid < kH) {
        float s = 0.0f;
        for (int r = 0; r < kGradRows; ++r) s = __fmaf_rn(h2[r * kHPad + tid], gy[r], s);
        atomicAdd(grad + kOffW3 + tid, s);
    }
    if (tid == kH) {
        float s = 0.0f;
        for (int r = 0; r < kGradRows; ++r) s += gy[r];
        atomicAdd(grad + kOffB3, s);
    }
    __syncthreads();
    // ga2 = gy w3 [h2 > 0], in place of h2
    for (int j = 0; j < kH; ++j) {
        float &v = h2[tid * kHPad + j];
        v = v > 0.0f ? gy[tid] * sw[kOffW3 + j] : 0.0f;
    }
    __syncthreads();
    // gW2[i][j] = sum_r h1[r][i] ga2[r][j]; gb2[j] = sum_r ga2[r][j]
    for (int o = tid; o < kH * kH; o += blockDim.x) {
        const int i = o / kH, j = o % kH;
        float s = 0.0f;
        for (int r = 0; r < kGradRows; ++r) s = __fmaf_rn(h1[r * kHPad + i], h2[r * kHPad + j], s);
        atomicAdd(grad + kOffW2 + o, s);
    }
    if (tid < kH) {
        float s = 0.0f;
        for (int r = 0; r < kGradRows; ++r) s += h2[r * kHPad + tid];
        atomicAdd(grad + kOffB2 + tid, s);
    }
    __syncthreads();
    // ga1 = (ga2 W2^T) [h1 > 0], in place of h1 (each thread its own row)
    {
        float g1[kH];
        for (int i = 0; i < kH; ++i) {
            float s = 0.0f;
            for (int j = 0; j < kH; ++j) s = __fmaf_rn(h2[tid * kHPad + j], sw[kOffW2 + i * kH + j], s);
            g1[i] = h1[tid * kHPad + i] > 0.0f ? s : 0.0f;
        }
        for (int i = 0; i < kH; ++i) h1[tid * kHPad + i] = g1[i];
    }
    __syncthreads();
    for (int o = tid; o < kF * kH; o += blockDim.x) {
        const int f = o / kH, i = o % kH;
        float s = 0.0f;
        for (int r = 0; r < kGradRows; ++r) s = __fmaf_rn(sx[r * kF + f], h1[r * kHPad + i], s);
        atomicAdd(grad + kOffW1 + o, s);
    }
    if (tid < kH) {
        float s = 0.0f;
        for (int r = 0; r < kGradRows; ++r) s += h1[r * kHPad + tid];
        atomicAdd(grad + kOffB1 + tid, s);
    }
    // loss
    float e2 = err * err;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e2 += __shfl_xor_sync(FULLMASK, e2, o);
    if ((tid & 31) == 0) atomicAdd(loss, e2);
}

// Adam on FP32 master parameters; writes the BF16 copy and clears the gradient.
__global__ void k_adam(float *w32, __nv_bfloat16 *wbf, float *m, float *v, float *g, int n, float lr, float b1,
                       float b2, float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w32[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w32[i] = wi;
    wbf[i] = __float2bfloat16_rn(wi);
    g[i] = 0.0f;
}

// ------------------------------------------------------------------- top-k

__device__ __forceinline__ unsigned fkey(float v)
{
    const unsigned b = __float_as_uint(v);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// Histogram of one digit of the keys that match the digits fixed so far.
// level 0: bits 31..21, level 1: bits 20..10, level 2: bits 9..0.
__global__ void k_topk_hist(Dev d, Learn L, const float *y, int n, int level, int gate)
{
    if (gate && done_gate(d)) return;
    __shared__ unsigned h[2048];
    for (int i = threadIdx.x; i < 2048; i += blockDim.x) h[i] = 0u;
    __syncthreads();
    const unsigned prefix = L.lc->prefix;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const unsigned k = fkey(y[j]);
        bool match;
        unsigned dig;
        if (level == 0) { match = true; dig = k >> 21; }
        else if (level == 1) { match = (k >> 21) == (prefix >> 21); dig = (k >> 10) & 0x7ffu; }
        else { match = (k >> 10) == (prefix >> 10); dig = k & 0x3ffu; }
        if (match) atomicAdd(&h[dig], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 2048; i += blockDim.x)
        if (h[i]) atomicAdd(&L.hist[i], h[i]);
}

// Fix the digit of this level: the largest digit whose count from the top
// reaches the elements still needed (a block-wide suffix scan of the 2048
// bins); clears the histogram for the next level.
__global__ void __launch_bounds__(256) k_topk_pick(Dev d, Learn L, int level, int k, int n, int gate)
{
    if (gate && done_gate(d)) return;
    constexpr int PER = 2048 / 256;
    __shared__ int wsum[8];
    __shared__ int s_dig, s_need;
    LearnCtl *c = L.lc;
    const int need0 = level == 0 ? min(k, n) : c->need;
    const int nb = level == 2 ? 1024 : 2048;
    // thread t owns bins [2048 - (t+1) PER, 2048 - t PER): higher bins first
    const int hi = 2048 - threadIdx.x * PER;
    int cnt[PER];
    int tot = 0;
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int b = hi - 1 - u;
        cnt[u] = b < nb ? (int)L.hist[b] : 0;
        tot += cnt[u];
    }
    // exclusive prefix of the per-thread totals in thread order (= from the top)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(FULLMASK, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[wid] = incl;
    if (threadIdx.x == 0) { s_dig = 0; s_need = need0; }
    __syncthreads();
    int before = incl - tot;
    for (int w = 0; w < wid; ++w) before += wsum[w];
    // the thread whose range contains the need0-th element from the top fixes the digit
    if (before < need0 && before + tot >= need0) {
        int acc = before;
        for (int u = 0; u < PER; ++u) {
            if (acc + cnt[u] >= need0) { s_dig = hi - 1 - u; s_need = need0 - acc; break; }
            acc += cnt[u];
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int dig = s_dig;
        c->need = s_need;
        const unsigned p = level == 0 ? ((unsigned)dig << 21) : level == 1 ? (c->prefix | ((unsigned)dig << 10))
                                                                           : (c->prefix | (unsigned)dig);
        c->prefix = p;
        if (level == 2) c->thr = p;
    }
    for (int i = threadIdx.x; i < 2048; i += blockDim.x) L.hist[i] = 0u;
}

__global__ void __launch_bounds__(256) k_topk_count(Dev d, Learn L, const float *y, int n, int gate)
{
    if (gate && done_gate(d)) return;
    const unsigned thr = L.lc->thr;
    int gt = 0, eq = 0;
    const int base = blockIdx.x * kTopkBlock + threadIdx.x * kTopkPerThread;
    for (int u = 0; u < kTopkPerThread; ++u) {
        const int j = base + u;
        if (j < n) {
            const unsigned k = fkey(y[j]);
            gt += k > thr;
            eq += k == thr;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        gt += __shfl_xor_sync(FULLMASK, gt, o);
        eq += __shfl_xor_sync(FULLMASK, eq, o);
    }
    __shared__ int sg[8], se[8];
    if ((threadIdx.x & 31) == 0) { sg[threadIdx.x >> 5] = gt; se[threadIdx.x >> 5] = eq; }
    __syncthreads();
    if (threadIdx.x == 0) {
        int a = 0, b = 0;
        for (int w = 0; w < 8; ++w) { a += sg[w]; b += se[w]; }
        L.bcnt[2 * blockIdx.x] = a;
        L.bcnt[2 * blockIdx.x + 1] = b;
    }
}

__global__ void k_topk_scan(Dev d, Learn L, int gate)
{
    if (gate && done_gate(d)) return;
    if (threadIdx.x != 0) return;
    int a = 0, b = 0;
    for (int i = 0; i < L.nblocks; ++i) {
        L.bpre[2 * i] = a;
        L.bpre[2 * i + 1] = b;
        a += L.bcnt[2 * i];
        b += L.bcnt[2 * i + 1];
    }
    L.lc->total_gt = a;
}

// Stable compaction: every key above the threshold, then the first `need`
// keys equal to it in index order.
__global__ void __launch_bounds__(256) k_topk_write(Dev d, Learn L, const float *y, int n, int gate)
{
    if (gate && done_gate(d)) return;
    const unsigned thr = L.lc->thr;
    const int need = L.lc->need, total_gt = L.lc->total_gt;
    const int base = blockIdx.x * kTopkBlock + threadIdx.x * kTopkPerThread;
    unsigned kk[kTopkPerThread];
    int gt = 0, eq = 0;
    for (int u = 0; u < kTopkPerThread; ++u) {
        const int j = base + u;
        kk[u] = j < n ? fkey(y[j]) : 0u;
        gt += j < n && kk[u] > thr;
        eq += j < n && kk[u] == thr;
    }
    // block exclusive scan of (gt, eq) in thread order
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int sgt = gt, seq = eq;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int a = __shfl_up_sync(FULLMASK, sgt, o), b = __shfl_up_sync(FULLMASK, seq, o);
        if (lane >= o) { sgt += a; seq += b; }
    }
    __shared__ int wg[8], we[8];
    if (lane == 31) { wg[wid] = sgt; we[wid] = seq; }
    __syncthreads();
    int og = 0, oe = 0;
    for (int w = 0; w < wid; ++w) { og += wg[w]; oe += we[w]; }
    int pg = L.bpre[2 * blockIdx.x] + og + sgt - gt;
    int pe = L.bpre[2 * blockIdx.x + 1] + oe + seq - eq;
    for (int u = 0; u < kTopkPerThread; ++u) {
        const int j = base + u;
        if (j >= n) break;
        if (kk[u] > thr) L.list[pg++] = j;
        else if (kk[u] == thr) {
            if (pe < need) L.list[total_gt + pe] = j;
            ++pe;
        }
    }
}

// ------------------------------------------------ exact scores of the subset

__device__ __forceinline__ int lflip_f(bool v0, bool v1, bool dec)
{
    return 2 * ((int)v0 - (int)v1) + ((v0 && v1) ? (dec ? 1 : -1) : 0);
}

__device__ __forceinline__ unsigned long long dkey_bits(long long b)
{
    const unsigned long long u = (unsigned long long)b;
    return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}

__device__ __forceinline__ long long flip_sign(long long b)
{
    long long r;
    asm("xor.b64 %0, %1, 0x8000000000000000;" : "=l"(r) : "l"(b));
    return r;
}

// Flip score of every listed binary variable (8 lanes per variable, as the
// exact binary kernel); the best admissible positive flip is folded into
// lc->key with one 64-bit atomicMax (larger score, then lower variable).
__global__ void __launch_bounds__(256) k_subset_eval(Dev d, Learn L, int k, int gate)
{
    if (gate && done_gate(d)) return;
    const int lane = threadIdx.x & 31, g = lane >> 3, sub = lane & 7;
    const long long iter = d.ctl->iter, nviol = d.ctl->nviol, bestnv = d.ctl->best_nviol;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int base = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 4; base < k; base += nwarps * 4) {
        const int idx = base + g;
        const int jl = idx < k ? L.list[idx] : 0;
        const bool live = idx < k && d.vtype[jl] == kVarBin;   // other columns: k_subset_eval_nb
        const int j = live ? jl : 0;
        const int q = d.vpos[j];
        const bool up = __double_as_longlong(d.x[j]) == 0;
        long long s = 0;
        int dc = 0;
        // integral rows
        {
            const int e0 = d.ci_ptr[q], e1 = live ? d.ci_ptr[q + 1] : e0;
            int len = e1 - e0, lmax = len;
#pragma unroll
            for (int o = 16; o >= 8; o >>= 1) lmax = max(lmax, __shfl_xor_sync(FULLMASK, lmax, o));
            for (int v0 = 0; v0 < lmax; v0 += 8) {
                const int v = v0 + sub;
                if (v < len) {
                    const int e = e0 + v;
                    const int4 st = __ldg(reinterpret_cast<const int4 *>(d.rs + d.ci_row[e]));
                    const long long r = i4_r(st);
                    const int ad = up ? d.ci_val[e] : -d.ci_val[e];
                    const long long r1 = r + ad;
                    s += (long long)lflip_f(r > 0, r1 > 0, ad < 0) * st.z;
                    dc += (int)(r1 > 0) - (int)(r > 0);
                    if (st.w >= 0) {
                        s += (long long)lflip_f(r < 0, r1 < 0, ad > 0) * st.w;
                        dc += (int)(r1 < 0) - (int)(r < 0);
                    }
                }
            }
        }
        // other rows: violated <=> m < 0; violated after the move <=> change > m
        {
            const int e0 = d.cf_ptr[q], e1 = live ? d.cf_ptr[q + 1] : e0;
            int len = e1 - e0, lmax = len;
#pragma unroll
            for (int o = 16; o >= 8; o >>= 1) lmax = max(lmax, __shfl_xor_sync(FULLMASK, lmax, o));
            for (int v0 = 0; v0 < lmax; v0 += 8) {
                const int v = v0 + sub;
                if (v < len) {
                    const int e = e0 + v;
                    const RowState st = d.rs[d.cf_row[e]];
                    const long long ab = __double_as_longlong(d.cf_val[e]);
                    const long long ad = up ? ab : flip_sign(ab);
                    const long long m1 = __double_as_longlong(st.m1), m2 = __double_as_longlong(st.m2);
                    const bool neg = ad < 0;
                    const bool v0b = m1 < 0, v1b = dkey_bits(ad) > dkey_bits(m1);
                    s += (long long)lflip_f(v0b, v1b, neg) * st.w1;
                    dc += (int)v1b - (int)v0b;
                    if (st.w2 >= 0) {
                        const bool u0 = m2 < 0, u1 = dkey_bits(flip_sign(ad)) > dkey_bits(m2);
                        s += (long long)lflip_f(u0, u1, !neg) * st.w2;
                        dc += (int)u1 - (int)u0;
                    }
                }
            }
        }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
            s += __shfl_xor_sync(FULLMASK, s, o);
            dc += __shfl_xor_sync(FULLMASK, dc, o);
        }
        if (sub == 0 && live && s > 0) {
            const int stamp = up ? d.tabu_inc[j] : d.tabu_dec[j];
            if (iter >= (long long)stamp || nviol + (long long)dc < bestnv) {
                const unsigned long long key =
                    ((unsigned long long)s << kVarBits) | (unsigned long long)((1 << kVarBits) - 1 - j);
                atomicMax(&L.lc->key, key);
            }
        }
    }
}

// Hand the proposal's move to the apply kernel of the exact path.
__global__ void k_learn_select(Dev d, Learn L, int gate)
{
    if (gate && done_gate(d)) return;
    Ctl *c = d.ctl;
    const unsigned long long key = L.lc->key;
    L.lc->key = 0ull;
    if (key != 0ull) {
        const int j = (1 << kVarBits) - 1 - (int)(key & ((1ull << kVarBits) - 1));
        const double x = d.x[j];
        c->mv_var = j;
        c->mv_s = (long long)(key >> kVarBits);
        c->mv_dc = 0;
        c->mv_old = x;
        c->mv_new = d.vtype[j] == kVarBin ? (__double_as_longlong(x) == 0 ? 1.0 : 0.0) : L.xh[j];
    } else {
        c->mv_var = -1;
        c->mv_s = 0;
        c->mv_dc = 0;
        c->mv_new = 0.0;
        c->mv_old = 0.0;
    }
}

// At an exact pass: the proposal misses when the exact best score exceeds the
// best score found in the proposed subset.
__global__ void k_learn_miss(Dev d, Learn L, int gate)
{
    if (gate && done_gate(d)) return;
    const unsigned long long key = L.lc->key;
    L.lc->key = 0ull;
    const long long ls = key ? (long long)(key >> kVarBits) : 0;
    const Ctl *c = d.ctl;
    L.lc->passes += 1;
    if (c->mv_var >= 0 && c->mv_s > ls) L.lc->misses += 1;
}

}  // namespace
}  // namespace chap

// ------------------------------------------------------------------ host

namespace chap {

struct LearnHost {
    Learn L{};
    std::vector<void *> allocs;
    cudaGraphExec_t gexec = nullptr;
    int g_key[4] = {0, 0, 0, 0};   // topk, exact_every, propose_every, graph weights pointer (low bits)
    const void *g_w = nullptr;
    LearnCtl *h_lc = nullptr;      // pinned
    float cmax = 0.0f;
};

void learn_free(chap_bs *h)
{
    if (!h || !h->learn) return;
    LearnHost *lh = static_cast<LearnHost *>(h->learn);
    if (lh->gexec) cudaGraphExecDestroy(lh->gexec);
    for (void *p : lh->allocs) cudaFree(p);
    if (lh->h_lc) cudaFreeHost(lh->h_lc);
    delete lh;
    h->learn = nullptr;
}

namespace {

template <class T>
T *lalloc(LearnHost *lh, size_t count)
{
    void *p = nullptr;
    if (cudaMalloc(&p, sizeof(T) * std::max<size_t>(count, 1)) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    lh->allocs.push_back(p);
    return static_cast<T *>(p);
}

chap_status lfail(chap_bs *h, chap_status s, const std::string &msg)
{
    h->err = msg;
    return s;
}

#define LCK(h, expr, what)                                                                   \
    do {                                                                                     \
        cudaError_t e_ = (expr);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            cudaGetLastError();                                                              \
            return lfail(h, CHAP_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e_)); \
        }                                                                                    \
    } while (0)

// Learned-driver state of the handle, created on first use.
chap_status ensure_learn(chap_bs *h, LearnHost **out)
{
    if (h->learn) {
        *out = static_cast<LearnHost *>(h->learn);
        return CHAP_OK;
    }
    LearnHost *lh = new (std::nothrow) LearnHost();
    if (!lh) return CHAP_E_OOM;
    const int n = h->n;
    Learn &L = lh->L;
    L.nblocks = (n + kTopkBlock - 1) / kTopkBlock;
    L.colviol = lalloc<float>(lh, n);
    L.colwv = lalloc<float>(lh, n);
    L.s_last = lalloc<long long>(lh, n);
    L.feat = lalloc<__nv_bfloat16>(lh, (size_t)n * kF);
    L.y = lalloc<float>(lh, n);
    L.hist = lalloc<unsigned>(lh, 2048);
    L.bcnt = lalloc<int>(lh, 2 * (size_t)std::max(1, L.nblocks));
    L.bpre = lalloc<int>(lh, 2 * (size_t)std::max(1, L.nblocks));
    L.list = lalloc<int>(lh, n);
    L.xh = lalloc<double>(lh, n);
    L.lc = lalloc<LearnCtl>(lh, 1);
    bool ok = L.colviol && L.colwv && L.s_last && L.feat && L.y && L.hist && L.bcnt && L.bpre && L.list && L.xh && L.lc &&
              cudaMallocHost(&lh->h_lc, sizeof(LearnCtl)) == cudaSuccess;
    cudaError_t e = cudaSuccess;
    if (ok) {
        e = cudaMemsetAsync(L.colviol, 0, sizeof(float) * std::max(1, n), h->st);
        if (e == cudaSuccess) e = cudaMemsetAsync(L.colwv, 0, sizeof(float) * std::max(1, n), h->st);
        if (e == cudaSuccess) e = cudaMemsetAsync(L.s_last, 0, sizeof(long long) * std::max(1, n), h->st);
        if (e == cudaSuccess) e = cudaMemsetAsync(L.hist, 0, sizeof(unsigned) * 2048, h->st);
        if (e == cudaSuccess) e = cudaMemsetAsync(L.lc, 0, sizeof(LearnCtl), h->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    }
    if (!ok || e != cudaSuccess) {
        cudaGetLastError();
        h->learn = lh;
        learn_free(h);
        return ok ? CHAP_E_CUDA : CHAP_E_OOM;
    }
    for (int j = 0; j < n; ++j) lh->cmax = std::max(lh->cmax, (float)std::fabs(h->obj[j]));
    h->learn = lh;
    *out = lh;
    return CHAP_OK;
}

int grid_n(long long n, int threads, int cap = 152 * 8)
{
    long long g = (n + threads - 1) / threads;
    return (int)std::max<long long>(1, std::min<long long>(g, cap));
}

// exact scores into s_last and the pass-time column features
cudaError_t launch_refresh(chap_bs *h, LearnHost *lh, int gate, cudaStream_t st)
{
    const Dev &d = h->dev;
    VarOut o{nullptr, lh->L.s_last, nullptr};
    cudaError_t e = launch_eval_gated(d, h->plan, o, gate, st);
    if (e == cudaSuccess) e = launch_select_gated(d, h->plan, gate, st);
    if (e != cudaSuccess) return e;
    k_refresh_begin<<<1, 1, 0, st>>>(d, lh->L, gate);
    // the refresh reads the state before the move; gated like the rest
    if (!gate) k_refresh<<<grid_n(d.n, 256), 256, 0, st>>>(d, lh->L);
    else k_refresh<<<grid_n(d.n, 256), 256, 0, st>>>(d, lh->L);
    return cudaGetLastError();
}

cudaError_t launch_propose(chap_bs *h, LearnHost *lh, const __nv_bfloat16 *w, int k, int gate, cudaStream_t st)
{
    const Dev &d = h->dev;
    const Learn &L = lh->L;
    const int n = d.n;
    k_features<<<grid_n(n, 256), 256, 0, st>>>(d, L, lh->cmax, gate);
    k_mlp_forward_tc<<<grid_n((n + 15) / 16 * 32, 256, 152 * 4), 256, 0, st>>>(w, L.feat, n, L.y,
                                                                             gate ? &d.ctl->done : nullptr);
    for (int level = 0; level < 3; ++level) {
        k_topk_hist<<<grid_n(n, 256, 152 * 2), 256, 0, st>>>(d, L, L.y, n, level, gate);
        k_topk_pick<<<1, 256, 0, st>>>(d, L, level, k, n, gate);
    }
    k_topk_count<<<std::max(1, L.nblocks), 256, 0, st>>>(d, L, L.y, n, gate);
    k_topk_scan<<<1, 32, 0, st>>>(d, L, gate);
    k_topk_write<<<std::max(1, L.nblocks), 256, 0, st>>>(d, L, L.y, n, gate);
    return cudaGetLastError();
}

cudaError_t launch_subset(chap_bs *h, LearnHost *lh, int k, int gate, cudaStream_t st)
{
    if (h->info.n_bin > 0) k_subset_eval<<<grid_n((long long)k * 8, 256, 152 * 4), 256, 0, st>>>(h->dev, lh->L, k, gate);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && h->info.n_bin < h->n - h->info.n_fixed)
        e = launch_subset_nb(h->dev, h->plan, lh->L.list, k, lh->L.xh, &lh->L.lc->key, gate, st);
    return e;
}

}  // namespace
}  // namespace chap

using namespace chap;

extern "C" {

chap_status chap_bs_refresh_features(chap_bs *h)
{
    if (!h) return CHAP_E_INVALID;
    if (h->broken) return lfail(h, CHAP_E_STATE, "handle unusable after a CUDA fault");
    if (own_scratch_ok(h) != CHAP_OK || whole_instance_ok(h) != CHAP_OK) return CHAP_E_STATE;
    LearnHost *lh = nullptr;
    chap_status s = ensure_learn(h, &lh);
    if (s != CHAP_OK) return lfail(h, s, "learned-driver state");
    LCK(h, launch_refresh(h, lh, 0, h->st), "refresh");
    LCK(h, cudaStreamSynchronize(h->st), "synchronise");
    return CHAP_OK;
}

chap_status chap_bs_features(chap_bs *h, uint16_t *feat, float *target)
{
    if (!h) return CHAP_E_INVALID;
    if (h->broken) return lfail(h, CHAP_E_STATE, "handle unusable after a CUDA fault");
    LearnHost *lh = nullptr;
    chap_status s = ensure_learn(h, &lh);
    if (s != CHAP_OK) return lfail(h, s, "learned-driver state");
    k_features<<<grid_n(h->n, 256), 256, 0, h->st>>>(h->dev, lh->L, lh->cmax, 0);
    LCK(h, cudaGetLastError(), "features");
    if (feat && h->n)
        LCK(h, cudaMemcpyAsync(feat, lh->L.feat, sizeof(uint16_t) * kF * (size_t)h->n, cudaMemcpyDeviceToDevice, h->st),
            "copy features");
    if (target && h->n) {
        // targets: the last exact scores scaled by 1 / (1 + max |score|)
        LCK(h, cudaMemcpyAsync(lh->h_lc, lh->L.lc, sizeof(LearnCtl), cudaMemcpyDeviceToHost, h->st), "read state");
        LCK(h, cudaStreamSynchronize(h->st), "synchronise");
        std::vector<long long> sl(h->n);
        LCK(h, cudaMemcpy(sl.data(), lh->L.s_last, sizeof(long long) * h->n, cudaMemcpyDeviceToHost), "copy scores");
        std::vector<float> t(h->n);
        const double sc = 1.0 / (1.0 + (double)lh->h_lc->smax);
        for (int j = 0; j < h->n; ++j) t[j] = (float)((double)sl[j] * sc);
        LCK(h, cudaMemcpy(target, t.data(), sizeof(float) * h->n, cudaMemcpyHostToDevice), "copy targets");
    }
    LCK(h, cudaStreamSynchronize(h->st), "synchronise");
    return CHAP_OK;
}

chap_status chap_bs_propose(chap_bs *h, const uint16_t *weights, int32_t k, int32_t *list, float *pred)
{
    if (!h || !weights || k < 1) return h ? lfail(h, CHAP_E_INVALID, "bad proposal arguments") : CHAP_E_INVALID;
    if (h->broken) return lfail(h, CHAP_E_STATE, "handle unusable after a CUDA fault");
    LearnHost *lh = nullptr;
    chap_status s = ensure_learn(h, &lh);
    if (s != CHAP_OK) return lfail(h, s, "learned-driver state");
    k = std::min(k, h->n);
    LCK(h, launch_propose(h, lh, reinterpret_cast<const __nv_bfloat16 *>(weights), k, 0, h->st), "proposal");
    if (list) LCK(h, cudaMemcpyAsync(list, lh->L.list, sizeof(int) * k, cudaMemcpyDeviceToDevice, h->st), "copy list");
    if (pred) LCK(h, cudaMemcpyAsync(pred, lh->L.y, sizeof(float) * h->n, cudaMemcpyDeviceToDevice, h->st), "copy predictions");
    LCK(h, cudaStreamSynchronize(h->st), "synchronise");
    return CHAP_OK;
}

chap_status chap_learned_run(chap_bs *h, const uint16_t *weights, const chap_learned_options *lo,
                             chap_learned_result *res)
{
    if (!h || !weights || !lo || !res) return h ? lfail(h, CHAP_E_INVALID, "NULL argument") : CHAP_E_INVALID;
    if (h->broken) return lfail(h, CHAP_E_STATE, "handle unusable after a CUDA fault");
    if (lo->topk < 1 || lo->exact_every < 1 || lo->propose_every < 1 || lo->max_iters < 0)
        return lfail(h, CHAP_E_INVALID, "bad learned-run options");
    if (own_scratch_ok(h) != CHAP_OK || whole_instance_ok(h) != CHAP_OK) return CHAP_E_STATE;
    if (h->n >= (1 << kVarBits))
        return lfail(h, CHAP_E_UNSUPPORTED, "the learned driver handles instances below 2^22 variables");
    LearnHost *lh = nullptr;
    chap_status s = ensure_learn(h, &lh);
    if (s != CHAP_OK) return lfail(h, s, "learned-driver state");
    const int k = std::min<int>(lo->topk, h->n);
    const auto t0 = std::chrono::steady_clock::now();
    LCK(h, cudaMemcpyAsync(h->h_ctl, h->dev.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->st), "read control");
    LCK(h, cudaStreamSynchronize(h->st), "synchronise");
    const long long iter0 = h->h_ctl->iter, moves0 = h->h_ctl->moves;
    if (iter0 + lo->max_iters + h->opt.tenure + 1 >= (long long)INT_MAX)
        return lfail(h, CHAP_E_UNSUPPORTED, "iteration counter would exceed the 32-bit tabu stamps");
    LCK(h, cudaMemsetAsync(&lh->L.lc->passes, 0, 2 * sizeof(long long), h->st), "reset counters");
    LCK(h, launch_begin_run(h->dev, lo->max_iters, lo->stop_at_feasible, h->st), "begin run");
    const __nv_bfloat16 *w = reinterpret_cast<const __nv_bfloat16 *>(weights);
    const int key[4] = {k, lo->exact_every, lo->propose_every, 0};
    if (!lh->gexec || lh->g_w != weights || !std::equal(key, key + 3, lh->g_key)) {
        if (lh->gexec) { cudaGraphExecDestroy(lh->gexec); lh->gexec = nullptr; }
        cudaGraph_t g = nullptr;
        cudaStream_t cs = h->cap_st;
        LCK(h, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "begin capture");
        cudaError_t e = cudaSuccess;
        // one block: the exact iteration, then exact_every - 1 proposal iterations
        e = launch_propose(h, lh, w, k, 1, cs);
        if (e == cudaSuccess) e = launch_subset(h, lh, k, 1, cs);
        if (e == cudaSuccess) e = launch_refresh(h, lh, 1, cs);
        if (e == cudaSuccess) { k_learn_miss<<<1, 1, 0, cs>>>(h->dev, lh->L, 1); e = cudaGetLastError(); }
        if (e == cudaSuccess) e = launch_apply_gated(h->dev, h->plan, 1, cs);
        for (int i = 1; i < lo->exact_every && e == cudaSuccess; ++i) {
            if (i % lo->propose_every == 0) e = launch_propose(h, lh, w, k, 1, cs);
            if (e == cudaSuccess) e = launch_subset(h, lh, k, 1, cs);
            if (e == cudaSuccess) { k_learn_select<<<1, 1, 0, cs>>>(h->dev, lh->L, 1); e = cudaGetLastError(); }
            if (e == cudaSuccess) e = launch_apply_gated(h->dev, h->plan, 1, cs);
        }
        cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); LCK(h, e, "capture"); }
        LCK(h, e2, "end capture");
        cudaError_t e3 = cudaGraphInstantiate(&lh->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e3 != cudaSuccess) { lh->gexec = nullptr; LCK(h, e3, "instantiate graph"); }
        std::copy(key, key + 3, lh->g_key);
        lh->g_w = weights;
    }
    const long long max_replays = lo->max_iters / lo->exact_every + 2;
    for (long long r = 0; r < max_replays; ++r) {
        LCK(h, cudaGraphLaunch(lh->gexec, h->st), "graph launch");
        LCK(h, cudaMemcpyAsync(h->h_ctl, h->dev.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->st), "read control");
        LCK(h, cudaStreamSynchronize(h->st), "synchronise");
        if (h->h_ctl->done) break;
    }
    const auto t1 = std::chrono::steady_clock::now();
    LCK(h, cudaMemcpyAsync(lh->h_lc, lh->L.lc, sizeof(LearnCtl), cudaMemcpyDeviceToHost, h->st), "read state");
    LCK(h, cudaStreamSynchronize(h->st), "synchronise");
    const Ctl c = *h->h_ctl;
    res->iters = c.iter - iter0;
    res->moves = c.moves - moves0;
    res->feasible_iter = c.feasible_iter;
    res->final_nviol = c.nviol;
    res->best_nviol = c.best_nviol;
    res->seconds = std::chrono::duration<double>(t1 - t0).count();
    res->time_to_feasible_s = c.feasible_iter >= 0 ? (double)(c.t_feas_ns - c.t_start_ns) * 1e-9 : -1.0;
    res->exact_passes = lh->h_lc->passes;
    res->misses = lh->h_lc->misses;
    return CHAP_OK;
}

chap_status chap_mlp_forward(const uint16_t *weights, const uint16_t *x, int64_t n, float *y, void *stream)
{
    if (!weights || !x || !y || n < 0) return CHAP_E_INVALID;
    if (n == 0) return CHAP_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_mlp_forward<<<grid_n(n, 256, 152 * 4), 256, 0, st>>>(reinterpret_cast<const __nv_bfloat16 *>(weights),
                                                           reinterpret_cast<const __nv_bfloat16 *>(x), n, y, nullptr);
    return cudaGetLastError() == cudaSuccess ? CHAP_OK : CHAP_E_CUDA;
}

chap_status chap_mlp_loss_grad(const uint16_t *weights, const uint16_t *x, const float *target, int64_t n, float *grad,
                               float *loss, void *stream)
{
    if (!weights || !x || !target || !grad || !loss || n < 1) return CHAP_E_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int smem = (int)sizeof(float) * (((kNParams + 3) & ~3) + kGradRows * kF + 2 * kGradRows * kHPad + kGradRows);
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) {
            cudaGetLastError();
            return CHAP_E_CUDA;
        }
        attr = true;
    }
    const long long tiles = (n + kGradRows - 1) / kGradRows;
    k_mlp_grad<<<(unsigned)tiles, kGradRows, smem, st>>>(reinterpret_cast<const __nv_bfloat16 *>(weights),
                                                         reinterpret_cast<const __nv_bfloat16 *>(x), target, n,
                                                         2.0f / (float)n, grad, loss);
    return cudaGetLastError() == cudaSuccess ? CHAP_OK : CHAP_E_CUDA;
}

chap_status chap_mlp_adam(float *w32, uint16_t *wbf, float *m, float *v, float *grad, int32_t step, float lr,
                          void *stream)
{
    if (!w32 || !wbf || !m || !v || !grad || step < 1 || !(lr > 0.0f)) return CHAP_E_INVALID;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - std::pow(b1, (float)step), c2 = 1.0f - std::pow(b2, (float)step);
    k_adam<<<(kNParams + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        w32, reinterpret_cast<__nv_bfloat16 *>(wbf), m, v, grad, kNParams, lr, b1, b2, 1e-8f, c1, c2);
    return cudaGetLastError() == cudaSuccess ? CHAP_OK : CHAP_E_CUDA;
}

}  // extern "C"
