// boundary.cu -- the exact top-k of Alg. 6 (lines 19-23) of arXiv 2412.03301 over
// the refine's candidates: the k smallest (Hausdorff distance of Def. 4, id), with
// the distance decided in FP32 and, where FP32 cannot order two candidates, in FP64.
//
// Every refine form leaves, per candidate, a value whose distance to the true
// Hausdorff value H has a stated bound, so each candidate gets an interval
// [lo, hi] that holds H (bounds below; every step rounds outward):
//   FP32 forms: the pair that attains the FP32 GEMM-form value (|q|^2 + |v|^2 -
//     2 q.v), re-scored directly as r = |q - v|.  The GEMM form's squared distance
//     is off by at most D = (d + 8) 2^-23 (N_Q + N_V)^2 (N = largest norm), so the
//     GEMM-form Hausdorff value is within D of H^2 and r^2 within 2D of it:
//     lo = sqrt(r^2 - 2D) (1 - eta_d), hi = sqrt(r^2 + 2D) (1 + 2 eta_d).
//   (The FP8 form by default replaces e by a stated tolerance, below: its rigorous
//   band would hold nearly every candidate.)
//   BF16 / FP8 forms: the GEMM-form Hausdorff value h of the rounded copies, packed
//     into the pair record by the refine.  Rounding moves a vector x by e_x = |x - x'|
//     and every pair distance by at most e_q + e_v (triangle inequality), so the
//     Hausdorff value of the rounded sets is within e = max e_q + max e_v of H
//     (max and min are 1-Lipschitz), and h is within D of that value squared:
//     lo = sqrt(h - D) - e, hi = sqrt(h + D) + e.
//   eta_d = (d + 4) 2^-24 bounds the relative error of a direct FP32 distance summed
//     in one chain over d dimensions (the re-scored pairs, norms, rounding errors).
//   eta = (40 + ceil(d / 32)) 2^-24 bounds that of this stage's own FP32 distances:
//     each lane sums at most ceil(d / 32) squared differences (each within 2u of
//     (q - v)^2) and a 5-level shuffle tree adds the lanes' sums (the CTA-tile form
//     for d > 1024 sums 32 dimensions per chunk and then the chunks); the square
//     root halves the relative error and adds u (u = 2^-24).
// k_boundary, one CTA per query set (k' = min(k, candidates)):
//   1. tau = the k'-th smallest hi; the band B = {lo <= tau} holds every candidate
//      that can be among the k' nearest;
//   2. the direct FP32 Hausdorff value H32 of every member of B over all pairs, one
//      warp per member (lanes over the dimensions, the query set staged in shared
//      memory, coalesced 16-byte row loads, shuffle sums);
//   3. S = the members whose interval H32 (1 +- eta) reaches the k'-th smallest H32,
//      sorted by (H32, id); neighbours in S whose intervals overlap at or above rank
//      k' are re-scored in FP64 the same way (one warp each);
//   4. S ordered by (value, id); the first k' are the result.
// Members of B get their exact FP32 (or FP64) value as their candidate distance;
// the others keep the refine's value.  Returned distances are within eta (relative)
// of the FP64 Hausdorff value, or are its FP32 rounding where FP64 decided.
// S is held in shared memory with room for max(256, 4 k) candidates; more near-ties
// than that at the k-th set a device status bit.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <math.h>

#include "block_util.cuh"
#include "bvss_internal.cuh"
#include "ptx_util.cuh"

namespace bvss {

namespace {

constexpr int kBT = 256;          // threads of the boundary kernel
constexpr int kBW = kBT / 32;     // its warps
constexpr int kTile = 32;         // CTA-tile form: query vectors x rows per pair tile
constexpr int kTP = kTile + 1;    // padded smem row
constexpr int kMaxS = 4096;       // candidates that may tie with the k-th (sorted in smem)
constexpr int kWarpMaxD = 1024;   // warp form up to this dimension (8 float4 per lane)
constexpr int kHausSmem = 2 * kTile * kTP + BVSS_MAX_QSET + kTile + 2;   // CTA-tile T's

__device__ __forceinline__ float inf_f() { return __int_as_float(0x7f800000); }

// shared-memory minimum / maximum of non-negative values through their bit patterns
__device__ __forceinline__ void smem_min(float *p, float v) {
    atomicMin(reinterpret_cast<unsigned *>(p), __float_as_uint(v));
}
__device__ __forceinline__ void smem_min(double *p, double v) {
    atomicMin(reinterpret_cast<unsigned long long *>(p),
              (unsigned long long)__double_as_longlong(v));
}
__device__ __forceinline__ void smem_max(float *p, float v) {
    atomicMax(reinterpret_cast<unsigned *>(p), __float_as_uint(v));
}
__device__ __forceinline__ void smem_max(double *p, double v) {
    atomicMax(reinterpret_cast<unsigned long long *>(p),
              (unsigned long long)__double_as_longlong(v));
}
template <class T> __device__ __forceinline__ T inf_of();
template <> __device__ __forceinline__ float inf_of<float>() { return inf_f(); }
template <> __device__ __forceinline__ double inf_of<double>() {
    return __longlong_as_double(0x7ff0000000000000ll);
}
__device__ __forceinline__ float root(float x) { return sqrtf(x); }
__device__ __forceinline__ double root(double x) { return sqrt(x); }

// Hausdorff distance (Def. 4) of the query set Q (mq x d) and the set V (mv x d),
// every pair |q - v|^2 summed directly over the dimensions in T, by the whole CTA
// (kBT threads, every thread must call).  sm: 2 * kTile * kTP + kMaxQ + kTile + 2 T.
template <class T>
__device__ T haus_exact(const float *__restrict__ Q, int mq, const float *__restrict__ V, int mv,
                        int d, T *sm) {
    constexpr int kMaxQ = BVSS_MAX_QSET;
    T *Qs = sm, *Vs = sm + kTile * kTP, *qmin = Vs + kTile * kTP, *vmin = qmin + kMaxQ;
    T *red = vmin + kTile;   // [0] max over rows of the row minima, [1] the answer
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    for (int a = tid; a < mq; a += kBT) qmin[a] = inf_of<T>();
    if (tid == 0) red[0] = (T)0;
    const int lr = tid >> 3, lc = (tid & 7) * 4;   // this thread's load: row, 4 dims
    for (int v0 = 0; v0 < mv; v0 += kTile) {
        __syncthreads();
        if (tid < kTile) vmin[tid] = inf_of<T>();
        for (int a0 = 0; a0 < mq; a0 += kTile) {
            T acc[2][2] = {{0, 0}, {0, 0}};
            for (int k0 = 0; k0 < d; k0 += kTile) {
                __syncthreads();
                const int k = k0 + lc;
                float4 x = make_float4(0.f, 0.f, 0.f, 0.f), y = x;
                if (k < d) {   // d % 4 == 0: the whole float4 is inside the row
                    if (a0 + lr < mq)
                        x = *reinterpret_cast<const float4 *>(Q + (int64_t)(a0 + lr) * d + k);
                    if (v0 + lr < mv)
                        y = *reinterpret_cast<const float4 *>(V + (int64_t)(v0 + lr) * d + k);
                }
                T *qs = Qs + lr * kTP + lc, *vs = Vs + lr * kTP + lc;
                qs[0] = (T)x.x; qs[1] = (T)x.y; qs[2] = (T)x.z; qs[3] = (T)x.w;
                vs[0] = (T)y.x; vs[1] = (T)y.y; vs[2] = (T)y.z; vs[3] = (T)y.w;
                __syncthreads();
                // each chunk of 32 dimensions is summed on its own, then added: the
                // rounding bound grows with 32 + d/32 terms instead of d
                T part[2][2] = {{0, 0}, {0, 0}};
#pragma unroll 8
                for (int kk = 0; kk < kTile; ++kk) {
                    const T q0 = Qs[tx * kTP + kk], q1 = Qs[(tx + 16) * kTP + kk];
                    const T w0 = Vs[ty * kTP + kk], w1 = Vs[(ty + 16) * kTP + kk];
                    const T d00 = q0 - w0, d01 = q0 - w1, d10 = q1 - w0, d11 = q1 - w1;
                    part[0][0] = fma(d00, d00, part[0][0]);
                    part[0][1] = fma(d01, d01, part[0][1]);
                    part[1][0] = fma(d10, d10, part[1][0]);
                    part[1][1] = fma(d11, d11, part[1][1]);
                }
#pragma unroll
                for (int i = 0; i < 2; ++i)
#pragma unroll
                    for (int j = 0; j < 2; ++j) acc[i][j] += part[i][j];
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int a = a0 + tx + 16 * i, b = ty + 16 * j;
                    if (a < mq && v0 + b < mv) {
                        smem_min(&qmin[a], acc[i][j]);
                        smem_min(&vmin[b], acc[i][j]);
                    }
                }
        }
        __syncthreads();
        if (tid < 32) {
            T m = v0 + tid < mv ? vmin[tid] : (T)0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const T y = __shfl_xor_sync(0xffffffffu, m, o);
                m = y > m ? y : m;
            }
            if (tid == 0 && m > red[0]) red[0] = m;
        }
    }
    __syncthreads();
    if (tid == 0) red[1] = red[0];
    __syncthreads();
    for (int a = tid; a < mq; a += kBT) smem_max(&red[1], qmin[a]);
    __syncthreads();
    const T h2 = red[1];
    __syncthreads();   // sm may be reused by the caller right away
    return root(h2);
}

// k-th smallest (1-based, 1 <= k <= n) of the n keys in shared memory, by the whole
// CTA: radix select over four 8-bit digits, the digit found with a block-wide scan.
// sh: kBW + 3 ints.
__device__ uint32_t block_kth(const uint32_t *keys, int n, int k, int *hist, int *sh) {
    uint32_t prefix = 0, mask = 0;
    for (int shift = 24; shift >= 0; shift -= 8) {
        for (int b = threadIdx.x; b < 256; b += kBT) hist[b] = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += kBT) {
            const uint32_t key = keys[i];
            if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1);
        }
        __syncthreads();
        // kBT == 256: one bin per thread
        const int c = hist[threadIdx.x];
        int tot;
        const int before = block_excl_scan<kBT>(c, sh, &tot);
        if (before < k && before + c >= k) {
            sh[kBW + 1] = threadIdx.x;
            sh[kBW + 2] = k - before;
        }
        __syncthreads();
        prefix |= (uint32_t)sh[kBW + 1] << shift;
        mask |= 0xFFu << shift;
        k = sh[kBW + 2];
        __syncthreads();
    }
    return prefix;
}

// relative error bound of a direct FP32 distance summed in one chain over d dimensions
__device__ __forceinline__ float eta_of(int d) { return (float)(d + 4) * 5.9604645e-8f; }
// the same for this stage's own FP32 distances (warp and CTA-tile forms)
__device__ __forceinline__ float eta_exact(int d) {
    return (float)(40 + (d + 31) / 32) * 5.9604645e-8f;
}

// Binary digits below the point that x needs: x = integer * 2^-g for this g and no
// smaller one (0 for integers and zero; subnormals report 200, beyond any usable grid).
__device__ __forceinline__ int frac_bits(float x) {
    const uint32_t u = __float_as_uint(x) & 0x7fffffffu;
    if (u == 0) return 0;
    const int ex = (int)(u >> 23);
    if (ex == 0) return 200;
    const uint32_t mant = (u & 0x7fffffu) | 0x800000u;   // x = mant * 2^(ex - 150)
    const int g = 150 - ex - (__ffs(mant) - 1);
    return g > 0 ? g : 0;
}

// A query vector's norm and the norm of its rounding error in the refine's copy:
// form 1 BF16 (round to nearest), form 2 FP8 E4M3 with the vector's own scale
// (largest magnitude -> 448, round to nearest, saturating), form 3 TF32 (to nearest, ties
// away from zero, as the refine rounds its query operand), form 0 none.  One warp.
// gbits: the largest frac_bits of its values.
__device__ void query_round_err(const float *x, int d, int form, float &norm, float &err,
                                int &gbits) {
    const int lane = threadIdx.x & 31;
    float mx = 0.0f;
    if (form == 2) {
        for (int k = lane; k < d; k += 32) mx = fmaxf(mx, fabsf(x[k]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    const float sc = mx > 0.0f ? mx / 448.0f : 1.0f;
    const float inv = 1.0f / sc;
    float s = 0.0f, e = 0.0f;
    int g = 0;
    for (int k = lane; k < d; k += 32) {
        const float v = x[k];
        g = max(g, frac_bits(v));
        float r = v;
        if (form == 1) {
            r = __bfloat162float(__float2bfloat16_rn(v));
        } else if (form == 3) {
            r = __uint_as_float(f32_to_tf32(v));
        } else if (form == 2) {
            const __nv_fp8_storage_t f8 = __nv_cvt_float_to_fp8(v * inv, __NV_SATFINITE, __NV_E4M3);
            const __half_raw hr = __nv_cvt_fp8_to_halfraw(f8, __NV_E4M3);
            r = __half2float(*reinterpret_cast<const __half *>(&hr)) * sc;
        }
        s = fmaf(v, v, s);
        e = fmaf(v - r, v - r, e);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        e += __shfl_xor_sync(0xffffffffu, e, o);
    }
    // outward: the sums' own rounding is within eta (relative)
    const float up = 1.0f + 2.0f * eta_of(d);
    norm = __fmul_ru(__fsqrt_ru(s), up);
    err = __fmul_ru(__fsqrt_ru(e), up);
    gbits = __reduce_max_sync(0xffffffffu, (unsigned)g);
}

// NJ: float4 of a row per lane (dimensions 4 lane + 128 j, j < NJ): d <= 128 NJ
constexpr int kNI = BVSS_MAX_QSET / 32;   // query vectors per lane (row-minimum owners)

// one database row into the lane's registers: dimensions 4 lane + 128 j
template <int NJ>
__device__ __forceinline__ void load_row(const float *__restrict__ v, int d, float4 (&r)[NJ]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        const int k = 4 * lane + 128 * j;
        if (k < d) r[j] = *reinterpret_cast<const float4 *>(v + k);
    }
}

// |q_a - v|^2 for the four query vectors a0 .. a0 + 3 (those below mq) and the row in r,
// each lane summing its dimensions in FP32 and a shuffle tree adding the lanes: four
// independent chains, so their latencies overlap.  Warp-uniform results.
template <int NJ>
__device__ __forceinline__ void pair4_sq(const float *Q, int a0, int mq, int d,
                                         const float4 (&r)[NJ], float (&s)[4]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int g = 0; g < 4; ++g) s[g] = 0.0f;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        const int k = 4 * lane + 128 * j;
        if (k < d) {
#pragma unroll
            for (int g = 0; g < 4; ++g)
                if (a0 + g < mq) {
                    const float4 x = *reinterpret_cast<const float4 *>(Q + (int64_t)(a0 + g) * d + k);
                    float t = x.x - r[j].x;
                    s[g] = fmaf(t, t, s[g]);
                    t = x.y - r[j].y;
                    s[g] = fmaf(t, t, s[g]);
                    t = x.z - r[j].z;
                    s[g] = fmaf(t, t, s[g]);
                    t = x.w - r[j].w;
                    s[g] = fmaf(t, t, s[g]);
                }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int g = 0; g < 4; ++g) s[g] += __shfl_xor_sync(0xffffffffu, s[g], o);
}

// The same for one query vector in FP64 (each difference and square in double).
template <int NJ>
__device__ __forceinline__ double pair_sq64(const float *q, int d, const float4 (&r)[NJ]) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        const int k = 4 * lane + 128 * j;
        if (k < d) {
            const float4 x = *reinterpret_cast<const float4 *>(q + k);
            double t = (double)x.x - (double)r[j].x;
            s = fma(t, t, s);
            t = (double)x.y - (double)r[j].y;
            s = fma(t, t, s);
            t = (double)x.z - (double)r[j].z;
            s = fma(t, t, s);
            t = (double)x.w - (double)r[j].w;
            s = fma(t, t, s);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

__device__ __forceinline__ float warp_max(float m) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    return m;
}

// One FP32 pass of a warp over V's rows against Q (mq x d, row stride d): the row
// minima of the squared distances of query vectors 32 i + lane go to rm[i] (owner
// lanes), the return value is the largest column minimum.  The next row's loads are in
// flight while a row is scored.  d % 4 == 0, d <= kWarpMaxD, 1 <= mq <= BVSS_MAX_QSET.
template <int NJ>
__device__ float warp_scan32(const float *Q, int mq, const float *__restrict__ V, int mv, int d,
                             float (&rm)[kNI]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < kNI; ++i) rm[i] = inf_f();
    float cmax = 0.0f;
    float4 rn[NJ];
    load_row<NJ>(V, d, rn);
    for (int b = 0; b < mv; ++b) {
        float4 r[NJ];
#pragma unroll
        for (int j = 0; j < NJ; ++j) r[j] = rn[j];
        if (b + 1 < mv) load_row<NJ>(V + (int64_t)(b + 1) * d, d, rn);
        float cmin = inf_f();
#pragma unroll
        for (int i = 0; i < kNI; ++i)
            for (int l = 0; l < 32; l += 4) {
                const int a0 = 32 * i + l;
                if (a0 >= mq) break;   // uniform over the warp
                float s[4];
                pair4_sq<NJ>(Q, a0, mq, d, r, s);
#pragma unroll
                for (int g = 0; g < 4; ++g)
                    if (a0 + g < mq) {
                        cmin = fminf(cmin, s[g]);
                        if (lane == l + g) rm[i] = fminf(rm[i], s[g]);
                    }
            }
        cmax = fmaxf(cmax, cmin);
    }
    return cmax;
}

// the largest row minimum over the valid query vectors
__device__ __forceinline__ float rows_max(const float (&rm)[kNI], int mq) {
    const int lane = threadIdx.x & 31;
    float m = 0.0f;
#pragma unroll
    for (int i = 0; i < kNI; ++i)
        if (32 * i + lane < mq) m = fmaxf(m, rm[i]);
    return warp_max(m);
}

// Hausdorff distance (Def. 4) of Q and V in FP32 by one warp (warp-uniform).
template <int NJ>
__device__ float warp_haus32(const float *Q, int mq, const float *__restrict__ V, int mv, int d) {
    float rm[kNI];
    const float cmax = warp_scan32<NJ>(Q, mq, V, mv, d, rm);
    return sqrtf(fmaxf(cmax, rows_max(rm, mq)));
}

// Hausdorff distance of Q and V decided in FP64 on the pairs that can attain it.  With
// the FP32 squared distances s' within a factor (1 +- e) of the true s: a row (query
// vector) whose FP32 minimum is below H'^2 (1 - e) / (1 + e) cannot attain the maximum,
// nor a column (row of V) likewise, and inside a row or column only pairs with
// s' (1 - e) <= min' (1 + e) can be its minimum.  A first FP32 pass gives the row
// minima and H'^2, a second one recomputes every pair, and the pairs that pass both
// tests are re-scored in FP64; the maximum over the surviving rows and columns of their
// FP64 minima is H^2.
template <int NJ>
__device__ __noinline__ double warp_haus64(const float *Q, int mq, const float *__restrict__ V,
                                           int mv, int d) {
    const int lane = threadIdx.x & 31;
    float rm[kNI];
    const float c32 = warp_scan32<NJ>(Q, mq, V, mv, d, rm);
    const float h2 = fmaxf(c32, rows_max(rm, mq));
    const float e = 2.0f * eta_exact(d);
    const float lo_reach = __fdiv_rd(__fmul_rd(h2, 1.0f - e), 1.0f + e);
    double rm64[kNI];
#pragma unroll
    for (int i = 0; i < kNI; ++i) rm64[i] = __longlong_as_double(0x7ff0000000000000ll);
    double best = 0.0;
    float4 r[NJ];
    for (int b = 0; b < mv; ++b) {
        load_row<NJ>(V + (int64_t)b * d, d, r);
        float sv[kNI];
        float cmin = inf_f();
#pragma unroll
        for (int i = 0; i < kNI; ++i) {
            sv[i] = inf_f();
            for (int l = 0; l < 32; l += 4) {
                const int a0 = 32 * i + l;
                if (a0 >= mq) break;
                float s[4];
                pair4_sq<NJ>(Q, a0, mq, d, r, s);
#pragma unroll
                for (int g = 0; g < 4; ++g)
                    if (a0 + g < mq) {
                        cmin = fminf(cmin, s[g]);
                        if (lane == l + g) sv[i] = s[g];
                    }
            }
        }
        const bool col_rel = cmin >= lo_reach;
        const float col_cut = __fmul_ru(cmin, 1.0f + e);
        double cm64 = __longlong_as_double(0x7ff0000000000000ll);
#pragma unroll
        for (int i = 0; i < kNI; ++i)
            for (int l = 0; l < 32; ++l) {
                const int a = 32 * i + l;
                if (a >= mq) break;
                const float sa = __shfl_sync(0xffffffffu, sv[i], l);
                const float ra = __shfl_sync(0xffffffffu, rm[i], l);
                const float sl = __fmul_rd(sa, 1.0f - e);
                const bool row_pair = ra >= lo_reach && sl <= __fmul_ru(ra, 1.0f + e);
                const bool col_pair = col_rel && sl <= col_cut;
                if (row_pair || col_pair) {   // uniform over the warp
                    const double s64 = pair_sq64<NJ>(Q + (int64_t)a * d, d, r);
                    if (row_pair && lane == l) rm64[i] = fmin(rm64[i], s64);
                    if (col_pair) cm64 = fmin(cm64, s64);
                }
            }
        if (col_rel) best = fmax(best, cm64);
    }
    // rows that can attain the maximum hold a finite FP64 minimum (their own arg-min pair
    // passed both tests); the others are left out
    double m = best;
#pragma unroll
    for (int i = 0; i < kNI; ++i)
        if (32 * i + lane < mq && rm[i] >= lo_reach) m = fmax(m, rm64[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    return sqrt(m);
}

// S's room: max(256, 4 k) rounded up to a power of two, at most kMaxS
__host__ __device__ inline int s_cap(int k) {
    int c = 256;
    while (c < 4 * k && c < kMaxS) c <<= 1;
    return c;
}

// Bytes of k_boundary's dynamic shared memory: the CTA-tile form's doubles (d >
// kWarpMaxD only), S's values, keys and slots, the staged query set (q_floats), and
// per candidate its hi key (then a band slot) and its lo (then the band's exact values).
__host__ __device__ inline size_t boundary_smem(int C, int k, int q_floats, bool tiles) {
    return (tiles ? sizeof(double) * kHausSmem : 0) +
           (sizeof(double) + sizeof(unsigned long long) + sizeof(int)) * s_cap(k) +
           sizeof(float) * (size_t)q_floats + 2 * sizeof(uint32_t) * (size_t)C;
}

// NJ: the warp form's float4 per lane and row (d <= 128 NJ); NJ = 0: the CTA-tile form
template <int NJ>
__global__ void __launch_bounds__(kBT, NJ >= 8 ? 1 : 2)
k_boundary(const float *__restrict__ qvec, const int64_t *__restrict__ qoff, int d, int form,
           const float *__restrict__ stats, const float *__restrict__ vec,
           const int64_t *__restrict__ set_off, const int32_t *__restrict__ cand,
           const int32_t *__restrict__ thr, int C, int k, const longlong2 *__restrict__ pair,
           float *__restrict__ cand_dist, int64_t *__restrict__ out_ids,
           float *__restrict__ out_dist, int *__restrict__ err, int q_floats, int exact_band) {
    constexpr bool tiles = NJ == 0;
    constexpr int NJW = NJ > 0 ? NJ : 1;   // the warp form's width (unused when tiles)
    extern __shared__ __align__(16) unsigned char bsm[];
    const int cap = s_cap(k);
    double *hsm = reinterpret_cast<double *>(bsm);
    double *sval = hsm + (tiles ? kHausSmem : 0);
    unsigned long long *skey = reinterpret_cast<unsigned long long *>(sval + cap);
    float *Qs = reinterpret_cast<float *>(skey + cap);
    uint32_t *hik = reinterpret_cast<uint32_t *>(Qs + q_floats);
    float *lov = reinterpret_cast<float *>(hik + C);
    int *mem = reinterpret_cast<int *>(hik);   // the band's slots, once tau is known
    int *sslot = reinterpret_cast<int *>(lov + C);
    __shared__ int hist[256];
    __shared__ int sh[kBW + 3];
    // largest norm of a rounded query vector, largest rounding error, largest frac_bits
    __shared__ float qst[3];
    const int q = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n_sel = thr[q * 4 + 3];
    const int kp = k < n_sel ? k : n_sel;
    float *cd = cand_dist + (int64_t)q * C;
    const int32_t *cq = cand + (int64_t)q * C;
    for (int j = n_sel + tid; j < C; j += kBT) cd[j] = inf_f();
    for (int t = kp + tid; t < k; t += kBT) {
        out_ids[(int64_t)q * k + t] = -1;
        out_dist[(int64_t)q * k + t] = inf_f();
    }
    if (kp <= 0) return;   // uniform over the CTA
    const int64_t a0 = qoff[q];
    const int mq = (int)(qoff[q + 1] - a0);
    const float *Q = qvec + a0 * d;
    if (mq * d <= q_floats) {
        for (int e = tid; e < mq * d / 4; e += kBT)
            reinterpret_cast<float4 *>(Qs)[e] = reinterpret_cast<const float4 *>(Q)[e];
        Q = Qs;
    }
    if (tid < 3) qst[tid] = 0.0f;
    __syncthreads();
    // ---- 1. intervals, tau and the band ----------------------------------------------
    for (int a = warp; a < mq; a += kBW) {
        float nrm, er;
        int gb;
        query_round_err(Q + (int64_t)a * d, d, form, nrm, er, gb);
        if (lane == 0) {
            smem_max(&qst[0], __fadd_ru(nrm, er));
            smem_max(&qst[1], er);
            smem_max(&qst[2], (float)gb);
        }
    }
    __syncthreads();
    // Exactness certificate: with every value a multiple of 2^-g, every product, partial
    // sum, norm and difference of the GEMM form and of the re-scored pair is a multiple of
    // 2^-2g no larger than (N_Q + N_V)^2 in magnitude.  Below 2^(22 - 2g) FP32 holds each
    // one exactly, in any order of accumulation, so the refine's value is the exact
    // Hausdorff value up to its final square root, and two such square roots are equal
    // only when the exact values are.  (The BF16 copy must be lossless, e = 0; the FP8
    // copy's scaling is never exact.)
    bool cert;
    {
        const float eV0 = form == 1 ? stats[1] : form == 2 ? stats[2] : form == 3 ? stats[4] : 0.0f;
        const float ns0 = __fadd_ru(qst[0], __fadd_ru(stats[0], eV0));
        const int g = (int)fmaxf(qst[2], stats[3]);
        cert = form != 2 && qst[1] == 0.0f && eV0 == 0.0f && g <= 10 &&
               __fmul_ru(ns0, ns0) < ldexpf(1.0f, 22 - 2 * g);
    }
    {
        const float eta_d = eta_of(d);
        const float eV = form == 1 ? stats[1] : form == 2 ? stats[2] : form == 3 ? stats[4] : 0.0f;
        const float nsum = __fadd_ru(qst[0], __fadd_ru(stats[0], eV));
        // GEMM-form squared-distance error bound (d + 8) 2^-23 (N_Q + N_V)^2
        const float D = __fmul_ru((float)(d + 8) * 1.1920929e-7f, __fmul_ru(nsum, nsum));
        // the rounding's effect on a distance: at most e_q + e_v (rigorous); for the FP8
        // form by default 3 standard deviations of the rounding model, in which the
        // per-value errors are independent and zero-mean, so a pair distance moves by
        // about sqrt(e_q^2 + e_v^2) / sqrt(d)
        // the TF32 form reads the FP32 rows as TF32 inside the tensor core but takes their
        // FP32 norms, so its GEMM-form value is |q~|^2 + |v|^2 - 2 q~.v~ = |q~ - v|^2 +
        // 2 q~.(v - v~): an extra additive term of at most 2 N_Q e_v on the squared value,
        // and only the query's rounding e_q moves the distance itself
        const float e = form == 2 && !exact_band
                            ? __fmul_ru(3.0f, __fdiv_ru(__fsqrt_ru(__fadd_ru(
                                  __fmul_ru(qst[1], qst[1]), __fmul_ru(eV, eV))), sqrtf((float)d) *
                                  (1.0f - 1e-6f)))
                        : form == 3 ? qst[1]
                                    : __fadd_ru(qst[1], eV);
        const float Dv = form == 3 ? __fadd_ru(D, __fmul_ru(2.0f, __fmul_ru(qst[0], eV))) : D;
        const longlong2 *pq = pair + (int64_t)q * C;
        for (int j = tid; j < n_sel; j += kBT) {
            float lo, hi;
            if (cert) {   // exact up to the square root's rounding
                const float v = form == 0 ? cd[j]
                                          : sqrtf(__uint_as_float(
                                                (uint32_t)((unsigned long long)pq[j].x >> 32)));
                lo = __fmul_rd(v, 1.0f - 1.1920929e-7f);
                hi = __fmul_ru(v, 1.0f + 1.1920929e-7f);
            } else if (form == 0) {
                const float r = cd[j];
                const float rl = __fmul_rd(r, 1.0f - eta_d), rh = __fmul_ru(r, 1.0f + 2.0f * eta_d);
                const float D2 = __fmul_ru(2.0f, D);
                lo = __fsqrt_rd(fmaxf(__fsub_rd(__fmul_rd(rl, rl), D2), 0.0f));
                hi = __fsqrt_ru(__fadd_ru(__fmul_ru(rh, rh), D2));
            } else {
                const float h2 = __uint_as_float((uint32_t)((unsigned long long)pq[j].x >> 32));
                lo = fmaxf(__fsub_rd(__fsqrt_rd(fmaxf(__fsub_rd(h2, Dv), 0.0f)), e), 0.0f);
                hi = __fadd_ru(__fsqrt_ru(__fadd_ru(h2, Dv)), e);
            }
            if (form != 0) cd[j] = sqrtf(__uint_as_float(
                                       (uint32_t)((unsigned long long)pq[j].x >> 32)));
            hik[j] = __float_as_uint(hi);   // non-negative: bit order is value order
            lov[j] = lo;
        }
    }
    __syncthreads();
    const float tau = __uint_as_float(block_kth(hik, n_sel, kp, hist, sh));
    int nb = 0;   // mem[] overwrites hik[] from here on (block_kth has returned)
    for (int j0 = 0; j0 < n_sel; j0 += kBT) {
        const int j = j0 + tid;
        const int in = j < n_sel && lov[j] <= tau;
        int tot;
        const int pos = block_excl_scan<kBT>(in, sh, &tot);
        if (in) mem[nb + pos] = j;
        nb += tot;
    }
    __syncthreads();
    // ---- 2. the direct FP32 Hausdorff value of every band member -----------------------
    if (cert) {   // the refine's value is already exact (up to the square root's rounding)
        const longlong2 *pq = pair + (int64_t)q * C;
        for (int t = tid; t < nb; t += kBT) {
            const int j = mem[t];
            const float h = form == 0 ? cd[j]
                                      : sqrtf(__uint_as_float(
                                            (uint32_t)((unsigned long long)pq[j].x >> 32)));
            lov[t] = h;
            cd[j] = h;
        }
    } else if (!tiles) {
        for (int t = warp; t < nb; t += kBW) {
            const int j = mem[t];
            const int64_t r0 = set_off[cq[j]];
            const float h = warp_haus32<NJW>(Q, mq, vec + r0 * d, (int)(set_off[cq[j] + 1] - r0), d);
            if (lane == 0) {
                lov[t] = h;
                cd[j] = h;
            }
        }
    } else {
        float *fsm = reinterpret_cast<float *>(hsm);
        for (int t = 0; t < nb; ++t) {
            const int j = mem[t];
            const int64_t r0 = set_off[cq[j]];
            const float h = haus_exact<float>(Q, mq, vec + r0 * d,
                                              (int)(set_off[cq[j] + 1] - r0), d, fsm);
            if (tid == 0) {
                lov[t] = h;
                cd[j] = h;
            }
        }
    }
    __syncthreads();
    // ---- 3. S: the members that can reach rank k', sorted by (H32, id) ----------------
    // the exact values are non-negative: their bits order as they do
    const float vk =
        __uint_as_float(block_kth(reinterpret_cast<const uint32_t *>(lov), nb, kp, hist, sh));
    const float eta = cert ? 0.0f : eta_exact(d);   // certified values: equal iff equal
    const float reach = __fmul_ru(vk, 1.0f + eta);
    int ns = 0;
    for (int t0 = 0; t0 < nb; t0 += kBT) {
        const int t = t0 + tid;
        const int in = t < nb && __fmul_rd(lov[t], 1.0f - eta) <= reach;
        int tot;
        const int pos = block_excl_scan<kBT>(in, sh, &tot);
        if (in && ns + pos < cap) {
            skey[ns + pos] = ((unsigned long long)__float_as_uint(lov[t]) << 32) |
                             (uint32_t)cq[mem[t]];
            sslot[ns + pos] = mem[t];
        }
        ns += tot;
    }
    if (ns > cap) {
        if (tid == 0) atomicOr(err, kErrBandOverflow);
        ns = cap;
    }
    int np = 1;
    while (np < ns) np <<= 1;
    for (int t = ns + tid; t < np; t += kBT) {
        skey[t] = ~0ull;
        sslot[t] = -1;
    }
    __syncthreads();
    for (int size = 2; size <= np; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = tid; t < np; t += kBT) {
                const int u = t ^ stride;
                if (u > t) {
                    const bool asc = (t & size) == 0;
                    const unsigned long long a = skey[t], b = skey[u];
                    if ((a > b) == asc) {
                        skey[t] = b;
                        skey[u] = a;
                        const int sl = sslot[t];
                        sslot[t] = sslot[u];
                        sslot[u] = sl;
                    }
                }
            }
            __syncthreads();
        }
    // neighbours that FP32 cannot order, at or above rank k': both marked (slot bit 30)
    for (int t = tid; t < ns; t += kBT) sval[t] = (double)__uint_as_float((uint32_t)(skey[t] >> 32));
    __syncthreads();
    for (int t = tid; t + 1 < ns && t < kp; t += kBT) {
        const float a = __uint_as_float((uint32_t)(skey[t] >> 32));
        const float b = __uint_as_float((uint32_t)(skey[t + 1] >> 32));
        if (__fmul_ru(a, 1.0f + eta) >= __fmul_rd(b, 1.0f - eta)) {
            atomicOr(&sslot[t], 1 << 30);
            atomicOr(&sslot[t + 1], 1 << 30);
        }
    }
    __syncthreads();
    // ---- FP64 for the marked members: the u-th marked one on warp u mod kBW --------------
    // (certified values are marked only when exactly equal: no FP64, the id decides)
    if (cert) {
    } else if (!tiles) {
        int u = 0;
        for (int t = 0; t < ns; ++t) {
            const int sl = sslot[t];
            if (!(sl & (1 << 30))) continue;
            if (u++ % kBW != warp) continue;
            const int j = sl & 0x3fffffff;
            const int64_t r0 = set_off[cq[j]];
            const double h = warp_haus64<NJW>(Q, mq, vec + r0 * d, (int)(set_off[cq[j] + 1] - r0), d);
            if (lane == 0) {
                sval[t] = h;
                cd[j] = (float)h;
            }
        }
    } else {
        for (int t = 0; t < ns; ++t) {
            const int sl = sslot[t];
            if (!(sl & (1 << 30))) continue;
            const int j = sl & 0x3fffffff;
            const int64_t r0 = set_off[cq[j]];
            const double h = haus_exact<double>(Q, mq, vec + r0 * d,
                                                (int)(set_off[cq[j] + 1] - r0), d, hsm);
            if (tid == 0) {
                sval[t] = h;
                cd[j] = (float)h;
            }
        }
    }
    __syncthreads();
    // ---- 4. order by (value, id): FP64 reorders only inside runs of overlapping
    // neighbours, so an insertion sort does no work elsewhere ------------------------------
    if (tid == 0) {
        for (int t = 1; t < ns; ++t) {
            const double v = sval[t];
            const unsigned long long kk = skey[t];
            const uint32_t id = (uint32_t)kk;
            int u = t - 1;
            while (u >= 0 && (sval[u] > v || (sval[u] == v && (uint32_t)skey[u] > id))) {
                sval[u + 1] = sval[u];
                skey[u + 1] = skey[u];
                --u;
            }
            sval[u + 1] = v;
            skey[u + 1] = kk;
        }
    }
    __syncthreads();
    for (int t = tid; t < kp; t += kBT) {
        out_ids[(int64_t)q * k + t] = (int64_t)(uint32_t)skey[t];
        out_dist[(int64_t)q * k + t] = (float)sval[t];
    }
}

}  // namespace

constexpr size_t kSmemLimit = 232448;    // 227 KB opt-in per CTA

cudaError_t launch_band_topk(const float *qvec, const int64_t *qoff, int n_q, int max_mq, int d,
                             int form, const float *stats, const float *vec,
                             const int64_t *set_off, const int32_t *cand, const int32_t *thr,
                             int C, int k, const longlong2 *pair, float *cand_dist,
                             int64_t *out_ids, float *out_dist, int *err, int exact_band,
                             cudaStream_t st) {
    if (n_q <= 0) return cudaSuccess;
    if (C > BVSS_MAX_C || k < 1 || k > BVSS_MAX_K || form < 0 || form > 3 || d % 4 != 0 ||
        max_mq < 1 || max_mq > BVSS_MAX_QSET)
        return cudaErrorInvalidValue;
    // the query set in shared memory whenever it fits beside the rest (else read in place)
    int q_floats = max_mq * d;
    const bool tiles = d > kWarpMaxD;
    if (boundary_smem(C, k, q_floats, tiles) > kSmemLimit) q_floats = 0;
    const size_t smem = boundary_smem(C, k, q_floats, tiles);
    if (smem > kSmemLimit) return cudaErrorInvalidValue;
    auto kern = tiles ? k_boundary<0> : d <= 128 ? k_boundary<1> : d <= 256 ? k_boundary<2>
              : d <= 512 ? k_boundary<4> : k_boundary<8>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<n_q, kBT, smem, st>>>(qvec, qoff, d, form, stats, vec, set_off, cand, thr, C, k, pair,
                                 cand_dist, out_ids, out_dist, err, q_floats, exact_band);
    return cudaGetLastError();
}

// The largest vector norm of the database and the largest rounding-error norm of its
// BF16 and FP8 copies (stats[0..2]), each rounded up, read from the stored copies, the
// largest frac_bits of its values (stats[3]), and a bound on the largest rounding-error
// norm of the vectors read as TF32 (stats[4]).  A tensor core that reads an FP32 value as
// TF32 keeps 10 of its 23 mantissa bits; whichever way it rounds (to nearest or toward
// zero), a value it cannot hold moves by less than one TF32 unit in the last place,
// 2^(e - 10) <= 2^-10 |x| for x = 1.m 2^e, and a value it can hold (low 13 bits zero) does
// not move.  A subnormal counts with its whole magnitude (it may be flushed to zero).
__global__ void k_round_stats(const float *__restrict__ x, int64_t n, int d,
                              const __nv_bfloat16 *__restrict__ x16,
                              const uint8_t *__restrict__ x8, const float *__restrict__ sc8,
                              float *__restrict__ stats) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const float up = 1.0f + 2.0f * eta_of(d);
    float m0 = 0.0f, m1 = 0.0f, m2 = 0.0f, m4 = 0.0f;
    int g = 0;
    for (int64_t v = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); v < n;
         v += warps) {
        float s = 0.0f, e16 = 0.0f, e8 = 0.0f, e32 = 0.0f;
        const float sc = x8 ? sc8[v] : 1.0f;
        for (int k = lane; k < d; k += 32) {
            const float a = x[v * d + k];
            g = max(g, frac_bits(a));
            s = fmaf(a, a, s);
            const uint32_t ua = __float_as_uint(a) & 0x7fffffffu;
            if ((ua >> 23) == 0) e32 = fmaf(a, a, e32);
            else if (ua & 0x1fffu) e32 = fmaf(a, a * 0x1p-20f, e32);
            if (x16) {
                const float b = __bfloat162float(x16[v * d + k]);
                e16 = fmaf(a - b, a - b, e16);
            }
            if (x8) {
                const __half_raw hr = __nv_cvt_fp8_to_halfraw(x8[v * d + k], __NV_E4M3);
                const float b = __half2float(*reinterpret_cast<const __half *>(&hr)) * sc;
                e8 = fmaf(a - b, a - b, e8);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s += __shfl_xor_sync(0xffffffffu, s, o);
            e16 += __shfl_xor_sync(0xffffffffu, e16, o);
            e8 += __shfl_xor_sync(0xffffffffu, e8, o);
            e32 += __shfl_xor_sync(0xffffffffu, e32, o);
        }
        m0 = fmaxf(m0, __fmul_ru(__fsqrt_ru(s), up));
        m1 = fmaxf(m1, __fmul_ru(__fsqrt_ru(e16), up));
        m2 = fmaxf(m2, __fmul_ru(__fsqrt_ru(e8), up));
        m4 = fmaxf(m4, __fmul_ru(__fsqrt_ru(e32), up));
    }
    g = (int)__reduce_max_sync(0xffffffffu, (unsigned)g);
    if (lane == 0) {
        atomicMax(reinterpret_cast<unsigned *>(&stats[3]), __float_as_uint((float)g));
        atomicMax(reinterpret_cast<unsigned *>(&stats[0]), __float_as_uint(m0));
        atomicMax(reinterpret_cast<unsigned *>(&stats[1]), __float_as_uint(m1));
        atomicMax(reinterpret_cast<unsigned *>(&stats[2]), __float_as_uint(m2));
        atomicMax(reinterpret_cast<unsigned *>(&stats[4]), __float_as_uint(m4));
    }
}

cudaError_t launch_round_stats(const float *x, int64_t n, int d, const __nv_bfloat16 *x16,
                               const uint8_t *x8, const float *sc8, float *stats,
                               cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(stats, 0, kRoundStats * sizeof(float), st);
    if (e != cudaSuccess || n <= 0) return e;
    int64_t g = (n + 7) / 8;
    if (g > 152 * 16) g = 152 * 16;
    k_round_stats<<<(unsigned)g, 256, 0, st>>>(x, n, d, x16, x8, sc8, stats);
    return cudaGetLastError();
}

}  // namespace bvss
