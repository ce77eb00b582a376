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
//     lo = sqrt(r^2 - 2D) (1 - eta), hi = sqrt(r^2 + 2D) (1 + eta).
//   BF16 / FP8 forms: the GEMM-form Hausdorff value h of the rounded copies, packed
//     into the pair record by the refine.  Rounding moves a vector x by e_x = |x - x'|
//     and every pair distance by at most e_q + e_v (triangle inequality), so the
//     Hausdorff value of the rounded sets is within e = max e_q + max e_v of H
//     (max and min are 1-Lipschitz), and h is within D of that value squared:
//     lo = sqrt(h - D) - e, hi = sqrt(h + D) + e.
//   eta = (d + 4) 2^-24 bounds the relative error of a direct FP32 distance
//     (d squared differences summed with FMA, then a square root).
// Then (k' = min(k, candidates)):
//   k_band_sel    tau = the k'-th smallest hi; the band B = {lo <= tau} holds every
//                 candidate that can be among the k' nearest;
//   k_band_exact  the direct FP32 Hausdorff value H32 of every member of B, all pairs
//                 (one CTA per candidate, 32 x 32 pair tiles, 32 dimensions at a time);
//   k_band_order  S = the members whose interval H32 (1 +- eta) reaches the k'-th
//                 smallest H32, sorted by (H32, id); members of S whose interval
//                 overlaps a neighbour's at or above rank k' are re-scored in FP64
//                 (the same tiles in double), then S is ordered by (value, id) and
//                 the first k' are the result.
// Members of B get their exact FP32 (or FP64) value as their candidate distance;
// the others keep the refine's value.  Returned distances are within eta (relative)
// of the FP64 Hausdorff value, or its FP32 rounding where FP64 decided.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <math.h>

#include "block_util.cuh"
#include "bvss_internal.cuh"

namespace bvss {

namespace {

constexpr int kBT = 256;          // threads of every boundary kernel (16 x 16 pair grid)
constexpr int kTile = 32;         // query vectors x rows per pair tile
constexpr int kTP = kTile + 1;    // padded smem row
constexpr int kMaxS = 4096;       // candidates that may tie with the k-th (sorted in smem)
constexpr int kExactCTAs = 8;     // CTAs per query set in k_band_exact

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
#pragma unroll 8
                for (int kk = 0; kk < kTile; ++kk) {
                    const T q0 = Qs[tx * kTP + kk], q1 = Qs[(tx + 16) * kTP + kk];
                    const T w0 = Vs[ty * kTP + kk], w1 = Vs[(ty + 16) * kTP + kk];
                    const T d00 = q0 - w0, d01 = q0 - w1, d10 = q1 - w0, d11 = q1 - w1;
                    acc[0][0] = fma(d00, d00, acc[0][0]);
                    acc[0][1] = fma(d01, d01, acc[0][1]);
                    acc[1][0] = fma(d10, d10, acc[1][0]);
                    acc[1][1] = fma(d11, d11, acc[1][1]);
                }
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

// k-th smallest (1-based) of the n keys in shared memory, by the whole CTA: radix
// select over four 8-bit digits.  hist: 256 ints; sh: 2 ints.
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
        if (threadIdx.x == 0) {
            int cum = 0, sel = 255;
            for (int b = 0; b < 256; ++b) {
                if (cum + hist[b] >= k) {
                    sel = b;
                    break;
                }
                cum += hist[b];
            }
            sh[0] = sel;
            sh[1] = k - cum;
        }
        __syncthreads();
        prefix |= (uint32_t)sh[0] << shift;
        mask |= 0xFFu << shift;
        k = sh[1];
        __syncthreads();
    }
    return prefix;
}

// eta: relative error bound of a direct FP32 distance in d dimensions
__device__ __forceinline__ float eta_of(int d) { return (float)(d + 4) * 5.9604645e-8f; }

// A query vector's norm and the norm of its rounding error in the refine's copy:
// form 1 BF16 (round to nearest), form 2 FP8 E4M3 with the vector's own scale
// (largest magnitude -> 448, round to nearest, saturating), form 0 none.  One warp.
__device__ void query_round_err(const float *x, int d, int form, float &norm, float &err) {
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
    for (int k = lane; k < d; k += 32) {
        const float v = x[k];
        float r = v;
        if (form == 1) {
            r = __bfloat162float(__float2bfloat16_rn(v));
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
}

// per query set: every candidate's interval, tau and the band (ascending candidate slot)
__global__ void __launch_bounds__(kBT)
k_band_sel(const float *__restrict__ qvec, const int64_t *__restrict__ qoff, int d, int form,
           const float *__restrict__ stats, float *__restrict__ cand_dist,
           const longlong2 *__restrict__ pair, const int32_t *__restrict__ thr, int C, int k,
           int32_t *__restrict__ band, int32_t *__restrict__ band_n) {
    extern __shared__ uint32_t bsm[];
    uint32_t *hik = bsm;                                      // C keys: bits of hi
    float *lov = reinterpret_cast<float *>(bsm + C);          // C values: lo
    __shared__ int hist[256];
    __shared__ int sh[kBT / 32 + 2];
    __shared__ float qst[2];                                  // max norm, max rounding error
    const int q = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n_sel = thr[q * 4 + 3];
    float *cd = cand_dist + (int64_t)q * C;
    for (int j = n_sel + tid; j < C; j += kBT) cd[j] = inf_f();
    if (n_sel <= 0) {
        if (tid == 0) band_n[q] = 0;
        return;
    }
    if (tid < 2) qst[tid] = 0.0f;
    __syncthreads();
    const int64_t a0 = qoff[q];
    const int mq = (int)(qoff[q + 1] - a0);
    for (int a = warp; a < mq; a += kBT / 32) {
        float nrm, err;
        query_round_err(qvec + (a0 + a) * d, d, form, nrm, err);
        if (lane == 0) {
            smem_max(&qst[0], __fadd_ru(nrm, err));   // norm of the rounded vector, at most
            smem_max(&qst[1], err);
        }
    }
    __syncthreads();
    const float eta = eta_of(d);
    const float eV = form == 1 ? stats[1] : (form == 2 ? stats[2] : 0.0f);
    const float nsum = __fadd_ru(qst[0], __fadd_ru(stats[0], eV));
    // GEMM-form squared-distance error bound (d + 8) 2^-23 (N_Q + N_V)^2
    const float D = __fmul_ru((float)(d + 8) * 1.1920929e-7f, __fmul_ru(nsum, nsum));
    const float e = __fadd_ru(qst[1], eV);
    const longlong2 *pq = pair + (int64_t)q * C;
    for (int j = tid; j < n_sel; j += kBT) {
        float lo, hi;
        if (form == 0) {
            const float r = cd[j];
            const float rl = __fmul_rd(r, 1.0f - eta), rh = __fmul_ru(r, 1.0f + 2.0f * eta);
            const float D2 = __fmul_ru(2.0f, D);
            lo = __fsqrt_rd(fmaxf(__fsub_rd(__fmul_rd(rl, rl), D2), 0.0f));
            hi = __fsqrt_ru(__fadd_ru(__fmul_ru(rh, rh), D2));
        } else {
            const float h2 = __uint_as_float((uint32_t)((unsigned long long)pq[j].x >> 32));
            lo = fmaxf(__fsub_rd(__fsqrt_rd(fmaxf(__fsub_rd(h2, D), 0.0f)), e), 0.0f);
            hi = __fadd_ru(__fsqrt_ru(__fadd_ru(h2, D)), e);
        }
        hik[j] = __float_as_uint(hi);   // non-negative: bit order is value order
        lov[j] = lo;
    }
    __syncthreads();
    const int kp = k < n_sel ? k : n_sel;
    const float tau = __uint_as_float(block_kth(hik, n_sel, kp, hist, sh));
    // the band, in slot order
    int base = 0;
    for (int j0 = 0; j0 < n_sel; j0 += kBT) {
        const int j = j0 + tid;
        const int in = j < n_sel && lov[j] <= tau;
        int tot;
        const int pos = block_excl_scan<kBT>(in, sh, &tot);
        if (in) band[(int64_t)q * C + base + pos] = j;
        base += tot;
    }
    if (tid == 0) band_n[q] = base;
}

// direct FP32 Hausdorff value of every band member
__global__ void __launch_bounds__(kBT)
k_band_exact(const float *__restrict__ qvec, const int64_t *__restrict__ qoff,
             const float *__restrict__ vec, const int64_t *__restrict__ set_off, int d,
             const int32_t *__restrict__ cand, int C, const int32_t *__restrict__ band,
             const int32_t *__restrict__ band_n, float *__restrict__ cand_dist) {
    __shared__ float sm[2 * kTile * kTP + BVSS_MAX_QSET + kTile + 2];
    const int q = blockIdx.y;
    const int nb = band_n[q];
    const int64_t a0 = qoff[q];
    const int mq = (int)(qoff[q + 1] - a0);
    for (int t = blockIdx.x; t < nb; t += gridDim.x) {
        const int j = band[(int64_t)q * C + t];
        const int64_t id = cand[(int64_t)q * C + j];
        const int64_t r0 = set_off[id];
        const int mv = (int)(set_off[id + 1] - r0);
        const float h = haus_exact<float>(qvec + a0 * d, mq, vec + r0 * d, mv, d, sm);
        if (threadIdx.x == 0) cand_dist[(int64_t)q * C + j] = h;
    }
}

// Bytes of k_band_order's dynamic shared memory: the FP64 pair tiles, S's values
// (double), sort keys (uint64) and slots (int), and one radix-select key per candidate.
__host__ __device__ inline size_t order_smem(int C) {
    return sizeof(double) * (2 * kTile * kTP + BVSS_MAX_QSET + kTile + 2) +
           (sizeof(double) + sizeof(unsigned long long) + sizeof(int)) * kMaxS +
           sizeof(uint32_t) * (size_t)C;
}

// per query set: S, FP64 where FP32 cannot order, the k' smallest (value, id)
__global__ void __launch_bounds__(kBT)
k_band_order(const float *__restrict__ qvec, const int64_t *__restrict__ qoff,
             const float *__restrict__ vec, const int64_t *__restrict__ set_off, int d,
             const int32_t *__restrict__ cand, const int32_t *__restrict__ thr, int C, int k,
             const int32_t *__restrict__ band, const int32_t *__restrict__ band_n,
             float *__restrict__ cand_dist, int64_t *__restrict__ out_ids,
             float *__restrict__ out_dist, int *__restrict__ err) {
    extern __shared__ double osm[];
    double *hsm = osm;                                        // haus_exact<double> tiles
    double *sval = hsm + (2 * kTile * kTP + BVSS_MAX_QSET + kTile + 2);
    unsigned long long *skey = reinterpret_cast<unsigned long long *>(sval + kMaxS);
    int *sslot = reinterpret_cast<int *>(skey + kMaxS);
    uint32_t *keys = reinterpret_cast<uint32_t *>(sslot + kMaxS);
    __shared__ int hist[256];
    __shared__ int sh[kBT / 32 + 2];
    const int q = blockIdx.x, tid = threadIdx.x;
    const int n_sel = thr[q * 4 + 3];
    const int kp = k < n_sel ? k : n_sel;
    for (int t = kp + tid; t < k; t += kBT) {
        out_ids[(int64_t)q * k + t] = -1;
        out_dist[(int64_t)q * k + t] = inf_f();
    }
    if (kp <= 0) return;
    const int nb = band_n[q];
    const int32_t *bq = band + (int64_t)q * C;
    const int32_t *cq = cand + (int64_t)q * C;
    float *cd = cand_dist + (int64_t)q * C;
    for (int t = tid; t < nb; t += kBT) keys[t] = __float_as_uint(cd[bq[t]]);
    __syncthreads();
    const float vk = __uint_as_float(block_kth(keys, nb, kp, hist, sh));
    const float eta = eta_of(d);
    const float reach = __fmul_ru(vk, 1.0f + eta);
    // S: members whose interval reaches the k'-th value, in band order
    int ns = 0;
    for (int t0 = 0; t0 < nb; t0 += kBT) {
        const int t = t0 + tid;
        float h = 0.0f;
        int in = 0;
        if (t < nb) {
            h = __uint_as_float(keys[t]);
            in = __fmul_rd(h, 1.0f - eta) <= reach;
        }
        int tot;
        const int pos = block_excl_scan<kBT>(in, sh, &tot);
        if (in && ns + pos < kMaxS) {
            skey[ns + pos] = ((unsigned long long)__float_as_uint(h) << 32) |
                             (uint32_t)cq[bq[t]];
            sslot[ns + pos] = bq[t];
        }
        ns += tot;
    }
    if (ns > kMaxS) {
        if (tid == 0) atomicOr(err, kErrBandOverflow);
        ns = kMaxS;
    }
    // sort S by (H32, id): bitonic over the next power of two, padded with the largest key
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
                        const int s = sslot[t];
                        sslot[t] = sslot[u];
                        sslot[u] = s;
                    }
                }
            }
            __syncthreads();
        }
    // neighbours that FP32 cannot order, at or above rank k': mark both (slot bit 30)
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
    const int64_t a0 = qoff[q];
    const int mq = (int)(qoff[q + 1] - a0);
    for (int t = 0; t < ns; ++t) {
        const int sl = sslot[t];   // uniform over the CTA
        if (!(sl & (1 << 30))) continue;
        const int j = sl & 0x3fffffff;
        const int64_t id = cq[j];
        const int64_t r0 = set_off[id];
        const double h = haus_exact<double>(qvec + a0 * d, mq, vec + r0 * d,
                                            (int)(set_off[id + 1] - r0), d, hsm);
        if (tid == 0) {
            sval[t] = h;
            cd[j] = (float)h;
        }
    }
    __syncthreads();
    if (tid == 0) {
        // FP64 reorders only inside runs of overlapping neighbours: insertion sort by
        // (value, id) does no work elsewhere
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

size_t band_workspace_ints(int64_t n_q, int C) { return (size_t)n_q * C + (size_t)n_q; }

cudaError_t launch_band_topk(const float *qvec, const int64_t *qoff, int n_q, int d, int form,
                             const float *stats, const float *vec, const int64_t *set_off,
                             const int32_t *cand, const int32_t *thr, int C, int k,
                             const longlong2 *pair, float *cand_dist, int32_t *band,
                             int64_t *out_ids, float *out_dist, int *err, cudaStream_t st) {
    if (n_q <= 0) return cudaSuccess;
    if (C > BVSS_MAX_C || form < 0 || form > 2 || d % 4 != 0) return cudaErrorInvalidValue;
    int32_t *band_n = band + (size_t)n_q * C;
    const size_t sel_smem = 2 * sizeof(uint32_t) * (size_t)C;
    cudaError_t e = cudaFuncSetAttribute(k_band_sel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sel_smem);
    if (e != cudaSuccess) return e;
    k_band_sel<<<n_q, kBT, sel_smem, st>>>(qvec, qoff, d, form, stats, cand_dist, pair, thr, C,
                                           k, band, band_n);
    k_band_exact<<<dim3(kExactCTAs, n_q), kBT, 0, st>>>(qvec, qoff, vec, set_off, d, cand, C,
                                                        band, band_n, cand_dist);
    const size_t ord_smem = order_smem(C);
    e = cudaFuncSetAttribute(k_band_order, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)ord_smem);
    if (e != cudaSuccess) return e;
    k_band_order<<<n_q, kBT, ord_smem, st>>>(qvec, qoff, vec, set_off, d, cand, thr, C, k, band,
                                             band_n, cand_dist, out_ids, out_dist, err);
    return cudaGetLastError();
}

// The largest vector norm of the database and the largest rounding-error norm of its
// BF16 and FP8 copies (stats[0..2]), each rounded up, read from the stored copies.
__global__ void k_round_stats(const float *__restrict__ x, int64_t n, int d,
                              const __nv_bfloat16 *__restrict__ x16,
                              const uint8_t *__restrict__ x8, const float *__restrict__ sc8,
                              float *__restrict__ stats) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const float up = 1.0f + 2.0f * eta_of(d);
    float m0 = 0.0f, m1 = 0.0f, m2 = 0.0f;
    for (int64_t v = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); v < n;
         v += warps) {
        float s = 0.0f, e16 = 0.0f, e8 = 0.0f;
        const float sc = x8 ? sc8[v] : 1.0f;
        for (int k = lane; k < d; k += 32) {
            const float a = x[v * d + k];
            s = fmaf(a, a, s);
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
        }
        m0 = fmaxf(m0, __fmul_ru(__fsqrt_ru(s), up));
        m1 = fmaxf(m1, __fmul_ru(__fsqrt_ru(e16), up));
        m2 = fmaxf(m2, __fmul_ru(__fsqrt_ru(e8), up));
    }
    if (lane == 0) {
        atomicMax(reinterpret_cast<unsigned *>(&stats[0]), __float_as_uint(m0));
        atomicMax(reinterpret_cast<unsigned *>(&stats[1]), __float_as_uint(m1));
        atomicMax(reinterpret_cast<unsigned *>(&stats[2]), __float_as_uint(m2));
    }
}

cudaError_t launch_round_stats(const float *x, int64_t n, int d, const __nv_bfloat16 *x16,
                               const uint8_t *x8, const float *sc8, float *stats,
                               cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(stats, 0, 4 * sizeof(float), st);
    if (e != cudaSuccess || n <= 0) return e;
    int64_t g = (n + 7) / 8;
    if (g > 152 * 16) g = 152 * 16;
    k_round_stats<<<(unsigned)g, 256, 0, st>>>(x, n, d, x16, x8, sc8, stats);
    return cudaGetLastError();
}

}  // namespace bvss
