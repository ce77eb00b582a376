// refine.cu -- exact re-rank of Alg. 6 (lines 19-23) of arXiv 2412.03301:
// Hausdorff distance (Def. 4) between the query set and each candidate set,
// then the k smallest (distance, id).
//
// k_refine: one warp per candidate, lanes over the query vectors (32 per
// chunk), candidate rows streamed 8 at a time as warp-uniform (broadcast)
// loads.  Squared distances use the GEMM form |q|^2 + |v|^2 - 2 q.v in FP32
// with precomputed norms; the row-min / column-max reductions pick the pair
// that attains the Hausdorff value, and that single pair is re-scored
// directly as sum((q - v)^2) in FP32 before the square root.  (On inputs that
// are multiples of 2^-8 every one of these FP32 sums is exact.)
#include "bvss_internal.cuh"

namespace bvss {

namespace {

constexpr int kRefThreads = 256;
constexpr int kRefWarps = kRefThreads / 32;
constexpr int kRows = 8;
constexpr int kMaxAChunks = BVSS_MAX_QSET / 32;

__global__ void __launch_bounds__(kRefThreads)
k_refine(const float *__restrict__ qvec, const int64_t *__restrict__ qoff,
         const float *__restrict__ vec, const float *__restrict__ vnorm,
         const int64_t *__restrict__ set_off, int d, int staged,
         const int32_t *__restrict__ cand, const int32_t *__restrict__ thr, int C,
         float *__restrict__ cand_dist) {
    extern __shared__ float smem[];
    const int q = blockIdx.y;
    const int n_sel = thr[q * 4 + 3];
    if (blockIdx.x * kRefWarps >= n_sel) return;   // uniform over the CTA
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t a0 = qoff[q];
    const int mq = (int)(qoff[q + 1] - a0);
    const int d4 = d / 4;
    // query rows: staged in shared memory (rows padded by 4 floats to spread
    // banks) or read in place from global memory
    const int dp = staged ? d + 4 : d;
    float *qn = smem;                                  // mq norms
    const float *qbase;
    if (staged) {
        float *qs = smem + BVSS_MAX_QSET;
        for (int e = tid; e < mq * d4; e += kRefThreads) {
            const int r = e / d4, c = e % d4;
            reinterpret_cast<float4 *>(qs + (size_t)r * dp)[c] =
                reinterpret_cast<const float4 *>(qvec + (a0 + r) * d)[c];
        }
        qbase = qs;
    } else {
        qbase = qvec + a0 * d;
    }
    for (int a = warp; a < mq; a += kRefWarps) {
        const float4 *row = reinterpret_cast<const float4 *>(qvec + (a0 + a) * d);
        float s = 0.0f;
        for (int k = lane; k < d4; k += 32) {
            const float4 t = row[k];
            s = fmaf(t.x, t.x, s);
            s = fmaf(t.y, t.y, s);
            s = fmaf(t.z, t.z, s);
            s = fmaf(t.w, t.w, s);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) qn[a] = s;
    }
    __syncthreads();

    const int nac = (mq + 31) / 32;
    const float INF = __int_as_float(0x7f800000);
    for (int c = blockIdx.x * kRefWarps + warp; c < n_sel; c += gridDim.x * kRefWarps) {
        const int64_t i = cand[(int64_t)q * C + c];
        const int64_t r0 = set_off[i], r1 = set_off[i + 1];
        float rmin[kMaxAChunks];
        int rarg[kMaxAChunks];
#pragma unroll
        for (int ac = 0; ac < kMaxAChunks; ++ac) {
            rmin[ac] = INF;
            rarg[ac] = 0;
        }
        float cmax = -1.0f;
        int cmax_r = 0, cmax_a = 0;
        for (int64_t rb = r0; rb < r1; rb += kRows) {
            const int nr = (int)(r1 - rb < kRows ? r1 - rb : kRows);
            float cmin[kRows];
            int carg[kRows];
#pragma unroll
            for (int r = 0; r < kRows; ++r) {
                cmin[r] = INF;
                carg[r] = 0;
            }
#pragma unroll
            for (int ac = 0; ac < kMaxAChunks; ++ac) {
                if (ac >= nac) break;
                const int a = ac * 32 + lane;
                const bool va = a < mq;
                const float *qa = qbase + (size_t)(va ? a : 0) * dp;
                float acc[kRows];
#pragma unroll
                for (int r = 0; r < kRows; ++r) acc[r] = 0.0f;
                for (int k = 0; k < d; k += 4) {
                    const float4 qv = *reinterpret_cast<const float4 *>(qa + k);
#pragma unroll
                    for (int r = 0; r < kRows; ++r) {
                        if (r < nr) {
                            const float4 vv =
                                __ldg(reinterpret_cast<const float4 *>(vec + (rb + r) * d + k));
                            acc[r] = fmaf(qv.x, vv.x, acc[r]);
                            acc[r] = fmaf(qv.y, vv.y, acc[r]);
                            acc[r] = fmaf(qv.z, vv.z, acc[r]);
                            acc[r] = fmaf(qv.w, vv.w, acc[r]);
                        }
                    }
                }
                const float qna = va ? qn[a] : 0.0f;
#pragma unroll
                for (int r = 0; r < kRows; ++r) {
                    if (r < nr) {
                        float d2 = qna + vnorm[rb + r] - 2.0f * acc[r];
                        d2 = d2 > 0.0f ? d2 : 0.0f;
                        if (!va) d2 = INF;
                        if (d2 < rmin[ac]) {          // min over the set's rows
                            rmin[ac] = d2;
                            rarg[ac] = (int)(rb + r - r0);
                        }
                        const uint32_t bits = __float_as_uint(d2);
                        const uint32_t mn = __reduce_min_sync(0xffffffffu, bits);
                        const uint32_t who = __ballot_sync(0xffffffffu, bits == mn);
                        const float mnf = __uint_as_float(mn);
                        if (mnf < cmin[r]) {          // min over the query's rows
                            cmin[r] = mnf;
                            carg[r] = ac * 32 + __ffs(who) - 1;
                        }
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < kRows; ++r) {
                if (r < nr && cmin[r] > cmax) {
                    cmax = cmin[r];
                    cmax_r = (int)(rb + r - r0);
                    cmax_a = carg[r];
                }
            }
        }
        // max over the query's rows of the row minima
        float rbest = -1.0f;
        int rbest_a = 0, rbest_r = 0;
#pragma unroll
        for (int ac = 0; ac < kMaxAChunks; ++ac) {
            const int a = ac * 32 + lane;
            if (ac < nac && a < mq && rmin[ac] > rbest) {
                rbest = rmin[ac];
                rbest_a = a;
                rbest_r = rarg[ac];
            }
        }
        const bool vl = lane < mq;
        const uint32_t rbits = vl ? __float_as_uint(rbest) : 0u;
        const uint32_t mb = __reduce_max_sync(0xffffffffu, rbits);
        const uint32_t who = __ballot_sync(0xffffffffu, vl && rbits == mb);
        const int src = __ffs(who) - 1;
        const int ra = __shfl_sync(0xffffffffu, rbest_a, src);
        const int rr = __shfl_sync(0xffffffffu, rbest_r, src);
        const float rowmax = __uint_as_float(mb);
        const int pa = rowmax >= cmax ? ra : cmax_a;
        const int pr = rowmax >= cmax ? rr : cmax_r;
        // direct re-score of the pair that attains the Hausdorff value
        const float4 *x4 = reinterpret_cast<const float4 *>(qvec + (a0 + pa) * d);
        const float4 *y4 = reinterpret_cast<const float4 *>(vec + (r0 + pr) * d);
        float s = 0.0f;
        for (int k = lane; k < d4; k += 32) {
            const float4 x = x4[k], y = y4[k];
            float t = x.x - y.x;
            s = fmaf(t, t, s);
            t = x.y - y.y;
            s = fmaf(t, t, s);
            t = x.z - y.z;
            s = fmaf(t, t, s);
            t = x.w - y.w;
            s = fmaf(t, t, s);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) cand_dist[(int64_t)q * C + c] = sqrtf(s);
    }
}

}  // namespace

cudaError_t launch_refine(const float *qvec, const int64_t *qoff, int n_q, int max_mq,
                          const float *vec, const float *vnorm, const int64_t *set_off, int d,
                          const int32_t *cand, const int32_t *thr, int C, float *cand_dist,
                          cudaStream_t st) {
    if (n_q <= 0) return cudaSuccess;
    const size_t staged_bytes =
        sizeof(float) * ((size_t)BVSS_MAX_QSET + (size_t)max_mq * (d + 4));
    const int staged = staged_bytes <= 96 * 1024 ? 1 : 0;
    const size_t smem = staged ? staged_bytes : sizeof(float) * BVSS_MAX_QSET;
    cudaError_t e = cudaFuncSetAttribute(k_refine, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    // about four candidates per warp
    int gx = (C + 4 * kRefWarps - 1) / (4 * kRefWarps);
    if (gx < 1) gx = 1;
    k_refine<<<dim3(gx, n_q), kRefThreads, smem, st>>>(qvec, qoff, vec, vnorm, set_off, d, staged,
                                                        cand, thr, C, cand_dist);
    return cudaGetLastError();
}

}  // namespace bvss
