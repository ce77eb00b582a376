// encode.cu -- FlyHash encoder (Def. 7, Alg. 1) and the query-side filters
// of Alg. 6 (lines 1-4) for the BioVSS++ query path of arXiv 2412.03301.
//
// k_encode: one CTA per vector.  The vector is staged in shared memory, each
// output j sums the F input dims listed in row j of the sparse binary
// projection W (FP32 adds in row order, starting from +0.0), and the
// winner-take-all keeps the L largest activations under the strict order
// (value desc, index asc).  The L-th largest key is found exactly by a
// three-pass MSB-first radix select over order-preserving uint32 keys
// (11 + 11 + 10 bits); ties at that key are taken in index order.
#include "block_util.cuh"
#include "bvss_internal.cuh"

namespace bvss {

namespace {

constexpr int kEncThreads = 128;   // divides every valid m (m % 128 == 0)

template <int THREADS>
__global__ void __launch_bounds__(THREADS)
k_encode(const float *__restrict__ x, int64_t n, const int64_t *__restrict__ n_dev, int d,
         int dpad, const uint16_t *__restrict__ proj, int m, int F, int L,
         uint16_t *__restrict__ pos, uint32_t *__restrict__ mask) {
    extern __shared__ uint32_t sm[];
    float *xs = reinterpret_cast<float *>(sm);       // dpad floats
    uint32_t *key = sm + dpad;                       // m keys
    uint32_t *hist = key + m;                        // 2048 bins
    uint32_t *mw = hist + 2048;                      // m/32 code words
    __shared__ int scan_sh[THREADS / 32 + 1];
    __shared__ uint32_t sel_digit;
    __shared__ int sel_need;

    const int tid = threadIdx.x;
    const int W = m >> 5;
    if (n_dev && *n_dev < n) n = *n_dev;   // the vector count, when it lives on the device
    for (int64_t v = blockIdx.x; v < n; v += gridDim.x) {
        const float *xv = x + v * (int64_t)d;
        for (int k = tid; k < d; k += THREADS) xs[k] = xv[k];
        __syncthreads();

        // activations a_j (Def. 7: W v with W sparse binary), as sortable keys
        if (F == 8) {
            for (int j = tid; j < m; j += THREADS) {
                const uint4 r = *reinterpret_cast<const uint4 *>(proj + (int64_t)j * 8);
                const uint32_t w4[4] = {r.x, r.y, r.z, r.w};
                float a = 0.0f;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    a = __fadd_rn(a, xs[w4[t] & 0xFFFFu]);
                    a = __fadd_rn(a, xs[w4[t] >> 16]);
                }
                key[j] = order_key(a);
            }
        } else {
            for (int j = tid; j < m; j += THREADS) {
                const uint16_t *row = proj + (int64_t)j * F;
                float a = 0.0f;
                for (int t = 0; t < F; ++t) a = __fadd_rn(a, xs[row[t]]);
                key[j] = order_key(a);
            }
        }

        // exact L-th largest key: radix select, most significant digit first
        uint32_t prefix = 0, pmask = 0;
        int need = L;
#pragma unroll 1
        for (int pass = 0; pass < 3; ++pass) {
            const int shift = pass == 0 ? 21 : (pass == 1 ? 10 : 0);
            const int nb = pass == 2 ? 1024 : 2048;
            for (int b = tid; b < nb; b += THREADS) hist[b] = 0;
            __syncthreads();
            for (int j = tid; j < m; j += THREADS) {
                const uint32_t k = key[j];
                if ((k & pmask) == prefix) atomicAdd(&hist[(k >> shift) & (nb - 1)], 1u);
            }
            __syncthreads();
            const int B = nb / THREADS;          // bins owned by this thread
            int s = 0;
            for (int b = 0; b < B; ++b) s += (int)hist[tid * B + b];
            int tot;
            const int excl = block_excl_scan<THREADS>(s, scan_sh, &tot);
            const int above = tot - excl - s;    // keys in higher bins
            if (above < need && above + s >= need) {
                int cum = above;
                for (int b = B - 1; b >= 0; --b) {
                    const int c = (int)hist[tid * B + b];
                    if (cum + c >= need) {
                        sel_digit = (uint32_t)(tid * B + b);
                        sel_need = need - cum;
                        break;
                    }
                    cum += c;
                }
            }
            __syncthreads();
            prefix |= sel_digit << shift;
            pmask |= (uint32_t)(nb - 1) << shift;
            need = sel_need;
        }
        const uint32_t T = prefix;                 // key of the L-th winner
        const int n_eq = (int)hist[T & 1023u];     // keys equal to T
        const bool all_ties = (need == n_eq);

        // code bits: 32 consecutive outputs per warp
        for (int j = tid; j < m; j += THREADS) {
            const uint32_t k = key[j];
            const bool sel = k > T || (k == T && all_ties);
            const uint32_t b = __ballot_sync(0xffffffffu, sel);
            if ((tid & 31) == 0) mw[j >> 5] = b;
        }
        __syncthreads();
        if (!all_ties) {
            // several outputs share the L-th value: lower indices win
            const int E = m / THREADS;
            const int e0 = tid * E;
            int c = 0;
            for (int j = e0; j < e0 + E; ++j) c += key[j] == T;
            int tot;
            int r = block_excl_scan<THREADS>(c, scan_sh, &tot);
            for (int j = e0; j < e0 + E && r < need; ++j) {
                if (key[j] == T) {
                    atomicOr(&mw[j >> 5], 1u << (j & 31));
                    ++r;
                }
            }
            __syncthreads();
        }

        // winner positions in ascending order
        const int WE = (W + THREADS - 1) / THREADS;
        const int w0 = tid * WE, w1 = min(W, w0 + WE);
        int c = 0;
        for (int w = w0; w < w1; ++w) c += __popc(mw[w]);
        int tot;
        int off = block_excl_scan<THREADS>(c, scan_sh, &tot);
        if (pos) {
            uint16_t *pv = pos + v * (int64_t)L;
            for (int w = w0; w < w1; ++w) {
                uint32_t b = mw[w];
                while (b) {
                    const int bit = __ffs(b) - 1;
                    b &= b - 1;
                    if (off < L) pv[off] = (uint16_t)((w << 5) + bit);
                    ++off;
                }
            }
        }
        if (mask)
            for (int w = tid; w < W; w += THREADS) mask[v * (int64_t)W + w] = mw[w];
        __syncthreads();
    }
}

template <int THREADS>
__global__ void __launch_bounds__(THREADS)
k_query_prep(const uint16_t *__restrict__ qpos, const int64_t *__restrict__ qoff, int m,
             int L, int A, uint32_t *__restrict__ sq, uint16_t *__restrict__ plist,
             int32_t *__restrict__ cq_trace) {
    extern __shared__ int32_t cnt[];   // m
    __shared__ uint32_t red[THREADS / 32];
    __shared__ uint32_t best;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int q = blockIdx.x;
    const int W = m >> 5;
    const int64_t v0 = qoff[q], v1 = qoff[q + 1];
    for (int p = tid; p < m; p += THREADS) cnt[p] = 0;
    __syncthreads();
    // C_Q = sum of the query codes (Alg. 6 line 1, Alg. 3)
    const uint16_t *src = qpos + v0 * L;
    const int64_t tot = (v1 - v0) * L;
    for (int64_t i = tid; i < tot; i += THREADS) atomicAdd(&cnt[src[i]], 1);
    __syncthreads();
    // S_Q = OR of the query codes (line 2, Alg. 5)
    for (int w = warp; w < W; w += THREADS / 32) {
        const uint32_t b = __ballot_sync(0xffffffffu, cnt[(w << 5) + lane] > 0);
        if (lane == 0) sq[(int64_t)q * W + w] = b;
    }
    if (cq_trace)
        for (int p = tid; p < m; p += THREADS) cq_trace[(int64_t)q * m + p] = cnt[p];
    // P = first A positions by (C_Q desc, position asc) (lines 3-4)
    for (int a = 0; a < A; ++a) {
        uint32_t mk = 0;
        for (int p = tid; p < m; p += THREADS) {
            const int c = cnt[p];
            const uint32_t k = c < 0 ? 0u : (((uint32_t)c << 16) | (0xFFFFu - (uint32_t)p));
            mk = max(mk, k);
        }
        mk = __reduce_max_sync(0xffffffffu, mk);
        if (lane == 0) red[warp] = mk;
        __syncthreads();
        if (warp == 0) {
            uint32_t z = lane < THREADS / 32 ? red[lane] : 0u;
            z = __reduce_max_sync(0xffffffffu, z);
            if (lane == 0) best = z;
        }
        __syncthreads();
        if (tid == 0) {
            const int p = (int)(0xFFFFu - (best & 0xFFFFu));
            plist[(int64_t)q * A + a] = (uint16_t)p;
            cnt[p] = -1;
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_encode(const float *x, int64_t n, int d, const uint16_t *proj, int m,
                          int F, int L, uint16_t *pos, uint32_t *mask, cudaStream_t st,
                          const int64_t *n_dev) {
    if (n <= 0) return cudaSuccess;
    const int dpad = (d + 3) & ~3;
    const size_t smem = sizeof(uint32_t) * ((size_t)dpad + m + 2048 + m / 32);
    auto kern = k_encode<kEncThreads>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = n < (int64_t)1 << 30 ? n : (int64_t)1 << 30;
    kern<<<(unsigned)grid, kEncThreads, smem, st>>>(x, n, n_dev, d, dpad, proj, m, F, L, pos,
                                                     mask);
    return cudaGetLastError();
}

cudaError_t launch_query_prep(const uint16_t *qpos, const int64_t *qoff, int n_q, int m,
                              int L, int A, uint32_t *sq, uint16_t *plist,
                              int32_t *cq_trace, cudaStream_t st) {
    if (n_q <= 0) return cudaSuccess;
    const size_t smem = sizeof(int32_t) * (size_t)m;
    auto kern = k_query_prep<256>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<n_q, 256, smem, st>>>(qpos, qoff, m, L, A, sq, plist, cq_trace);
    return cudaGetLastError();
}

}  // namespace bvss
