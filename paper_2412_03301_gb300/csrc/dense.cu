// dense.cu -- the learned projection of arXiv 2412.03301 (BioHash in place of FlyHash
// in Def. 7: h = WTA(W v) with a learned dense W) and its training on neighbour pairs.
//
// k_dense_gemm: the BF16 layer a = W x for a block of vectors on the tensor cores
//   (tcgen05, FP32 accumulation in tensor memory): D (n x m) = X (n x d) W^T, tiles of
//   128 vectors x 128 outputs, K in blocks of 64 BF16 values staged by coalesced 16-byte
//   cp.async copies into the 128-byte swizzle layout (3-stage ring, copies arriving on
//   the stage's mbarrier themselves), one thread issuing the MMAs, four warps reading
//   the accumulator out of tensor memory.  The WTA of the encoder then reads the
//   activations (the block is sized to stay in L2).
// k_pair_grad: per training pair, the WTA thresholds, soft codes, loss and its gradient
//   in the activations (the threshold held fixed), as the oracle defines them.
// k_wgrad: d W = (1/n) sum_i g_x,i x_i^T + g_y,i y_i^T (register-tiled FP32).
// k_absmax, k_apply: the normalized step, the row rescaling and the 2^-8-grid BF16
//   forward weights.
// k_nearest: for pair mining, the nearest database vector of each query vector in each
//   of its query set's neighbour sets.
#include <cuda_bf16.h>

#include "block_util.cuh"
#include "bvss_internal.cuh"
#include "ptx_util.cuh"

namespace bvss {

namespace {

constexpr int kGM = 128;              // vectors per tile (MMA M, TMEM lanes)
constexpr int kGN = 128;              // outputs per tile (MMA N, TMEM columns)
constexpr int kGStages = 3;          // 99 KB of shared memory: two CTAs per SM
constexpr int kGStage = (kGM + kGN) * 128;   // one K-block of A and B: 32 KB
constexpr int kGThreads = 6 * 32;     // warps 0-3 epilogue, 4 producer, 5 MMA
constexpr uint64_t kGWaitNs = 2000000000ull;
constexpr int kGSmem = kGStages * kGStage + 1024 + 256;

// wait for a phase, or give up (error bit 4) when the limit passes or another role gave up
__device__ __forceinline__ bool gwait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                      int *err) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort_flag) return false;
        if (global_timer_ns() - t0 > kGWaitNs) {
            *abort_flag = 1;
            atomicOr(err, 4);
            return false;
        }
    }
    return true;
}

__global__ void __launch_bounds__(kGThreads, 2)
k_dense_gemm(const __nv_bfloat16 *__restrict__ X, int64_t n, int d,
             const __nv_bfloat16 *__restrict__ Wt, int m, float *__restrict__ D, int64_t ldd,
             int *__restrict__ err) {
    extern __shared__ unsigned char gsm_raw[];
    unsigned char *gsm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(gsm_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t *full = reinterpret_cast<uint64_t *>(gsm + kGStages * kGStage);
    uint64_t *empty = full + kGStages;
    uint64_t *done = empty + kGStages;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row0 = (int64_t)blockIdx.y * kGM;
    const int col0 = blockIdx.x * kGN;
    const int KB = d / 64;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kGStages; ++s) {
            mbar_init(&full[s], 32);   // one arrival per producer lane, when its copies land
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 5) tmem_alloc(tmem_slot, kGN);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    if (warp == 4) {
        // ---- producer: A rows (vectors) and B rows (outputs) of each K-block ---------
        for (int kb = 0; kb < KB; ++kb) {
            const int s = kb % kGStages;
            if (kb >= kGStages &&
                !gwait(&empty[s], (uint32_t)(((kb / kGStages) - 1) & 1), abort_flag, err))
                break;
            unsigned char *sa = gsm + s * kGStage, *sb = sa + kGM * 128;
#pragma unroll 4
            for (int e = lane; e < kGM * 8; e += 32) {
                const int r = e >> 3, c = e & 7;
                const int64_t row = row0 + r < n ? row0 + r : n - 1;   // past n: any row
                cp_async16(sa + sw128_off(r, c), X + row * d + kb * 64 + c * 8);
            }
#pragma unroll 4
            for (int e = lane; e < kGN * 8; e += 32) {
                const int r = e >> 3, c = e & 7;
                cp_async16(sb + sw128_off(r, c), Wt + (int64_t)(col0 + r) * d + kb * 64 + c * 8);
            }
            cp_async_mbar_arrive(&full[s]);
        }
        cp_async_wait<0>();
    } else if (warp == 5) {
        // ---- MMA issue: one thread ---------------------------------------------------
        if (lane == 0) {
            constexpr uint32_t idesc = umma_idesc_bf16(kGM, kGN);
            const uint32_t base = smem_u32(gsm);
            bool ok = true;
            for (int kb = 0; kb < KB && ok; ++kb) {
                const int s = kb % kGStages;
                ok = gwait(&full[s], (uint32_t)((kb / kGStages) & 1), abort_flag, err);
                if (!ok) break;
                fence_proxy_async();
                tc_fence_after();
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint64_t ad = umma_desc_sw128(base + s * kGStage + 32 * k);
                    const uint64_t bd = umma_desc_sw128(base + s * kGStage + kGM * 128 + 32 * k);
                    umma_bf16(tmem, ad, bd, idesc, (kb | k) != 0 ? 1u : 0u);
                }
                umma_commit(&empty[s]);
            }
            if (ok) umma_commit(done);
        }
    } else {
        // ---- epilogue: lane = vector, 32 outputs per tensor-memory load ---------------
        if (gwait(done, 0u, abort_flag, err)) {
            tc_fence_after();
            const int64_t row = row0 + warp * 32 + lane;
#pragma unroll 1
            for (int c = 0; c < kGN; c += 32) {
                uint32_t v[32];
                tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
                if (row < n) {
                    float4 *dst = reinterpret_cast<float4 *>(D + row * ldd + col0 + c);
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        dst[i] = make_float4(__uint_as_float(v[4 * i]), __uint_as_float(v[4 * i + 1]),
                                             __uint_as_float(v[4 * i + 2]),
                                             __uint_as_float(v[4 * i + 3]));
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 5) tmem_dealloc(tmem, kGN);
}

constexpr int kPT = 256;   // threads of the per-pair and per-row kernels

// k-th smallest (1-based) of the n keys in shared memory, by the whole CTA (kPT threads):
// radix select over four 8-bit digits.  hist: 256 ints; sh: kPT / 32 + 3 ints.
__device__ uint32_t kth_key(const uint32_t *keys, int n, int k, int *hist, int *sh) {
    uint32_t prefix = 0, mask = 0;
    for (int shift = 24; shift >= 0; shift -= 8) {
        for (int b = threadIdx.x; b < 256; b += kPT) hist[b] = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += kPT) {
            const uint32_t key = keys[i];
            if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1);
        }
        __syncthreads();
        const int c = hist[threadIdx.x];
        int tot;
        const int before = block_excl_scan<kPT>(c, sh, &tot);
        if (before < k && before + c >= k) {
            sh[kPT / 32 + 1] = threadIdx.x;
            sh[kPT / 32 + 2] = k - before;
        }
        __syncthreads();
        prefix |= (uint32_t)sh[kPT / 32 + 1] << shift;
        mask |= 0xFFu << shift;
        k = sh[kPT / 32 + 2];
        __syncthreads();
    }
    return prefix;
}

// the FP32 value of an order_key
__device__ __forceinline__ float key_value(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// one activation row's WTA threshold: midway between its L-th and (L+1)-th largest
__device__ float wta_threshold(const float *a, int m, int L, uint32_t *keys, int *hist, int *sh) {
    for (int j = threadIdx.x; j < m; j += kPT) keys[j] = order_key(a[j]);
    __syncthreads();
    const float hi = key_value(kth_key(keys, m, m - L + 1, hist, sh));   // L-th largest
    const float lo = key_value(kth_key(keys, m, m - L, hist, sh));       // (L+1)-th largest
    return 0.5f * (hi + lo);
}

__device__ __forceinline__ float sigm(float z) { return 1.0f / (1.0f + __expf(-z)); }

// per pair: soft codes, overlap, logistic loss and d loss / d a (thresholds fixed)
__global__ void __launch_bounds__(kPT)
k_pair_grad(const float *__restrict__ act_x, const float *__restrict__ act_y, int64_t lda,
            const uint8_t *__restrict__ labels, int m, int L, float T, float s, float mu,
            float *__restrict__ g_x, float *__restrict__ g_y, int64_t ldg,
            double *__restrict__ loss_sum) {
    extern __shared__ uint32_t psm[];   // m keys
    __shared__ int hist[256];
    __shared__ int sh[kPT / 32 + 3];
    __shared__ float red[kPT / 32];
    const int64_t i = blockIdx.x;
    const float *ax = act_x + i * lda, *ay = act_y + i * lda;
    const float tx = wta_threshold(ax, m, L, psm, hist, sh);
    const float ty = wta_threshold(ay, m, L, psm, hist, sh);
    const float inv_t = 1.0f / T;
    float o = 0.0f;
    for (int j = threadIdx.x; j < m; j += kPT)
        o += sigm((ax[j] - tx) * inv_t) * sigm((ay[j] - ty) * inv_t);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) o += __shfl_xor_sync(0xffffffffu, o, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = o;
    __syncthreads();
    o = 0.0f;
#pragma unroll
    for (int w = 0; w < kPT / 32; ++w) o += red[w];
    o /= (float)L;
    const float sg = labels[i] ? 1.0f : -1.0f;
    const float z = sg * s * (o - mu);
    const float dl_do = -sg * s * sigm(-z);
    for (int j = threadIdx.x; j < m; j += kPT) {
        const float cx = sigm((ax[j] - tx) * inv_t), cy = sigm((ay[j] - ty) * inv_t);
        g_x[i * ldg + j] = dl_do * (cy / L) * cx * (1.0f - cx) * inv_t;
        g_y[i * ldg + j] = dl_do * (cx / L) * cy * (1.0f - cy) * inv_t;
    }
    if (threadIdx.x == 0) {
        const double zz = z;
        atomicAdd(loss_sum, zz >= 0.0 ? log1p(exp(-zz)) : -zz + log1p(exp(zz)));
    }
}

// d W (m x d) = (1/n) sum_i g_x,i x_i^T + g_y,i y_i^T: 64 x 64 outputs per CTA, 4 x 4 per
// thread, the 2n rows of (g_x; g_y) and (x; y) in chunks of 16
constexpr int kWT = 64, kWK = 16;
__global__ void __launch_bounds__(kPT)
k_wgrad(const float *__restrict__ g_x, const float *__restrict__ g_y, int64_t ldg,
        const __nv_bfloat16 *__restrict__ x, const __nv_bfloat16 *__restrict__ y, int64_t n,
        int m, int d, float *__restrict__ dw) {
    __shared__ float As[kWK][kWT + 4];
    __shared__ float Bs[kWK][kWT + 4];
    const int j0 = blockIdx.y * kWT, k0 = blockIdx.x * kWT;
    const int tj = threadIdx.x >> 4, tk = threadIdx.x & 15;
    float acc[4][4] = {};
    for (int64_t r0 = 0; r0 < 2 * n; r0 += kWK) {
        // 16 rows x 64 columns of each operand: 4 values per thread
        for (int e = threadIdx.x; e < kWK * kWT; e += kPT) {
            const int rr = e / kWT, cc = e % kWT;
            const int64_t r = r0 + rr;
            float a = 0.0f, b = 0.0f;
            if (r < 2 * n) {
                const int64_t i = r < n ? r : r - n;
                a = (r < n ? g_x : g_y)[i * ldg + j0 + cc];
                b = __bfloat162float((r < n ? x : y)[i * d + k0 + cc]);
            }
            As[rr][cc] = a;
            Bs[rr][cc] = b;
        }
        __syncthreads();
#pragma unroll
        for (int rr = 0; rr < kWK; ++rr) {
            float av[4], bv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                av[u] = As[rr][tj * 4 + u];
                bv[u] = Bs[rr][tk * 4 + u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
        }
        __syncthreads();
    }
    const float inv_n = 1.0f / (float)n;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v)
            dw[(int64_t)(j0 + tj * 4 + u) * d + k0 + tk * 4 + v] = acc[u][v] * inv_n;
}

// the largest |d W| (non-negative: its bits order as it does)
__global__ void k_absmax(const float *__restrict__ v, int64_t n, float *__restrict__ out) {
    float mx = 0.0f;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x)
        mx = fmaxf(mx, fabsf(v[e]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<unsigned *>(out), __float_as_uint(mx));
}

// one warp per row: w <- w - eta dw / max|dw|, rescaled to row_norm; the forward weights
// are w rounded to the nearest multiple of 2^-8 (ties to even), clamped to [-1, 1]
__global__ void k_apply(float *__restrict__ w, const float *__restrict__ dw, int m, int d,
                        float eta, float row_norm, const float *__restrict__ absmax,
                        __nv_bfloat16 *__restrict__ wq) {
    const int lane = threadIdx.x & 31;
    const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j >= m) return;
    const float mx = *absmax;
    const float step = mx > 0.0f ? eta / mx : 0.0f;
    float *wr = w + (int64_t)j * d;
    const float *gr = dw + (int64_t)j * d;
    float ss = 0.0f;
    for (int k = lane; k < d; k += 32) {
        const float v = wr[k] - step * gr[k];
        wr[k] = v;
        ss = fmaf(v, v, ss);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, off);
    const float sc = ss > 0.0f ? row_norm / sqrtf(ss) : 1.0f;
    for (int k = lane; k < d; k += 32) {
        const float v = wr[k] * sc;
        wr[k] = v;
        const float q = fminf(fmaxf(rintf(v * 256.0f) * (1.0f / 256.0f), -1.0f), 1.0f);
        wq[(int64_t)j * d + k] = __float2bfloat16_rn(q);
    }
}

// For pair mining: rows[a][t] = the global row of the vector of set sets[q][t] nearest to
// query vector a of query set q (direct FP32 distance, ties to the lower row), -1 for a
// negative set id.  One CTA per query set, one warp per (query vector, neighbour).
__global__ void __launch_bounds__(kPT)
k_nearest(const float *__restrict__ qvec, const int64_t *__restrict__ qoff, int d,
          const float *__restrict__ vec, const int64_t *__restrict__ set_off, int64_t n_sets,
          const int64_t *__restrict__ sets, int k, int64_t *__restrict__ rows) {
    const int q = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t a0 = qoff[q];
    const int mq = (int)(qoff[q + 1] - a0);
    for (int u = warp; u < mq * k; u += kPT / 32) {
        const int a = u / k, t = u % k;
        const int64_t sid = sets[(int64_t)q * k + t];
        int64_t best = -1;
        if (sid >= 0 && sid < n_sets) {
            const float *qa = qvec + (a0 + a) * d;
            float bd = __int_as_float(0x7f800000);
            for (int64_t r = set_off[sid]; r < set_off[sid + 1]; ++r) {
                float ssum = 0.0f;
                for (int kk = lane; kk < d; kk += 32) {
                    const float df = qa[kk] - vec[r * d + kk];
                    ssum = fmaf(df, df, ssum);
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1)
                    ssum += __shfl_xor_sync(0xffffffffu, ssum, off);
                if (ssum < bd) {
                    bd = ssum;
                    best = r;
                }
            }
        }
        if (lane == 0) rows[(a0 + a) * k + t] = best;
    }
}

// BF16 copies of FP32 rows (rows == nullptr: rows 0..n-1 of x; else the listed rows of the
// n_src rows of x, a row id outside [0, n_src) giving a row of zeros)
__global__ void k_rows_bf16(const float *__restrict__ x, int d, const int64_t *__restrict__ rows,
                            int64_t n, int64_t n_src, __nv_bfloat16 *__restrict__ out) {
    const int64_t total = n * d;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / d, k = e - i * d;
        const int64_t r = rows ? rows[i] : i;
        out[e] = __float2bfloat16_rn(r >= 0 && r < n_src ? x[r * d + k] : 0.0f);
    }
}

}  // namespace

cudaError_t launch_dense_gemm(const __nv_bfloat16 *X, int64_t n, int d, const __nv_bfloat16 *W,
                              int m, float *D, int64_t ldd, int *err, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (d % 64 != 0 || m % kGN != 0 || ldd % 4 != 0 || ldd < m || n > ((int64_t)65535 * kGM))
        return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_dense_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kGSmem);
    if (e != cudaSuccess) return e;
    const dim3 grid(m / kGN, (unsigned)((n + kGM - 1) / kGM));
    k_dense_gemm<<<grid, kGThreads, kGSmem, st>>>(X, n, d, W, m, D, ldd, err);
    return cudaGetLastError();
}

cudaError_t launch_rows_bf16(const float *x, int d, const int64_t *rows, int64_t n,
                             __nv_bfloat16 *out, cudaStream_t st, int64_t n_src) {
    if (n <= 0) return cudaSuccess;
    int64_t g = (n * d + 255) / 256;
    if (g > 152 * 32) g = 152 * 32;
    k_rows_bf16<<<(unsigned)g, 256, 0, st>>>(x, d, rows, n, rows ? n_src : n, out);
    return cudaGetLastError();
}

cudaError_t launch_nearest(const float *qvec, const int64_t *qoff, int n_q, int d,
                           const float *vec, const int64_t *set_off, int64_t n_sets,
                           const int64_t *sets, int k, int64_t *rows, cudaStream_t st) {
    if (n_q <= 0) return cudaSuccess;
    k_nearest<<<n_q, kPT, 0, st>>>(qvec, qoff, d, vec, set_off, n_sets, sets, k, rows);
    return cudaGetLastError();
}

}  // namespace bvss

// ---------------------------------------------------------------------------
// C ABI of the learned projection (include/bvss.h)
// ---------------------------------------------------------------------------
using namespace bvss;

namespace {

// status word of the dense GEMM's bounded waits (bit 4: a wait gave up), per device
__device__ int g_dense_status;

cudaError_t dense_status_ptr(int **p) {
    return cudaGetSymbolAddress(reinterpret_cast<void **>(p), g_dense_status);
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

}  // namespace

extern "C" int bvss_dense_forward(const void *x_bf16, int64_t n, int32_t d, const void *w_bf16,
                                  int32_t m, float *act, int64_t ld_act, void *stream) {
    if (n < 0 || d < 64 || d % 64 != 0 || m < 128 || m % 128 != 0 || ld_act < m ||
        ld_act % 4 != 0)
        return record_error(BVSS_EINVAL, "bvss_dense_forward: need n >= 0, d %% 64 == 0, "
                                         "m %% 128 == 0, ld_act >= m and ld_act %% 4 == 0");
    if (n == 0) return BVSS_OK;
    if (!x_bf16 || !w_bf16 || !act || !aligned16(x_bf16) || !aligned16(w_bf16) || !aligned16(act))
        return record_error(BVSS_EINVAL, "bvss_dense_forward: pointers must be non-NULL and "
                                         "16-byte aligned");
    int *status = nullptr;
    cudaError_t e = dense_status_ptr(&status);
    if (e == cudaSuccess)
        e = launch_dense_gemm(static_cast<const __nv_bfloat16 *>(x_bf16), n, d,
                              static_cast<const __nv_bfloat16 *>(w_bf16), m, act, ld_act, status,
                              reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess)
        return record_error(BVSS_ECUDA, "bvss_dense_forward: %s", cudaGetErrorString(e));
    return BVSS_OK;
}

extern "C" int bvss_learn_sync(void *stream) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int *status = nullptr;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = dense_status_ptr(&status);
    int v = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&v, status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && v) e = cudaMemset(status, 0, sizeof(int));
    if (e != cudaSuccess) return record_error(BVSS_ECUDA, "bvss_learn_sync: %s", cudaGetErrorString(e));
    if (v) return record_error(BVSS_ETIMEOUT, "a dense-layer kernel's bounded wait gave up");
    return BVSS_OK;
}

extern "C" int bvss_learn_pair_grad(const float *act_x, const float *act_y, int64_t ld_act,
                                    const uint8_t *labels, int64_t n, int32_t m, int32_t L,
                                    float temperature, float scale, float margin, float *g_x,
                                    float *g_y, int64_t ld_g, double *loss_sum, void *stream) {
    if (n < 0 || m < 2 || L < 1 || L >= m || ld_act < m || ld_g < m || !(temperature > 0.0f))
        return record_error(BVSS_EINVAL, "bvss_learn_pair_grad: need n >= 0, 1 <= L < m, "
                                         "ld_act, ld_g >= m and temperature > 0");
    if (n == 0) return BVSS_OK;
    if (!act_x || !act_y || !labels || !g_x || !g_y || !loss_sum)
        return record_error(BVSS_EINVAL, "bvss_learn_pair_grad: NULL pointer");
    if (n > 0x7fffffffLL)
        return record_error(BVSS_EINVAL, "bvss_learn_pair_grad: at most 2^31 - 1 pairs");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t smem = sizeof(uint32_t) * (size_t)m;
    cudaError_t e = cudaFuncSetAttribute(k_pair_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e == cudaSuccess) {
        k_pair_grad<<<(unsigned)n, kPT, smem, st>>>(act_x, act_y, ld_act, labels, m, L,
                                                    temperature, scale, margin, g_x, g_y, ld_g,
                                                    loss_sum);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess)
        return record_error(BVSS_ECUDA, "bvss_learn_pair_grad: %s", cudaGetErrorString(e));
    return BVSS_OK;
}

extern "C" int bvss_learn_weight_grad(const float *g_x, const float *g_y, int64_t ld_g,
                                      const void *x_bf16, const void *y_bf16, int64_t n,
                                      int32_t m, int32_t d, float *dw, void *stream) {
    if (n < 1 || m % kWT != 0 || d % kWT != 0 || m < kWT || d < kWT || ld_g < m)
        return record_error(BVSS_EINVAL, "bvss_learn_weight_grad: need n >= 1, m and d "
                                         "multiples of 64, ld_g >= m");
    if (!g_x || !g_y || !x_bf16 || !y_bf16 || !dw)
        return record_error(BVSS_EINVAL, "bvss_learn_weight_grad: NULL pointer");
    const dim3 grid(d / kWT, m / kWT);
    k_wgrad<<<grid, kPT, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        g_x, g_y, ld_g, static_cast<const __nv_bfloat16 *>(x_bf16),
        static_cast<const __nv_bfloat16 *>(y_bf16), n, m, d, dw);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return record_error(BVSS_ECUDA, "bvss_learn_weight_grad: %s", cudaGetErrorString(e));
    return BVSS_OK;
}

extern "C" int bvss_learn_update(float *w, const float *dw, int32_t m, int32_t d, float eta,
                                 float row_norm, float *absmax, void *wq_bf16, void *stream) {
    if (m < 1 || d < 1 || !(eta >= 0.0f) || !(row_norm > 0.0f))
        return record_error(BVSS_EINVAL, "bvss_learn_update: need m, d >= 1, eta >= 0 and "
                                         "row_norm > 0");
    if (!w || !dw || !absmax || !wq_bf16)
        return record_error(BVSS_EINVAL, "bvss_learn_update: NULL pointer");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(absmax, 0, sizeof(float), st);
    if (e == cudaSuccess) {
        const int64_t tot = (int64_t)m * d;
        int64_t g = (tot + 255) / 256;
        if (g > 152 * 8) g = 152 * 8;
        k_absmax<<<(unsigned)g, 256, 0, st>>>(dw, tot, absmax);
        k_apply<<<(unsigned)((m + 7) / 8), 256, 0, st>>>(w, dw, m, d, eta, row_norm, absmax,
                                                         static_cast<__nv_bfloat16 *>(wq_bf16));
        e = cudaGetLastError();
    }
    if (e != cudaSuccess)
        return record_error(BVSS_ECUDA, "bvss_learn_update: %s", cudaGetErrorString(e));
    return BVSS_OK;
}

extern "C" int bvss_to_bf16(const float *x, int64_t n, int32_t d, void *out, void *stream) {
    if (n < 0 || d < 1) return record_error(BVSS_EINVAL, "bvss_to_bf16: need n >= 0, d >= 1");
    if (n == 0) return BVSS_OK;
    if (!x || !out) return record_error(BVSS_EINVAL, "bvss_to_bf16: NULL pointer");
    const cudaError_t e = launch_rows_bf16(x, d, nullptr, n, static_cast<__nv_bfloat16 *>(out),
                                           reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return record_error(BVSS_ECUDA, "bvss_to_bf16: %s", cudaGetErrorString(e));
    return BVSS_OK;
}
