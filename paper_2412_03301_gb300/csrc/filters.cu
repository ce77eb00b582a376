// filters.cu -- per-set filters of the BioVSS++ index (arXiv 2412.03301):
// the binary Bloom filter / sketch S_i = OR of the member codes (Def. 10,
// Alg. 5) and the count Bloom filter C_i = sum of the member codes (Def. 8,
// Alg. 3), stored position-major (row p = C_.[p] over all sets), which is the
// dense form of the inverted index of Def. 9 / Alg. 4.  Also the first-layer
// gate planes, squared norms for the refine, and gathers used for exports.
#include "bvss_internal.cuh"

namespace bvss {

namespace {

__global__ void k_check_finite(const float4 *__restrict__ x, int64_t n4, int *flag) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float4 v = x[i];
        if (!(isfinite(v.x) && isfinite(v.y) && isfinite(v.z) && isfinite(v.w))) *flag = 1;
    }
}

// squared norm of every vector; one warp per vector
__global__ void k_norms(const float *__restrict__ x, int64_t n, int d, float *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t v = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); v < n;
         v += warps) {
        const float4 *row = reinterpret_cast<const float4 *>(x + v * d);
        float s = 0.0f;
        for (int k = lane; k < d / 4; k += 32) {
            const float4 t = row[k];
            s = fmaf(t.x, t.x, s);
            s = fmaf(t.y, t.y, s);
            s = fmaf(t.z, t.z, s);
            s = fmaf(t.w, t.w, s);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) out[v] = s;
    }
}

// one CTA per set: counts in shared memory, then the sketch words and the
// position-major count column (saturated at 255)
__global__ void __launch_bounds__(256)
k_build_filters(const uint16_t *__restrict__ codes, const int64_t *__restrict__ set_off,
                int64_t n_sets, int m, int L, uint32_t *__restrict__ sketch,
                uint8_t *__restrict__ count) {
    extern __shared__ uint32_t cnt[];   // m
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int W = m >> 5;
    for (int64_t i = blockIdx.x; i < n_sets; i += gridDim.x) {
        for (int p = tid; p < m; p += 256) cnt[p] = 0;
        __syncthreads();
        const int64_t v0 = set_off[i], v1 = set_off[i + 1];
        const uint16_t *src = codes + v0 * L;
        const int64_t tot = (v1 - v0) * L;
        for (int64_t e = tid; e < tot; e += 256) atomicAdd(&cnt[src[e]], 1u);
        __syncthreads();
        for (int w = warp; w < W; w += 8) {
            const uint32_t b = __ballot_sync(0xffffffffu, cnt[(w << 5) + lane] > 0);
            if (lane == 0) sketch[i * W + w] = b;
        }
        for (int p = tid; p < m; p += 256)
            count[(int64_t)p * n_sets + i] = (uint8_t)min(cnt[p], 255u);
        __syncthreads();
    }
}

// plane[p][w] bit b = (count[p][32w + b] >= M); one warp per output word
__global__ void k_gate_plane(const uint8_t *__restrict__ count, int m, int64_t n_sets,
                             int64_t NW, int M, uint32_t *__restrict__ plane) {
    const int lane = threadIdx.x & 31;
    const int64_t total = (int64_t)m * NW;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t g = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); g < total;
         g += warps) {
        const int64_t p = g / NW, w = g % NW;
        const int64_t i = w * 32 + lane;
        const bool on = i < n_sets && (int)count[p * n_sets + i] >= M;
        const uint32_t b = __ballot_sync(0xffffffffu, on);
        if (lane == 0) plane[g] = b;
    }
}

__global__ void k_gather_rows(const uint32_t *__restrict__ src, int W, int64_t n_rows,
                              const int64_t *__restrict__ ids, int64_t n,
                              uint32_t *__restrict__ out) {
    const int64_t total = n * W;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / W, w = e % W;
        const int64_t i = ids[j];
        out[e] = (i >= 0 && i < n_rows) ? src[i * W + w] : 0u;
    }
}

__global__ void k_gather_counts(const uint8_t *__restrict__ count, int m, int64_t n_sets,
                                const int64_t *__restrict__ ids, int64_t n,
                                uint8_t *__restrict__ out) {
    const int64_t total = n * m;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / m, p = e % m;
        const int64_t i = ids[j];
        out[e] = (i >= 0 && i < n_sets) ? count[p * n_sets + i] : (uint8_t)0;
    }
}

unsigned grid_for(int64_t work, int threads) {
    int64_t g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > (int64_t)1 << 20) g = (int64_t)1 << 20;
    return (unsigned)g;
}

}  // namespace

cudaError_t launch_check_finite(const float *x, int64_t n, int *flag, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int64_t n4 = n / 4;
    k_check_finite<<<grid_for(n4, 256), 256, 0, st>>>(reinterpret_cast<const float4 *>(x),
                                                       n4, flag);
    return cudaGetLastError();
}

cudaError_t launch_norms(const float *x, int64_t n, int d, float *norm, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_norms<<<grid_for(n * 32, 256), 256, 0, st>>>(x, n, d, norm);
    return cudaGetLastError();
}

cudaError_t launch_build_filters(const uint16_t *codes, const int64_t *set_off,
                                 int64_t n_sets, int m, int L, uint32_t *sketch,
                                 uint8_t *count, cudaStream_t st) {
    if (n_sets <= 0) return cudaSuccess;
    const size_t smem = sizeof(uint32_t) * (size_t)m;
    cudaError_t e = cudaFuncSetAttribute(k_build_filters,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = n_sets < (int64_t)1 << 30 ? n_sets : (int64_t)1 << 30;
    k_build_filters<<<(unsigned)grid, 256, smem, st>>>(codes, set_off, n_sets, m, L, sketch,
                                                       count);
    return cudaGetLastError();
}

cudaError_t launch_gate_plane(const uint8_t *count, int m, int64_t n_sets, int64_t NW, int M,
                              uint32_t *plane, cudaStream_t st) {
    k_gate_plane<<<grid_for((int64_t)m * NW * 32, 256), 256, 0, st>>>(count, m, n_sets, NW, M,
                                                                      plane);
    return cudaGetLastError();
}

cudaError_t launch_gather_sketches(const uint32_t *sketch, int W, int64_t n_sets,
                                   const int64_t *ids, int64_t n, uint32_t *out,
                                   cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_gather_rows<<<grid_for(n * W, 256), 256, 0, st>>>(sketch, W, n_sets, ids, n, out);
    return cudaGetLastError();
}

cudaError_t launch_gather_counts(const uint8_t *count, int m, int64_t n_sets,
                                 const int64_t *ids, int64_t n, uint8_t *out,
                                 cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_gather_counts<<<grid_for(n * m, 256), 256, 0, st>>>(count, m, n_sets, ids, n, out);
    return cudaGetLastError();
}

}  // namespace bvss
