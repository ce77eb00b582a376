// scan.cu -- both filter layers of Alg. 6 (arXiv 2412.03301) over every set
// of the database for a batch of query sets.
//
// Layer 1 (lines 5-9): set i is in F1 when C_i[p] >= M for one of the A
// positions p in P.  The inverted lists of Def. 9 are held as bit planes
// (row p, bit i = [C_i[p] >= M]), so F1 for 32 consecutive sets is the OR of
// A plane words.  Layer 2 (line 12): h_i = popcount(S_Q xor S_i).
//
// Each CTA stages a tile of 32 consecutive sketches (32 x m/8 bytes) in shared
// memory once and scores it against every query of the batch (one warp per
// query at a time; one set per warp step, lanes across the sketch words), so
// the sketch matrix is read from HBM once per batch and the kernel is bound
// by the popcount rate.  Output h[q][i] (uint16), 0xFFFF for sets outside F1.
#include "bvss_internal.cuh"

namespace bvss {

namespace {

constexpr int kScanThreads = 256;

__device__ __forceinline__ uint32_t popc_xor(uint4 a, uint4 b) {
    return __popc(a.x ^ b.x) + __popc(a.y ^ b.y) + __popc(a.z ^ b.z) + __popc(a.w ^ b.w);
}

// CH = ceil(G / 32) uint4 chunks per lane, G = m / 128 uint4 per sketch
template <int CH>
__global__ void __launch_bounds__(kScanThreads)
k_scan(const uint4 *__restrict__ sk4, int64_t n_sets, int G,
       const uint32_t *__restrict__ plane, int64_t NW, int gate_mode,
       const uint4 *__restrict__ sq4, const uint16_t *__restrict__ plist, int A, int n_q,
       uint16_t *__restrict__ h, int64_t hs) {
    extern __shared__ uint4 tile[];   // 32 x G
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t n_tiles = (n_sets + 31) / 32;
    const uint4 zero = make_uint4(0, 0, 0, 0);
    for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const int64_t i0 = t * 32;
        const int valid = (int)(n_sets - i0 < 32 ? n_sets - i0 : 32);
        const uint32_t vmask = valid == 32 ? 0xffffffffu : ((1u << valid) - 1u);
        __syncthreads();   // the previous tile is no longer read
        const uint4 *src = sk4 + i0 * G;
        for (int e = threadIdx.x; e < valid * G; e += kScanThreads) tile[e] = src[e];
        __syncthreads();
        for (int q = warp; q < n_q; q += kScanThreads / 32) {
            uint32_t g;
            if (gate_mode == 1) {
                g = 0;
                for (int a = 0; a < A; ++a)
                    g |= plane[(int64_t)plist[(int64_t)q * A + a] * NW + t];
            } else {
                g = gate_mode == 0 ? 0xffffffffu : 0u;
            }
            g &= vmask;
            uint4 qv[CH];
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const int k = lane + 32 * c;
                qv[c] = k < G ? sq4[(int64_t)q * G + k] : zero;
            }
            uint32_t myh = kGatedOut;
            uint32_t rem = g;
            while (rem) {
                const int s = __ffs(rem) - 1;
                rem &= rem - 1;
                uint32_t cnt = 0;
#pragma unroll
                for (int c = 0; c < CH; ++c) {
                    const int k = lane + 32 * c;
                    const uint4 x = k < G ? tile[s * G + k] : zero;
                    cnt += popc_xor(x, qv[c]);
                }
                cnt = __reduce_add_sync(0xffffffffu, cnt);
                if (lane == s) myh = cnt;
            }
            if (lane < valid) h[(int64_t)q * hs + i0 + lane] = (uint16_t)myh;
        }
    }
}

int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
            n = 1;
    }
    return n;
}

template <int CH>
cudaError_t launch_scan_t(const uint32_t *sketch, int64_t n_sets, int W, const uint32_t *plane,
                          int64_t NW, int gate_mode, const uint32_t *sq, const uint16_t *plist,
                          int A, int n_q, uint16_t *h, int64_t hs, cudaStream_t st) {
    const int G = W / 4;
    const size_t smem = sizeof(uint4) * 32 * (size_t)G;
    cudaError_t e = cudaFuncSetAttribute(k_scan<CH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scan<CH>, kScanThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const int64_t n_tiles = (n_sets + 31) / 32;
    int64_t grid = (int64_t)sm_count() * per_sm;
    if (grid > n_tiles) grid = n_tiles;
    k_scan<CH><<<(unsigned)grid, kScanThreads, smem, st>>>(
        reinterpret_cast<const uint4 *>(sketch), n_sets, G, plane, NW, gate_mode,
        reinterpret_cast<const uint4 *>(sq), plist, A, n_q, h, hs);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_scan(const uint32_t *sketch, int64_t n_sets, int W, const uint32_t *plane,
                        int64_t NW, int gate_mode, const uint32_t *sq, const uint16_t *plist,
                        int A, int n_q, uint16_t *h, int64_t hs, cudaStream_t st) {
    if (n_q <= 0 || n_sets <= 0) return cudaSuccess;
    const int G = W / 4;
    const int CH = (G + 31) / 32;
    switch (CH) {
        case 1: return launch_scan_t<1>(sketch, n_sets, W, plane, NW, gate_mode, sq, plist, A, n_q, h, hs, st);
        case 2: return launch_scan_t<2>(sketch, n_sets, W, plane, NW, gate_mode, sq, plist, A, n_q, h, hs, st);
        case 3: return launch_scan_t<3>(sketch, n_sets, W, plane, NW, gate_mode, sq, plist, A, n_q, h, hs, st);
        case 4: return launch_scan_t<4>(sketch, n_sets, W, plane, NW, gate_mode, sq, plist, A, n_q, h, hs, st);
        case 5: return launch_scan_t<5>(sketch, n_sets, W, plane, NW, gate_mode, sq, plist, A, n_q, h, hs, st);
        case 6: return launch_scan_t<6>(sketch, n_sets, W, plane, NW, gate_mode, sq, plist, A, n_q, h, hs, st);
        case 7: return launch_scan_t<7>(sketch, n_sets, W, plane, NW, gate_mode, sq, plist, A, n_q, h, hs, st);
        case 8: return launch_scan_t<8>(sketch, n_sets, W, plane, NW, gate_mode, sq, plist, A, n_q, h, hs, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace bvss
