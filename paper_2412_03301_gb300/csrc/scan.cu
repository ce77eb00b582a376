// scan.cu -- both filter layers of Alg. 6 (arXiv 2412.03301) over every set
// of the database for a batch of query sets.
//
// Layer 1 (lines 5-9): set i is in F1 when C_i[p] >= M for one of the A
// positions p in P.  The inverted lists of Def. 9 are held as bit planes
// (row p, bit i = [C_i[p] >= M]), so F1 for 32 consecutive sets is the OR of
// A plane words; k_gate writes that word once per (query, 32-set tile).
// Layer 2 (line 12): h_i = popcount(S_Q xor S_i).
//
// Each CTA of k_scan stages a tile of 32 consecutive sketches (32 x m/8 bytes)
// in shared memory once and scores it against every query of the batch (one
// warp per query at a time, lanes across the sketch words), so the sketch
// matrix is read from HBM once per batch and the kernel is bound by the
// popcount rate.  Two gated sets share one warp reduction (their partial
// counts packed in the halves of a word; a count is at most m <= 32768), and
// the next query's gate word and sketch are loaded while the current one is
// scored.  Output h[q][i] (uint16), 0xFFFF for sets outside F1.
#include "bvss_internal.cuh"

namespace bvss {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanWarps = kScanThreads / 32;

__device__ __forceinline__ uint32_t popc_xor(uint4 a, uint4 b) {
    return __popc(a.x ^ b.x) + __popc(a.y ^ b.y) + __popc(a.z ^ b.z) + __popc(a.w ^ b.w);
}

// gate[q][t] = OR over the A positions of plane word t (layer 1 for sets 32t..32t+31)
__global__ void k_gate(const uint32_t *__restrict__ plane, int64_t NW,
                       const uint16_t *__restrict__ plist, int A, int n_q,
                       uint32_t *__restrict__ gate) {
    const int64_t total = (int64_t)n_q * NW;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = e / NW, t = e - q * NW;
        uint32_t g = 0;
        for (int a = 0; a < A; ++a) g |= plane[(int64_t)plist[q * A + a] * NW + t];
        gate[e] = g;
    }
}

// CH = ceil(G / 32) uint4 chunks per lane, G = m / 128 uint4 per sketch;
// FULL when G == 32 * CH (no lane runs past the sketch)
template <int CH, bool FULL>
__global__ void __launch_bounds__(kScanThreads, CH == 1 ? 6 : 1)
k_scan(const uint4 *__restrict__ sk4, int64_t n_sets, int G,
       const uint32_t *__restrict__ gate, int64_t NW, int gate_mode,
       const uint4 *__restrict__ sq4, int n_q, uint16_t *__restrict__ h, int64_t hs) {
    extern __shared__ uint4 tile[];   // 32 x G
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t n_tiles = (n_sets + 31) / 32;
    const uint4 zero = make_uint4(0, 0, 0, 0);
    const uint32_t g_const = gate_mode == 0 ? 0xffffffffu : 0u;
    auto load_q = [&](int q, int64_t t, uint32_t &g, uint4 (&qv)[CH]) {
        g = gate_mode == 1 ? gate[(int64_t)q * NW + t] : g_const;
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const int k = lane + 32 * c;
            qv[c] = (FULL || k < G) ? sq4[(int64_t)q * G + k] : zero;
        }
    };
    for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const int64_t i0 = t * 32;
        const int valid = (int)(n_sets - i0 < 32 ? n_sets - i0 : 32);
        const uint32_t vmask = valid == 32 ? 0xffffffffu : ((1u << valid) - 1u);
        __syncthreads();   // the previous tile is no longer read
        const uint4 *src = sk4 + i0 * G;
        for (int e = threadIdx.x; e < valid * G; e += kScanThreads) tile[e] = src[e];
        uint32_t g_n = 0;
        uint4 qv_n[CH];
        if (warp < n_q) load_q(warp, t, g_n, qv_n);
        __syncthreads();
        for (int q = warp; q < n_q; q += kScanWarps) {
            const uint32_t g = g_n & vmask;
            uint4 qv[CH];
#pragma unroll
            for (int c = 0; c < CH; ++c) qv[c] = qv_n[c];
            if (q + kScanWarps < n_q) load_q(q + kScanWarps, t, g_n, qv_n);
            uint32_t myh = kGatedOut;
            uint32_t rem = g;
            while (rem) {
                const int s1 = __ffs(rem) - 1;
                rem &= rem - 1;
                int s2 = s1;
                if (rem) {
                    s2 = __ffs(rem) - 1;
                    rem &= rem - 1;
                }
                uint32_t c1 = 0, c2 = 0;
#pragma unroll
                for (int c = 0; c < CH; ++c) {
                    const int k = lane + 32 * c;
                    const uint4 x1 = (FULL || k < G) ? tile[s1 * G + k] : zero;
                    const uint4 x2 = (FULL || k < G) ? tile[s2 * G + k] : zero;
                    c1 += popc_xor(x1, qv[c]);
                    c2 += popc_xor(x2, qv[c]);
                }
                const uint32_t tot = __reduce_add_sync(0xffffffffu, c1 | (c2 << 16));
                if (lane == s1) myh = tot & 0xffffu;
                if (lane == s2) myh = tot >> 16;
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

template <int CH, bool FULL>
cudaError_t launch_scan_t(const uint32_t *sketch, int64_t n_sets, int W, const uint32_t *gate,
                          int64_t NW, int gate_mode, const uint32_t *sq, int n_q, uint16_t *h,
                          int64_t hs, cudaStream_t st) {
    const int G = W / 4;
    const size_t smem = sizeof(uint4) * 32 * (size_t)G;
    cudaError_t e = cudaFuncSetAttribute(k_scan<CH, FULL>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scan<CH, FULL>, kScanThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const int64_t n_tiles = (n_sets + 31) / 32;
    int64_t grid = (int64_t)sm_count() * per_sm;
    if (grid > n_tiles) grid = n_tiles;
    k_scan<CH, FULL><<<(unsigned)grid, kScanThreads, smem, st>>>(
        reinterpret_cast<const uint4 *>(sketch), n_sets, G, gate, NW, gate_mode,
        reinterpret_cast<const uint4 *>(sq), n_q, h, hs);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gate(const uint32_t *plane, int64_t NW, const uint16_t *plist, int A, int n_q,
                        uint32_t *gate, cudaStream_t st) {
    if (n_q <= 0 || NW <= 0) return cudaSuccess;
    const int64_t total = (int64_t)n_q * NW;
    int64_t g = (total + 255) / 256;
    if (g > (int64_t)sm_count() * 16) g = (int64_t)sm_count() * 16;
    k_gate<<<(unsigned)g, 256, 0, st>>>(plane, NW, plist, A, n_q, gate);
    return cudaGetLastError();
}

cudaError_t launch_scan(const uint32_t *sketch, int64_t n_sets, int W, const uint32_t *gate,
                        int64_t NW, int gate_mode, const uint32_t *sq, int n_q, uint16_t *h,
                        int64_t hs, cudaStream_t st) {
    if (n_q <= 0 || n_sets <= 0) return cudaSuccess;
    const int G = W / 4;
    const int CH = (G + 31) / 32;
    const bool full = G == 32 * CH;
#define BVSS_SCAN_CASE(n)                                                                      \
    case n:                                                                                    \
        return full ? launch_scan_t<n, true>(sketch, n_sets, W, gate, NW, gate_mode, sq, n_q,  \
                                             h, hs, st)                                        \
                    : launch_scan_t<n, false>(sketch, n_sets, W, gate, NW, gate_mode, sq, n_q, \
                                              h, hs, st);
    switch (CH) {
        BVSS_SCAN_CASE(1)
        BVSS_SCAN_CASE(2)
        BVSS_SCAN_CASE(3)
        BVSS_SCAN_CASE(4)
        BVSS_SCAN_CASE(5)
        BVSS_SCAN_CASE(6)
        BVSS_SCAN_CASE(7)
        BVSS_SCAN_CASE(8)
        default: return cudaErrorInvalidValue;
    }
#undef BVSS_SCAN_CASE
}

}  // namespace bvss
