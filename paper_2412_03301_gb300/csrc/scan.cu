// scan.cu -- both filter layers of Alg. 6 (arXiv 2412.03301) over every set
// of the database for a batch of query sets.
//
// Layer 1 (lines 5-9): set i is in F1 when C_i[p] >= M for one of the A
// positions p in P.  The inverted lists of Def. 9 are held as bit planes
// (row p, bit i = [C_i[p] >= M]), so F1 for 32 consecutive sets is the OR of
// A plane words.  Layer 2 (line 12): h_i = popcount(S_Q xor S_i).
//
// Each CTA stages a tile of 128 consecutive sketches (64 or 32 for sketches
// too long for that) in shared memory once and scores it against every query
// of the batch, one warp per query at a time.  For one set the lanes split the
// sketch words (conflict-free 16-byte reads of one row), each lane XORs its
// words with the query's, which it keeps in registers, and counts bits; one
// warp reduction gives the distance.  Two gated sets are scored per loop step
// for instruction-level parallelism.  The sketch matrix is read from HBM once
// per batch.  Output h[q][i] (uint16), 0xFFFF for sets outside F1.
#include "bvss_internal.cuh"

namespace bvss {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanWarps = kScanThreads / 32;
constexpr int kMaxTileSets = 128;

__device__ __forceinline__ uint32_t popc_xor(uint4 a, uint4 b) {
    return __popc(a.x ^ b.x) + __popc(a.y ^ b.y) + __popc(a.z ^ b.z) + __popc(a.w ^ b.w);
}

// CH = ceil(G / 32) uint4 per lane, G = m / 128 uint4 per sketch, TS sets per tile
template <int CH>
__global__ void __launch_bounds__(kScanThreads)
k_scan(const uint4 *__restrict__ sk4, int64_t n_sets, int G, int TS,
       const uint32_t *__restrict__ plane, int64_t NW, int gate_mode,
       const uint4 *__restrict__ sq4, const uint16_t *__restrict__ plist, int A, int n_q,
       uint16_t *__restrict__ h, int64_t hs) {
    extern __shared__ uint4 tile[];   // TS x G
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int TW = TS / 32;
    const int64_t n_tiles = (n_sets + TS - 1) / TS;
    const uint4 zero = make_uint4(0, 0, 0, 0);
    for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const int64_t i0 = t * TS;
        const int valid = (int)(n_sets - i0 < TS ? n_sets - i0 : TS);
        __syncthreads();   // the previous tile is no longer read
        const uint4 *src = sk4 + i0 * G;
        for (int e = threadIdx.x; e < valid * G; e += kScanThreads) tile[e] = src[e];
        __syncthreads();
        for (int q = warp; q < n_q; q += kScanWarps) {
            uint4 qv[CH];
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const int k = lane + 32 * c;
                qv[c] = k < G ? sq4[(int64_t)q * G + k] : zero;
            }
            const uint16_t *pl = plist + (int64_t)q * A;
            for (int w = 0; w < TW; ++w) {
                const int64_t wi = t * TW + w;
                uint32_t g;
                if (gate_mode == 1) {
                    g = 0;
                    if (wi < NW)
                        for (int a = 0; a < A; ++a) g |= plane[(int64_t)pl[a] * NW + wi];
                } else {
                    g = gate_mode == 0 ? 0xffffffffu : 0u;
                }
                const int nv = valid - 32 * w;
                if (nv <= 0) break;
                g &= nv >= 32 ? 0xffffffffu : ((1u << nv) - 1u);
                uint32_t myh = kGatedOut;
                while (g) {
                    const int s0 = __ffs(g) - 1;
                    g &= g - 1;
                    const bool two = g != 0;
                    const int s1 = two ? __ffs(g) - 1 : s0;
                    if (two) g &= g - 1;
                    const uint4 *r0 = tile + (32 * w + s0) * G;
                    const uint4 *r1 = tile + (32 * w + s1) * G;
                    uint32_t c0 = 0, c1 = 0;
#pragma unroll
                    for (int c = 0; c < CH; ++c) {
                        const int k = lane + 32 * c;
                        const uint4 x0 = k < G ? r0[k] : zero;
                        const uint4 x1 = k < G ? r1[k] : zero;
                        c0 += popc_xor(x0, qv[c]);
                        c1 += popc_xor(x1, qv[c]);
                    }
                    c0 = __reduce_add_sync(0xffffffffu, c0);
                    c1 = __reduce_add_sync(0xffffffffu, c1);
                    if (lane == s0) myh = c0;
                    if (two && lane == s1) myh = c1;
                }
                if (lane < nv) h[(int64_t)q * hs + i0 + 32 * w + lane] = (uint16_t)myh;
            }
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
cudaError_t launch_scan_t(const uint32_t *sketch, int64_t n_sets, int G, const uint32_t *plane,
                          int64_t NW, int gate_mode, const uint32_t *sq, const uint16_t *plist,
                          int A, int n_q, uint16_t *h, int64_t hs, cudaStream_t st) {
    // the largest tile (128, 64 or 32 sets) whose sketches fit in shared memory
    int TS = kMaxTileSets;
    while (TS > 32 && sizeof(uint4) * (size_t)TS * G > 200 * 1024) TS /= 2;
    const size_t smem = sizeof(uint4) * (size_t)TS * G;
    cudaError_t e = cudaFuncSetAttribute(k_scan<CH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scan<CH>, kScanThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int64_t n_tiles = (n_sets + TS - 1) / TS;
    int64_t grid = (int64_t)sm_count() * per_sm;
    if (grid > n_tiles) grid = n_tiles;
    k_scan<CH><<<(unsigned)grid, kScanThreads, smem, st>>>(
        reinterpret_cast<const uint4 *>(sketch), n_sets, G, TS, plane, NW, gate_mode,
        reinterpret_cast<const uint4 *>(sq), plist, A, n_q, h, hs);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_scan(const uint32_t *sketch, int64_t n_sets, int W, const uint32_t *plane,
                        int64_t NW, int gate_mode, const uint32_t *sq, const uint16_t *plist,
                        int A, int n_q, uint16_t *h, int64_t hs, cudaStream_t st) {
    if (n_q <= 0 || n_sets <= 0) return cudaSuccess;
    const int G = W / 4;
    switch ((G + 31) / 32) {
        case 1: return launch_scan_t<1>(sketch, n_sets, G, plane, NW, gate_mode, sq, plist, A, n_q, h, hs, st);
        case 2: return launch_scan_t<2>(sketch, n_sets, G, plane, NW, gate_mode, sq, plist, A, n_q, h, hs, st);
        case 3: return launch_scan_t<3>(sketch, n_sets, G, plane, NW, gate_mode, sq, plist, A, n_q, h, hs, st);
        case 4: return launch_scan_t<4>(sketch, n_sets, G, plane, NW, gate_mode, sq, plist, A, n_q, h, hs, st);
        case 5: return launch_scan_t<5>(sketch, n_sets, G, plane, NW, gate_mode, sq, plist, A, n_q, h, hs, st);
        case 6: return launch_scan_t<6>(sketch, n_sets, G, plane, NW, gate_mode, sq, plist, A, n_q, h, hs, st);
        case 7: return launch_scan_t<7>(sketch, n_sets, G, plane, NW, gate_mode, sq, plist, A, n_q, h, hs, st);
        case 8: return launch_scan_t<8>(sketch, n_sets, G, plane, NW, gate_mode, sq, plist, A, n_q, h, hs, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace bvss
