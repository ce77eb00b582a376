// scan.cu -- both filter layers of Alg. 6 (arXiv 2412.03301) over every set
// of the database for a batch of query sets.
//
// Layer 1 (lines 5-9): set i is in F1 when C_i[p] >= M for one of the A
// positions p in P.  The inverted lists of Def. 9 are held as bit planes
// (row p, bit i = [C_i[p] >= M]), so F1 for 32 consecutive sets is the OR of
// A plane words.  Layer 2 (line 12): h_i = popcount(S_Q xor S_i).
//
// Each CTA stages a tile of 128 consecutive sketches (rows padded by 16 bytes;
// 64 or 32 sets for sketches too long for that)
// in shared memory once and scores it against every query of the batch, one
// warp per query at a time.  The gated sets of the tile are compacted onto
// the lanes, so a lane computes a whole Hamming distance (128 popcounts for
// m = 4096) on its own: no cross-lane reduction, the query sketch is read as
// a broadcast, and the kernel runs at the popcount rate.  The sketch matrix
// is read from HBM once per batch.  Output h[q][i] (uint16), 0xFFFF for sets
// outside F1, written as whole 256-byte rows.
#include "bvss_internal.cuh"

namespace bvss {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanWarps = kScanThreads / 32;
constexpr int kMaxTileSets = 128;

// G = m / 128 uint4 per sketch; rows of the staged tile have G + 1 uint4.
// TS = sets per tile (128, 64 or 32; smaller for long sketches).
__global__ void __launch_bounds__(kScanThreads)
k_scan(const uint4 *__restrict__ sk4, int64_t n_sets, int G, int TS,
       const uint32_t *__restrict__ plane, int64_t NW, int gate_mode,
       const uint4 *__restrict__ sq4, const uint16_t *__restrict__ plist, int A, int n_q,
       uint16_t *__restrict__ h, int64_t hs) {
    extern __shared__ uint4 sm4[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int RS = G + 1;
    const int TW = TS / 32;                                       // gate words per tile
    uint4 *tile = sm4;                                            // TS x RS
    uint4 *qsk = sm4 + TS * RS + warp * G;                        // this warp's query sketch
    uint16_t *hrow = reinterpret_cast<uint16_t *>(sm4 + TS * RS + kScanWarps * G) +
                     warp * TS;                                   // this warp's output row
    const int64_t n_tiles = (n_sets + TS - 1) / TS;
    for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const int64_t i0 = t * TS;
        const int valid = (int)(n_sets - i0 < TS ? n_sets - i0 : TS);
        __syncthreads();   // the previous tile is no longer read
        const uint4 *src = sk4 + i0 * G;
        for (int e = threadIdx.x; e < valid * G; e += kScanThreads) {
            const int r = e / G, c = e - (e / G) * G;
            tile[r * RS + c] = src[e];
        }
        __syncthreads();
        for (int q = warp; q < n_q; q += kScanWarps) {
            // F1 bits of the tile's sets: lane w < TW holds word w
            uint32_t gw = 0;
            if (lane < TW) {
                const int64_t wi = t * TW + lane;
                if (gate_mode == 0) {
                    gw = 0xffffffffu;
                } else if (gate_mode == 1 && wi < NW) {
                    for (int a = 0; a < A; ++a)
                        gw |= plane[(int64_t)plist[(int64_t)q * A + a] * NW + wi];
                }
                const int nv = valid - lane * 32;
                gw &= nv >= 32 ? 0xffffffffu : (nv > 0 ? (1u << nv) - 1u : 0u);
            }
            for (int c = lane; c < G; c += 32) qsk[c] = sq4[(int64_t)q * G + c];
            for (int e = lane; e < TS; e += 32) hrow[e] = kGatedOut;
            __syncwarp();
            const uint32_t w0 = __shfl_sync(0xffffffffu, gw, 0), w1 = __shfl_sync(0xffffffffu, gw, 1);
            const uint32_t w2 = __shfl_sync(0xffffffffu, gw, 2), w3 = __shfl_sync(0xffffffffu, gw, 3);
            const int c0 = __popc(w0), c1 = c0 + __popc(w1), c2 = c1 + __popc(w2);
            const int total = c2 + __popc(w3);
            for (int base = 0; base < total; base += 32) {
                const int j = base + lane;
                if (j < total) {
                    int s;
                    if (j < c0) s = (int)__fns(w0, 0, j + 1);
                    else if (j < c1) s = 32 + (int)__fns(w1, 0, j - c0 + 1);
                    else if (j < c2) s = 64 + (int)__fns(w2, 0, j - c1 + 1);
                    else s = 96 + (int)__fns(w3, 0, j - c2 + 1);
                    const uint4 *row = tile + s * RS;
                    uint32_t cnt = 0;
#pragma unroll 4
                    for (int c = 0; c < G; ++c) {
                        const uint4 x = row[c], y = qsk[c];
                        cnt += __popc(x.x ^ y.x) + __popc(x.y ^ y.y) + __popc(x.z ^ y.z) +
                               __popc(x.w ^ y.w);
                    }
                    hrow[s] = (uint16_t)cnt;
                }
            }
            __syncwarp();
            uint16_t *dst = h + (int64_t)q * hs + i0;
            if (valid == TS) {
                if (lane < TS / 4)
                    reinterpret_cast<uint2 *>(dst)[lane] = reinterpret_cast<const uint2 *>(hrow)[lane];
            } else {
                for (int e = lane; e < valid; e += 32) dst[e] = hrow[e];
            }
            __syncwarp();
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

}  // namespace

cudaError_t launch_scan(const uint32_t *sketch, int64_t n_sets, int W, const uint32_t *plane,
                        int64_t NW, int gate_mode, const uint32_t *sq, const uint16_t *plist,
                        int A, int n_q, uint16_t *h, int64_t hs, cudaStream_t st) {
    if (n_q <= 0 || n_sets <= 0) return cudaSuccess;
    const int G = W / 4;
    // the largest tile whose shared memory fits next to the per-warp buffers
    int TS = kMaxTileSets;
    auto bytes = [&](int ts) {
        return sizeof(uint4) * ((size_t)ts * (G + 1) + (size_t)kScanWarps * G) +
               sizeof(uint16_t) * kScanWarps * ts;
    };
    while (TS > 32 && bytes(TS) > 227 * 1024) TS /= 2;
    const size_t smem = bytes(TS);
    cudaError_t e = cudaFuncSetAttribute(k_scan, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scan, kScanThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int64_t n_tiles = (n_sets + TS - 1) / TS;
    int64_t grid = (int64_t)sm_count() * per_sm;
    if (grid > n_tiles) grid = n_tiles;
    k_scan<<<(unsigned)grid, kScanThreads, smem, st>>>(
        reinterpret_cast<const uint4 *>(sketch), n_sets, G, TS, plane, NW, gate_mode,
        reinterpret_cast<const uint4 *>(sq), plist, A, n_q, h, hs);
    return cudaGetLastError();
}

}  // namespace bvss
