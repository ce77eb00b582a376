// select.cu -- the candidate stage of Alg. 6 (lines 10-18) of arXiv 2412.03301.
//
// The bounded max-heap over (Hamming distance, set id) keeps the T smallest
// pairs of F1.  Here it is computed as an exact threshold select over the
// scores of all sets:
//   1. histogram of h over [0, m] per query                    (k_hist)
//   2. H* = smallest value whose cumulative count reaches
//      C' = min(C, |F1|); sets with h < H* all qualify, and the
//      first (C' - #{h < H*}) sets with h == H* in id order      (k_thresh)
//   3. per warp range of sets: counts of h < H* and h == H*     (k_count)
//   4. per query: exclusive scans over chunks                     (k_offsets)
//   5. stable compaction in id order                              (k_write)
// The result lists the C' candidate ids in ascending id order, -1 padded.
//
// With the minimum score of every block of kSelBlock sets (written by the scan),
// the passes read only blocks that can hold a candidate.  k_bound takes U = the
// C-th smallest block minimum: C blocks each hold a set with h <= U, so
// H* <= U, and a block whose minimum exceeds U (for k_hist) or H* (for k_count
// and k_write) holds no candidate and no score the threshold depends on.  With
// fewer than C blocks in F1 there is no bound and every such block is read.
#include <mutex>

#include "block_util.cuh"
#include "bvss_internal.cuh"

namespace bvss {

namespace {

constexpr int kSelThreads = 256;

// U per query: the C-th smallest block minimum below kGatedOut, or kGatedOut - 1
// (every block of F1) when fewer than C blocks hold a set of F1
__global__ void __launch_bounds__(kSelThreads)
k_bound(const uint16_t *__restrict__ bmin, int64_t n_blk, int m, int C,
        int32_t *__restrict__ bound) {
    extern __shared__ uint32_t sh[];   // m + 1 bins
    __shared__ int scan_sh[kSelThreads / 32 + 1];
    __shared__ int res;
    const int q = blockIdx.x, tid = threadIdx.x;
    for (int b = tid; b <= m; b += kSelThreads) sh[b] = 0;
    if (tid == 0) res = (int)kGatedOut - 1;
    __syncthreads();
    const uint16_t *bq = bmin + (int64_t)q * n_blk;
    for (int64_t b = tid; b < n_blk; b += kSelThreads) {
        const int v = bq[b];
        if (v <= m) atomicAdd(&sh[v], 1u);
    }
    __syncthreads();
    const int nb = m + 1;
    const int B = (nb + kSelThreads - 1) / kSelThreads;
    const int b0 = tid * B, b1 = min(nb, b0 + B);
    int s = 0;
    for (int b = b0; b < b1; ++b) s += (int)sh[b];
    int tot;
    const int excl = block_excl_scan<kSelThreads>(s, scan_sh, &tot);
    if (tot >= C && excl < C && excl + s >= C) {
        int cum = excl;
        for (int b = b0; b < b1; ++b) {
            cum += (int)sh[b];
            if (cum >= C) {
                res = b;
                break;
            }
        }
    }
    __syncthreads();
    if (tid == 0) bound[q] = res;
}

__global__ void __launch_bounds__(kSelThreads)
k_hist(const uint16_t *__restrict__ h, int64_t n_sets, int64_t hs, int m,
       const uint16_t *__restrict__ bmin, const int32_t *__restrict__ bound,
       uint32_t *__restrict__ hist) {
    extern __shared__ uint32_t sh[];   // m + 1 bins
    constexpr int kBlkPerChunk = kSelChunk / kSelBlock;
    __shared__ int act[kBlkPerChunk];
    __shared__ int n_act;
    const int q = blockIdx.y, tid = threadIdx.x, lane = tid & 31;
    const int64_t c0 = (int64_t)blockIdx.x * kSelChunk;
    const int64_t end = c0 + kSelChunk < n_sets ? c0 + kSelChunk : n_sets;
    const int nb = (int)((end - c0 + kSelBlock - 1) / kSelBlock);
    const int64_t n_blk = (n_sets + kSelBlock - 1) / kSelBlock;
    const uint16_t *bq = bmin ? bmin + (int64_t)q * n_blk + c0 / kSelBlock : nullptr;
    const int U = bmin ? bound[q] : 0xFFFF;
    for (int b = tid; b <= m; b += kSelThreads) sh[b] = 0;
    if (tid < 32) {
        // the chunk's blocks that can hold a score at or below U, in order (the minima
        // are loaded together, before the first comparison)
        constexpr int kR = kBlkPerChunk / 32;
        int bmv[kR];
#pragma unroll
        for (int i = 0; i < kR; ++i) {
            const int b = 32 * i + lane;
            bmv[i] = b < nb ? (bq ? (int)bq[b] : 0) : 0x10000;
        }
        int base = 0;
#pragma unroll
        for (int i = 0; i < kR; ++i) {
            const bool a = bmv[i] <= U;
            const uint32_t bal = __ballot_sync(0xffffffffu, a);
            if (a) act[base + __popc(bal & ((1u << lane) - 1u))] = 32 * i + lane;
            base += __popc(bal);
        }
        if (lane == 0) n_act = base;
    }
    __syncthreads();
    const uint4 *row4 = reinterpret_cast<const uint4 *>(h + (int64_t)q * hs);
    // half a warp per block: 16 lanes x 8 scores
    const int hw = tid >> 4, hl = tid & 15;
    const int na = n_act;
#pragma unroll 2
    for (int i = hw; i < na; i += kSelThreads / 16) {
        const int64_t s0 = c0 + (int64_t)act[i] * kSelBlock + hl * 8;
        if (s0 >= end) continue;
        const uint4 v = row4[s0 / 8];
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const uint32_t val = (w[e >> 1] >> ((e & 1) * 16)) & 0xFFFFu;
            // a score above m (only a caller of bvss_select_noalloc can pass one) counts
            // as outside F1, as in k_count and k_write, which never match it against H* <= m
            if (s0 + e < end && val <= (uint32_t)m) atomicAdd(&sh[val], 1u);
        }
    }
    __syncthreads();
    uint32_t *hq = hist + (int64_t)q * (m + 1);
    for (int b = tid; b <= m; b += kSelThreads)
        if (sh[b]) atomicAdd(&hq[b], sh[b]);
}

__global__ void __launch_bounds__(kSelThreads)
k_thresh(const uint32_t *__restrict__ hist, int m, int C, int32_t *__restrict__ thr,
         int32_t *__restrict__ cand) {
    __shared__ int scan_sh[kSelThreads / 32 + 1];
    __shared__ int res[4];
    const int q = blockIdx.x, tid = threadIdx.x;
    const uint32_t *hq = hist + (int64_t)q * (m + 1);
    const int nb = m + 1;
    const int B = (nb + kSelThreads - 1) / kSelThreads;
    const int b0 = tid * B, b1 = min(nb, b0 + B);
    int s = 0;
    for (int b = b0; b < b1; ++b) s += (int)hq[b];
    int tot;
    const int excl = block_excl_scan<kSelThreads>(s, scan_sh, &tot);
    const int cp = min(C, tot);
    if (tid == 0) {
        res[0] = -1;
        res[1] = 0;
        res[2] = 0;
        res[3] = cp;
    }
    __syncthreads();
    if (cp > 0 && excl < cp && excl + s >= cp) {
        int cum = excl;
        for (int b = b0; b < b1; ++b) {
            const int c = (int)hq[b];
            if (cum + c >= cp) {
                res[0] = b;
                res[1] = cum;
                res[2] = cp - cum;
                break;
            }
            cum += c;
        }
    }
    __syncthreads();
    if (tid < 4) thr[q * 4 + tid] = res[tid];
    for (int j = cp + tid; j < C; j += kSelThreads) cand[(int64_t)q * C + j] = -1;
}

// Each chunk of kSelChunk sets is split into kSelWarps ranges of kSelSpan
// sets, one per warp; counts and output slots are kept per range.
constexpr int kSelWarps = kSelThreads / 32;
constexpr int kSelSpan = kSelChunk / kSelWarps;
static_assert(kSelRangeWords == kSelWarps * 4, "per-chunk record size");

__device__ __forceinline__ void sel_range(int64_t n_sets, int warp, int64_t &w0, int64_t &w1) {
    const int64_t c0 = (int64_t)blockIdx.x * kSelChunk;
    const int64_t chunk_end = c0 + kSelChunk < n_sets ? c0 + kSelChunk : n_sets;
    w0 = c0 + (int64_t)warp * kSelSpan;
    w1 = w0 + kSelSpan < chunk_end ? w0 + kSelSpan : chunk_end;
}

static_assert(kSelSpan / kSelBlock <= 32, "a warp's blocks fit one ballot");

// minimum score of block `lane` of the warp's range [w0, w1) (0 without block minima,
// 0xFFFF past the range); loaded before the threshold is known
__device__ __forceinline__ int lane_block_min(const uint16_t *bq, int64_t w0, int64_t w1) {
    const int lane = threadIdx.x & 31;
    const int nb = w1 > w0 ? (int)((w1 - w0 + kSelBlock - 1) / kSelBlock) : 0;
    if (lane >= nb) return 0x10000;
    return bq ? (int)bq[w0 / kSelBlock + lane] : 0;
}

// bit i set: block i of the warp's range can hold a score <= H
__device__ __forceinline__ uint32_t active_blocks(int bm, int H) {
    return __ballot_sync(0xffffffffu, bm <= H);
}

// the next two active blocks, in order: lanes 0-15 take the first, 16-31 the second
// (-1 when there is none); returns false when none is left
__device__ __forceinline__ bool next_pair(uint32_t &act, int &mine) {
    if (!act) return false;
    const int b0 = __ffs(act) - 1;
    act &= act - 1;
    int b1 = -1;
    if (act) {
        b1 = __ffs(act) - 1;
        act &= act - 1;
    }
    mine = (threadIdx.x & 16) ? b1 : b0;
    return true;
}

// this lane's eight scores of block `mine` of the range [w0, w1) (lanes 0-15 and 16-31
// each cover one block); all 0xFFFF when there is no such block
__device__ __forceinline__ uint4 lane_block_scores(const uint4 *row4, int64_t w0, int64_t w1,
                                                   int mine) {
    const int64_t i0 = w0 + (int64_t)(mine < 0 ? 0 : mine) * kSelBlock + (threadIdx.x & 15) * 8;
    if (mine < 0 || i0 >= w1) return make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu);
    return row4[i0 / 8];
}

__global__ void __launch_bounds__(kSelThreads)
k_count(const uint16_t *__restrict__ h, int64_t n_sets, int64_t hs,
        const int32_t *__restrict__ thr, const uint16_t *__restrict__ bmin,
        int32_t *__restrict__ ranges) {
    const int q = blockIdx.y;
    const int n_chunks = gridDim.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int H = thr[q * 4];
    const int64_t n_blk = (n_sets + kSelBlock - 1) / kSelBlock;
    const uint16_t *bq = bmin ? bmin + (int64_t)q * n_blk : nullptr;
    int64_t w0, w1;
    sel_range(n_sets, warp, w0, w1);
    const int bm = lane_block_min(bq, w0, w1);
    int lt = 0, eq = 0;
    if (H >= 0) {
        const uint4 *row4 = reinterpret_cast<const uint4 *>(h + (int64_t)q * hs);
        // blocks whose minimum is above H* count nothing
        uint32_t act = active_blocks(bm, H);
        int mine = -1;
        bool have = next_pair(act, mine);
        uint4 v = lane_block_scores(row4, w0, w1, have ? mine : -1);
        while (have) {
            // the next pair's scores are in flight while this pair is counted
            int nmine = -1;
            const bool nhave = next_pair(act, nmine);
            const uint4 nv = lane_block_scores(row4, w0, w1, nhave ? nmine : -1);
            const int64_t i0 = w0 + (int64_t)(mine < 0 ? 0 : mine) * kSelBlock + (lane & 15) * 8;
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int val = (int)((w[e >> 1] >> ((e & 1) * 16)) & 0xFFFFu);
                const bool in = mine >= 0 && i0 + e < w1;
                lt += in && val < H;
                eq += in && val == H;
            }
            v = nv;
            mine = nmine;
            have = nhave;
        }
    }
    lt = (int)__reduce_add_sync(0xffffffffu, (uint32_t)lt);
    eq = (int)__reduce_add_sync(0xffffffffu, (uint32_t)eq);
    if (lane == 0) {
        int32_t *o = ranges + (((int64_t)q * n_chunks + blockIdx.x) * kSelWarps + warp) * 4;
        o[0] = lt;
        o[1] = eq;
    }
}

// per query: in id order over all ranges, the rank of each range's first tie
// and its first output slot (the first `take` ties by id are selected)
__global__ void __launch_bounds__(kSelThreads)
k_offsets(const int32_t *__restrict__ thr, int n_ranges, int32_t *__restrict__ ranges) {
    __shared__ int scan_sh[kSelThreads / 32 + 1];
    const int q = blockIdx.x;
    const int take = thr[q * 4 + 2];
    int run_eq = 0, run_sel = 0;
    for (int base = 0; base < n_ranges; base += kSelThreads) {
        const int r = base + threadIdx.x;
        int32_t *o = ranges + ((int64_t)q * n_ranges + r) * 4;
        int lt = 0, eq = 0;
        if (r < n_ranges) {
            lt = o[0];
            eq = o[1];
        }
        int te;
        const int ex_eq = block_excl_scan<kSelThreads>(eq, scan_sh, &te);
        const int eqb = run_eq + ex_eq;
        const int sel = lt + max(0, min(take - eqb, eq));
        int ts;
        const int ex_sel = block_excl_scan<kSelThreads>(sel, scan_sh, &ts);
        if (r < n_ranges) {
            o[2] = eqb;
            o[3] = run_sel + ex_sel;
        }
        run_eq += te;
        run_sel += ts;
    }
}

// inclusive prefix sum over the warp
__device__ __forceinline__ int warp_incl_scan(int x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Stable compaction: warp w of a chunk walks its range 256 sets at a time and
// writes the selected ids from the range's first output slot on, with
// warp-shuffle scans only where the warp's ballot shows a candidate.
__global__ void __launch_bounds__(kSelThreads)
k_write(const uint16_t *__restrict__ h, int64_t n_sets, int64_t hs,
        const int32_t *__restrict__ thr, const int32_t *__restrict__ ranges, int C,
        const uint16_t *__restrict__ bmin, int32_t *__restrict__ cand) {
    const int q = blockIdx.y;
    const int n_chunks = gridDim.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t w0, w1;
    sel_range(n_sets, warp, w0, w1);
    // the threshold, this range's record and the block minima, all in flight together
    const int H = thr[q * 4];
    const int take = thr[q * 4 + 2];
    const int32_t *o = ranges + (((int64_t)q * n_chunks + blockIdx.x) * kSelWarps + warp) * 4;
    const int4 rec = *reinterpret_cast<const int4 *>(o);
    const int64_t n_blk = (n_sets + kSelBlock - 1) / kSelBlock;
    const uint16_t *bq = bmin ? bmin + (int64_t)q * n_blk : nullptr;
    const int bm = lane_block_min(bq, w0, w1);
    if (H < 0) return;   // uniform over the CTA
    if (rec.x == 0 && (rec.y == 0 || rec.z >= take)) return;   // nothing selected in this range
    int rank = rec.z, pos = rec.w;
    const uint4 *row4 = reinterpret_cast<const uint4 *>(h + (int64_t)q * hs);
    int32_t *out = cand + (int64_t)q * C;
    // blocks whose minimum is above H* hold no candidate; the others two at a time, in
    // id order over the lanes
    uint32_t act = active_blocks(bm, H);
    int mine = -1;
    bool have = next_pair(act, mine);
    uint4 v = lane_block_scores(row4, w0, w1, have ? mine : -1);
    while (have) {
        // the next pair's scores are in flight while this pair is written
        int nmine = -1;
        const bool nhave = next_pair(act, nmine);
        const uint4 nv = lane_block_scores(row4, w0, w1, nhave ? nmine : -1);
        const int cur = mine;
        const uint4 cv = v;
        v = nv;
        mine = nmine;
        have = nhave;
        const int64_t i0 = w0 + (int64_t)(cur < 0 ? 0 : cur) * kSelBlock + (lane & 15) * 8;
        int val[8];
        {
            const uint32_t w[4] = {cv.x, cv.y, cv.z, cv.w};
#pragma unroll
            for (int e = 0; e < 8; ++e)
                val[e] = cur >= 0 && i0 + e < w1 ? (int)((w[e >> 1] >> ((e & 1) * 16)) & 0xFFFFu)
                                                 : 0xFFFF;
        }
        int n_lt = 0, n_eq = 0;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            n_lt += val[e] < H;
            n_eq += val[e] == H;
        }
        if (!__any_sync(0xffffffffu, (n_lt | n_eq) != 0)) continue;
        const int inc_eq = warp_incl_scan(n_eq);
        int r = rank + inc_eq - n_eq;   // id-order rank of my first tie
        const int n_sel = n_lt + max(0, min(take - r, n_eq));
        const int inc_sel = warp_incl_scan(n_sel);
        int p = pos + inc_sel - n_sel;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            bool sel = val[e] < H;
            if (val[e] == H) {
                sel = r < take;
                ++r;
            }
            if (sel && p < C) out[p++] = (int32_t)(i0 + e);
        }
        rank += __shfl_sync(0xffffffffu, inc_eq, 31);
        pos += __shfl_sync(0xffffffffu, inc_sel, 31);
    }
}

}  // namespace

cudaError_t launch_select(const uint16_t *h, int64_t n_sets, int64_t hs, int m, int n_q, int C,
                          uint32_t *hist, int32_t *thr, int32_t *chunk, int32_t *cand,
                          cudaStream_t st, const uint16_t *bmin, int32_t *bound) {
    if (n_q <= 0) return cudaSuccess;
    if (bmin && !bound) return cudaErrorInvalidValue;
    const int n_chunks = (int)((n_sets + kSelChunk - 1) / kSelChunk);
    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(uint32_t) * (size_t)n_q * (m + 1), st);
    if (e != cudaSuccess) return e;
    const size_t smem = sizeof(uint32_t) * (size_t)(m + 1);
    e = cudaFuncSetAttribute(k_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const dim3 g2(n_chunks, n_q);
    if (bmin) {
        e = cudaFuncSetAttribute(k_bound, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_bound<<<n_q, kSelThreads, smem, st>>>(bmin, (n_sets + kSelBlock - 1) / kSelBlock, m, C,
                                                bound);
    }
    k_hist<<<g2, kSelThreads, smem, st>>>(h, n_sets, hs, m, bmin, bound, hist);
    k_thresh<<<n_q, kSelThreads, 0, st>>>(hist, m, C, thr, cand);
    k_count<<<g2, kSelThreads, 0, st>>>(h, n_sets, hs, thr, bmin, chunk);
    k_offsets<<<n_q, kSelThreads, 0, st>>>(thr, n_chunks * kSelWarps, chunk);
    k_write<<<g2, kSelThreads, 0, st>>>(h, n_sets, hs, thr, chunk, C, bmin, cand);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Candidate select that allocates nothing (bvss_select_noalloc).
//
// Its scratch -- the per-query histograms, thresholds and per-chunk counts
// that launch_select needs -- lives in one file-scope device array of fixed
// size instead of memory obtained from cudaMalloc.  Every GPU that loads the
// library holds this array until the process exits.  Host code must not pass
// the array's name to a kernel (on the host it is only a stand-in); the
// device address is looked up once per device with cudaGetSymbolAddress.
// ---------------------------------------------------------------------------
namespace {

constexpr int kNoAllocMaxQ = 32;
constexpr int kNoAllocMaxM = 8192;
constexpr int kNoAllocMaxChunks = 1024;
constexpr size_t kNoAllocHistWords = (size_t)kNoAllocMaxQ * (kNoAllocMaxM + 1);
constexpr size_t kNoAllocThrWords = (size_t)kNoAllocMaxQ * 4;
constexpr size_t kNoAllocChunkWords = (size_t)kNoAllocMaxQ * kNoAllocMaxChunks * kSelRangeWords;
constexpr size_t kNoAllocWords = kNoAllocHistWords + kNoAllocThrWords + kNoAllocChunkWords;
constexpr int kNoAllocMaxDevices = 64;

static_assert(BVSS_NOALLOC_MAX_QUERIES == kNoAllocMaxQ, "header limit");
static_assert(BVSS_NOALLOC_MAX_M == kNoAllocMaxM, "header limit");
static_assert(BVSS_NOALLOC_MAX_SETS == (int64_t)kNoAllocMaxChunks * kSelChunk, "header limit");

static __device__ __align__(256) uint32_t g_select_scratch[kNoAllocWords];

std::mutex g_scratch_mu;
uint32_t *g_scratch_ptr[kNoAllocMaxDevices] = {};

// device address of g_select_scratch on the current device (looked up once)
cudaError_t scratch_for_current_device(uint32_t **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_select_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<uint32_t *>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

}  // namespace bvss

extern "C" int bvss_select_noalloc(const uint16_t *h, int64_t n_sets, int64_t h_stride,
                                   int32_t m, int32_t n_queries, int32_t C, int32_t *cand,
                                   int32_t *n_cand, void *stream) {
    using namespace bvss;
    if (n_queries < 0 || n_queries > kNoAllocMaxQ)
        return record_error(BVSS_EINVAL, "bvss_select_noalloc: n_queries = %d, limit %d",
                            n_queries, kNoAllocMaxQ);
    if (m < 1 || m > kNoAllocMaxM)
        return record_error(BVSS_EINVAL, "bvss_select_noalloc: m = %d, limit %d", m, kNoAllocMaxM);
    if (n_sets < 1 || n_sets > (int64_t)kNoAllocMaxChunks * kSelChunk)
        return record_error(BVSS_EINVAL, "bvss_select_noalloc: n_sets = %lld, limit %lld",
                            (long long)n_sets, (long long)kNoAllocMaxChunks * kSelChunk);
    if (h_stride < n_sets || h_stride % 8 != 0)
        return record_error(BVSS_EINVAL,
                            "bvss_select_noalloc: h_stride must be >= n_sets and a multiple of 8");
    if (C < 1 || C > BVSS_MAX_C)
        return record_error(BVSS_EINVAL, "bvss_select_noalloc: C = %d, need 1..%d", C, BVSS_MAX_C);
    if (n_queries == 0) return BVSS_OK;
    if (!h || !cand || (reinterpret_cast<uintptr_t>(h) & 15) != 0)
        return record_error(BVSS_EINVAL, "bvss_select_noalloc: h must be 16-byte aligned, "
                                         "h and cand non-NULL");
    uint32_t *scratch = nullptr;
    cudaError_t e = scratch_for_current_device(&scratch);
    if (e != cudaSuccess)
        return record_error(BVSS_ECUDA, "bvss_select_noalloc: scratch lookup failed: %s",
                            cudaGetErrorString(e));
    uint32_t *hist = scratch;
    int32_t *thr = reinterpret_cast<int32_t *>(scratch + kNoAllocHistWords);
    int32_t *chunk = thr + kNoAllocThrWords;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // launch_select clears the histograms it uses before counting
    e = launch_select(h, n_sets, h_stride, m, n_queries, C, hist, thr, chunk, cand, st);
    if (e == cudaSuccess && n_cand)
        e = cudaMemcpy2DAsync(n_cand, sizeof(int32_t), thr + 3, 4 * sizeof(int32_t),
                              sizeof(int32_t), n_queries, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess)
        return record_error(BVSS_ECUDA, "bvss_select_noalloc: %s", cudaGetErrorString(e));
    return BVSS_OK;
}
