// refine_mma.cu -- exact re-rank of Alg. 6 (lines 19-22) of arXiv 2412.03301 on
// the 5th-generation tensor cores (tcgen05), from BF16 copies of the vectors.
//
// One CTA takes one query set (at most 32 vectors) and up to 128 of its
// candidates, whose rows, concatenated in candidate order, are cut into tiles
// of 128 rows.  For every tile the dot products of all (query vector, row)
// pairs are one 128 x 128 x d GEMM: the query vectors are the A operand
// (M = 128 rows of shared memory, of which the first 32 hold the query; the
// rest are never read back), the tile rows the B operand (N = 128), both
// K-major in the 128-byte swizzle layout, accumulated in FP32 in tensor memory
// (TMEM lane = query vector, column = row).
//
// The same stage also feeds a second, four times smaller MMA with the roles
// swapped (rows as M = 128, the 32 query vectors as N), so tensor memory holds
// the tile both ways round and every reduction of the epilogue stays inside a
// thread.
//
// Warp roles (no block-wide barrier between set-up and tear-down):
//   warps 4-7  producers: each thread gathers one row of every tile, one
//              64-dimension block at a time, with 16-byte cp.async copies
//              straight into the swizzled stage (a ring of 8 stages, 5 kept in
//              flight per thread), then signals the stage's mbarrier;
//   warp 8     one thread issues the MMAs (K = 16 each) and commits them to the
//              stage's "empty" mbarrier and, per tile, to a "full" mbarrier of
//              one of two pairs of TMEM accumulators;
//   warps 0-3  epilogue.  Warp w reads the swapped tile for rows 32w..32w+31
//              and takes each row's minimum over the query vectors of
//              |q|^2 + |v|^2 - 2 q.v (with its arg-min).  Warp 0 then reads the
//              tile with lane = query vector and walks the rows in order,
//              keeping for the open candidate the minimum over its rows per
//              query vector and the maximum of the rows' minima; when a
//              candidate ends it records the pair attaining the candidate's
//              Hausdorff value (Def. 4).
// k_rescore then computes that pair's distance directly in FP32 from the
// original vectors (one warp per candidate, many rows in flight) and writes
// the square root as the candidate's distance.
// Every wait gives up after 2 s (or when another role gave up), sets the error
// word and lets all roles reach tear-down, where TMEM is released.
#include <cuda_bf16.h>

#include "bvss_internal.cuh"
#include "ptx_util.cuh"

namespace bvss {

namespace {

constexpr int kRowsN = 128;          // candidate rows per tile (MMA N)
constexpr int kKB = 64;              // BF16 values per K-block (one 128-byte swizzle row)
constexpr int kNS = 8;               // stages in the ring
constexpr int kLag = 5;              // stages a producer thread keeps in flight
constexpr int kCandCTA = 128;        // candidates per CTA
constexpr int kMaxMeta = 12;         // tiles of row metadata in flight, at most
constexpr int kThreads = 9 * 32;     // warps 0-3 epilogue, 4-7 producers, 8 MMA
constexpr int kProd = 128;
constexpr int kEpi = 128;
constexpr uint32_t kTmemCols = 512;  // D: 2 x 128 columns at 0; swapped D: 2 x 32 at 256
constexpr uint32_t kTmemT = 256;
constexpr uint64_t kWaitNs = 2000000000ull;
constexpr int kStageBytes = kRowsN * 128;
constexpr int kQBlock = 4096;        // 32 query rows x 128 bytes per K-block
constexpr int kMaxQ = 32;

struct Meta {
    int slot;     // candidate slot of the row, -1 past the end
    int row_in;   // row index inside its set
    float vn;     // squared norm of the row's BF16 values
    int pad;
};

struct Layout {
    int q, stages, meta, colkey, bars, grow0, vrow0, qn, misc, total;
};

// Tiles of row metadata the ring must hold: producers run at most kNS stages
// ahead of the MMA, which runs at most two tiles ahead of the epilogue.
__host__ __device__ inline int meta_ring(int KB) { return (kNS + 1 + KB - 1) / KB + 3; }

__host__ __device__ inline Layout make_layout(int d) {
    Layout L;
    const int KB = d / kKB;
    const int MR = meta_ring(KB);
    int o = 0;
    L.q = o;       o += KB * kQBlock;              // rows 32..127 of a block read on into the next
    o = (o + 1023) & ~1023;
    L.stages = o;  o += kNS * kStageBytes;         // >= 12 KB follow the last Q block
    L.meta = o;    o += MR * kRowsN * (int)sizeof(Meta);
    L.colkey = o;  o += 2 * kRowsN * 8;            // per-row minima over the query, 2 tiles
    L.bars = o;    o += (2 * kNS + 4 + kMaxMeta) * 8;
    L.grow0 = o;   o += kCandCTA * 8;
    L.vrow0 = o;   o += (kCandCTA + 4) * 4;
    L.qn = o;      o += kMaxQ * 4;
    L.misc = o;    o += 16;                        // TMEM address, abort flag
    L.total = o + 1024;                            // slack to align the base to 1024 bytes
    return L;
}

// wait for a phase, or give up when the limit passes or another role gave up
__device__ __forceinline__ bool wait_or_abort(uint64_t *bar, uint32_t parity,
                                              volatile int *abort_flag, int *err) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort_flag) return false;
        if (global_timer_ns() - t0 > kWaitNs) {
            *abort_flag = 1;
            atomicOr(err, 2);
            return false;
        }
    }
    return true;
}

__global__ void __launch_bounds__(kThreads, 1)
k_refine_mma(const float *__restrict__ qvec, const int64_t *__restrict__ qoff,
             const float *__restrict__ vec, const __nv_bfloat16 *__restrict__ vec16,
             const float *__restrict__ vnorm16, const int64_t *__restrict__ set_off, int d,
             const int32_t *__restrict__ cand, const int32_t *__restrict__ thr, int C,
             int2 *__restrict__ pair, int *__restrict__ err) {
    extern __shared__ unsigned char smem_raw[];
    const int q = blockIdx.y;
    const int n_sel = thr[q * 4 + 3];
    const int c0 = blockIdx.x * kCandCTA;
    if (c0 >= n_sel) return;                       // uniform over the CTA
    const int ncand = min(kCandCTA, n_sel - c0);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t a0 = qoff[q];
    const int mq = (int)(qoff[q + 1] - a0);
    const int KB = d / kKB;
    const int MR = meta_ring(KB);
    const Layout Lo = make_layout(d);
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    unsigned char *Qs = smem + Lo.q;
    unsigned char *stages = smem + Lo.stages;
    Meta *meta = reinterpret_cast<Meta *>(smem + Lo.meta);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + Lo.bars);
    uint64_t *full = bars, *empty = bars + kNS, *tfull = bars + 2 * kNS,
             *tempty = bars + 2 * kNS + 2, *mfull = bars + 2 * kNS + 4;
    int64_t *grow0 = reinterpret_cast<int64_t *>(smem + Lo.grow0);
    int *vrow0 = reinterpret_cast<int *>(smem + Lo.vrow0);
    float *qn = reinterpret_cast<float *>(smem + Lo.qn);
    unsigned long long *colkey = reinterpret_cast<unsigned long long *>(smem + Lo.colkey);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + Lo.misc);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + Lo.misc + 4);

    // ---- set-up -------------------------------------------------------------
    if (warp == 0) {
        // candidate table: sizes, exclusive prefix of the rows, first global rows
        int n4[4], s = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int c = lane * 4 + i;
            n4[i] = 0;
            if (c < ncand) {
                const int64_t id = cand[(int64_t)q * C + c0 + c];
                const int64_t g = set_off[id];
                grow0[c] = g;
                n4[i] = (int)(set_off[id + 1] - g);
            }
            s += n4[i];
        }
        int incl = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        int run = incl - s;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            vrow0[lane * 4 + i] = run;
            run += n4[i];
        }
        if (lane == 31) vrow0[kCandCTA] = incl;    // rows of the CTA
        tmem_alloc(tmem_slot, kTmemCols);
    }
    // query rows 0..31 in BF16, K-major 128-byte swizzle (rows >= mq are zero)
    const int nch = d / 8;                         // 16-byte chunks per row
    for (int e = tid; e < kMaxQ * nch; e += kThreads) {
        const int a = e / nch, ch = e - (e / nch) * nch;
        float x[8];
        if (a < mq) {
            const float4 *src = reinterpret_cast<const float4 *>(qvec + (a0 + a) * d + ch * 8);
            const float4 u = src[0], w = src[1];
            x[0] = u.x; x[1] = u.y; x[2] = u.z; x[3] = u.w;
            x[4] = w.x; x[5] = w.y; x[6] = w.z; x[7] = w.w;
        } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) x[i] = 0.0f;
        }
        uint4 pk;
        __nv_bfloat162 b0 = __floats2bfloat162_rn(x[0], x[1]), b1 = __floats2bfloat162_rn(x[2], x[3]);
        __nv_bfloat162 b2 = __floats2bfloat162_rn(x[4], x[5]), b3 = __floats2bfloat162_rn(x[6], x[7]);
        pk.x = *reinterpret_cast<uint32_t *>(&b0);
        pk.y = *reinterpret_cast<uint32_t *>(&b1);
        pk.z = *reinterpret_cast<uint32_t *>(&b2);
        pk.w = *reinterpret_cast<uint32_t *>(&b3);
        *reinterpret_cast<uint4 *>(Qs + (ch >> 3) * kQBlock + sw128_off(a, ch & 7)) = pk;
    }
    fence_proxy_async();
    if (tid == 0) {
        for (int s = 0; s < kNS; ++s) {
            mbar_init(&full[s], kProd);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 1);
        }
        for (int i = 0; i < MR; ++i) mbar_init(&mfull[i], kProd);
        *abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();
    // squared norms of the staged BF16 query rows, one warp per row
    for (int a = warp; a < kMaxQ; a += kThreads / 32) {
        float sq = 0.0f;
        for (int ch = lane; ch < nch; ch += 32) {
            const uint4 pk =
                *reinterpret_cast<const uint4 *>(Qs + (ch >> 3) * kQBlock + sw128_off(a, ch & 7));
            const uint32_t w4[4] = {pk.x, pk.y, pk.z, pk.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w4[i]));
                sq = fmaf(f.x, f.x, sq);
                sq = fmaf(f.y, f.y, sq);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
        if (lane == 0) qn[a] = sq;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int R = vrow0[kCandCTA];
    const int n_tiles = (R + kRowsN - 1) / kRowsN;
    const int total = n_tiles * KB;

    if (warp >= 4 && warp <= 7) {
        // ---- producers: thread p fills row p of every tile ----------------------
        const int p = tid - 128;
        // where row p of tile t lives; its norm is loaded one tile ahead of use
        int n_slot = -1, n_row = 0;
        int64_t n_grow = 0;
        float n_vn = 0.0f;
        auto locate = [&](int t) {
            const int v = t * kRowsN + p;
            n_slot = -1;
            n_row = 0;
            n_vn = 0.0f;
            if (v < R) {
                int c = 0;
#pragma unroll
                for (int b = 64; b > 0; b >>= 1)
                    if (c + b < ncand && vrow0[c + b] <= v) c += b;
                n_slot = c;
                n_row = v - vrow0[c];
                n_grow = grow0[c] + n_row;
                n_vn = vnorm16[n_grow];
            }
        };
        locate(0);
        int64_t grow = 0;
        bool rv = false;
        bool ok = true;
        for (int u = 0; u < total && ok; ++u) {
            const int t = u / KB, kb = u - (u / KB) * KB, s = u % kNS;
            if (kb == 0) {
                Meta m;
                m.slot = n_slot;
                m.row_in = n_row;
                m.vn = n_vn;
                m.pad = 0;
                rv = n_slot >= 0;
                grow = n_grow;
                meta[(t % MR) * kRowsN + p] = m;
                mbar_arrive(&mfull[t % MR]);
                if (t + 1 < n_tiles) locate(t + 1);
            }
            ok = wait_or_abort(&empty[s], (uint32_t)(((u / kNS) & 1) ^ 1), abort_flag, err);
            if (ok && rv) {
                const unsigned char *src =
                    reinterpret_cast<const unsigned char *>(vec16 + grow * d + kb * kKB);
                unsigned char *dst = stages + s * kStageBytes;
#pragma unroll
                for (int c = 0; c < 8; ++c) cp_async16(dst + sw128_off(p, c), src + c * 16);
            }
            cp_async_commit();
            if (u >= kLag) {
                cp_async_wait<kLag>();
                fence_proxy_async();
                mbar_arrive(&full[(u - kLag) % kNS]);
            }
        }
        cp_async_wait<0>();
        fence_proxy_async();
        if (ok)
            for (int u = total > kLag ? total - kLag : 0; u < total; ++u) mbar_arrive(&full[u % kNS]);
    } else if (warp == 8) {
        // ---- MMA issue: one thread ----------------------------------------------
        if (lane == 0) {
            constexpr uint32_t idesc = umma_idesc_bf16(128, kRowsN);
            constexpr uint32_t idesc_t = umma_idesc_bf16(kRowsN, kMaxQ);
            const uint32_t qaddr = smem_u32(Qs), saddr = smem_u32(stages);
            bool ok = true;
            for (int t = 0; t < n_tiles && ok; ++t) {
                const int buf = t & 1;
                ok = wait_or_abort(&tempty[buf], (uint32_t)(((t >> 1) & 1) ^ 1), abort_flag, err);
                if (!ok) break;
                tc_fence_after();
                const uint32_t dt = tmem + (uint32_t)(buf * kRowsN);
                const uint32_t dtt = tmem + kTmemT + (uint32_t)(buf * kMaxQ);
                for (int kb = 0; kb < KB && ok; ++kb) {
                    const int u = t * KB + kb, s = u % kNS;
                    ok = wait_or_abort(&full[s], (uint32_t)((u / kNS) & 1), abort_flag, err);
                    if (!ok) break;
                    tc_fence_after();
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint64_t dq = umma_desc_sw128(qaddr + kb * kQBlock + 32 * k);
                        const uint64_t dv = umma_desc_sw128(saddr + s * kStageBytes + 32 * k);
                        const uint32_t acc = (kb | k) != 0 ? 1u : 0u;
                        umma_bf16(dt, dq, dv, idesc, acc);      // lane = query vector
                        umma_bf16(dtt, dv, dq, idesc_t, acc);   // lane = row
                    }
                    umma_commit(&empty[s]);
                }
                if (ok) umma_commit(&tfull[buf]);
            }
        }
    } else {
        // ---- epilogue: warps 0-3 ---------------------------------------------------
        const float INF = __int_as_float(0x7f800000);
        const bool va = lane < mq;
        int open = -1;
        float rmin = INF;
        int rrow = 0;
        long long cmax_key = -1;   // (d2 bits << 32) | (row << 8) | query vector
        auto finalize = [&](int c) {
            const uint32_t bits = va ? __float_as_uint(rmin) : 0u;
            const uint32_t mx = __reduce_max_sync(0xffffffffu, bits);
            const uint32_t who = __ballot_sync(0xffffffffu, va && bits == mx);
            const int src = __ffs(who) - 1;
            int pa = src, pr = __shfl_sync(0xffffffffu, rrow, src);
            if ((long long)mx < (cmax_key >> 32)) {
                pa = (int)(cmax_key & 0xff);
                pr = (int)((cmax_key >> 8) & 0xffffff);
            }
            if (lane == 0) pair[(int64_t)q * C + c0 + c] = make_int2(pa, pr);
        };
        bool ok = true;
        for (int t = 0; t < n_tiles && ok; ++t) {
            const int buf = t & 1;
            ok = wait_or_abort(&mfull[t % MR], (uint32_t)((t / MR) & 1), abort_flag, err) &&
                 wait_or_abort(&tfull[buf], (uint32_t)((t >> 1) & 1), abort_flag, err);
            // all four epilogue warps take the same exit
            if (!named_barrier_and(1, kEpi, ok)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const Meta *mt = meta + (t % MR) * kRowsN;
            const int rows_t = min(kRowsN, R - t * kRowsN);
            unsigned long long *ck = colkey + buf * kRowsN;
            {
                // row 32w + lane: minimum over the query vectors, from the swapped tile
                const int r = warp * 32 + lane;
                const Meta m = mt[r];
                uint32_t v[32];
                tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + kTmemT + (uint32_t)(buf * kMaxQ), v);
                float best = INF;
                int ba = 0;
#pragma unroll
                for (int a = 0; a < kMaxQ; ++a) {
                    float d2 = qn[a] + m.vn - 2.0f * __uint_as_float(v[a]);
                    d2 = d2 > 0.0f ? d2 : 0.0f;
                    if (a < mq && d2 < best) {
                        best = d2;
                        ba = a;
                    }
                }
                ck[r] = ((unsigned long long)__float_as_uint(best) << 32) |
                        ((unsigned long long)(m.row_in & 0xffffff) << 8) | (unsigned)ba;
            }
            tc_fence_before();
            named_barrier_sync(2, kEpi);
            if (warp == 0) {
                tc_fence_after();
                const float qna = qn[lane];
                for (int cc = 0; cc < (rows_t + 31) / 32; ++cc) {
                    uint32_t v[32];
                    tmem_ld32(tmem + (uint32_t)(buf * kRowsN + cc * 32), v);
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int r = cc * 32 + j;
                        const int slot = mt[r].slot;
                        if (slot < 0) break;
                        if (slot != open) {
                            if (open >= 0) finalize(open);
                            open = slot;
                            rmin = INF;
                            rrow = 0;
                            cmax_key = -1;
                        }
                        float d2 = qna + mt[r].vn - 2.0f * __uint_as_float(v[j]);
                        d2 = d2 > 0.0f ? d2 : 0.0f;
                        if (va && d2 < rmin) {
                            rmin = d2;
                            rrow = mt[r].row_in;
                        }
                        const long long key = (long long)ck[r];
                        if (key > cmax_key) cmax_key = key;
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty[buf]);
            }
        }
        if (warp == 0 && ok && open >= 0) finalize(open);
    }

    // ---- tear-down --------------------------------------------------------------
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// distance of each candidate's recorded pair, directly in FP32; one warp per candidate
__global__ void __launch_bounds__(256)
k_rescore(const float *__restrict__ qvec, const int64_t *__restrict__ qoff,
          const float *__restrict__ vec, const int64_t *__restrict__ set_off,
          const int32_t *__restrict__ cand, const int32_t *__restrict__ thr,
          const int2 *__restrict__ pair, int C, int d, float *__restrict__ cand_dist) {
    const int q = blockIdx.y;
    const int n_sel = thr[q * 4 + 3];
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (c >= n_sel) return;
    int2 pr = pair[(int64_t)q * C + c];
    const int64_t id = cand[(int64_t)q * C + c];
    // keep the pair inside its sets whatever the array holds
    pr.x = min(max(pr.x, 0), (int)(qoff[q + 1] - qoff[q]) - 1);
    pr.y = min(max(pr.y, 0), (int)(set_off[id + 1] - set_off[id]) - 1);
    const float4 *x4 = reinterpret_cast<const float4 *>(qvec + (qoff[q] + pr.x) * d);
    const float4 *y4 = reinterpret_cast<const float4 *>(vec + (set_off[id] + pr.y) * d);
    float s = 0.0f;
    for (int k = lane; k < d / 4; k += 32) {
        const float4 x = x4[k], y = y4[k];
        float u = x.x - y.x;
        s = fmaf(u, u, s);
        u = x.y - y.y;
        s = fmaf(u, u, s);
        u = x.z - y.z;
        s = fmaf(u, u, s);
        u = x.w - y.w;
        s = fmaf(u, u, s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) cand_dist[(int64_t)q * C + c] = sqrtf(s);
}

// FP32 -> BF16 copy of the vectors and the squared norms of the BF16 values
__global__ void k_to_bf16(const float *__restrict__ x, int64_t n, int d,
                          __nv_bfloat16 *__restrict__ y, float *__restrict__ norm) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t v = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); v < n;
         v += warps) {
        const float4 *src = reinterpret_cast<const float4 *>(x + v * d);
        __nv_bfloat162 *dst = reinterpret_cast<__nv_bfloat162 *>(y + v * d);
        float s = 0.0f;
        for (int k = lane; k < d / 4; k += 32) {
            const float4 f = src[k];
            const __nv_bfloat162 lo = __floats2bfloat162_rn(f.x, f.y);
            const __nv_bfloat162 hi = __floats2bfloat162_rn(f.z, f.w);
            dst[2 * k] = lo;
            dst[2 * k + 1] = hi;
            const float2 a = __bfloat1622float2(lo), b = __bfloat1622float2(hi);
            s = fmaf(a.x, a.x, s);
            s = fmaf(a.y, a.y, s);
            s = fmaf(b.x, b.x, s);
            s = fmaf(b.y, b.y, s);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) norm[v] = s;
    }
}

}  // namespace

bool refine_mma_supported(int d, int max_mq) {
    if (d % kKB != 0 || d < kKB || max_mq < 1 || max_mq > kMaxQ) return false;
    if (meta_ring(d / kKB) > kMaxMeta) return false;
    return make_layout(d).total <= 232448;
}

cudaError_t launch_to_bf16(const float *x, int64_t n, int d, __nv_bfloat16 *y, float *norm,
                           cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int64_t g = (n * 32 + 255) / 256;
    if (g > (1 << 20)) g = 1 << 20;
    k_to_bf16<<<(unsigned)g, 256, 0, st>>>(x, n, d, y, norm);
    return cudaGetLastError();
}

cudaError_t launch_refine_mma(const float *qvec, const int64_t *qoff, int n_q,
                              const float *vec, const __nv_bfloat16 *vec16,
                              const float *vnorm16, const int64_t *set_off, int d,
                              const int32_t *cand, const int32_t *thr, int C, int2 *pair,
                              float *cand_dist, int *err, cudaStream_t st) {
    if (n_q <= 0) return cudaSuccess;
    const Layout Lo = make_layout(d);
    cudaError_t e = cudaFuncSetAttribute(k_refine_mma,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, Lo.total);
    if (e != cudaSuccess) return e;
    const int gx = (C + kCandCTA - 1) / kCandCTA;
    k_refine_mma<<<dim3(gx, n_q), kThreads, Lo.total, st>>>(qvec, qoff, vec, vec16, vnorm16,
                                                            set_off, d, cand, thr, C, pair, err);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_rescore<<<dim3((C + 7) / 8, n_q), 256, 0, st>>>(qvec, qoff, vec, set_off, cand, thr, pair,
                                                       C, d, cand_dist);
    return cudaGetLastError();
}

}  // namespace bvss
