// refine_mma.cu -- exact re-rank of Alg. 6 (lines 19-22) of arXiv 2412.03301 on
// the 5th-generation tensor cores (tcgen05), from BF16 copies of the vectors.
//
// One CTA takes one query set (at most MQ = 32 or 64 vectors, one kernel
// instance each) and up to 512 of its candidates, whose rows, concatenated in
// candidate order, are cut into tiles of 128 rows.  For every tile the dot
// products of all (row, query vector) pairs are one 128 x MQ x d GEMM: the tile
// rows are the A operand (M = 128), the query vectors the B operand (N = MQ),
// both K-major in the 128-byte
// swizzle layout, accumulated in FP32 in tensor memory (TMEM lane = row,
// column = query vector).
//
// Warp roles (no block-wide barrier between set-up and tear-down):
//   warps 4-7  producers: gather the tile rows one 64-dimension block at a
//              time with 16-byte cp.async copies straight into the swizzled
//              stage (8 lanes per 128-byte row segment, so copies coalesce),
//              each lane's copies arriving on the stage's mbarrier when they
//              land (cp.async.mbarrier.arrive), so producers never wait for
//              their own copies and the whole ring (4-10 stages) is in flight;
//   warp 8     one thread waits for a stage, fences the producers' copies
//              into the async proxy, issues the MMAs (K = 16 each) and
//              commits them to the stage's "empty" mbarrier and, per tile, to
//              a "full" mbarrier of one of two TMEM accumulators;
//   warps 0-3  epilogue (for the 32-wide instances the column phase below runs
//              in warps 9-12 instead, on double-buffered distance blocks, so it
//              overlaps the next tile's row phase).  Row phase (lane = row 32w + lane): squared
//              distances |q|^2 + |v|^2 - 2 q.v to all query vectors from
//              MQ / 32 tensor-memory loads, their minimum with its arg-min
//              (the row's key), the distances written to a swizzled
//              shared-memory block.  After a barrier over the four warps,
//              column phase (lane = query vector, and lane + 32 when
//              MQ = 64): warp w walks, whole, the candidates whose first row in
//              the tile lies in rows 32w..32w+31, keeping per query vector the
//              minimum over the candidate's rows (with the row) and the maximum
//              of the rows' keys; when a candidate ends, the larger of the two
//              directed values (Def. 4) gives the pair that attains its
//              Hausdorff value, which is recorded.  The one candidate that runs
//              past the end of a tile carries its state in shared memory to the
//              next tile (double-buffered), so no atomics are needed.
// The record holds the pair (query vector, global row of the database vector) and, in
// the high word of its first field, the candidate's squared Hausdorff value over the
// stored copies; the boundary stage (boundary.cu) takes it from there.
// Every wait gives up after 2 s (or when another role gave up), sets the error
// word and lets all roles reach tear-down, where TMEM is released.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "block_util.cuh"
#include "bvss_internal.cuh"
#include "ptx_util.cuh"

namespace bvss {

namespace {

constexpr int kRowsN = 128;          // candidate rows per tile (MMA M)
constexpr int kMaxNS = 10;           // stages in the ring, at most
constexpr int kCandCTA = 512;        // candidates per CTA
constexpr int kMaxMeta = 14;         // tiles of row metadata in flight, at most
// warps 0-3 epilogue (row phase, and the column phase unless split), 4-7 producers, 8 MMA,
// and with a split epilogue 9-12 the column phase
__host__ __device__ constexpr int threads_for(bool split) { return (split ? 13 : 9) * 32; }
// the column phase gets warps of its own (and double-buffered distance blocks) in the
// 32-wide instances and in the 64-wide ones that stream their query operand (holding it,
// a 64-wide instance has no room for a second distance block)
__host__ __device__ constexpr bool split_for(int MQ, bool qs) { return MQ == 32 || qs; }
constexpr int kProd = 128;
constexpr int kEpi = 128;
constexpr int kMaxQ = 64;            // query vectors per query set, at most
constexpr uint64_t kWaitNs = 2000000000ull;
constexpr int kStageBytes = kRowsN * 128;
constexpr int kQOpRows = 64;         // rows of a query set's staged operand block (k_query_op)
constexpr int kQOpBlock = kQOpRows * 128;   // bytes of one K-block of it
constexpr int kSmemMax = 232448;

struct Meta {
    int slot;     // candidate slot of the row, -1 past the end
    int row_in;   // row index inside its set
    float vn;     // squared norm of the row's stored values (BF16, or FP8 times its scale)
    float sc;     // FP8 copy: the row's scale (1 for BF16)
};

struct Layout {
    int q, stages, meta, dist, rkey, carry, head, bars, grow0, vrow0, qn, qsc, misc, total;
};

constexpr float kE4M3Max = 448.0f;   // largest finite FP8 E4M3 value

// Tiles of row metadata the ring must hold: producers run at most ns stages
// ahead of the MMA, which runs at most two tiles ahead of the row phase, which with a
// split epilogue runs at most two tiles ahead of the column phase.
__host__ __device__ inline int meta_ring(int KB, int ns, bool split) {
    return (ns + KB) / KB + 3 + (split ? 2 : 0);
}

// bytes of one ring stage: a K-block of 128 rows, and with a streamed query operand the
// same K-block of the MQ query rows
__host__ __device__ inline int stage_bytes(int MQ, bool qs) {
    return kStageBytes + (qs ? MQ * 128 : 0);
}

// KB K-blocks of 128 bytes per row (64 BF16, 128 FP8 or 32 TF32 values); MQ query rows x
// 128 bytes per K-block, held whole (qs false) or streamed through the ring (qs true)
__host__ __device__ inline Layout make_layout(int KB, int ns, int MQ, bool qs) {
    Layout L;
    const bool split = split_for(MQ, qs);
    const int nd = split ? 2 : 1;                  // distance blocks
    const int MR = meta_ring(KB, ns, split);
    int o = 0;
    L.q = o;       o += qs ? 0 : KB * MQ * 128;
    L.stages = o;  o += ns * stage_bytes(MQ, qs);  // 1024-byte aligned (4 KB multiples)
    L.meta = o;    o += MR * kRowsN * (int)sizeof(Meta);
    L.dist = o;    o += nd * kRowsN * MQ * 4;      // row-phase distances, MQ per row
    L.rkey = o;    o += nd * kRowsN * 8;           // per row minimum (the row's key), per block
    L.carry = o;   o += 2 * (MQ + 1) * 8;          // state of a candidate continuing into the next tile
    L.head = o;    o += split ? 0 : 4 * (MQ + 1) * 8;   // 64-wide: the warps' head segments
    L.bars = o;    o += (2 * kMaxNS + 8 + kMaxMeta) * 8;
    L.grow0 = o;   o += kCandCTA * 8;
    L.vrow0 = o;   o += (kCandCTA + 4) * 4;
    L.qn = o;      o += MQ * 4;
    L.qsc = o;     o += MQ * 4;                    // FP8: scale of each query vector
    L.misc = o;    o += 16;                        // TMEM address, abort flag
    L.total = o + 1024;                            // slack to align the base to 1024 bytes
    return L;
}

constexpr int kMinNS = 4;   // smallest ring a caller may ask for

// most stages that fit, at least 5 with the query operand held whole, 4 streamed
inline int pick_stages(int KB, int MQ, bool qs) {
    for (int ns = kMaxNS; ns >= (qs ? 4 : 5); --ns)
        if (make_layout(KB, ns, MQ, qs).total <= kSmemMax &&
            meta_ring(KB, ns, split_for(MQ, qs)) <= kMaxMeta)
            return ns;
    return 0;
}

// 16 FP8 E4M3 values (16 bytes) -> floats
__device__ __forceinline__ void fp8x16_to_float(const uint4 pk, float (&f)[16]) {
    const uint32_t w[4] = {pk.x, pk.y, pk.z, pk.w};
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const __nv_fp8x2_storage_t two = (__nv_fp8x2_storage_t)(w[i >> 1] >> (16 * (i & 1)));
        const __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2(two, __NV_E4M3);
        const float2 v = __half22float2(*reinterpret_cast<const __half2 *>(&hr));
        f[2 * i] = v.x;
        f[2 * i + 1] = v.y;
    }
}

// 16 floats -> 16 FP8 E4M3 values (round to nearest, saturating)
__device__ __forceinline__ uint4 float16_to_fp8(const float (&f)[16]) {
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(f[4 * i], f[4 * i + 1]),
                                                     __NV_SATFINITE, __NV_E4M3);
        const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(f[4 * i + 2], f[4 * i + 3]),
                                                     __NV_SATFINITE, __NV_E4M3);
        w[i] = (lo & 0xFFFFu) | (hi << 16);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// 16-byte chunk ch of query row x (d FP32 values) in the refine's operand form: FP8 of
// x / scale (16 values), TF32 (4 values, to nearest) or BF16 (8 values, to nearest)
template <int EK>
__device__ __forceinline__ uint4 query_chunk(const float *__restrict__ x, int ch, float inv) {
    if (EK == (int)Elem::FP8) {
        const float4 *src = reinterpret_cast<const float4 *>(x + ch * 16);
        float f[16];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float4 u = src[i];
            f[4 * i] = u.x * inv;
            f[4 * i + 1] = u.y * inv;
            f[4 * i + 2] = u.z * inv;
            f[4 * i + 3] = u.w * inv;
        }
        return float16_to_fp8(f);
    } else if (EK == (int)Elem::TF32) {
        const float4 u = reinterpret_cast<const float4 *>(x)[ch];
        return make_uint4(f32_to_tf32(u.x), f32_to_tf32(u.y), f32_to_tf32(u.z), f32_to_tf32(u.w));
    } else {
        const float4 *src = reinterpret_cast<const float4 *>(x + ch * 8);
        const float4 u = src[0], w = src[1];
        __nv_bfloat162 b0 = __floats2bfloat162_rn(u.x, u.y), b1 = __floats2bfloat162_rn(u.z, u.w);
        __nv_bfloat162 b2 = __floats2bfloat162_rn(w.x, w.y), b3 = __floats2bfloat162_rn(w.z, w.w);
        return make_uint4(*reinterpret_cast<uint32_t *>(&b0), *reinterpret_cast<uint32_t *>(&b1),
                          *reinterpret_cast<uint32_t *>(&b2), *reinterpret_cast<uint32_t *>(&b3));
    }
}

// sum of squares of one operand chunk, added to sq in value order
template <int EK>
__device__ __forceinline__ float chunk_sq(const uint4 pk, float sq) {
    if (EK == (int)Elem::FP8) {
        float f[16];
        fp8x16_to_float(pk, f);
#pragma unroll
        for (int i = 0; i < 16; ++i) sq = fmaf(f[i], f[i], sq);
    } else if (EK == (int)Elem::TF32) {
        const float f[4] = {__uint_as_float(pk.x), __uint_as_float(pk.y), __uint_as_float(pk.z),
                            __uint_as_float(pk.w)};
#pragma unroll
        for (int i = 0; i < 4; ++i) sq = fmaf(f[i], f[i], sq);
    } else {
        const uint32_t w4[4] = {pk.x, pk.y, pk.z, pk.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w4[i]));
            sq = fmaf(f.x, f.x, sq);
            sq = fmaf(f.y, f.y, sq);
        }
    }
    return sq;
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

__device__ __forceinline__ unsigned long long dkey(float d2, uint32_t low) {
    return ((unsigned long long)__float_as_uint(d2) << 32) | low;
}

// EK = Elem::FP8: the database rows are the FP8 copy (vecb: d bytes per row, with scale
// vscale and squared norm vnorm of the scaled values) and the query vectors are quantised
// the same way in the CTA; Elem::BF16: both are BF16 (vecb: 2d bytes per row, vnorm the
// squared norms of the BF16 values); Elem::TF32: the rows are the FP32 vectors themselves
// (vecb: 4d bytes per row, vnorm their FP32 squared norms), which the tensor core reads
// as TF32, and the query vectors are rounded to TF32 (to nearest) in the CTA.
template <int MQ, int EK, bool QS>
__global__ void __launch_bounds__(threads_for(split_for(MQ, QS)), 1)
k_refine_mma(const float *__restrict__ qvec, const int64_t *__restrict__ qoff,
             const unsigned char *__restrict__ vecb, const float *__restrict__ vscale,
             const float *__restrict__ vnorm,
             const int64_t *__restrict__ set_off, int d, int ns,
             const int32_t *__restrict__ cand, const int32_t *__restrict__ thr, int C, int cpc,
             longlong2 *__restrict__ pair, int *__restrict__ err,
             const int32_t *__restrict__ qlist, const int32_t *__restrict__ qcount,
             const unsigned char *__restrict__ qop, const float *__restrict__ qop_n,
             const float *__restrict__ qop_sc) {
    extern __shared__ unsigned char smem_raw[];
    // with a list, CTA row y takes query set qlist[y] (rows past *qcount have none)
    if (qcount && (int)blockIdx.y >= *qcount) return;   // uniform over the CTA
    const int q = qlist ? qlist[blockIdx.y] : (int)blockIdx.y;
    const int n_sel = thr[q * 4 + 3];
    const int c0 = blockIdx.x * cpc;               // cpc <= kCandCTA candidates per CTA
    if (c0 >= n_sel) return;                       // uniform over the CTA
    const int ncand = min(cpc, n_sel - c0);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t a0 = qoff[q];
    const int mq = (int)(qoff[q + 1] - a0);
    constexpr int kQBlock = MQ * 128;               // query rows x 128 bytes per K-block
    constexpr int kRowB = MQ * 4;                    // bytes of one row's distances
    constexpr uint32_t kTmemCols = 2 * MQ;           // two accumulators of MQ columns
    constexpr bool F8 = EK == (int)Elem::FP8, TF = EK == (int)Elem::TF32;
    const int RB = F8 ? d : (TF ? 4 * d : 2 * d);   // bytes of one stored row
    const int KB = RB / 128;
    constexpr bool SPLIT = split_for(MQ, QS);
    constexpr int kThreads = threads_for(SPLIT);
    constexpr int kDistBytes = kRowsN * MQ * 4;      // one distance block
    const int MR = meta_ring(KB, ns, SPLIT);
    const Layout Lo = make_layout(KB, ns, MQ, QS);
    const int SB = stage_bytes(MQ, QS);
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    unsigned char *Qs = smem + Lo.q;
    unsigned char *stages = smem + Lo.stages;
    Meta *meta = reinterpret_cast<Meta *>(smem + Lo.meta);
    unsigned char *dist = smem + Lo.dist;
    unsigned long long *carry = reinterpret_cast<unsigned long long *>(smem + Lo.carry);
    unsigned long long *head = reinterpret_cast<unsigned long long *>(smem + Lo.head);
    unsigned long long *rkey = reinterpret_cast<unsigned long long *>(smem + Lo.rkey);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + Lo.bars);
    uint64_t *full = bars, *empty = bars + kMaxNS, *tfull = bars + 2 * kMaxNS,
             *tempty = bars + 2 * kMaxNS + 2, *dfull = bars + 2 * kMaxNS + 4,
             *dempty = bars + 2 * kMaxNS + 6, *mfull = bars + 2 * kMaxNS + 8;
    int64_t *grow0 = reinterpret_cast<int64_t *>(smem + Lo.grow0);
    int *vrow0 = reinterpret_cast<int *>(smem + Lo.vrow0);
    float *qn = reinterpret_cast<float *>(smem + Lo.qn);
    float *qsc = reinterpret_cast<float *>(smem + Lo.qsc);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + Lo.misc);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + Lo.misc + 4);

    // ---- set-up -------------------------------------------------------------
    // candidate table: first global row and size of each candidate (sizes are
    // turned into an exclusive prefix of the rows below)
    for (int c = tid; c < kCandCTA; c += kThreads) {
        int n = 0;
        if (c < ncand) {
            const int64_t id = cand[(int64_t)q * C + c0 + c];
            const int64_t g = set_off[id];
            grow0[c] = g;
            n = (int)(set_off[id + 1] - g);
        }
        vrow0[c] = n;
    }
    if (warp == 0) tmem_alloc(tmem_slot, kTmemCols);
    if (F8 && !QS) {
        // scale of each query vector: its largest magnitude maps to the largest E4M3 value
        for (int a = warp; a < MQ; a += kThreads / 32) {
            float mx = 0.0f;
            if (a < mq)
                for (int k = lane; k < d; k += 32) mx = fmaxf(mx, fabsf(qvec[(a0 + a) * d + k]));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (lane == 0) qsc[a] = mx > 0.0f ? mx / kE4M3Max : 1.0f;
        }
        __syncthreads();
    }
    // query rows 0..MQ-1 (BF16, or FP8 over their scales), K-major 128-byte swizzle
    // (rows >= mq are zero)
    const int nch = RB / 16;                       // 16-byte chunks per row
    for (int e = tid; e < MQ * nch && !QS; e += kThreads) {
        const int a = e / nch, ch = e - (e / nch) * nch;
        const uint4 pk = a < mq ? query_chunk<EK>(qvec + (a0 + a) * d, ch, F8 ? 1.0f / qsc[a] : 1.0f)
                                : make_uint4(0u, 0u, 0u, 0u);
        *reinterpret_cast<uint4 *>(Qs + (ch >> 3) * kQBlock + sw128_off(a, ch & 7)) = pk;
    }
    if (QS) {
        // the operand was staged in global memory by k_query_op: its norms and scales
        for (int a = tid; a < MQ; a += kThreads) {
            qn[a] = qop_n[(int64_t)q * kQOpRows + a];
            qsc[a] = qop_sc[(int64_t)q * kQOpRows + a];
        }
    }
    fence_proxy_async();
    if (tid == 0) {
        for (int s = 0; s < ns; ++s) {
            mbar_init(&full[s], kProd);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], kEpi / 32);
            mbar_init(&dfull[b], kEpi / 32);    // split epilogue: row phase -> column phase
            mbar_init(&dempty[b], kEpi / 32);   // and back
        }
        for (int i = 0; i < MR; ++i) mbar_init(&mfull[i], kProd);
        *abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (warp == 0) {
        // exclusive prefix of the candidate sizes, 16 per lane
        constexpr int kPer = kCandCTA / 32;
        int n[kPer], sum = 0;
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            n[i] = vrow0[lane * kPer + i];
            sum += n[i];
        }
        int incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        int run = incl - sum;
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            vrow0[lane * kPer + i] = run;
            run += n[i];
        }
        if (lane == 31) vrow0[kCandCTA] = incl;
    }
    // squared norms of the staged query rows, one warp per row (warps 1-8)
    for (int a = warp - 1; !QS && warp > 0 && a < MQ; a += kThreads / 32 - 1) {
        float sq = 0.0f;
        for (int ch = lane; ch < nch; ch += 32)
            sq = chunk_sq<EK>(
                *reinterpret_cast<const uint4 *>(Qs + (ch >> 3) * kQBlock + sw128_off(a, ch & 7)),
                sq);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
        if (lane == 0) qn[a] = F8 ? sq * qsc[a] * qsc[a] : sq;   // of the stored values
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int R = vrow0[ncand];
    const int n_tiles = (R + kRowsN - 1) / kRowsN;

    if (warp >= 4 && warp <= 7) {
        // ---- producers ----------------------------------------------------------
        // Thread p locates row p of every tile (its candidate, row and norm, for
        // the row metadata); the copies are coalesced instead: lane group p / 8
        // copies rows p / 8 + 16 k (k = 0..7), lane p % 8 one 16-byte chunk of
        // each, so a warp instruction moves four whole 128-byte row segments.
        const int p = tid - 128;
        const int pc = p & 7, pg = p >> 3;
        int n_slot = -1, n_row = 0;
        float n_vn = 0.0f, n_sc = 1.0f;
        auto locate = [&](int t) {
            const int v = t * kRowsN + p;
            n_slot = -1;
            n_row = 0;
            n_vn = 0.0f;
            n_sc = 1.0f;
            if (v < R) {
                int c = 0;
#pragma unroll
                for (int b = kCandCTA / 2; b > 0; b >>= 1)
                    if (c + b < ncand && vrow0[c + b] <= v) c += b;
                n_slot = c;
                n_row = v - vrow0[c];
                n_vn = vnorm[grow0[c] + n_row];
                if (F8) n_sc = vscale[grow0[c] + n_row];
            }
        };
        locate(0);
        bool ok = true;
        int u = 0;
        for (int t = 0; t < n_tiles; ++t) {
            Meta m;
            m.slot = n_slot;
            m.row_in = n_row;
            m.vn = n_vn;
            m.sc = n_sc;
            Meta *mt = meta + (t % MR) * kRowsN;
            mt[p] = m;
            mbar_arrive(&mfull[t % MR]);
            // every producer's row metadata of this tile is visible after this barrier,
            // which all producers also leave together if one of them gave up
            if (!named_barrier_and(4, kProd, ok)) break;
            const unsigned char *src[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const Meta mk = mt[pg + 16 * k];
                src[k] = mk.slot >= 0 ? vecb + (grow0[mk.slot] + mk.row_in) * RB + pc * 16 : nullptr;
            }
            if (t + 1 < n_tiles) locate(t + 1);
            for (int kb = 0; kb < KB; ++kb, ++u) {
                const int s = u % ns;
                ok = wait_or_abort(&empty[s], (uint32_t)(((u / ns) & 1) ^ 1), abort_flag, err);
                if (!ok) break;
                unsigned char *dst = stages + s * SB;
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    if (src[k]) cp_async16(dst + sw128_off(pg + 16 * k, pc), src[k] + kb * 128);
                if (QS) {
                    // the query operand's K-block: its first MQ rows, already swizzled
                    const unsigned char *qs_src = qop + ((int64_t)q * KB + kb) * kQOpBlock;
#pragma unroll
                    for (int c = p; c < MQ * 8; c += kProd)
                        cp_async16(dst + kStageBytes + 16 * c, qs_src + 16 * c);
                }
                cp_async_mbar_arrive(&full[s]);   // fires when these copies have landed
            }
        }
        cp_async_wait<0>();
    } else if (warp == 8) {
        // ---- MMA issue: one thread ----------------------------------------------
        if (lane == 0) {
            constexpr uint32_t idesc = F8   ? umma_idesc_e4m3(kRowsN, MQ)
                                       : TF ? umma_idesc_tf32(kRowsN, MQ)
                                            : umma_idesc_bf16(kRowsN, MQ);
            const uint32_t qaddr = smem_u32(Qs), saddr = smem_u32(stages);
            bool ok = true;
            for (int t = 0; t < n_tiles && ok; ++t) {
                const int buf = t & 1;
                ok = wait_or_abort(&tempty[buf], (uint32_t)(((t >> 1) & 1) ^ 1), abort_flag, err);
                if (!ok) break;
                tc_fence_after();
                const uint32_t dt = tmem + (uint32_t)(buf * MQ);
                for (int kb = 0; kb < KB && ok; ++kb) {
                    const int u = t * KB + kb, s = u % ns;
                    ok = wait_or_abort(&full[s], (uint32_t)((u / ns) & 1), abort_flag, err);
                    if (!ok) break;
                    fence_proxy_async();   // the producers' copies, seen by the tensor core
                    tc_fence_after();
                    // four MMAs per 128-byte K-block: K = 16 BF16, 32 FP8 or 8 TF32 values each
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint64_t ad = umma_desc_sw128(saddr + s * SB + 32 * k);
                        const uint64_t bd =
                            QS ? umma_desc_sw128(saddr + s * SB + kStageBytes + 32 * k)
                               : umma_desc_sw128(qaddr + kb * kQBlock + 32 * k);
                        if (F8)
                            umma_f8(dt, ad, bd, idesc, (kb | k) != 0 ? 1u : 0u);
                        else if (TF)
                            umma_tf32(dt, ad, bd, idesc, (kb | k) != 0 ? 1u : 0u);
                        else
                            umma_bf16(dt, ad, bd, idesc, (kb | k) != 0 ? 1u : 0u);
                    }
                    umma_commit(&empty[s]);
                }
                if (ok) umma_commit(&tfull[buf]);
            }
        }
    } else {
        // ---- epilogue ----------------------------------------------------------------
        const float INF = __int_as_float(0x7f800000);
        constexpr int H = MQ / 32;                   // query vectors per lane in the column phase
        const int coff = ((lane >> 2) << 4) + (lane & 3) * 4;   // column phase: my query vector's word
        // A candidate's pair and value from its per-query-vector row minima (bmin, brow)
        // and the largest row key kmax: the larger of the two directed values (Def. 4);
        // the query side's pair is the lowest query vector attaining it.
        auto finish = [&](int c, const float (&bmin)[H], const int (&brow)[H],
                          unsigned long long kmax) {
            uint32_t bits[H], lmx = 0;
#pragma unroll
            for (int h = 0; h < H; ++h) {
                bits[h] = 32 * h + lane < mq ? __float_as_uint(bmin[h]) : 0u;
                lmx = bits[h] > lmx ? bits[h] : lmx;
            }
            const uint32_t mx = __reduce_max_sync(0xffffffffu, lmx);
            int pa = -1, pr = 0;
#pragma unroll
            for (int h = 0; h < H; ++h) {
                const uint32_t who = __ballot_sync(0xffffffffu, 32 * h + lane < mq && bits[h] == mx);
                const int src = __ffs(who) - 1;
                const int rsrc = (int)__shfl_sync(0xffffffffu, (uint32_t)brow[h], src < 0 ? 0 : src);
                if (pa < 0 && who != 0u) {
                    pa = 32 * h + src;
                    pr = rsrc;
                }
            }
            uint32_t hbits = mx;   // the candidate's squared value, as bits
            if (mx < (uint32_t)(kmax >> 32)) {
                pa = (int)(kmax & 0xff);
                pr = (int)((kmax >> 8) & 0xffffff);
                hbits = (uint32_t)(kmax >> 32);
            }
            // the pair as (query vector, global row of the database vector), with the
            // squared Hausdorff value of the stored copies in the high word of .x
            if (lane == 0)
                pair[(int64_t)q * C + c0 + c] = make_longlong2(
                    (long long)(((unsigned long long)hbits << 32) | (uint32_t)pa), grow0[c] + pr);
        };
        // Column phase of the 32-wide instances, which run it in warps of their own on
        // double-buffered distance blocks: warp gw walks, whole, the candidates whose
        // first row in the tile lies in rows 32gw..32gw+31 (lane = query vector), from the
        // tile's distance block dblk and row keys kblk.
        auto column_walk = [&](int t, const Meta *mt, const unsigned char *dblk,
                               const unsigned long long *kblk, int gw) {
            const int t0 = t * kRowsN;
            const int rows_t = min(kRowsN, R - t0);
            const int lo = gw * 32, hi = min(lo + 32, rows_t);
            int c = mt[lo].slot;
            int j = lo;
            if (lo > 0 && vrow0[c] - t0 < lo) {   // begun in an earlier warp's rows
                j = vrow0[c + 1] - t0;
                ++c;
            }
            const unsigned long long *cin = carry + ((t + 1) & 1) * (MQ + 1);
            unsigned long long *cout = carry + (t & 1) * (MQ + 1);
            while (j < hi) {
                const int cs = vrow0[c] - t0;   // < 0: continues from the last tile
                const int je = min(vrow0[c + 1] - t0, rows_t);
                float bmin[H];
                int brow[H];
#pragma unroll
                for (int h = 0; h < H; ++h) {
                    bmin[h] = INF;
                    brow[h] = 0;
                }
                unsigned long long kmax = 0;
                if (cs < 0) {
#pragma unroll
                    for (int h = 0; h < H; ++h) {
                        const unsigned long long k0 = cin[32 * h + lane];
                        bmin[h] = __uint_as_float((uint32_t)(k0 >> 32));
                        brow[h] = (int)(uint32_t)k0;
                    }
                    kmax = cin[MQ];
                }
                for (int j0 = j; j0 < je; j0 += 4) {
                    float x[4][H];
                    unsigned long long kk[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int jr = min(j0 + i, je - 1);   // rows past je repeat the last one
#pragma unroll
                        for (int h = 0; h < H; ++h)
                            x[i][h] = *reinterpret_cast<const float *>(
                                dblk + jr * kRowB + h * 128 + (coff ^ ((jr & 7) << 4)));
                        kk[i] = kblk[jr];
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
#pragma unroll
                        for (int h = 0; h < H; ++h)
                            if (x[i][h] < bmin[h]) {
                                bmin[h] = x[i][h];
                                brow[h] = j0 + i - cs;   // row inside the candidate's set
                            }
                        kmax = kk[i] > kmax ? kk[i] : kmax;
                    }
                }
                if (vrow0[c + 1] - t0 <= rows_t) {
                    finish(c, bmin, brow, kmax);
                } else {
                    // continues into the next tile
#pragma unroll
                    for (int h = 0; h < H; ++h) cout[32 * h + lane] = dkey(bmin[h], (uint32_t)brow[h]);
                    if (lane == 0) cout[MQ] = kmax;
                }
                j = je;
                ++c;
            }
        };
        // Column phase of the 64-wide instances (run by the row-phase warps after their
        // row phase) for tile t and warp gw (lane = query vector), from the tile's
        // distance block dblk and row keys kblk.  Each warp walks exactly its own rows
        // 32gw..32gw+31, so a long candidate does not leave one warp with the tile's work:
        // it finishes the candidates that start and end there, publishes in head[gw] the
        // minima of the segment that continues a candidate begun before its rows, and keeps
        // the candidate that runs past them.  After a barrier of the four warps the owner
        // of such a candidate (the warp where it starts, or warp 0 for one carried from the
        // last tile) merges the later warps' heads in row order and finishes it, or carries
        // it into the next tile.  active false: the warp only meets the barrier.
        auto column_phase = [&](int t, const Meta *mt, const unsigned char *dblk,
                                const unsigned long long *kblk, int gw, bool active) {
            const int t0 = t * kRowsN;
            const int rows_t = min(kRowsN, R - t0);
            const int lo = gw * 32, hi = min(lo + 32, rows_t);
            const unsigned long long *cin = carry + ((t + 1) & 1) * (MQ + 1);
            unsigned long long *cout = carry + (t & 1) * (MQ + 1);
            int pc = -1;   // the candidate this warp owns that runs past its rows
            float pmin[H];
            int prow[H];
            unsigned long long pkmax = 0;
#pragma unroll
            for (int h = 0; h < H; ++h) {
                pmin[h] = INF;
                prow[h] = 0;
            }
            if (active && lo < hi) {
                int c = mt[lo].slot;
                int j = lo;
                while (j < hi) {
                    const int cs = vrow0[c] - t0;   // < 0: continues from the last tile
                    const int ce = vrow0[c + 1] - t0;
                    const int je = min(ce, hi);
                    const bool owned = cs >= lo || gw == 0;
                    // per query vector lane + 32 h: minimum over the segment's rows, with
                    // the row inside the candidate's set
                    float bmin[H];
                    int brow[H];
#pragma unroll
                    for (int h = 0; h < H; ++h) {
                        bmin[h] = INF;
                        brow[h] = 0;
                    }
                    unsigned long long kmax = 0;
                    if (cs < 0 && gw == 0) {
#pragma unroll
                        for (int h = 0; h < H; ++h) {
                            const unsigned long long k0 = cin[32 * h + lane];
                            bmin[h] = __uint_as_float((uint32_t)(k0 >> 32));
                            brow[h] = (int)(uint32_t)k0;
                        }
                        kmax = cin[MQ];
                    }
                    for (int j0 = j; j0 < je; j0 += 4) {
                        float x[4][H];
                        unsigned long long kk[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const int jr = min(j0 + i, je - 1);   // rows past je repeat the last
#pragma unroll
                            for (int h = 0; h < H; ++h)
                                x[i][h] = *reinterpret_cast<const float *>(
                                    dblk + jr * kRowB + h * 128 + (coff ^ ((jr & 7) << 4)));
                            kk[i] = kblk[jr];
                        }
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
#pragma unroll
                            for (int h = 0; h < H; ++h)
                                if (x[i][h] < bmin[h]) {
                                    bmin[h] = x[i][h];
                                    brow[h] = j0 + i - cs;
                                }
                            kmax = kk[i] > kmax ? kk[i] : kmax;
                        }
                    }
                    if (!owned) {
                        // the head: a candidate begun in an earlier warp's rows
                        unsigned long long *hd = head + gw * (MQ + 1);
#pragma unroll
                        for (int h = 0; h < H; ++h) hd[32 * h + lane] = dkey(bmin[h], (uint32_t)brow[h]);
                        if (lane == 0) hd[MQ] = kmax;
                    } else if (ce <= hi) {
                        finish(c, bmin, brow, kmax);
                    } else {
                        pc = c;
#pragma unroll
                        for (int h = 0; h < H; ++h) {
                            pmin[h] = bmin[h];
                            prow[h] = brow[h];
                        }
                        pkmax = kmax;
                    }
                    j = je;
                    ++c;
                }
            }
            named_barrier_sync(5, kEpi);   // every warp's head is visible
            if (pc >= 0) {
                const int ce = vrow0[pc + 1] - t0;
                for (int w2 = gw + 1; w2 < 4 && 32 * w2 < min(ce, rows_t); ++w2) {
                    const unsigned long long *hd = head + w2 * (MQ + 1);
#pragma unroll
                    for (int h = 0; h < H; ++h) {
                        const unsigned long long k0 = hd[32 * h + lane];
                        const float v = __uint_as_float((uint32_t)(k0 >> 32));
                        if (v < pmin[h]) {
                            pmin[h] = v;
                            prow[h] = (int)(uint32_t)k0;
                        }
                    }
                    const unsigned long long km = hd[MQ];
                    pkmax = km > pkmax ? km : pkmax;
                }
                if (ce <= rows_t) {
                    finish(pc, pmin, prow, pkmax);
                } else {
                    // continues into the next tile
#pragma unroll
                    for (int h = 0; h < H; ++h) cout[32 * h + lane] = dkey(pmin[h], (uint32_t)prow[h]);
                    if (lane == 0) cout[MQ] = pkmax;
                }
            }
        };
        if (!SPLIT || warp < 4) {
            // ---- row phase (and, unless split, the column phase): warps 0-3 ----------
            // the query norms (+inf past the set) in registers for 32 query vectors; the
            // 64-wide instances read them from shared memory (broadcast) to stay within
            // their registers
            constexpr bool kQnReg = MQ == 32;
            float qreg[kQnReg ? MQ : 1];
#pragma unroll
            for (int a = 0; a < (kQnReg ? MQ : 1); ++a) qreg[a] = a < mq ? qn[a] : INF;
            // FP8: q.v = (query scale) (row scale) x accumulator; BF16: scales of 1.  The
            // 64-wide FP8 instance reads the scales from shared memory (broadcast) to stay
            // within its registers
            constexpr bool kQsReg = F8 && MQ == 32;
            float qs2[kQsReg ? MQ : 1];
#pragma unroll
            for (int a = 0; a < (kQsReg ? MQ : 1); ++a) qs2[a] = kQsReg ? 2.0f * qsc[a] : 2.0f;
            const int r = warp * 32 + lane;
            bool ok = true;
            for (int t = 0; t < n_tiles; ++t) {
                // all four warps leave together if one of them gave up
                if (!named_barrier_and(1, kEpi, ok)) break;
                const int buf = t & 1;
                const int db = SPLIT ? buf : 0;      // this tile's distance block
                ok = wait_or_abort(&mfull[t % MR], (uint32_t)((t / MR) & 1), abort_flag, err) &&
                     wait_or_abort(&tfull[buf], (uint32_t)((t >> 1) & 1), abort_flag, err) &&
                     (!SPLIT || wait_or_abort(&dempty[buf], (uint32_t)(((t >> 1) & 1) ^ 1),
                                              abort_flag, err));
                ok = __all_sync(0xffffffffu, ok);   // the tensor-memory load below is warp-wide
                const Meta *mt = meta + (t % MR) * kRowsN;
                const int rows_t = min(kRowsN, R - t * kRowsN);
                unsigned char *dblk = dist + db * kDistBytes;
                unsigned long long *kblk = rkey + db * kRowsN;
                if (ok) {
                    tc_fence_after();
                    const int rows_w = min(32, rows_t - warp * 32);
                    uint32_t v[MQ];
                    if (rows_w > 0) {
#pragma unroll
                        for (int h = 0; h < H; ++h)
                            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) +
                                          (uint32_t)(buf * MQ + 32 * h),
                                      *reinterpret_cast<uint32_t(*)[32]>(v + 32 * h));
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&tempty[buf]);
                    if (rows_w > 0) {
                        // row phase: lane = row r
                        const Meta m = mt[r];
                        unsigned char *dw = dblk + warp * 32 * kRowB;
                        float best = INF;
                        int ba = 0;
#pragma unroll
                        for (int c4 = 0; c4 < MQ / 4; ++c4) {
                            float x[4];
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                const int a = c4 * 4 + i;
                                // qreg is +inf past the query, which keeps those entries out
                                const float w2 =
                                    F8 ? (kQsReg ? qs2[kQsReg ? a : 0] : 2.0f * qsc[a]) * m.sc
                                       : 2.0f;
                                const float qa = kQnReg ? qreg[kQnReg ? a : 0] : (a < mq ? qn[a] : INF);
                                const float d2 =
                                    fmaxf(qa + m.vn - w2 * __uint_as_float(v[a]), 0.0f);
                                x[i] = d2;
                                if (d2 < best) {
                                    best = d2;
                                    ba = a;
                                }
                            }
                            // 128-byte halves of the row, 16-byte chunks swizzled by the row
                            *reinterpret_cast<float4 *>(dw + lane * kRowB + (c4 >> 3) * 128 +
                                                        (((c4 & 7) ^ (lane & 7)) << 4)) =
                                make_float4(x[0], x[1], x[2], x[3]);
                        }
                        kblk[r] = dkey(best, ((uint32_t)(m.row_in & 0xffffff) << 8) | (uint32_t)ba);
                    }
                }
                if (SPLIT) {
                    // hand the block to the column warps
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&dfull[buf]);
                    continue;
                }
                named_barrier_sync(2, kEpi);   // the tile's distances and row keys are visible
                column_phase(t, mt, dblk, kblk, warp, ok);
            }
        } else if (warp >= 9) {
            // ---- column phase: warps 9-12 (split epilogue) ----------------------------
            const int gw = warp - 9;
            bool ok = true;
            for (int t = 0; t < n_tiles; ++t) {
                // the previous tile's carry is visible after this barrier, which all four
                // warps also leave together if one of them gave up
                if (!named_barrier_and(3, kEpi, ok)) break;
                const int buf = t & 1;
                ok = __all_sync(0xffffffffu, wait_or_abort(&dfull[buf], (uint32_t)((t >> 1) & 1),
                                                           abort_flag, err));
                if (ok && gw * 32 < min(kRowsN, R - t * kRowsN))
                    column_walk(t, meta + (t % MR) * kRowsN, dist + buf * kDistBytes,
                                rkey + buf * kRowsN, gw);
                __syncwarp();
                if (lane == 0) mbar_arrive(&dempty[buf]);
            }
        }
    }

    // ---- tear-down --------------------------------------------------------------
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
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

// FP8 E4M3 copy of the vectors with one FP32 scale per vector (its largest magnitude
// maps to the largest finite E4M3 value), and the squared norms of the scaled values
__global__ void k_to_fp8(const float *__restrict__ x, int64_t n, int d, uint8_t *__restrict__ y,
                         float *__restrict__ scale, float *__restrict__ norm) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t v = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); v < n;
         v += warps) {
        const float *xv = x + v * d;
        float mx = 0.0f;
        for (int k = lane; k < d; k += 32) mx = fmaxf(mx, fabsf(xv[k]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        const float sc = mx > 0.0f ? mx / kE4M3Max : 1.0f;
        const float inv = 1.0f / sc;
        float s = 0.0f;
        for (int c = lane; c < d / 16; c += 32) {
            float f[16];
            const float4 *src = reinterpret_cast<const float4 *>(xv + 16 * c);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float4 u = src[i];
                f[4 * i] = u.x * inv;
                f[4 * i + 1] = u.y * inv;
                f[4 * i + 2] = u.z * inv;
                f[4 * i + 3] = u.w * inv;
            }
            const uint4 pk = float16_to_fp8(f);
            *reinterpret_cast<uint4 *>(y + v * d + 16 * c) = pk;
            float g[16];
            fp8x16_to_float(pk, g);
#pragma unroll
            for (int i = 0; i < 16; ++i) s = fmaf(g[i], g[i], s);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            scale[v] = sc;
            norm[v] = s * sc * sc;
        }
    }
}

}  // namespace

// query-set width of the kernel instance for the batch's largest query set
inline int mq_for(int max_mq) { return max_mq <= 32 ? 32 : 64; }

// values per 128-byte K-block of a stored row
inline int kb_values(Elem e) { return e == Elem::FP8 ? 128 : (e == Elem::TF32 ? 32 : 64); }
// K-blocks of 128 bytes per stored row
inline int kblocks(int d, Elem e) { return d / kb_values(e); }

// the shape's basic limits (query-set width, whole K-blocks)
inline bool shape_ok(int d, int max_mq, Elem e) {
    if (max_mq < 1 || max_mq > kMaxQ) return false;
    const int kv = kb_values(e);
    return d % kv == 0 && d >= kv;
}

bool refine_mma_streams(int d, int max_mq, Elem e, int mode) {
    if (!shape_ok(d, max_mq, e)) return false;
    const int res = pick_stages(kblocks(d, e), mq_for(max_mq), false);
    const int str = pick_stages(kblocks(d, e), mq_for(max_mq), true);
    if (str == 0) return false;   // cannot stream
    if (res == 0) return true;    // cannot hold the operand
    if (mode == 1) return false;
    if (mode == 2) return true;
    // by default a ring left shallow by the resident operand streams it when that buys
    // two or more stages (more row bytes in flight)
    return res <= 5 && str >= res + 2;
}

bool refine_mma_supported(int d, int max_mq, Elem e) {
    return shape_ok(d, max_mq, e) && (pick_stages(kblocks(d, e), mq_for(max_mq), false) > 0 ||
                                      pick_stages(kblocks(d, e), mq_for(max_mq), true) > 0);
}

size_t refine_mma_qop_bytes(int d, Elem e) { return (size_t)kblocks(d, e) * kQOpBlock; }

cudaError_t launch_to_bf16(const float *x, int64_t n, int d, __nv_bfloat16 *y, float *norm,
                           cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int64_t g = (n * 32 + 255) / 256;
    if (g > (1 << 20)) g = 1 << 20;
    k_to_bf16<<<(unsigned)g, 256, 0, st>>>(x, n, d, y, norm);
    return cudaGetLastError();
}

cudaError_t launch_to_fp8(const float *x, int64_t n, int d, uint8_t *y, float *scale,
                          float *norm, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (d % 16 != 0) return cudaErrorInvalidValue;
    int64_t g = (n * 32 + 255) / 256;
    if (g > (1 << 20)) g = 1 << 20;
    k_to_fp8<<<(unsigned)g, 256, 0, st>>>(x, n, d, y, scale, norm);
    return cudaGetLastError();
}

int refine_mma_stages(int d, int max_mq, Elem e, int mode) {
    return refine_mma_supported(d, max_mq, e)
               ? pick_stages(kblocks(d, e), mq_for(max_mq), refine_mma_streams(d, max_mq, e, mode))
               : 0;
}

int refine_mma_ring(int d, int max_mq, int stages, Elem e, int mode) {
    const int ns = refine_mma_stages(d, max_mq, e, mode);
    return stages >= kMinNS && stages < ns ? stages : ns;
}

cudaError_t launch_refine_mma(const float *qvec, const int64_t *qoff, int n_q, int max_mq,
                              const void *vecb, const float *vscale, const float *vnorm,
                              Elem el, const int64_t *set_off, int d, const int32_t *cand,
                              const int32_t *thr, int C, longlong2 *pair, int *err, cudaStream_t st,
                              int cand_cta, int stages, const int32_t *qlist,
                              const int32_t *qcount, const unsigned char *qop,
                              const float *qop_n, const float *qop_sc, int qs_mode) {
    if (n_q <= 0) return cudaSuccess;
    if (!refine_mma_supported(d, max_mq, el)) return cudaErrorInvalidValue;
    if (el == Elem::FP8 && !vscale) return cudaErrorInvalidValue;
    if ((qlist == nullptr) != (qcount == nullptr)) return cudaErrorInvalidValue;
    // without an operand buffer only the shapes that cannot hold the operand stream
    const int mode = qop && qop_n && qop_sc ? qs_mode : 1;
    const bool qs = refine_mma_streams(d, max_mq, el, mode);
    if (qs && (!qop || !qop_n || !qop_sc)) return cudaErrorInvalidValue;
    const int MQ = mq_for(max_mq);
    const int ns = refine_mma_ring(d, max_mq, stages, el, mode);
    const Layout Lo = make_layout(kblocks(d, el), ns, MQ, qs);
    const int cpc = cand_cta >= 1 && cand_cta <= kCandCTA ? cand_cta : kCandCTA;
    const int gx = (C + cpc - 1) / cpc;
    constexpr int kB = (int)Elem::BF16, kF = (int)Elem::FP8, kT = (int)Elem::TF32;
    using Kern = decltype(&k_refine_mma<32, kB, false>);
    Kern kern;
    if (el == Elem::FP8)
        kern = MQ == 32 ? (qs ? k_refine_mma<32, kF, true> : k_refine_mma<32, kF, false>)
                        : (qs ? k_refine_mma<64, kF, true> : k_refine_mma<64, kF, false>);
    else if (el == Elem::TF32)
        kern = MQ == 32 ? (qs ? k_refine_mma<32, kT, true> : k_refine_mma<32, kT, false>)
                        : (qs ? k_refine_mma<64, kT, true> : k_refine_mma<64, kT, false>);
    else
        kern = MQ == 32 ? (qs ? k_refine_mma<32, kB, true> : k_refine_mma<32, kB, false>)
                        : (qs ? k_refine_mma<64, kB, true> : k_refine_mma<64, kB, false>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Lo.total);
    if (e != cudaSuccess) return e;
    kern<<<dim3(gx, n_q), threads_for(split_for(MQ, qs)), Lo.total, st>>>(
        qvec, qoff, static_cast<const unsigned char *>(vecb), vscale, vnorm, set_off, d, ns, cand,
        thr, C, cpc, pair, err, qlist, qcount, qop, qop_n, qop_sc);
    return cudaGetLastError();
}

namespace {

// A query set's refine operand in global memory, for the streamed instances: one warp
// per (query set, row < kQOpRows); row a of K-block kb at ((q KB + kb) kQOpBlock +
// sw128_off(a, .)), zero past the set; the squared norm of the stored values (times the
// scale squared for FP8) and the FP8 scale per row (1 elsewhere).  The same arithmetic as
// the resident staging in k_refine_mma.
template <int EK>
__global__ void k_query_op(const float *__restrict__ qvec, const int64_t *__restrict__ qoff,
                           int n_q, int d, unsigned char *__restrict__ qop,
                           float *__restrict__ qop_n, float *__restrict__ qop_sc) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (wid >= (int64_t)n_q * kQOpRows) return;   // uniform over the warp
    const int q = (int)(wid / kQOpRows), a = (int)(wid % kQOpRows);
    constexpr bool F8 = EK == (int)Elem::FP8;
    const int RB = F8 ? d : (EK == (int)Elem::TF32 ? 4 * d : 2 * d);
    const int KB = RB / 128, nch = RB / 16;
    const int64_t a0 = qoff[q];
    const bool valid = a < (int)(qoff[q + 1] - a0);
    const float *x = qvec + (a0 + a) * d;
    float sc = 1.0f;
    if (F8 && valid) {
        float mx = 0.0f;
        for (int k = lane; k < d; k += 32) mx = fmaxf(mx, fabsf(x[k]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        sc = mx > 0.0f ? mx / kE4M3Max : 1.0f;
    }
    float sq = 0.0f;
    unsigned char *blk = qop + (int64_t)q * KB * kQOpBlock;
    for (int ch = lane; ch < nch; ch += 32) {
        const uint4 pk = valid ? query_chunk<EK>(x, ch, F8 ? 1.0f / sc : 1.0f)
                               : make_uint4(0u, 0u, 0u, 0u);
        *reinterpret_cast<uint4 *>(blk + (ch >> 3) * kQOpBlock + sw128_off(a, ch & 7)) = pk;
        sq = chunk_sq<EK>(pk, sq);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if (lane == 0) {
        qop_n[(int64_t)q * kQOpRows + a] = F8 ? sq * sc * sc : sq;
        qop_sc[(int64_t)q * kQOpRows + a] = sc;
    }
}

}  // namespace

cudaError_t launch_query_op(const float *qvec, const int64_t *qoff, int n_q, int d, Elem el,
                            unsigned char *qop, float *qop_n, float *qop_sc, cudaStream_t st) {
    if (n_q <= 0) return cudaSuccess;
    if (!qop || !qop_n || !qop_sc || d % kb_values(el) != 0) return cudaErrorInvalidValue;
    const int64_t warps = (int64_t)n_q * kQOpRows;
    const unsigned g = (unsigned)((warps + 7) / 8);
    if (el == Elem::FP8)
        k_query_op<(int)Elem::FP8><<<g, 256, 0, st>>>(qvec, qoff, n_q, d, qop, qop_n, qop_sc);
    else if (el == Elem::TF32)
        k_query_op<(int)Elem::TF32><<<g, 256, 0, st>>>(qvec, qoff, n_q, d, qop, qop_n, qop_sc);
    else
        k_query_op<(int)Elem::BF16><<<g, 256, 0, st>>>(qvec, qoff, n_q, d, qop, qop_n, qop_sc);
    return cudaGetLastError();
}

namespace {

// The query sets of a batch split by width: lists[0..) those of at most 32 vectors,
// lists[n_q..) the wider ones, both in order; counts[0], counts[1] their numbers.
__global__ void __launch_bounds__(1024)
k_width_lists(const int64_t *__restrict__ qoff, int n_q, int32_t *__restrict__ lists,
              int32_t *__restrict__ counts) {
    __shared__ int scan_sh[1024 / 32 + 1];
    int base_n = 0, base_w = 0;
    for (int q0 = 0; q0 < n_q; q0 += 1024) {
        const int q = q0 + threadIdx.x;
        const bool valid = q < n_q;
        const bool wide = valid && qoff[q + 1] - qoff[q] > 32;
        int tn, tw;
        const int pn = block_excl_scan<1024>(valid && !wide ? 1 : 0, scan_sh, &tn);
        const int pw = block_excl_scan<1024>(wide ? 1 : 0, scan_sh, &tw);
        if (valid && !wide) lists[base_n + pn] = q;
        if (wide) lists[n_q + base_w + pw] = q;
        base_n += tn;
        base_w += tw;
    }
    if (threadIdx.x == 0) {
        counts[0] = base_n;
        counts[1] = base_w;
    }
}

}  // namespace

cudaError_t launch_width_lists(const int64_t *qoff, int n_q, int32_t *lists, int32_t *counts,
                               cudaStream_t st) {
    if (n_q <= 0) return cudaSuccess;
    k_width_lists<<<1, 1024, 0, st>>>(qoff, n_q, lists, counts);
    return cudaGetLastError();
}

}  // namespace bvss
