// scan_mma.cu -- layer 2 of Alg. 6 (line 12) of arXiv 2412.03301 on the
// 5th-generation tensor cores: Hamming scores of a batch of query sketches
// against every database sketch as one dense binary contraction.
//
// For 0/1 vectors, popcount(S_Q xor S_i) = |S_Q| + |S_i| - 2 <S_Q, S_i>, and
// the inner products of all (query, set) pairs are a GEMM with K = m.  A set
// bit is encoded as the FP8 E4M3 value 2^-6 (byte 0x08), so each product is
// 2^-12 and every partial sum (at most m * 2^-12 <= 8) is exact in the FP32
// accumulator; <S_Q, S_i> = 4096 x accumulator.  Computing every pair and
// masking with layer 1 (line 9) gives the same h as scoring only the sets of
// F1: sets outside F1 get 0xFFFF.
//
// Tile: 256 query sketches (two MMAs of M = 128) x 128 set sketches (MMA N),
// so every expanded set row feeds 256 queries; K-blocks of 128 bits (one
// 128-byte swizzle row of FP8).  Persistent CTAs walk the tiles
// set-tile-major, so the query blocks of one set tile run side by side and
// share its packed words through L2.
//
// Warp roles:
//   warps 4-11 producers: per K-block, thread p copies 8 packed bytes (half
//              of set row p mod 128) into a private ring with cp.async (6
//              K-blocks ahead), expands each bit to one FP8 byte into the
//              swizzled stage, and thread 0 also starts the bulk copy of the
//              query block pair's pre-expanded 32 KB;
//   warp 12    one thread issues 2 x 4 MMAs (K = 32) per K-block into one of
//              two pairs of TMEM accumulators of 128 columns;
//   warps 0-3  epilogue: lane = query row of each block; per 32 sets, one
//              tensor-memory load, h = |S_Q| + |S_i| - 2 <S_Q, S_i>, the
//              layer-1 bit, and 64-byte row stores into h; per tile, the
//              minimum of the row's 128 scores (the candidate select reads
//              only tiles whose minimum can reach its threshold).
// Every wait gives up after 2 s (or when another role gave up), sets the error
// word and lets all roles reach tear-down, where TMEM is released.
#include "bvss_internal.cuh"
#include "ptx_util.cuh"

namespace bvss {

namespace {

constexpr int kQM = 128;              // query sketches per MMA (M); a tile holds two blocks
constexpr int kSN = 128;              // set sketches per tile (MMA N)
static_assert(kSN == kSelBlock, "one block minimum per tile");
constexpr int kNS = 4;                // stages
constexpr int kPR = 8;                // packed-word ring slots per producer thread
constexpr int kPLag = 6;              // packed-word copies in flight per producer thread
constexpr int kThreads = 13 * 32;     // warps 0-3 epilogue, 4-11 producers, 12 MMA
constexpr int kProd = 2 * kSN;        // two producer threads per set row (8 bytes each)
constexpr int kEpi = 128;
constexpr uint32_t kTmemCols = 512;   // two buffers x two query blocks x 128 columns
constexpr int kQBlk = kQM * 128;      // 16 KB: one query block's K-block
constexpr int kAStage = 2 * kQBlk;    // 32 KB: the pair
constexpr int kBStage = kSN * 128;    // 16 KB
constexpr float kDotScale = 4096.0f;  // 1 / (2^-6 * 2^-6)
constexpr uint64_t kWaitNs = 2000000000ull;

constexpr int kOffA = 0;
constexpr int kOffB = kOffA + kNS * kAStage;
constexpr int kOffRing = kOffB + kNS * kBStage;
constexpr int kOffSpop = kOffRing + kPR * kProd * 8;
constexpr int kOffBars = kOffSpop + kSN * 4;
constexpr int kOffMisc = kOffBars + (2 * kNS + 4) * 8;
constexpr int kSmemBytes = kOffMisc + 16 + 1024;   // slack to align the base to 1024 bytes

// 4 bits -> 4 bytes, each 0x08 (FP8 E4M3 2^-6) for a set bit, 0 otherwise.  The
// four partial products of the multiply land in disjoint bit ranges (no carries).
__device__ __forceinline__ uint32_t spread4(uint32_t nib) {
    return (nib * 0x01020408u) & 0x08080808u;
}
// 16 bits -> 16 FP8 bytes
__device__ __forceinline__ uint4 spread16(uint32_t x) {
    return make_uint4(spread4(x & 0xF), spread4((x >> 4) & 0xF), spread4((x >> 8) & 0xF),
                      spread4((x >> 12) & 0xF));
}

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


// Query sketches -> FP8 rows in the blocked, swizzled layout of the MMA's A
// operand: block (qp, kb) holds query rows 256 qp .. 256 qp + 255, bits
// 128 kb .. 128 kb + 127, as two 16 KB halves of 128 rows exactly as the stage
// expects.  Rows past n_q are zero.  Also |S_Q| per query.
__global__ void k_expand_q(const uint32_t *__restrict__ sq, int n_q, int W, int QP,
                           uint8_t *__restrict__ q8, int32_t *__restrict__ qpop) {
    const int KB = W / 4;
    const int64_t total = (int64_t)QP * 2 * kQM * KB;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / KB), kb = (int)(e - (e / KB) * KB);
        uint4 w = make_uint4(0, 0, 0, 0);
        if (r < n_q) w = *reinterpret_cast<const uint4 *>(sq + (int64_t)r * W + 4 * kb);
        uint8_t *blk = q8 + ((int64_t)(r / (2 * kQM)) * KB + kb) * kAStage +
                       ((r / kQM) & 1) * kQBlk;
        const int rr = r % kQM;
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int c = 0; c < 8; ++c)
            *reinterpret_cast<uint4 *>(blk + sw128_off(rr, c)) =
                spread16(ws[c >> 1] >> (16 * (c & 1)));
        if (kb == 0) {
            int pc = 0;
            if (r < n_q)
                for (int i = 0; i < W; ++i) pc += __popc(sq[(int64_t)r * W + i]);
            qpop[r] = pc;
        }
    }
}

__global__ void __launch_bounds__(kThreads, 1)
k_scan_mma(const uint32_t *__restrict__ sk, const int32_t *__restrict__ spop, int64_t n_sets,
           int W, const uint32_t *__restrict__ gate, int64_t NW, int gate_mode,
           const uint8_t *__restrict__ q8, const int32_t *__restrict__ qpop, int n_q, int QP,
           uint16_t *__restrict__ h, int64_t hs, uint16_t *__restrict__ bmin, int64_t n_blk,
           int *__restrict__ err) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    unsigned char *stA = smem + kOffA;
    unsigned char *stB = smem + kOffB;
    unsigned char *ring = smem + kOffRing;
    int32_t *sp_s = reinterpret_cast<int32_t *>(smem + kOffSpop);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kOffBars);
    uint64_t *full = bars, *empty = bars + kNS, *tfull = bars + 2 * kNS, *tempty = bars + 2 * kNS + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + kOffMisc);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + kOffMisc + 4);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int KB = W / 4;
    const int n_tiles = (int)((n_sets + kSN - 1) / kSN) * QP;   // < 2^31 (host check)
    const int n_it = n_tiles > (int)blockIdx.x ? (n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

    if (warp == 0) tmem_alloc(tmem_slot, kTmemCols);
    if (tid == 0) {
        for (int s = 0; s < kNS; ++s) {
            mbar_init(&full[s], kProd + 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], kEpi / 32);
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp >= 4 && warp <= 11) {
        // ---- producers: thread p expands half (p >> 7) of set row p & 127 ----------
        const int p = tid - 128;
        const int pr = p & (kSN - 1), ph = p >> 7;
        // the unit (tile, K-block) whose packed words are copied next
        int i_it = 0, i_kb = 0, i_u = 0;
        int64_t i_row = (int64_t)((int)blockIdx.x / QP) * kSN + pr;
        auto issue = [&]() {
            if (i_it < n_it) {
                if (i_row < n_sets)
                    cp_async8(ring + ((i_u % kPR) * kProd + p) * 8, sk + i_row * W + 4 * i_kb + 2 * ph);
                if (++i_kb == KB) {
                    i_kb = 0;
                    ++i_it;
                    i_row = (int64_t)(((int)blockIdx.x + i_it * (int)gridDim.x) / QP) * kSN + pr;
                }
            }
            ++i_u;
            cp_async_commit();
        };
        for (int i = 0; i < kPLag; ++i) issue();
        bool ok = true;
        int u = 0;
        for (int it = 0; it < n_it && ok; ++it) {
            const int tau = (int)blockIdx.x + it * (int)gridDim.x;
            const int st = tau / QP, qp = tau - st * QP;
            const bool row_ok = (int64_t)st * kSN + pr < n_sets;
            const uint8_t *qsrc = q8 + (int64_t)qp * KB * kAStage;
            for (int kb = 0; kb < KB; ++kb, ++u) {
                issue();
                cp_async_wait<kPLag>();
                const int s = u % kNS;
                ok = wait_or_abort(&empty[s], (uint32_t)(((u / kNS) & 1) ^ 1), abort_flag, err);
                if (!ok) break;
                if (p == 0) {
                    mbar_arrive_expect_tx(&full[s], kAStage);
                    bulk_g2s(stA + s * kAStage, qsrc + (int64_t)kb * kAStage, kAStage, &full[s]);
                }
                uint2 w = make_uint2(0, 0);
                if (row_ok) w = *reinterpret_cast<const uint2 *>(ring + ((u % kPR) * kProd + p) * 8);
                // The previous stage is signalled here, one step late: its stores were
                // issued an iteration ago, so the proxy fence does not wait on the
                // stores this iteration is about to make.
                if (u > 0) {
                    fence_proxy_async();
                    mbar_arrive(&full[(u - 1) % kNS]);
                }
                unsigned char *dst = stB + s * kBStage;
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    *reinterpret_cast<uint4 *>(dst + sw128_off(pr, 4 * ph + c)) =
                        spread16((c < 2 ? w.x : w.y) >> (16 * (c & 1)));
            }
        }
        if (ok && u > 0) {
            fence_proxy_async();
            mbar_arrive(&full[(u - 1) % kNS]);
        }
        cp_async_wait<0>();
        if (p == 0 && !ok) {
            // after giving up, let the query-block copies already issued land before the CTA exits
            for (int v = u > kNS ? u - kNS : 0; v < u; ++v)
                mbar_wait_bounded(&full[v % kNS], (uint32_t)((v / kNS) & 1), kWaitNs / 10);
        }
    } else if (warp == 12) {
        // ---- MMA issue: one thread ------------------------------------------------
        if (lane == 0) {
            constexpr uint32_t idesc = umma_idesc_e4m3(kQM, kSN);
            const uint32_t aaddr = smem_u32(stA), baddr = smem_u32(stB);
            bool ok = true;
            int u = 0;
            for (int it = 0; it < n_it && ok; ++it) {
                const int buf = it & 1;
                ok = wait_or_abort(&tempty[buf], (uint32_t)(((it >> 1) & 1) ^ 1), abort_flag, err);
                if (!ok) break;
                tc_fence_after();
                const uint32_t dt = tmem + (uint32_t)(buf * 2 * kSN);
                for (int kb = 0; kb < KB && ok; ++kb, ++u) {
                    const int s = u % kNS;
                    ok = wait_or_abort(&full[s], (uint32_t)((u / kNS) & 1), abort_flag, err);
                    if (!ok) break;
                    tc_fence_after();
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint64_t db = umma_desc_sw128(baddr + s * kBStage + 32 * k);
                        const uint32_t acc = (kb | k) != 0 ? 1u : 0u;
                        umma_f8(dt, umma_desc_sw128(aaddr + s * kAStage + 32 * k), db, idesc, acc);
                        umma_f8(dt + kSN, umma_desc_sw128(aaddr + s * kAStage + kQBlk + 32 * k), db,
                                idesc, acc);
                    }
                    umma_commit(&empty[s]);
                }
                if (ok) umma_commit(&tfull[buf]);
            }
        }
    } else {
        // ---- epilogue: warps 0-3, lane = query row 32w + lane of each block -------
        const int r = warp * 32 + lane;
        const uint32_t g_const = gate_mode == 0 ? 0xffffffffu : 0u;
        bool ok = true;
        for (int it = 0; it < n_it; ++it) {
            // all four warps leave together if one of them gave up
            if (!named_barrier_and(1, kEpi, ok)) break;
            const int tau = (int)blockIdx.x + it * (int)gridDim.x;
            const int st = tau / QP, qp = tau - st * QP;
            const int64_t s0 = (int64_t)st * kSN;
            if (r < kSN) sp_s[r] = s0 + r < n_sets ? spop[s0 + r] : 0;
            named_barrier_sync(2, kEpi);
            // layer-1 words of the tile's 4 groups of 32 sets for both queries, before the wait
            int qh[2], qpc[2];
            uint32_t gw[2][kSN / 32];
#pragma unroll
            for (int b2 = 0; b2 < 2; ++b2) {
                const int q = (2 * qp + b2) * kQM + r;
                const bool qv = q < n_q;
                qh[b2] = qv ? q : -1;
                qpc[b2] = qv ? qpop[q] : 0;
#pragma unroll
                for (int c = 0; c < kSN / 32; ++c)
                    gw[b2][c] = gate_mode == 1
                                    ? (qv && s0 + 32 * c < n_sets ? gate[(int64_t)q * NW + (s0 >> 5) + c] : 0u)
                                    : g_const;
            }
            const int buf = it & 1;
            ok = __all_sync(0xffffffffu,
                            wait_or_abort(&tfull[buf], (uint32_t)((it >> 1) & 1), abort_flag, err));
            if (!ok) continue;
            tc_fence_after();
#pragma unroll
            for (int b2 = 0; b2 < 2; ++b2) {
                uint32_t tmin = kGatedOut;   // minimum score of the row over the tile
#pragma unroll
                for (int c = 0; c < kSN / 32; ++c) {
                    uint32_t v[32];
                    tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) +
                                  (uint32_t)(buf * 2 * kSN + b2 * kSN + c * 32),
                              v);
                    const int64_t sb = s0 + 32 * c;
                    if (qh[b2] >= 0 && sb < n_sets) {
                        const uint32_t g = gw[b2][c];
                        const int qp_b = qpc[b2];
                        uint32_t pk[16];
#pragma unroll
                        for (int j = 0; j < 32; j += 2) {
                            const int d0 = __float2int_rn(__uint_as_float(v[j]) * kDotScale);
                            const int d1 = __float2int_rn(__uint_as_float(v[j + 1]) * kDotScale);
                            const uint32_t h0 = ((g >> j) & 1)
                                                    ? (uint32_t)(qp_b + sp_s[32 * c + j] - 2 * d0)
                                                    : (uint32_t)kGatedOut;
                            const uint32_t h1 = ((g >> (j + 1)) & 1)
                                                    ? (uint32_t)(qp_b + sp_s[32 * c + j + 1] - 2 * d1)
                                                    : (uint32_t)kGatedOut;
                            pk[j >> 1] = (h0 & 0xffffu) | (h1 << 16);
                            if (sb + j < n_sets) tmin = min(tmin, h0);
                            if (sb + j + 1 < n_sets) tmin = min(tmin, h1);
                        }
                        uint16_t *dst = h + (int64_t)qh[b2] * hs + sb;
                        if (sb + 32 <= n_sets) {
                            uint4 *d4 = reinterpret_cast<uint4 *>(dst);
#pragma unroll
                            for (int i = 0; i < 4; ++i)
                                d4[i] = make_uint4(pk[4 * i], pk[4 * i + 1], pk[4 * i + 2], pk[4 * i + 3]);
                        } else {
                            const int nv = (int)(n_sets - sb);
#pragma unroll
                            for (int j = 0; j < 32; ++j)
                                if (j < nv) dst[j] = (uint16_t)(pk[j >> 1] >> (16 * (j & 1)));
                        }
                    }
                    __syncwarp();
                }
                if (bmin && qh[b2] >= 0) bmin[(int64_t)qh[b2] * n_blk + st] = (uint16_t)tmin;
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[buf]);
        }
    }

    // ---- tear-down ----------------------------------------------------------------
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// ---- the same contraction with the set sketches in tensor memory -------------------
// Tile: 128 set sketches (MMA M, the A operand) x 128 query sketches (MMA N, the B
// operand).  The producers expand each K-block of the set rows straight into tensor
// memory (tcgen05.st: a warp writes its own 32 lanes, two warps per lane quarter split
// the block's 32 columns), so only the query block's 16 KB pass through shared memory
// (one bulk copy, one MMA read) per K-block, against 112 KB per twice the work in
// k_scan_mma.  Each expanded set block feeds 128 queries instead of 256, though, so
// the expansion costs twice the ALU work per pair; on a 1000-query batch over 1M sets
// this form takes 5.8 ms against k_scan_mma's 4.1 ms.  A batch of at most 128 query
// sets leaves no half-empty 256-query block here, which is where the tuner may prefer
// it.  The
// accumulator's lanes are sets and its columns queries, so the epilogue takes, per
// query column, one 2-byte score per lane (64 contiguous bytes per warp store) and the
// tile minimum per query from a warp reduction and four warps' partial minima.
constexpr int kTS = 128;                  // set sketches per tile (MMA M)
static_assert(kTS == kSelBlock, "one block minimum per tile");
constexpr int kTN = 128;                  // query sketches per tile (MMA N)
constexpr int kTNS = 8;                   // stages (A in tensor memory, B in shared memory)
constexpr int kTAcc = 2 * kTN;            // two accumulators of kTN columns
constexpr int kTACol = kTAcc;             // first tensor-memory column of the A stages
constexpr uint32_t kTTmemCols = 512;      // kTAcc + kTNS x 32
static_assert(kTAcc + kTNS * 32 <= (int)kTTmemCols, "tensor memory");
constexpr int kTBStage = kTN * 128;       // 16 KB: one query block's K-block
constexpr int kTOffB = 0;
constexpr int kTOffRing = kTOffB + kTNS * kTBStage;
constexpr int kTOffMin = kTOffRing + kPR * kProd * 8;
constexpr int kTOffBars = kTOffMin + 4 * kTN * 4;
constexpr int kTOffMisc = kTOffBars + (2 * kTNS + 4) * 8;
constexpr int kTSmemBytes = kTOffMisc + 16 + 1024;

__global__ void __launch_bounds__(kThreads, 1)
k_scan_tm(const uint32_t *__restrict__ sk, const int32_t *__restrict__ spop, int64_t n_sets,
          int W, const uint32_t *__restrict__ gate, int64_t NW, int gate_mode,
          const uint8_t *__restrict__ q8, const int32_t *__restrict__ qpop, int n_q, int QB,
          uint16_t *__restrict__ h, int64_t hs, uint16_t *__restrict__ bmin, int64_t n_blk,
          int *__restrict__ err) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    unsigned char *stB = smem + kTOffB;
    unsigned char *ring = smem + kTOffRing;
    uint32_t *tmin_s = reinterpret_cast<uint32_t *>(smem + kTOffMin);   // 4 warps x kTN
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kTOffBars);
    uint64_t *full = bars, *empty = bars + kTNS, *tfull = bars + 2 * kTNS,
             *tempty = bars + 2 * kTNS + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + kTOffMisc);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + kTOffMisc + 4);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int KB = W / 4;
    const int n_tiles = (int)((n_sets + kTS - 1) / kTS) * QB;   // < 2^31 (host check)
    const int n_it = n_tiles > (int)blockIdx.x ? (n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

    if (warp == 0) tmem_alloc(tmem_slot, kTTmemCols);
    if (tid == 0) {
        for (int s = 0; s < kTNS; ++s) {
            mbar_init(&full[s], kProd + 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], kEpi / 32);
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp >= 4 && warp <= 11) {
        // ---- producers: thread p expands half ph of set row pr into lane pr ----------
        // (warp w reaches lanes 32 (w % 4) .. + 31, and (w % 4) * 32 + lane == p % 128)
        const int p = tid - 128;
        const int pr = p & (kTS - 1), ph = p >> 7;
        const uint32_t a_lane = (uint32_t)((warp & 3) * 32) << 16;
        int i_it = 0, i_kb = 0, i_u = 0;
        int64_t i_row = (int64_t)((int)blockIdx.x / QB) * kTS + pr;
        auto issue = [&]() {
            if (i_it < n_it) {
                if (i_row < n_sets)
                    cp_async8(ring + ((i_u % kPR) * kProd + p) * 8, sk + i_row * W + 4 * i_kb + 2 * ph);
                if (++i_kb == KB) {
                    i_kb = 0;
                    ++i_it;
                    i_row = (int64_t)(((int)blockIdx.x + i_it * (int)gridDim.x) / QB) * kTS + pr;
                }
            }
            ++i_u;
            cp_async_commit();
        };
        for (int i = 0; i < kPLag; ++i) issue();
        bool ok = true;
        int u = 0;
        for (int it = 0; it < n_it && ok; ++it) {
            const int tau = (int)blockIdx.x + it * (int)gridDim.x;
            const int st = tau / QB, qb = tau - st * QB;
            const bool row_ok = (int64_t)st * kTS + pr < n_sets;
            // query block qb of the operand laid out in pairs of 128-row halves
            const uint8_t *qsrc = q8 + (int64_t)(qb >> 1) * KB * kAStage + (qb & 1) * kQBlk;
            for (int kb = 0; kb < KB; ++kb, ++u) {
                issue();
                cp_async_wait<kPLag>();
                const int s = u % kTNS;
                ok = wait_or_abort(&empty[s], (uint32_t)(((u / kTNS) & 1) ^ 1), abort_flag, err);
                if (!ok) break;
                tc_fence_after();   // the MMAs that read this A stage are complete
                if (p == 0) {
                    mbar_arrive_expect_tx(&full[s], kTBStage);
                    bulk_g2s(stB + s * kTBStage, qsrc + (int64_t)kb * kAStage, kTBStage, &full[s]);
                }
                uint2 w = make_uint2(0, 0);
                if (row_ok) w = *reinterpret_cast<const uint2 *>(ring + ((u % kPR) * kProd + p) * 8);
                // The previous stage is signalled here, one step late, once its
                // tensor-memory stores have completed.
                if (u > 0) {
                    tmem_wait_st();
                    tc_fence_before();
                    mbar_arrive(&full[(u - 1) % kTNS]);
                }
                uint32_t a[16];
#pragma unroll
                for (int c = 0; c < 16; ++c)
                    a[c] = spread4(((c < 8 ? w.x : w.y) >> (4 * (c & 7))) & 0xF);
                tmem_st16(tmem + a_lane + (uint32_t)(kTACol + s * 32 + ph * 16), a);
            }
        }
        if (ok && u > 0) {
            tmem_wait_st();
            tc_fence_before();
            mbar_arrive(&full[(u - 1) % kTNS]);
        }
        cp_async_wait<0>();
        if (p == 0 && !ok) {
            // after giving up, let the query-block copies already issued land before the CTA exits
            for (int v = u > kTNS ? u - kTNS : 0; v < u; ++v)
                mbar_wait_bounded(&full[v % kTNS], (uint32_t)((v / kTNS) & 1), kWaitNs / 10);
        }
    } else if (warp == 12) {
        // ---- MMA issue: one thread ------------------------------------------------
        if (lane == 0) {
            constexpr uint32_t idesc = umma_idesc_e4m3(kTS, kTN);
            const uint32_t baddr = smem_u32(stB);
            bool ok = true;
            int u = 0;
            for (int it = 0; it < n_it && ok; ++it) {
                const int buf = it & 1;
                ok = wait_or_abort(&tempty[buf], (uint32_t)(((it >> 1) & 1) ^ 1), abort_flag, err);
                if (!ok) break;
                tc_fence_after();
                const uint32_t dt = tmem + (uint32_t)(buf * kTN);
                for (int kb = 0; kb < KB && ok; ++kb, ++u) {
                    const int s = u % kTNS;
                    ok = wait_or_abort(&full[s], (uint32_t)((u / kTNS) & 1), abort_flag, err);
                    if (!ok) break;
                    tc_fence_after();
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        umma_f8_tmem_a(dt, tmem + (uint32_t)(kTACol + s * 32 + 8 * k),
                                       umma_desc_sw128(baddr + s * kTBStage + 32 * k), idesc,
                                       (kb | k) != 0 ? 1u : 0u);
                    umma_commit(&empty[s]);
                }
                if (ok) umma_commit(&tfull[buf]);
            }
        }
    } else {
        // ---- epilogue: warps 0-3, lane = set 32w + lane of the tile, column = query ----
        const uint32_t g_const = gate_mode == 0 ? 0xffffffffu : 0u;
        bool ok = true;
        for (int it = 0; it < n_it; ++it) {
            // all four warps leave together if one of them gave up
            if (!named_barrier_and(1, kEpi, ok)) break;
            const int tau = (int)blockIdx.x + it * (int)gridDim.x;
            const int st = tau / QB, qb = tau - st * QB;
            const int64_t s0 = (int64_t)st * kTS;
            const int64_t sidx = s0 + warp * 32 + lane;
            const bool vs = sidx < n_sets;
            const bool grp = s0 + warp * 32 < n_sets;
            const int spl = vs ? spop[sidx] : 0;
            // lane j of group c: query qb kTN + 32 c + j's layer-1 word for this warp's 32
            // sets and its |S_Q|, loaded before the wait
            uint32_t gw[kTN / 32];
            int qpl[kTN / 32];
#pragma unroll
            for (int c = 0; c < kTN / 32; ++c) {
                const int q = qb * kTN + 32 * c + lane;
                const bool qv = q < n_q;
                qpl[c] = qv ? qpop[q] : 0;
                gw[c] = gate_mode == 1 ? (qv && grp ? gate[(int64_t)q * NW + (s0 >> 5) + warp] : 0u)
                                       : g_const;
            }
            const int buf = it & 1;
            ok = __all_sync(0xffffffffu,
                            wait_or_abort(&tfull[buf], (uint32_t)((it >> 1) & 1), abort_flag, err));
            if (!ok) continue;
            tc_fence_after();
#pragma unroll
            for (int c = 0; c < kTN / 32; ++c) {
                uint32_t v[32];
                tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(buf * kTN + c * 32), v);
                const int q0 = qb * kTN + 32 * c;
                uint32_t mine = kGatedOut;   // lane j: this warp's minimum for query q0 + j
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const uint32_t g = __shfl_sync(0xffffffffu, gw[c], j);
                    const int qp_j = __shfl_sync(0xffffffffu, qpl[c], j);
                    const int dot = __float2int_rn(__uint_as_float(v[j]) * kDotScale);
                    const uint32_t hv =
                        ((g >> lane) & 1) ? (uint32_t)(qp_j + spl - 2 * dot) : (uint32_t)kGatedOut;
                    if (vs && q0 + j < n_q) h[(int64_t)(q0 + j) * hs + sidx] = (uint16_t)hv;
                    const uint32_t mn = __reduce_min_sync(0xffffffffu, vs ? hv : (uint32_t)kGatedOut);
                    if (lane == j) mine = mn;
                }
                tmin_s[warp * kTN + 32 * c + lane] = mine;
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[buf]);
            named_barrier_sync(2, kEpi);   // the four warps' partial minima are visible
            const int q = qb * kTN + tid;
            if (bmin && q < n_q) {
                uint32_t m4 = tmin_s[tid];
#pragma unroll
                for (int w2 = 1; w2 < 4; ++w2) m4 = min(m4, tmin_s[w2 * kTN + tid]);
                bmin[(int64_t)q * n_blk + st] = (uint16_t)m4;
            }
        }
    }

    // ---- tear-down ----------------------------------------------------------------
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, kTTmemCols);
}

// |S_i| per database sketch, one warp per set
__global__ void k_sketch_pop(const uint32_t *__restrict__ sk, int64_t n_sets, int W,
                             int32_t *__restrict__ spop) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < n_sets;
         i += warps) {
        int c = 0;
        for (int k = lane; k < W; k += 32) c += __popc(sk[i * W + k]);
        c = __reduce_add_sync(0xffffffffu, (uint32_t)c);
        if (lane == 0) spop[i] = c;
    }
}

int sm_count_mma() {
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

size_t scan_mma_q8_bytes(int64_t n_q, int m) {
    return (size_t)((n_q + 2 * kQM - 1) / (2 * kQM)) * 2 * kQM * (size_t)m;
}

cudaError_t launch_sketch_pop(const uint32_t *sketch, int64_t n_sets, int W, int32_t *spop,
                              cudaStream_t st) {
    if (n_sets <= 0) return cudaSuccess;
    int64_t g = (n_sets + 7) / 8;
    if (g > (1 << 16)) g = 1 << 16;
    k_sketch_pop<<<(unsigned)g, 256, 0, st>>>(sketch, n_sets, W, spop);
    return cudaGetLastError();
}

cudaError_t launch_expand_q(const uint32_t *sq, int n_q, int W, uint8_t *q8, int32_t *qpop,
                            cudaStream_t st) {
    if (n_q <= 0) return cudaSuccess;
    const int QP = (n_q + 2 * kQM - 1) / (2 * kQM);
    const int64_t total = (int64_t)QP * 2 * kQM * (W / 4);
    int64_t g = (total + 255) / 256;
    if (g > 4096) g = 4096;
    k_expand_q<<<(unsigned)g, 256, 0, st>>>(sq, n_q, W, QP, q8, qpop);
    return cudaGetLastError();
}

cudaError_t launch_scan_mma(const uint32_t *sketch, const int32_t *spop, int64_t n_sets, int W,
                            const uint32_t *gate, int64_t NW, int gate_mode, const uint8_t *q8,
                            const int32_t *qpop, int n_q, uint16_t *h, int64_t hs, int *err,
                            cudaStream_t st, uint16_t *bmin) {
    if (n_q <= 0 || n_sets <= 0) return cudaSuccess;
    const int QP = (n_q + 2 * kQM - 1) / (2 * kQM);
    cudaError_t e = cudaFuncSetAttribute(k_scan_mma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kSmemBytes);
    if (e != cudaSuccess) return e;
    const int64_t n_tiles = ((n_sets + kSN - 1) / kSN) * QP;
    if (n_tiles >= ((int64_t)1 << 31)) return cudaErrorInvalidValue;
    int64_t grid = sm_count_mma();
    if (grid > n_tiles) grid = n_tiles;
    k_scan_mma<<<(unsigned)grid, kThreads, kSmemBytes, st>>>(sketch, spop, n_sets, W, gate, NW,
                                                             gate_mode, q8, qpop, n_q, QP, h,
                                                             hs, bmin, (n_sets + kSN - 1) / kSN,
                                                             err);
    return cudaGetLastError();
}

cudaError_t launch_scan_tm(const uint32_t *sketch, const int32_t *spop, int64_t n_sets, int W,
                           const uint32_t *gate, int64_t NW, int gate_mode, const uint8_t *q8,
                           const int32_t *qpop, int n_q, uint16_t *h, int64_t hs, int *err,
                           cudaStream_t st, uint16_t *bmin) {
    if (n_q <= 0 || n_sets <= 0) return cudaSuccess;
    const int QB = (n_q + kTN - 1) / kTN;
    cudaError_t e = cudaFuncSetAttribute(k_scan_tm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kTSmemBytes);
    if (e != cudaSuccess) return e;
    const int64_t n_tiles = ((n_sets + kTS - 1) / kTS) * QB;
    if (n_tiles >= ((int64_t)1 << 31)) return cudaErrorInvalidValue;
    int64_t grid = sm_count_mma();
    if (grid > n_tiles) grid = n_tiles;
    k_scan_tm<<<(unsigned)grid, kThreads, kTSmemBytes, st>>>(sketch, spop, n_sets, W, gate, NW,
                                                            gate_mode, q8, qpop, n_q, QB, h, hs,
                                                            bmin, (n_sets + kTS - 1) / kTS, err);
    return cudaGetLastError();
}

}  // namespace bvss
