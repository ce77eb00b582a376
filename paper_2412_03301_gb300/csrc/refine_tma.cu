// refine_tma.cu -- exact re-rank of Alg. 6 (lines 19-22) of arXiv 2412.03301
// with candidate rows streamed by TMA bulk copies, one pipeline per warp.
//
// A CTA takes one query set (its vectors staged in shared memory once) and up
// to 32 candidates per warp.  Each warp walks the rows of its candidates,
// concatenated in candidate order, in tiles of 32 rows; a tile arrives in
// chunks of 64 dimensions, one cp.async.bulk per row and chunk, into a
// two-stage ring of the warp's own shared memory guarded by its own
// mbarriers, so the next chunk is in flight while the current one is used.
// There is no block-wide barrier after set-up: warps never wait for each
// other.
//
// Per tile a warp accumulates the dot products of (up to) 32 query vectors x
// 32 rows, 4 x 8 per lane, turns them into squared distances
// |q|^2 + |v|^2 - 2 q.v (Def. 4 in GEMM form) and walks the rows in order:
// lanes keep, for their query vector, the minimum over the open candidate's
// rows, and the warp keeps the maximum over those rows of the minimum over
// the query vectors.  When the walk leaves a candidate, the pair attaining its
// Hausdorff value is re-scored directly as sum((q - v)^2) and the square root
// is written.  mbarrier waits give up after 2 s and report an error.
#include "bvss_internal.cuh"
#include "ptx_util.cuh"

namespace bvss {

namespace {

constexpr int kRowsT = 32;        // rows per tile
constexpr int kKC = 64;           // dimensions per chunk
constexpr int kKCP = kKC + 4;     // padded stage row (floats): bank-conflict-free reads
constexpr int kCandW = 32;        // candidates per warp
constexpr int kMaxWarps = 8;
constexpr uint64_t kWaitNs = 2000000000ull;
constexpr int kSmemMax = 232448;  // 227 KB opt-in limit per CTA

__host__ __device__ constexpr int align16(int x) { return (x + 15) & ~15; }

__host__ __device__ inline int q_bytes(int d, int nat) {
    return align16((32 * nat * (d + 4) + 32 * nat) * 4);
}
__host__ __device__ inline int warp_bytes(int nat) {
    return align16(16 + 2 * kRowsT * kKCP * 4 + kRowsT * (32 * nat + 1) * 4);
}

template <int NAT>
__global__ void __launch_bounds__(kMaxWarps * 32, 1)
k_refine_tma(const float *__restrict__ qvec, const int64_t *__restrict__ qoff,
             const float *__restrict__ vec, const float *__restrict__ vnorm,
             const int64_t *__restrict__ set_off, int d, int nwarps,
             const int32_t *__restrict__ cand, const int32_t *__restrict__ thr, int C,
             float *__restrict__ cand_dist, int *__restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int q = blockIdx.y;
    const int n_sel = thr[q * 4 + 3];
    const int c_cta = blockIdx.x * kCandW * nwarps;
    if (c_cta >= n_sel) return;                      // uniform over the CTA
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t a0 = qoff[q];
    const int mq = (int)(qoff[q + 1] - a0);
    const int dq = d + 4, d4 = d / 4;
    float *Qs = reinterpret_cast<float *>(smem);
    float *qn = Qs + 32 * NAT * dq;
    unsigned char *wb = smem + q_bytes(d, NAT) + warp * warp_bytes(NAT);
    uint64_t *bars = reinterpret_cast<uint64_t *>(wb);
    float *stg = reinterpret_cast<float *>(wb + 16);
    float *D = stg + 2 * kRowsT * kKCP;
    constexpr int DS = 32 * NAT + 1;
    const float INF = __int_as_float(0x7f800000);

    // the query set, zero rows past its end, and its squared norms
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int e = tid; e < 32 * NAT * d4; e += blockDim.x) {
        const int r = e / d4, c = e % d4;
        const float4 v = r < mq ? reinterpret_cast<const float4 *>(qvec + (a0 + r) * d)[c] : zero4;
        reinterpret_cast<float4 *>(Qs + (size_t)r * dq)[c] = v;
    }
    __syncthreads();
    for (int a = warp; a < 32 * NAT; a += nwarps) {
        float s = 0.0f;
        for (int k = lane; k < d4; k += 32) {
            const float4 t = reinterpret_cast<const float4 *>(Qs + (size_t)a * dq)[k];
            s = fmaf(t.x, t.x, s);
            s = fmaf(t.y, t.y, s);
            s = fmaf(t.z, t.z, s);
            s = fmaf(t.w, t.w, s);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) qn[a] = s;
    }
    if (lane == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncthreads();   // the last block-wide barrier

    // this warp's candidates: lane c holds candidate c's first global row, size
    // and first row in the warp's concatenated row order
    const int cw0 = c_cta + warp * kCandW;
    const int ncw = min(kCandW, n_sel - cw0);
    if (ncw <= 0) return;
    int64_t g0 = 0;
    int n = 0;
    if (lane < ncw) {
        const int64_t id = cand[(int64_t)q * C + cw0 + lane];
        g0 = set_off[id];
        n = (int)(set_off[id + 1] - g0);
    }
    int incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const int vr0 = incl - n;
    const int R = __shfl_sync(0xffffffffu, incl, 31);
    const int n_tiles = (R + kRowsT - 1) / kRowsT;
    const int KCH = (d + kKC - 1) / kKC;
    const int total = n_tiles * KCH;

    // candidate slot and global row of concatenated row v (all lanes call it)
    auto locate = [&](int v, int &slot, int64_t &grow) {
        int s = 0;
#pragma unroll
        for (int b = 16; b > 0; b >>= 1) {
            const int c = s + b;
            const int vc = __shfl_sync(0xffffffffu, vr0, c & 31);
            if (c < ncw && vc <= v) s = c;
        }
        slot = s;
        grow = __shfl_sync(0xffffffffu, g0, s) + (v - __shfl_sync(0xffffffffu, vr0, s));
    };
    auto issue = [&](int u) {
        const int t = u / KCH, kc = u - (u / KCH) * KCH;
        const int nr = min(kRowsT, R - kRowsT * t);
        const int w = min(kKC, d - kc * kKC);
        float *dst = stg + (u & 1) * kRowsT * kKCP;
        int s;
        int64_t g;
        locate(min(kRowsT * t + lane, R - 1), s, g);
        if (lane == 0) mbar_arrive_expect_tx(&bars[u & 1], (uint32_t)(nr * w * 4));
        __syncwarp();
        if (lane < nr)
            bulk_g2s(dst + lane * kKCP, vec + g * d + kc * kKC, (uint32_t)(w * 4), &bars[u & 1]);
    };

    if (total > 0) issue(0);
    if (total > 1) issue(1);

    const int la = lane & 7, lr = lane >> 3;
    float acc[NAT][4][8];
    // the open candidate: per-lane row minima (query vector a = at*32 + lane)
    int open = -1;
    float rmin[NAT];
    int rrow[NAT];
    long long cmax_key = -1;   // max over rows of min over a: (d2 bits << 32) | (row << 8) | a
    auto finalize = [&](int c) {
        uint32_t best = 0;
        int best_a = 0, best_r = 0;
        bool have = false;
#pragma unroll
        for (int at = 0; at < NAT; ++at) {
            const int a = at * 32 + lane;
            const bool va = a < mq;
            const uint32_t bits = va ? __float_as_uint(rmin[at]) : 0u;
            const uint32_t mx = __reduce_max_sync(0xffffffffu, bits);
            const uint32_t who = __ballot_sync(0xffffffffu, va && bits == mx);
            if (who) {
                const int src = __ffs(who) - 1;
                const int rr = __shfl_sync(0xffffffffu, rrow[at], src);
                if (!have || mx > best) {
                    best = mx;
                    best_a = at * 32 + src;
                    best_r = rr;
                    have = true;
                }
            }
        }
        int pa = best_a, pr = best_r;
        if ((long long)best < (cmax_key >> 32)) {
            pa = (int)(cmax_key & 0xff);
            pr = (int)((cmax_key >> 8) & 0xffffff);
        }
        const int64_t grow = __shfl_sync(0xffffffffu, g0, c) + pr;
        const float4 *x4 = reinterpret_cast<const float4 *>(Qs + (size_t)pa * dq);
        const float4 *y4 = reinterpret_cast<const float4 *>(vec + grow * d);
        float s = 0.0f;
        for (int k = lane; k < d4; k += 32) {
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
        if (lane == 0) cand_dist[(int64_t)q * C + cw0 + c] = sqrtf(s);
    };

    bool failed = false;
    for (int u = 0; u < total; ++u) {
        const int t = u / KCH, kc = u - (u / KCH) * KCH;
        if (kc == 0) {
#pragma unroll
            for (int at = 0; at < NAT; ++at)
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[at][i][j] = 0.0f;
        }
        if (!mbar_wait_bounded(&bars[u & 1], (uint32_t)((u >> 1) & 1), kWaitNs)) failed = true;
        if (__any_sync(0xffffffffu, failed)) {
            failed = true;
            break;
        }
        const float *St = stg + (u & 1) * kRowsT * kKCP;
        const float *qb = Qs + kc * kKC;
        const int w4 = min(kKC, d - kc * kKC) / 4;
        for (int k4 = 0; k4 < w4; ++k4) {
            float4 vv[8];
#pragma unroll
            for (int j = 0; j < 8; ++j)
                vv[j] = *reinterpret_cast<const float4 *>(St + (lr + 4 * j) * kKCP + 4 * k4);
#pragma unroll
            for (int at = 0; at < NAT; ++at) {
                float4 qv[4];
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    qv[i] = *reinterpret_cast<const float4 *>(
                        qb + (size_t)(at * 32 + la + 8 * i) * dq + 4 * k4);
                // component-major: 32 independent accumulators between dependent FMAs
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[at][i][j] = fmaf(qv[i].x, vv[j].x, acc[at][i][j]);
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[at][i][j] = fmaf(qv[i].y, vv[j].y, acc[at][i][j]);
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[at][i][j] = fmaf(qv[i].z, vv[j].z, acc[at][i][j]);
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[at][i][j] = fmaf(qv[i].w, vv[j].w, acc[at][i][j]);
            }
        }
        __syncwarp();                  // every lane is done with this stage
        if (u + 2 < total) issue(u + 2);
        if (kc != KCH - 1) continue;

        // tile t complete: squared distances into D[row][a]
        const int nr = min(kRowsT, R - kRowsT * t);
        int my_slot;
        int64_t my_grow;
        locate(min(kRowsT * t + lane, R - 1), my_slot, my_grow);
        const float my_vn = lane < nr ? vnorm[my_grow] : 0.0f;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float vn = __shfl_sync(0xffffffffu, my_vn, lr + 4 * j);
#pragma unroll
            for (int at = 0; at < NAT; ++at)
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int a = at * 32 + la + 8 * i;
                    const float d2 = qn[a] + vn - 2.0f * acc[at][i][j];
                    D[(lr + 4 * j) * DS + a] = d2 > 0.0f ? d2 : 0.0f;
                }
        }
        __syncwarp();
        // walk the tile's rows in order
        for (int r = 0; r < nr; ++r) {
            const int slot = __shfl_sync(0xffffffffu, my_slot, r);
            if (slot != open) {
                if (open >= 0) finalize(open);
                open = slot;
#pragma unroll
                for (int at = 0; at < NAT; ++at) {
                    rmin[at] = INF;
                    rrow[at] = 0;
                }
                cmax_key = -1;
            }
            const int row_in = kRowsT * t + r - __shfl_sync(0xffffffffu, vr0, slot);
            uint32_t cm = 0xffffffffu;
            int cma = 0;
#pragma unroll
            for (int at = 0; at < NAT; ++at) {
                const int a = at * 32 + lane;
                const float v = a < mq ? D[r * DS + a] : INF;
                if (v < rmin[at]) {
                    rmin[at] = v;
                    rrow[at] = row_in;
                }
                const uint32_t b = __float_as_uint(v);
                const uint32_t mn = __reduce_min_sync(0xffffffffu, b);
                if (mn < cm) {
                    cm = mn;
                    cma = at * 32 + __ffs(__ballot_sync(0xffffffffu, b == mn)) - 1;
                }
            }
            const long long key = ((long long)cm << 32) | ((long long)row_in << 8) | cma;
            if (key > cmax_key) cmax_key = key;
        }
        __syncwarp();                  // D is rewritten by the next tile
    }
    if (failed) {
        if (lane == 0) {
            atomicOr(err, 1);
            // copies of this warp still in flight get one more bounded wait
            mbar_wait_bounded(&bars[0], 0u, kWaitNs);
        }
        __syncwarp();
        return;
    }
    if (open >= 0) finalize(open);
}

// waits for a phase that never completes (nothing arrives), bounded by limit_ns
__global__ void k_wait_selftest(int *err, uint64_t limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bar, 0u, limit_ns);
    if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicOr(err, 1);
}

int tma_warps(int d, int nat) {
    const int free = kSmemMax - q_bytes(d, nat);
    if (free <= 0) return 0;
    const int w = free / warp_bytes(nat);
    return w > kMaxWarps ? kMaxWarps : w;
}

}  // namespace

cudaError_t launch_wait_selftest(int *err, uint64_t limit_ns, cudaStream_t st) {
    k_wait_selftest<<<1, 32, 0, st>>>(err, limit_ns);
    return cudaGetLastError();
}

bool refine_tma_supported(int d, int max_mq) {
    if (d % 4 != 0 || max_mq < 1 || max_mq > 64) return false;
    return tma_warps(d, (max_mq + 31) / 32) >= 2;
}

cudaError_t launch_refine_tma(const float *qvec, const int64_t *qoff, int n_q, int max_mq,
                              const float *vec, const float *vnorm, const int64_t *set_off,
                              int d, const int32_t *cand, const int32_t *thr, int C,
                              float *cand_dist, int *err, cudaStream_t st) {
    if (n_q <= 0) return cudaSuccess;
    const int nat = (max_mq + 31) / 32;
    const int nw = tma_warps(d, nat);
    if (nw < 2 || nat > 2) return cudaErrorInvalidValue;
    const int smem = q_bytes(d, nat) + nw * warp_bytes(nat);
    const int gx = (C + kCandW * nw - 1) / (kCandW * nw);
    cudaError_t e;
    if (nat == 1) {
        e = cudaFuncSetAttribute(k_refine_tma<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem);
        if (e != cudaSuccess) return e;
        k_refine_tma<1><<<dim3(gx, n_q), nw * 32, smem, st>>>(qvec, qoff, vec, vnorm, set_off, d,
                                                              nw, cand, thr, C, cand_dist, err);
    } else {
        e = cudaFuncSetAttribute(k_refine_tma<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem);
        if (e != cudaSuccess) return e;
        k_refine_tma<2><<<dim3(gx, n_q), nw * 32, smem, st>>>(qvec, qoff, vec, vnorm, set_off, d,
                                                              nw, cand, thr, C, cand_dist, err);
    }
    return cudaGetLastError();
}

}  // namespace bvss
