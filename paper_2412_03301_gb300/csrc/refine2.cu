// refine2.cu -- exact re-rank of Alg. 6 (lines 19-22) of arXiv 2412.03301,
// staged through shared memory with TMA bulk copies.
//
// One CTA takes one query set and up to 32 of its candidates.  The rows of
// those candidates, concatenated in candidate order, are cut into tiles of
// 32 rows; every row of a tile is brought into shared memory by one
// cp.async.bulk (rows padded by 16 bytes so the compute reads are free of
// bank conflicts) into a ring of NS stages guarded by mbarriers, so NS - 1
// tiles are in flight while one is computed.
//
// Each of the 8 warps takes one eighth of the dimension d and accumulates the
// dot products of a 32 (query vectors) x 32 (tile rows) block, 4 x 8 per
// lane.  The eight partial blocks are summed through shared memory, turned
// into squared distances |q|^2 + |v|^2 - 2 q.v (Def. 4 in GEMM form), and
// folded into, per candidate, the row minima over its vectors (for every query
// vector) and the column maxima of the per-row minima over the query vectors.
// When a candidate's last row has been seen, the pair that attains its
// Hausdorff value is re-scored directly as sum((q - v)^2) and its square root
// written.  Waits on the mbarriers give up after 2 s and report an error.
#include "bvss_internal.cuh"
#include "ptx_util.cuh"

namespace bvss {

namespace {

constexpr int kT = 256;
constexpr int kW = kT / 32;
constexpr int kRowsT = 32;            // rows per tile
constexpr int kCandB = 32;            // candidates per CTA
constexpr int kMaxMq = 64;            // query vectors per set (two tiles of 32)
constexpr int kMaxNS = 4;
constexpr int kPStride = 40;          // row stride of the partial blocks (conflict-free)
constexpr int kPartialBytes = kW * kRowsT * kPStride * 4;
constexpr uint64_t kWaitNs = 2000000000ull;
constexpr int kSmemMax = 232448;      // 227 KB opt-in limit per CTA

__host__ __device__ constexpr int align128(int x) { return (x + 127) & ~127; }

// byte offsets of the shared-memory regions
struct Layout {
    int rowmin, colmax, colrun, grow0, vrow0, nrows, qn, q, stages, partial, total;
};

__host__ __device__ inline Layout make_layout(int d, int mq_pad, int NS, int alias) {
    Layout L;
    const int dp = d + 4;
    int o = 64;                                    // NS (<= 8) mbarriers
    L.rowmin = o;  o += kCandB * kMaxMq * 8;
    L.colmax = o;  o += kCandB * 8;
    L.colrun = o;  o += kRowsT * 8;
    L.grow0 = o;   o += kCandB * 8;
    L.vrow0 = o;   o += (kCandB + 4) * 4;
    L.nrows = o;   o += kCandB * 4;
    L.qn = o;      o += kMaxMq * 4;
    o = align128(o);
    L.q = o;       o += mq_pad * dp * 4;
    o = align128(o);
    L.stages = o;  o += NS * kRowsT * dp * 4;
    L.partial = alias ? -1 : o;
    if (!alias) o += kPartialBytes;
    L.total = o;
    return L;
}

__device__ __forceinline__ unsigned long long pack_hi(float v, unsigned lo) {
    return ((unsigned long long)__float_as_uint(v) << 32) | lo;
}

__global__ void __launch_bounds__(kT, 1)
k_refine2(const float *__restrict__ qvec, const int64_t *__restrict__ qoff,
          const float *__restrict__ vec, const float *__restrict__ vnorm,
          const int64_t *__restrict__ set_off, int d, int NS, int alias,
          const int32_t *__restrict__ cand, const int32_t *__restrict__ thr, int C,
          float *__restrict__ cand_dist, int *__restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int q = blockIdx.y;
    const int n_sel = thr[q * 4 + 3];
    const int c0 = blockIdx.x * kCandB;
    if (c0 >= n_sel) return;                      // uniform over the CTA
    const int ncand = min(kCandB, n_sel - c0);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t a0 = qoff[q];
    const int mq = (int)(qoff[q + 1] - a0);
    const int n_at = (mq + 31) / 32;
    const int mq_pad = n_at * 32;
    const int dp = d + 4, d4 = d / 4;
    const Layout Lo = make_layout(d, mq_pad, NS, alias);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    unsigned long long *rowmin = reinterpret_cast<unsigned long long *>(smem + Lo.rowmin);
    unsigned long long *colmax = reinterpret_cast<unsigned long long *>(smem + Lo.colmax);
    unsigned long long *colrun = reinterpret_cast<unsigned long long *>(smem + Lo.colrun);
    int64_t *s_grow0 = reinterpret_cast<int64_t *>(smem + Lo.grow0);
    int *s_vrow0 = reinterpret_cast<int *>(smem + Lo.vrow0);
    int *s_n = reinterpret_cast<int *>(smem + Lo.nrows);
    float *qn = reinterpret_cast<float *>(smem + Lo.qn);
    float *Qs = reinterpret_cast<float *>(smem + Lo.q);
    float *stages = reinterpret_cast<float *>(smem + Lo.stages);
    float *partial_sep = alias ? nullptr : reinterpret_cast<float *>(smem + Lo.partial);
    const float INF = __int_as_float(0x7f800000);

    if (tid == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        int n = 0;
        int64_t g0 = 0;
        if (lane < ncand) {
            const int64_t id = cand[(int64_t)q * C + c0 + lane];
            g0 = set_off[id];
            n = (int)(set_off[id + 1] - g0);
        }
        int x = n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        s_vrow0[lane] = x - n;
        s_n[lane] = n;
        s_grow0[lane] = g0;
        if (lane == 31) s_vrow0[kCandB] = x;      // total rows of the CTA
    }
    for (int e = tid; e < kCandB * kMaxMq; e += kT) rowmin[e] = ~0ull;
    for (int e = tid; e < kCandB; e += kT) colmax[e] = 0ull;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int e = tid; e < mq_pad * d4; e += kT) {
        const int r = e / d4, c = e % d4;
        const float4 v = r < mq ? reinterpret_cast<const float4 *>(qvec + (a0 + r) * d)[c] : zero4;
        reinterpret_cast<float4 *>(Qs + (size_t)r * dp)[c] = v;
    }
    __syncthreads();
    for (int a = warp; a < mq_pad; a += kW) {
        float s = 0.0f;
        for (int k = lane; k < d4; k += 32) {
            const float4 t = reinterpret_cast<const float4 *>(Qs + (size_t)a * dp)[k];
            s = fmaf(t.x, t.x, s);
            s = fmaf(t.y, t.y, s);
            s = fmaf(t.z, t.z, s);
            s = fmaf(t.w, t.w, s);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) qn[a] = s;
    }
    const int R = s_vrow0[kCandB];
    const int n_tiles = (R + kRowsT - 1) / kRowsT;

    // candidate slot of virtual row v (slots are in increasing row order)
    auto slot_of = [&](int v) {
        int c = 0;
#pragma unroll
        for (int b = 16; b > 0; b >>= 1)
            if (c + b < ncand && s_vrow0[c + b] <= v) c += b;
        return c;
    };
    // producer: warp 0 loads tile t into stage t % NS, one bulk copy per row
    auto issue = [&](int t) {
        const int s = t % NS;
        const int r0v = t * kRowsT;
        const int nr = min(kRowsT, R - r0v);
        if (lane == 0) mbar_arrive_expect_tx(&bars[s], (uint32_t)(nr * d * 4));
        __syncwarp();
        if (lane < nr) {
            const int v = r0v + lane;
            const int c = slot_of(v);
            const int64_t g = s_grow0[c] + (v - s_vrow0[c]);
            bulk_g2s(stages + ((size_t)s * kRowsT + lane) * dp, vec + g * d, (uint32_t)(d * 4),
                     &bars[s]);
        }
    };
    __syncthreads();
    if (warp == 0)
        for (int t = 0; t < NS && t < n_tiles; ++t) issue(t);

    const int la = lane & 7, lr = lane >> 3;
    const int k4_lo = warp * d4 / kW, k4_hi = (warp + 1) * d4 / kW;
    for (int t = 0; t < n_tiles; ++t) {
        const int s = t % NS;
        const bool ok = mbar_wait_bounded(&bars[s], (uint32_t)((t / NS) & 1), kWaitNs);
        if (__syncthreads_or(!ok)) {
            // give copies still in flight one more bounded chance to land, then report
            if (tid == 0) {
                atomicOr(err, 1);
                for (int u = t; u < t + NS && u < n_tiles; ++u)
                    mbar_wait_bounded(&bars[u % NS], (uint32_t)((u / NS) & 1), kWaitNs);
            }
            __syncthreads();
            return;
        }
        const int r0v = t * kRowsT;
        const int nr = min(kRowsT, R - r0v);
        const float *St = stages + (size_t)s * kRowsT * dp;
        float *Pt = alias ? const_cast<float *>(St) : partial_sep;
        for (int at = 0; at < n_at; ++at) {
            float acc[4][8];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
            const float *qa = Qs + (size_t)(at * 32 + la) * dp;
            const float *vr = St + (size_t)lr * dp;
            for (int k4 = k4_lo; k4 < k4_hi; ++k4) {
                float4 qv[4], vv[8];
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    qv[i] = *reinterpret_cast<const float4 *>(qa + (size_t)(8 * i) * dp + 4 * k4);
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    vv[j] = *reinterpret_cast<const float4 *>(vr + (size_t)(4 * j) * dp + 4 * k4);
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        acc[i][j] = fmaf(qv[i].x, vv[j].x, acc[i][j]);
                        acc[i][j] = fmaf(qv[i].y, vv[j].y, acc[i][j]);
                        acc[i][j] = fmaf(qv[i].z, vv[j].z, acc[i][j]);
                        acc[i][j] = fmaf(qv[i].w, vv[j].w, acc[i][j]);
                    }
            }
            __syncthreads();   // every warp is done reading the stage (it may hold the partials)
            // partial block of this warp: [r][a], row stride kPStride
            float *pw = Pt + (size_t)warp * kRowsT * kPStride;
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) pw[(lr + 4 * j) * kPStride + la + 8 * i] = acc[i][j];
            __syncthreads();
            {
                const int r = tid >> 3, ag = tid & 7;
                float4 sum = zero4;
#pragma unroll
                for (int w = 0; w < kW; ++w) {
                    const float4 pv = *reinterpret_cast<const float4 *>(
                        Pt + ((size_t)w * kRowsT + r) * kPStride + ag * 4);
                    sum.x += pv.x;
                    sum.y += pv.y;
                    sum.z += pv.z;
                    sum.w += pv.w;
                }
                const bool rv = r < nr;
                const int c = slot_of(r0v + (rv ? r : 0));
                const int row_in = r0v + r - s_vrow0[c];
                const float vn = rv ? vnorm[s_grow0[c] + row_in] : 0.0f;
                const float dots[4] = {sum.x, sum.y, sum.z, sum.w};
                float dmin = INF;
                int amin = 0;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int a = at * 32 + ag * 4 + i;
                    float d2 = qn[a] + vn - 2.0f * dots[i];
                    d2 = d2 > 0.0f ? d2 : 0.0f;
                    if (rv && a < mq) {
                        atomicMin(&rowmin[c * kMaxMq + a], pack_hi(d2, (unsigned)row_in));
                        if (d2 < dmin) {
                            dmin = d2;
                            amin = a;
                        }
                    }
                }
#pragma unroll
                for (int o = 1; o < 8; o <<= 1) {
                    const float od = __shfl_xor_sync(0xffffffffu, dmin, o);
                    const int oa = __shfl_xor_sync(0xffffffffu, amin, o);
                    if (od < dmin || (od == dmin && oa < amin)) {
                        dmin = od;
                        amin = oa;
                    }
                }
                if (ag == 0 && rv) {
                    const unsigned long long key = pack_hi(dmin, (unsigned)amin);
                    if (at == 0 || key < colrun[r]) colrun[r] = key;
                }
            }
            __syncthreads();
        }
        // fold each row's minimum over the query into its candidate's maximum
        if (tid < nr) {
            const int c = slot_of(r0v + tid);
            const int row_in = r0v + tid - s_vrow0[c];
            const unsigned long long cr = colrun[tid];
            atomicMax(&colmax[c], (cr & 0xffffffff00000000ull) |
                                      ((unsigned long long)row_in << 16) | (cr & 0xffffull));
        }
        __syncthreads();
        if (warp == 0 && t + NS < n_tiles) issue(t + NS);
        // candidates whose last row is in this tile: Hausdorff value and re-score
        for (int c = warp; c < ncand; c += kW) {
            const int end = s_vrow0[c] + s_n[c];
            if (end <= r0v || end > r0v + kRowsT) continue;
            unsigned long long best = 0ull;   // (d2 bits, a, row) of the largest row minimum
            for (int a = lane; a < mq; a += 32) {
                const unsigned long long v = rowmin[c * kMaxMq + a];
                const unsigned long long key = (v & 0xffffffff00000000ull) |
                                               ((unsigned long long)a << 16) | (v & 0xffffull);
                best = best > key ? best : key;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
                best = best > other ? best : other;
            }
            const unsigned long long cm = colmax[c];
            int pa, pr;
            if ((best >> 32) >= (cm >> 32)) {
                pa = (int)((best >> 16) & 0xffffull);
                pr = (int)(best & 0xffffull);
            } else {
                pa = (int)(cm & 0xffffull);
                pr = (int)((cm >> 16) & 0xffffull);
            }
            pa = min(max(pa, 0), mq - 1);
            pr = min(max(pr, 0), s_n[c] - 1);
            const float4 *x4 = reinterpret_cast<const float4 *>(Qs + (size_t)pa * dp);
            const float4 *y4 = reinterpret_cast<const float4 *>(vec + (s_grow0[c] + pr) * d);
            float sacc = 0.0f;
            for (int k = lane; k < d4; k += 32) {
                const float4 x = x4[k], y = y4[k];
                float u = x.x - y.x;
                sacc = fmaf(u, u, sacc);
                u = x.y - y.y;
                sacc = fmaf(u, u, sacc);
                u = x.z - y.z;
                sacc = fmaf(u, u, sacc);
                u = x.w - y.w;
                sacc = fmaf(u, u, sacc);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
            if (lane == 0) cand_dist[(int64_t)q * C + c0 + c] = sqrtf(sacc);
        }
    }
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

}  // namespace

cudaError_t launch_wait_selftest(int *err, uint64_t limit_ns, cudaStream_t st) {
    k_wait_selftest<<<1, 32, 0, st>>>(err, limit_ns);
    return cudaGetLastError();
}

bool refine2_supported(int d, int max_mq, int64_t max_set) {
    if (d % 4 != 0 || max_mq > kMaxMq || max_set > 0xffff || max_mq < 1) return false;
    return refine2_stages(d, max_mq) >= 2;
}

int refine2_stages(int d, int max_mq) {
    const int mq_pad = (max_mq + 31) / 32 * 32;
    const int stage = kRowsT * (d + 4) * 4;
    const int alias = (mq_pad == 32 && stage >= kPartialBytes) ? 1 : 0;
    for (int ns = kMaxNS; ns >= 2; --ns)
        if (make_layout(d, mq_pad, ns, alias).total <= kSmemMax) return ns;
    return 0;
}

cudaError_t launch_refine2(const float *qvec, const int64_t *qoff, int n_q, int max_mq,
                           const float *vec, const float *vnorm, const int64_t *set_off, int d,
                           const int32_t *cand, const int32_t *thr, int C, float *cand_dist,
                           int *err, cudaStream_t st) {
    if (n_q <= 0) return cudaSuccess;
    const int mq_pad = (max_mq + 31) / 32 * 32;
    const int stage = kRowsT * (d + 4) * 4;
    const int alias = (mq_pad == 32 && stage >= kPartialBytes) ? 1 : 0;
    const int NS = refine2_stages(d, max_mq);
    if (NS < 2) return cudaErrorInvalidValue;
    const Layout Lo = make_layout(d, mq_pad, NS, alias);
    cudaError_t e = cudaFuncSetAttribute(k_refine2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         Lo.total);
    if (e != cudaSuccess) return e;
    const int gx = (C + kCandB - 1) / kCandB;
    k_refine2<<<dim3(gx, n_q), kT, Lo.total, st>>>(qvec, qoff, vec, vnorm, set_off, d, NS, alias,
                                                   cand, thr, C, cand_dist, err);
    return cudaGetLastError();
}

}  // namespace bvss
