// encode.cu -- FlyHash encoder (Def. 7, Alg. 1) and the query-side filters
// of Alg. 6 (lines 1-4) for the BioVSS++ query path of arXiv 2412.03301.
//
// k_encode: one CTA per vector.  The vector is staged in shared memory, each
// output j sums the F input dims listed in row j of the sparse binary
// projection W (FP32 adds in row order, starting from +0.0), and the
// winner-take-all keeps the L largest activations under the strict order
// (value desc, index asc).  The L-th largest key is found exactly by a
// three-pass MSB-first radix select over order-preserving uint32 keys
// (11 + 11 + 10 bits); ties at that key are taken in index order.
#include "block_util.cuh"
#include "bvss_internal.cuh"

namespace bvss {

namespace {

constexpr int kEncThreads = 128;   // divides every valid m (m % 128 == 0)
constexpr int kEncWide = 256;      // used when it divides m
constexpr int kEncRepWords = 3072;  // 12 KB for the copies of the vector: 8 at d = 384,
                                    // which keeps 6 CTAs per SM (measured faster than 32
                                    // conflict-free copies at 3 CTAs per SM)

// eight 16-byte read-only loads issued back to back (one asm statement, so the
// compiler cannot interleave their uses and serialise the latencies)
__device__ __forceinline__ void ld_nc_v4x8(const void *const (&p)[8], uint4 (&v)[8]) {
    asm volatile(
        "ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%32];\n\t"
        "ld.global.nc.v4.u32 {%4, %5, %6, %7}, [%33];\n\t"
        "ld.global.nc.v4.u32 {%8, %9, %10, %11}, [%34];\n\t"
        "ld.global.nc.v4.u32 {%12, %13, %14, %15}, [%35];\n\t"
        "ld.global.nc.v4.u32 {%16, %17, %18, %19}, [%36];\n\t"
        "ld.global.nc.v4.u32 {%20, %21, %22, %23}, [%37];\n\t"
        "ld.global.nc.v4.u32 {%24, %25, %26, %27}, [%38];\n\t"
        "ld.global.nc.v4.u32 {%28, %29, %30, %31}, [%39];"
        : "=r"(v[0].x), "=r"(v[0].y), "=r"(v[0].z), "=r"(v[0].w), "=r"(v[1].x), "=r"(v[1].y),
          "=r"(v[1].z), "=r"(v[1].w), "=r"(v[2].x), "=r"(v[2].y), "=r"(v[2].z), "=r"(v[2].w),
          "=r"(v[3].x), "=r"(v[3].y), "=r"(v[3].z), "=r"(v[3].w), "=r"(v[4].x), "=r"(v[4].y),
          "=r"(v[4].z), "=r"(v[4].w), "=r"(v[5].x), "=r"(v[5].y), "=r"(v[5].z), "=r"(v[5].w),
          "=r"(v[6].x), "=r"(v[6].y), "=r"(v[6].z), "=r"(v[6].w), "=r"(v[7].x), "=r"(v[7].y),
          "=r"(v[7].z), "=r"(v[7].w)
        : "l"(p[0]), "l"(p[1]), "l"(p[2]), "l"(p[3]), "l"(p[4]), "l"(p[5]), "l"(p[6]),
          "l"(p[7]));
}

template <int THREADS>
__global__ void __launch_bounds__(THREADS)
k_encode(const float *__restrict__ x, int64_t n, const int64_t *__restrict__ n_dev, int d,
         int dpad, int rep, const uint16_t *__restrict__ proj, int m, int F, int L,
         uint16_t *__restrict__ pos, uint32_t *__restrict__ mask,
         const float *__restrict__ act, int64_t lda) {
    extern __shared__ uint32_t sm[];
    // rep (a power of two <= 32) copies of the vector, interleaved: value k of copy c
    // at xs[k * rep + c].  Lane l reads copy l % rep, so lanes l and l' can only meet in
    // a bank when l = l' mod rep: with rep = 32 the random gathers of W's rows never
    // conflict, with rep = 8 at most four lanes share a bank.
    float *xs = reinterpret_cast<float *>(sm);       // dpad * rep floats
    uint32_t *key = sm + dpad * rep;                 // m keys (first: a plain copy of x)
    uint32_t *hist = key + m;                        // 2048 bins
    uint32_t *mw = hist + 2048;                      // m/32 code words
    uint32_t *eqw = mw + (m >> 5);                   // m/32 words: outputs equal to the L-th
    __shared__ int scan_sh[THREADS / 32 + 1];
    __shared__ uint32_t sel_digit;
    __shared__ int sel_need;

    const int tid = threadIdx.x;
    const int W = m >> 5;
    if (n_dev && *n_dev < n) n = *n_dev;   // the vector count, when it lives on the device
    for (int64_t v = blockIdx.x; v < n; v += gridDim.x) {
      if (act) {
        // activations of a dense layer, computed elsewhere (the learned projection)
        const float *av = act + v * lda;
        for (int j = tid; j < m; j += THREADS) key[j] = order_key(av[j]);
        __syncthreads();
      } else {
        const float *xv = x + v * (int64_t)d;
        const int rs = __ffs(rep) - 1;
        float *x0 = reinterpret_cast<float *>(key);    // plain copy, until the keys are written
        for (int k = tid; k < d; k += THREADS) x0[k] = xv[k];
        __syncthreads();
        // replicate: a warp reads one value (broadcast) and writes its consecutive copies
#pragma unroll 4
        for (int e = tid; e < d * rep; e += THREADS) xs[e] = x0[e >> rs];
        __syncthreads();
        const float *xl = xs + (tid & 31 & (rep - 1));   // this lane's copy
        __syncthreads();

        // activations a_j (Def. 7: W v with W sparse binary), as sortable keys
        if (F == 8) {
            // eight rows of W per thread in flight (m is a multiple of THREADS)
            constexpr int kU = 8;
            for (int j0 = tid; j0 < m; j0 += kU * THREADS) {
                uint4 r[kU];
                const void *rp[kU];
#pragma unroll
                for (int i = 0; i < kU; ++i) {
                    const int j = j0 + i * THREADS;
                    rp[i] = proj + (int64_t)(j < m ? j : m - 1) * 8;   // past m: any valid row
                }
                ld_nc_v4x8(rp, r);
#pragma unroll
                for (int i = 0; i < kU; ++i) {
                    const int j = j0 + i * THREADS;
                    const uint32_t w4[4] = {r[i].x, r[i].y, r[i].z, r[i].w};
                    float a = 0.0f;
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        a = __fadd_rn(a, xl[(w4[t] & 0xFFFFu) << rs]);
                        a = __fadd_rn(a, xl[(w4[t] >> 16) << rs]);
                    }
                    if (j < m) key[j] = order_key(a);
                }
            }
        } else {
            for (int j = tid; j < m; j += THREADS) {
                const uint16_t *row = proj + (int64_t)j * F;
                float a = 0.0f;
                for (int t = 0; t < F; ++t) a = __fadd_rn(a, xl[(int)row[t] << rs]);
                key[j] = order_key(a);
            }
        }
      }

        // exact L-th largest key: radix select, most significant digit first
        uint32_t prefix = 0, pmask = 0;
        int need = L;
#pragma unroll 1
        for (int pass = 0; pass < 3; ++pass) {
            const int shift = pass == 0 ? 21 : (pass == 1 ? 10 : 0);
            const int nb = pass == 2 ? 1024 : 2048;
            for (int b = tid; b < nb; b += THREADS) hist[b] = 0;
            __syncthreads();
            for (int j = tid; j < m; j += THREADS) {
                const uint32_t k = key[j];
                if ((k & pmask) == prefix) atomicAdd(&hist[(k >> shift) & (nb - 1)], 1u);
            }
            __syncthreads();
            // bins owned by this thread, read 16 bytes at a time (B is a multiple of 4)
            constexpr int BMAX = 2048 / THREADS;
            const int B = nb / THREADS;
            uint32_t hv[BMAX];
            int s = 0;
#pragma unroll
            for (int i = 0; i < BMAX / 4; ++i) {
                uint4 q = make_uint4(0u, 0u, 0u, 0u);
                if (4 * i < B) q = reinterpret_cast<const uint4 *>(hist + tid * B)[i];
                hv[4 * i] = q.x;
                hv[4 * i + 1] = q.y;
                hv[4 * i + 2] = q.z;
                hv[4 * i + 3] = q.w;
                s += (int)(q.x + q.y + q.z + q.w);
            }
            int tot;
            const int excl = block_excl_scan<THREADS>(s, scan_sh, &tot);
            const int above = tot - excl - s;    // keys in higher bins
            if (above < need && above + s >= need) {
                int cum = above;
                bool found = false;
#pragma unroll
                for (int b = BMAX - 1; b >= 0; --b) {
                    if (b >= B || found) continue;
                    const int c = (int)hv[b];
                    if (cum + c >= need) {
                        sel_digit = (uint32_t)(tid * B + b);
                        sel_need = need - cum;
                        found = true;
                    }
                    cum += c;
                }
            }
            __syncthreads();
            prefix |= sel_digit << shift;
            pmask |= (uint32_t)(nb - 1) << shift;
            need = sel_need;
        }
        const uint32_t T = prefix;                 // key of the L-th winner
        const int n_eq = (int)hist[T & 1023u];     // keys equal to T
        const bool all_ties = (need == n_eq);

        // code bits and the outputs equal to the L-th value: 32 consecutive outputs per warp
        for (int j = tid; j < m; j += THREADS) {
            const uint32_t k = key[j];
            const uint32_t b = __ballot_sync(0xffffffffu, k > T || (k == T && all_ties));
            const uint32_t e = __ballot_sync(0xffffffffu, k == T);
            if ((tid & 31) == 0) {
                mw[j >> 5] = b;
                eqw[j >> 5] = e;
            }
        }
        __syncthreads();
        const int WE = (W + THREADS - 1) / THREADS;   // code words per thread
        const int w0 = tid * WE, w1 = min(W, w0 + WE);
        if (!all_ties) {
            // several outputs share the L-th value: the first `need` of them in index order win
            int c = 0;
            for (int w = w0; w < w1; ++w) c += __popc(eqw[w]);
            int tot;
            int r = block_excl_scan<THREADS>(c, scan_sh, &tot);
            for (int w = w0; w < w1 && r < need; ++w) {
                uint32_t e = eqw[w], take = 0u;
                while (e && r < need) {
                    const uint32_t low = e & (0u - e);
                    take |= low;
                    e ^= low;
                    ++r;
                }
                mw[w] |= take;
            }
            __syncthreads();
        }

        // winner positions in ascending order
        int c = 0;
        for (int w = w0; w < w1; ++w) c += __popc(mw[w]);
        int tot;
        int off = block_excl_scan<THREADS>(c, scan_sh, &tot);
        if (pos) {
            uint16_t *pv = pos + v * (int64_t)L;
            for (int w = w0; w < w1; ++w) {
                uint32_t b = mw[w];
                while (b) {
                    const int bit = __ffs(b) - 1;
                    b &= b - 1;
                    if (off < L) pv[off] = (uint16_t)((w << 5) + bit);
                    ++off;
                }
            }
        }
        if (mask)
            for (int w = tid; w < W; w += THREADS) mask[v * (int64_t)W + w] = mw[w];
        __syncthreads();
    }
}

template <int THREADS>
__global__ void __launch_bounds__(THREADS)
k_query_prep(const uint16_t *__restrict__ qpos, const int64_t *__restrict__ qoff, int m,
             int L, int A, uint32_t *__restrict__ sq, uint16_t *__restrict__ plist,
             int32_t *__restrict__ cq_trace) {
    extern __shared__ int32_t cnt[];   // m
    __shared__ uint32_t red[THREADS / 32];
    __shared__ uint32_t best;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int q = blockIdx.x;
    const int W = m >> 5;
    const int64_t v0 = qoff[q], v1 = qoff[q + 1];
    for (int p = tid; p < m; p += THREADS) cnt[p] = 0;
    __syncthreads();
    // C_Q = sum of the query codes (Alg. 6 line 1, Alg. 3)
    const uint16_t *src = qpos + v0 * L;
    const int64_t tot = (v1 - v0) * L;
    for (int64_t i = tid; i < tot; i += THREADS) atomicAdd(&cnt[src[i]], 1);
    __syncthreads();
    // S_Q = OR of the query codes (line 2, Alg. 5)
    for (int w = warp; w < W; w += THREADS / 32) {
        const uint32_t b = __ballot_sync(0xffffffffu, cnt[(w << 5) + lane] > 0);
        if (lane == 0) sq[(int64_t)q * W + w] = b;
    }
    if (cq_trace)
        for (int p = tid; p < m; p += THREADS) cq_trace[(int64_t)q * m + p] = cnt[p];
    // P = first A positions by (C_Q desc, position asc) (lines 3-4)
    for (int a = 0; a < A; ++a) {
        uint32_t mk = 0;
        for (int p = tid; p < m; p += THREADS) {
            const int c = cnt[p];
            const uint32_t k = c < 0 ? 0u : (((uint32_t)c << 16) | (0xFFFFu - (uint32_t)p));
            mk = max(mk, k);
        }
        mk = __reduce_max_sync(0xffffffffu, mk);
        if (lane == 0) red[warp] = mk;
        __syncthreads();
        if (warp == 0) {
            uint32_t z = lane < THREADS / 32 ? red[lane] : 0u;
            z = __reduce_max_sync(0xffffffffu, z);
            if (lane == 0) best = z;
        }
        __syncthreads();
        if (tid == 0) {
            const int p = (int)(0xFFFFu - (best & 0xFFFFu));
            plist[(int64_t)q * A + a] = (uint16_t)p;
            cnt[p] = -1;
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_encode(const float *x, int64_t n, int d, const uint16_t *proj, int m,
                          int F, int L, uint16_t *pos, uint32_t *mask, cudaStream_t st,
                          const int64_t *n_dev) {
    if (n <= 0) return cudaSuccess;
    const int dpad = (d + 3) & ~3;
    int rep = 32;                                   // copies of the vector that fit 48 KB
    while (rep > 1 && (size_t)dpad * rep > (size_t)kEncRepWords) rep >>= 1;
    // after the copies: the keys, histogram and code words, which also hold the plain
    // copy of the vector while the copies are made
    size_t tail = (size_t)m + 2048 + 2 * (m / 32);
    if (tail < (size_t)dpad) tail = dpad;
    const size_t smem = sizeof(uint32_t) * ((size_t)dpad * rep + tail);
    const bool wide = m % kEncWide == 0;
    auto kern = wide ? k_encode<kEncWide> : k_encode<kEncThreads>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = n < (int64_t)1 << 30 ? n : (int64_t)1 << 30;
    kern<<<(unsigned)grid, wide ? kEncWide : kEncThreads, smem, st>>>(x, n, n_dev, d, dpad, rep,
                                                                      proj, m, F, L, pos, mask,
                                                                      nullptr, 0);
    return cudaGetLastError();
}

cudaError_t launch_encode_dense(const float *act, int64_t n, int64_t lda, int m, int L,
                                uint16_t *pos, uint32_t *mask, cudaStream_t st,
                                const int64_t *n_dev) {
    if (n <= 0) return cudaSuccess;
    // the keys, histogram and code words only (no copies of the vector)
    const size_t smem = sizeof(uint32_t) * ((size_t)m + 2048 + 2 * (m / 32));
    const bool wide = m % kEncWide == 0;
    auto kern = wide ? k_encode<kEncWide> : k_encode<kEncThreads>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = n < (int64_t)1 << 30 ? n : (int64_t)1 << 30;
    kern<<<(unsigned)grid, wide ? kEncWide : kEncThreads, smem, st>>>(
        nullptr, n, n_dev, 0, 0, 1, nullptr, m, 0, L, pos, mask, act, lda);
    return cudaGetLastError();
}

cudaError_t launch_query_prep(const uint16_t *qpos, const int64_t *qoff, int n_q, int m,
                              int L, int A, uint32_t *sq, uint16_t *plist,
                              int32_t *cq_trace, cudaStream_t st) {
    if (n_q <= 0) return cudaSuccess;
    const size_t smem = sizeof(int32_t) * (size_t)m;
    auto kern = k_query_prep<256>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<n_q, 256, smem, st>>>(qpos, qoff, m, L, A, sq, plist, cq_trace);
    return cudaGetLastError();
}

}  // namespace bvss
