// alg2.cu -- candidate scores of the plain BioVSS search (Alg. 2 of arXiv
// 2412.03301, lines 6-8): Haus^H(Q^H, H_j) for every database set j, the
// Hausdorff distance of Def. 4 with the Hamming distance between per-vector
// codes in place of the norm.
//
// Every code has exactly L ones (WTA, Def. 7), so ham(a, r) = 2L - 2 o(a, r)
// with o the number of shared positions, and
//   Haus^H = 2L - 2 min( min_a max_r o(a, r), min_r max_a o(a, r) ).
// A CTA takes one query set (at most 32 vectors) and 1024 database sets.  It
// first builds, in shared memory, one word per code position p whose bit a says
// whether query vector a's code holds p.  A warp then scores one set at a time,
// one lane per database vector: the lane adds the words of its code's L
// positions into bit-sliced counters (bit a of counter plane b is bit b of
// o(a, r)), so one pass over L positions gives the overlaps with all query
// vectors at once.  The words are summed 16 at a time by a carry-save tree
// (Harley and Seal's popcount scheme: 15 three-to-two compressors of 5 logic
// operations per 16 words, the "sixteens" rippled into the upper planes), and
// both directed terms come from bit-sliced maxima: per lane over the query
// vectors (most significant plane first, keeping the query vectors that have
// the bit), and per query vector over the warp's rows (one warp OR per plane).  The scores
// (at most 2L) go to h[q][j], where the candidate select of the query path
// takes the C smallest (score, id).
#include "bvss_internal.cuh"

namespace bvss {

namespace {

constexpr int kA2Threads = 256;
constexpr int kA2Warps = kA2Threads / 32;
constexpr int kA2Sets = 1024;   // database sets per CTA

// add the 32 one-bit values of x into the bit-sliced counters c[B0..NB)
template <int NB, int B0 = 0>
__device__ __forceinline__ void add_bits(uint32_t (&c)[NB], uint32_t x) {
#pragma unroll
    for (int b = B0; b < NB; ++b) {
        const uint32_t t = c[b] & x;
        c[b] ^= x;
        x = t;
    }
}

// carry-save adder: a + b + c = 2 hi + lo, bitwise
__device__ __forceinline__ void csa(uint32_t &hi, uint32_t &lo, uint32_t a, uint32_t b,
                                    uint32_t c) {
    const uint32_t u = a ^ b;
    hi = (a & b) | (u & c);
    lo = u ^ c;
}

// add 16 one-bit words into the bit-sliced counters c[0..NB) (NB >= 5): the carry-save
// tree keeps c[0..3] as the ones, twos, fours and eights planes and ripples its
// sixteens into c[4..)
template <int NB>
__device__ __forceinline__ void add16(uint32_t (&c)[NB], const uint32_t (&w)[16]) {
    uint32_t twosA, twosB, foursA, foursB, eightsA, eightsB, sixteens;
    csa(twosA, c[0], c[0], w[0], w[1]);
    csa(twosB, c[0], c[0], w[2], w[3]);
    csa(foursA, c[1], c[1], twosA, twosB);
    csa(twosA, c[0], c[0], w[4], w[5]);
    csa(twosB, c[0], c[0], w[6], w[7]);
    csa(foursB, c[1], c[1], twosA, twosB);
    csa(eightsA, c[2], c[2], foursA, foursB);
    csa(twosA, c[0], c[0], w[8], w[9]);
    csa(twosB, c[0], c[0], w[10], w[11]);
    csa(foursA, c[1], c[1], twosA, twosB);
    csa(twosA, c[0], c[0], w[12], w[13]);
    csa(twosB, c[0], c[0], w[14], w[15]);
    csa(foursB, c[1], c[1], twosA, twosB);
    csa(eightsB, c[2], c[2], foursA, foursB);
    csa(sixteens, c[3], c[3], eightsA, eightsB);
    add_bits<NB, 4>(c, sixteens);
}

template <int NB>
__global__ void __launch_bounds__(kA2Threads)
k_haus_h(const uint16_t *__restrict__ qpos, const int64_t *__restrict__ qoff,
         const uint16_t *__restrict__ codes, const int64_t *__restrict__ set_off,
         int64_t n_sets, int m, int L, uint16_t *__restrict__ h, int64_t hs) {
    extern __shared__ uint32_t qbits[];   // m words
    const int q = blockIdx.y;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t a0 = qoff[q];
    const int mq = (int)(qoff[q + 1] - a0);   // 1..32 (host check)
    for (int p = threadIdx.x; p < m; p += kA2Threads) qbits[p] = 0;
    __syncthreads();
    for (int e = threadIdx.x; e < mq * L; e += kA2Threads) {
        const int a = e / L;
        atomicOr(&qbits[qpos[(a0 + a) * L + (e - a * L)]], 1u << a);
    }
    __syncthreads();
    const uint32_t vmask = mq >= 32 ? 0xffffffffu : (1u << mq) - 1u;   // valid query vectors
    const int64_t s_begin = (int64_t)blockIdx.x * kA2Sets;
    const int64_t s_end = s_begin + kA2Sets < n_sets ? s_begin + kA2Sets : n_sets;
    for (int64_t j = s_begin + warp; j < s_end; j += kA2Warps) {
        const int64_t r0 = set_off[j], nr = set_off[j + 1] - r0;
        uint32_t colmax = 0;             // lane a: max over rows of o(a, r)
        uint32_t rowmin = 0xFFFFFFFFu;   // min over this lane's rows of max_a o(a, r)
        for (int64_t rc = 0; rc < nr; rc += 32) {
            const bool rv = rc + lane < nr;
            uint32_t c[NB];
#pragma unroll
            for (int b = 0; b < NB; ++b) c[b] = 0;
            if (rv) {
                const uint16_t *pr = codes + (r0 + rc + lane) * L;
                int t0 = 0;
                if ((L & 7) == 0) {
                    // rows are 16-byte aligned: eight positions per load, 16 per tree
                    const uint4 *pr4 = reinterpret_cast<const uint4 *>(pr);
                    for (; t0 + 16 <= L; t0 += 16) {
                        const uint4 v0 = pr4[t0 / 8], v1 = pr4[t0 / 8 + 1];
                        const uint32_t p[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
                        uint32_t w[16];
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            w[2 * i] = qbits[p[i] & 0xFFFFu];
                            w[2 * i + 1] = qbits[p[i] >> 16];
                        }
                        add16<NB>(c, w);
                    }
                }
                for (int t = t0; t < L; ++t) add_bits<NB>(c, qbits[pr[t]]);
            }
            // this row's largest overlap over the valid query vectors: the planes from the
            // top, keeping the query vectors that have each bit while any does
            uint32_t rmax = 0;
            {
                uint32_t alive = vmask;
#pragma unroll
                for (int b = NB - 1; b >= 0; --b) {
                    const uint32_t t = c[b] & alive;
                    if (t) {
                        rmax |= 1u << b;
                        alive = t;
                    }
                }
            }
            // each query vector's largest overlap over the warp's rows (rows past nr hold
            // zero counters): per plane from the top, the warp's OR over the rows still in
            // the running for that query vector; lane a takes query vector a's value
            {
                uint32_t alive = 0xffffffffu;
                uint32_t cm = 0;
#pragma unroll
                for (int b = NB - 1; b >= 0; --b) {
                    const uint32_t t = c[b] & alive;
                    const uint32_t any = __reduce_or_sync(0xffffffffu, t);
                    alive &= t | ~any;
                    cm |= ((any >> lane) & 1u) << b;
                }
                if (cm > colmax) colmax = cm;
            }
            if (rv && rmax < rowmin) rowmin = rmax;
        }
        const uint32_t cmin = __reduce_min_sync(0xffffffffu, lane < mq ? colmax : 0xFFFFFFFFu);
        const uint32_t rmin = __reduce_min_sync(0xffffffffu, rowmin);
        const uint32_t best = cmin < rmin ? cmin : rmin;
        if (lane == 0) h[(int64_t)q * hs + j] = (uint16_t)(2 * L - 2 * (int)best);
    }
}

template <int NB>
cudaError_t launch_t(const uint16_t *qpos, const int64_t *qoff, int n_q, const uint16_t *codes,
                     const int64_t *set_off, int64_t n_sets, int m, int L, uint16_t *h,
                     int64_t hs, cudaStream_t st) {
    const size_t smem = sizeof(uint32_t) * (size_t)m;
    cudaError_t e = cudaFuncSetAttribute(k_haus_h<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)((n_sets + kA2Sets - 1) / kA2Sets), (unsigned)n_q);
    k_haus_h<NB><<<grid, kA2Threads, smem, st>>>(qpos, qoff, codes, set_off, n_sets, m, L, h, hs);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_haus_h(const uint16_t *qpos, const int64_t *qoff, int n_q,
                          const uint16_t *codes, const int64_t *set_off, int64_t n_sets, int m,
                          int L, uint16_t *h, int64_t hs, cudaStream_t st) {
    if (n_q <= 0 || n_sets <= 0) return cudaSuccess;
    // counter planes: enough bits for an overlap of up to L
    if (L < 64) return launch_t<6>(qpos, qoff, n_q, codes, set_off, n_sets, m, L, h, hs, st);
    if (L < 128) return launch_t<7>(qpos, qoff, n_q, codes, set_off, n_sets, m, L, h, hs, st);
    if (L < 256) return launch_t<8>(qpos, qoff, n_q, codes, set_off, n_sets, m, L, h, hs, st);
    if (L < 2048) return launch_t<11>(qpos, qoff, n_q, codes, set_off, n_sets, m, L, h, hs, st);
    return cudaErrorInvalidValue;
}

}  // namespace bvss
