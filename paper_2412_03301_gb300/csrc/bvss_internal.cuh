// bvss_internal.cuh -- index layout and kernel entry points shared by the
// CUDA translation units of the BioVSS++ query path (arXiv 2412.03301).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "bvss.h"

namespace bvss {

constexpr int kMaxPlanes = 8;          // cached first-layer gate planes (one per M)
constexpr uint16_t kGatedOut = 0xFFFF; // h of a set outside F1
constexpr int kSelChunk = 16384;       // sets per CTA in the candidate select
constexpr int kSelBlock = 128;         // sets per block minimum (the scan's tile width)
constexpr int kSelRangeWords = 32;     // per chunk: 8 warp ranges x (lt, eq, tie rank, slot)
constexpr int kOffRing = 4;            // pinned staging slots for query offsets
constexpr int kProfEvents = BVSS_N_STAGES + 1;  // events per profiled batch
constexpr int kErrBandOverflow = 16;   // device status: more near-ties at the k-th than fit

// A bit plane of the first-layer gate for one minimum count M:
// word w of row p holds bit b = (C_{32w+b}[p] >= M), for every set (Def. 9 in
// dense form: the union of Alg. 6 lines 5-9 is an OR of A rows).
struct GatePlane {
    int M = -1;
    uint32_t *words = nullptr;   // m x NW
};

// Scratch memory of one query batch (owned by the index, grown on demand).
struct Workspace {
    int64_t cap_q = 0, cap_vq = 0;
    int cap_C = 0, cap_A = 0;
    float *qvec = nullptr;        // staged query vectors (host input)   cap_vq x d
    int64_t *qoff = nullptr;      // query offsets, batch-relative       cap_q + 1
    uint16_t *qpos = nullptr;     // query codes                         cap_vq x L
    uint32_t *sq = nullptr;       // query sketches                      cap_q x W
    uint16_t *plist = nullptr;    // top-A positions                     cap_q x cap_A
    uint16_t *h = nullptr;        // Hamming scores                      cap_q x N
    uint32_t *gate = nullptr;     // layer-1 mask per 32-set tile        cap_q x NW
    uint8_t *q8 = nullptr;        // query sketches as FP8 MMA operand   scan_mma_q8_bytes
    int32_t *qpop = nullptr;      // |S_Q|                               cap_q rounded to 256
    uint32_t *hist = nullptr;     // histogram of h                      cap_q x (m + 1)
    int32_t *thr = nullptr;       // per query: H*, n_lt, take_eq, n_sel cap_q x 4
    int32_t *chunk = nullptr;     // per (query, chunk): lt, eq, eq_before, out_off
    uint16_t *bmin = nullptr;     // minimum h per block of kSelBlock sets  cap_q x n_blk
    int32_t *bound = nullptr;     // per query: bound on the select threshold  cap_q
    int32_t *cand = nullptr;      // candidate ids                       cap_q x cap_C
    float *cand_dist = nullptr;   // candidate distances                 cap_q x cap_C
    longlong2 *pair = nullptr;    // (query vector, global row) attaining each candidate's value
    int32_t *wlist = nullptr;     // query sets by width (<= 32, wider), then their two counts
    unsigned char *qop = nullptr; // refine operand of each query set when it is streamed
    float *qop_n = nullptr;       //   (k_query_op), with its rows' norms and FP8 scales
    float *qop_sc = nullptr;
    __nv_bfloat16 *enc_x = nullptr;  // dense projection: a block of query vectors in BF16
    float *enc_act = nullptr;        //   and their activations (kEncChunk x d, x m)
    int64_t *out_ids = nullptr;   // staged results (host output)        cap_q x k
    float *out_dist = nullptr;
    int cap_k = 0;
};

}  // namespace bvss

struct bvss_index {
    bvss_params p;
    int device = 0;
    int64_t n_sets = 0, n_vec = 0;
    int W = 0;                   // m / 32 words per code or sketch
    int64_t NW = 0;              // ceil(n_sets / 32) words per gate-plane row
    float *vec = nullptr;        // n_vec x d FP32 (set-contiguous)
    float *vnorm = nullptr;      // n_vec squared norms (FP32)
    __nv_bfloat16 *vec16 = nullptr;   // n_vec x d BF16 copy (BVSS_BUILD_BF16)
    float *vnorm16 = nullptr;         // squared norms of the BF16 values
    uint8_t *vec8 = nullptr;          // n_vec x d FP8 E4M3 copy (BVSS_BUILD_FP8)
    float *vscale8 = nullptr;         // its per-vector scales
    float *vnorm8 = nullptr;          // squared norms of the scaled FP8 values
    float *rstat = nullptr;           // kRoundStats entries: [0] largest norm, [1] / [2]
                                      // largest rounding-error norm of the BF16 / FP8 copy
                                      // (rounded up), [3] the largest frac_bits of the
                                      // values, [4] a bound on the largest rounding-error
                                      // norm of the vectors read as TF32
    __nv_bfloat16 *wproj16 = nullptr; // learned dense projection (m x d BF16), or null for
                                      // the sparse binary FlyHash projection proj
    int64_t *set_off = nullptr;  // n_sets + 1
    uint16_t *proj = nullptr;    // m x F
    uint16_t *codes = nullptr;   // n_vec x L, ascending positions
    uint32_t *sketch = nullptr;  // n_sets x W
    int32_t *spop = nullptr;     // |S_i| per set
    uint8_t *count = nullptr;    // m x n_sets, position-major, saturated at 255
    int *flag = nullptr;         // device status word (build-time checks)
    int *err = nullptr;          // device error word: set when a kernel's bounded wait gives up
    int64_t max_set = 0;         // largest set size (vectors)
    bvss::GatePlane planes[bvss::kMaxPlanes];
    int n_planes = 0;
    int n_plans = 0;             // live plans (their graphs hold plane pointers)
    bvss::Workspace ws;
    int64_t *off_host[bvss::kOffRing] = {};     // pinned, batch-relative offsets
    cudaEvent_t off_event[bvss::kOffRing] = {}; // last copy out of each slot
    int off_next = 0;
    int64_t off_cap = 0;
    // per-stage profiling: kProfEvents events per batch, summed on read
    bool prof_on = false;
    cudaEvent_t *prof_ev = nullptr;
    int64_t prof_cap = 0, prof_used = 0;
    double prof_ms[BVSS_N_STAGES] = {};
    int64_t prof_batches = 0;
    int64_t prof_launches = 0;     // kernels launched by the profiled batches
};

namespace bvss {

// ---- encode.cu --------------------------------------------------------------
constexpr int64_t kEncChunk = 4096;   // vectors per block of the dense projection
// FlyHash (Def. 7): pos[v] = ascending L winners, mask[v] = code bits.  With n_dev,
// the count is min(n, *n_dev) read on the device (n is then the capacity).
cudaError_t launch_encode(const float *x, int64_t n, int d, const uint16_t *proj,
                          int m, int F, int L, uint16_t *pos, uint32_t *mask,
                          cudaStream_t st, const int64_t *n_dev = nullptr);
// WTA of dense activations act (n x m, row stride lda) into codes, as launch_encode
cudaError_t launch_encode_dense(const float *act, int64_t n, int64_t lda, int m, int L,
                                uint16_t *pos, uint32_t *mask, cudaStream_t st,
                                const int64_t *n_dev = nullptr);
// ---- dense.cu: the learned projection's BF16 layer on the tensor cores -----------------
// D (n x m, row stride ldd) = X (n x d) W^T (W: m x d), BF16 in, FP32 out; d % 64 == 0,
// m % 128 == 0; a bounded wait that gives up sets bit 4 of *err
cudaError_t launch_dense_gemm(const __nv_bfloat16 *X, int64_t n, int d, const __nv_bfloat16 *W,
                              int m, float *D, int64_t ldd, int *err, cudaStream_t st);
// BF16 copies of FP32 rows: rows null -> rows 0..n-1, else the listed rows of the n_src
// rows of x (ids outside [0, n_src) give zero rows)
cudaError_t launch_rows_bf16(const float *x, int d, const int64_t *rows, int64_t n,
                             __nv_bfloat16 *out, cudaStream_t st, int64_t n_src = 0);
// rows[a][t]: the row nearest to query vector a in set sets[q][t] of its query set q
cudaError_t launch_nearest(const float *qvec, const int64_t *qoff, int n_q, int d,
                           const float *vec, const int64_t *set_off, int64_t n_sets,
                           const int64_t *sets, int k, int64_t *rows, cudaStream_t st);
// Alg. 6 lines 1-4 for n_q query sets (codes qpos, offsets qoff relative to qpos).
cudaError_t launch_query_prep(const uint16_t *qpos, const int64_t *qoff, int n_q,
                              int m, int L, int A, uint32_t *sq, uint16_t *plist,
                              int32_t *cq_trace, cudaStream_t st);

// ---- filters.cu -------------------------------------------------------------
cudaError_t launch_check_finite(const float *x, int64_t n, int *flag, cudaStream_t st);
cudaError_t launch_norms(const float *x, int64_t n, int d, float *norm, cudaStream_t st);
cudaError_t launch_build_filters(const uint16_t *codes, const int64_t *set_off,
                                 int64_t n_sets, int m, int L, uint32_t *sketch,
                                 uint8_t *count, cudaStream_t st);
cudaError_t launch_gate_plane(const uint8_t *count, int m, int64_t n_sets, int64_t NW,
                              int M, uint32_t *plane, cudaStream_t st);
// gathers write zeros for ids outside [0, n_sets)
cudaError_t launch_gather_sketches(const uint32_t *sketch, int W, int64_t n_sets,
                                   const int64_t *ids, int64_t n, uint32_t *out,
                                   cudaStream_t st);
cudaError_t launch_gather_counts(const uint8_t *count, int m, int64_t n_sets,
                                 const int64_t *ids, int64_t n, uint8_t *out,
                                 cudaStream_t st);

// ---- scan.cu ----------------------------------------------------------------
// Alg. 6 lines 5-9: gate[q][t] = OR over the A positions of plane word t, i.e.
// the first-layer mask of sets 32t .. 32t + 31 (n_q x NW words).
cudaError_t launch_gate(const uint32_t *plane, int64_t NW, const uint16_t *plist, int A, int n_q,
                        uint32_t *gate, cudaStream_t st);
// Alg. 6 line 12 with CUDA-core popcounts: h[q][i] = popc(S_Q ^ S_i) for sets
// passing the gate.  gate_mode: 0 = every set passes (M = 0), 1 = gate words,
// 2 = no set passes.  h rows have stride hs (a multiple of 64 elements).
cudaError_t launch_scan(const uint32_t *sketch, int64_t n_sets, int W, const uint32_t *gate,
                        int64_t NW, int gate_mode, const uint32_t *sq, int n_q, uint16_t *h,
                        int64_t hs, cudaStream_t st);

// ---- scan_mma.cu: the same h on the tensor cores ----------------------------
size_t scan_mma_q8_bytes(int64_t n_q, int m);
cudaError_t launch_sketch_pop(const uint32_t *sketch, int64_t n_sets, int W, int32_t *spop,
                              cudaStream_t st);
// query sketches -> FP8 MMA operand (q8 of scan_mma_q8_bytes(n_q, m) bytes) and
// |S_Q| (qpop, n_q rounded up to 256 ints)
cudaError_t launch_expand_q(const uint32_t *sq, int n_q, int W, uint8_t *q8, int32_t *qpop,
                            cudaStream_t st);
// bmin (may be null): n_q x ceil(n_sets / kSelBlock) minimum scores per block of sets
cudaError_t launch_scan_mma(const uint32_t *sketch, const int32_t *spop, int64_t n_sets, int W,
                            const uint32_t *gate, int64_t NW, int gate_mode, const uint8_t *q8,
                            const int32_t *qpop, int n_q, uint16_t *h, int64_t hs, int *err,
                            cudaStream_t st, uint16_t *bmin = nullptr);
// the same h and bmin with the set sketches as the MMA's A operand in tensor memory (128
// sets x 128 queries per tile); the same q8 and qpop
cudaError_t launch_scan_tm(const uint32_t *sketch, const int32_t *spop, int64_t n_sets, int W,
                           const uint32_t *gate, int64_t NW, int gate_mode, const uint8_t *q8,
                           const int32_t *qpop, int n_q, uint16_t *h, int64_t hs, int *err,
                           cudaStream_t st, uint16_t *bmin = nullptr);

// ---- alg2.cu: Haus^H scores of the plain BioVSS search (Alg. 2 lines 6-8) ----
// h[q][j] = Haus^H between query set q's codes (qpos, L positions per vector,
// at most 32 vectors per set) and set j's codes (codes, set_off)
cudaError_t launch_haus_h(const uint16_t *qpos, const int64_t *qoff, int n_q,
                          const uint16_t *codes, const int64_t *set_off, int64_t n_sets, int m,
                          int L, uint16_t *h, int64_t hs, cudaStream_t st);

// ---- select.cu
constexpr int kSelectKernels = 5;   // kernels launch_select runs --------------------------------------------------------------
// Alg. 6 lines 10-18: the min(C, |F1|) smallest (h, id), listed by ascending id.  With
// bmin (n_q x ceil(n_sets / kSelBlock) block minima of h) the passes over h skip blocks
// that cannot hold a candidate; bound is then n_q ints of scratch.
cudaError_t launch_select(const uint16_t *h, int64_t n_sets, int64_t hs, int m, int n_q,
                          int C, uint32_t *hist, int32_t *thr, int32_t *chunk,
                          int32_t *cand, cudaStream_t st, const uint16_t *bmin = nullptr,
                          int32_t *bound = nullptr);

// ---- refine.cu --------------------------------------------------------------
// Alg. 6 lines 19-23: exact Hausdorff of each candidate, then top-k.
cudaError_t launch_refine(const float *qvec, const int64_t *qoff, int n_q, int max_mq,
                          const float *vec, const float *vnorm, const int64_t *set_off,
                          int d, const int32_t *cand, const int32_t *thr, int C,
                          float *cand_dist, cudaStream_t st);
// refine_tma.cu: the same, candidate rows streamed by TMA bulk copies, one
// pipeline per warp (query sets of at most 64 vectors)
bool refine_tma_supported(int d, int max_mq);
cudaError_t launch_refine_tma(const float *qvec, const int64_t *qoff, int n_q, int max_mq,
                              const float *vec, const float *vnorm, const int64_t *set_off,
                              int d, const int32_t *cand, const int32_t *thr, int C,
                              float *cand_dist, int *err, cudaStream_t st);
// refine_mma.cu: the same on the tensor cores (query sets <= 64) from the BF16 copy
// (d % 64 == 0), the FP8 copy (d % 128 == 0) or the FP32 vectors read as TF32
// (d % 32 == 0); the values match the boundary stage's form numbers
enum class Elem : int { BF16 = 1, FP8 = 2, TF32 = 3 };
bool refine_mma_supported(int d, int max_mq, Elem e);
cudaError_t launch_to_bf16(const float *x, int64_t n, int d, __nv_bfloat16 *y, float *norm,
                           cudaStream_t st);
// FP8 E4M3 copy with one scale per vector and the squared norms of the scaled values
cudaError_t launch_to_fp8(const float *x, int64_t n, int d, uint8_t *y, float *scale,
                          float *norm, cudaStream_t st);
// records each candidate's attaining (query vector, row) pair and, in the high word of
// pair.x, its squared Hausdorff value over the stored copies (read by the boundary
// stage).  vecb: the BF16 copy, the FP8 copy (with its per-vector scales vscale) or the
// FP32 vectors, as el says; vnorm: squared norms of the stored values (of the FP32 values
// for TF32).  cand_cta: candidates per CTA (1..512, 0 = 512); stages: depth of the copy
// ring (4 up to the most that fit; otherwise, and for 0, the most that fit).
cudaError_t launch_refine_mma(const float *qvec, const int64_t *qoff, int n_q, int max_mq,
                              const void *vecb, const float *vscale, const float *vnorm,
                              Elem el, const int64_t *set_off, int d, const int32_t *cand,
                              const int32_t *thr, int C, longlong2 *pair, int *err, cudaStream_t st,
                              int cand_cta = 0, int stages = 0, const int32_t *qlist = nullptr,
                              const int32_t *qcount = nullptr, const unsigned char *qop = nullptr,
                              const float *qop_n = nullptr, const float *qop_sc = nullptr,
                              int qs_mode = 0);
// true when the refine streams the shape's query operand through its ring instead of
// holding it in shared memory: always when it does not fit there; otherwise as qs_mode
// asks (1 hold it, 2 stream it, 0 stream it when that deepens a ring of five stages or
// fewer by two or more).  A streaming launch needs launch_query_op to have written the
// batch's operand first (qop of n_q x refine_mma_qop_bytes(d, el) bytes, qop_n / qop_sc
// of n_q x 64 floats); without those buffers a launch holds the operand where it fits.
bool refine_mma_streams(int d, int max_mq, Elem e, int qs_mode = 0);
size_t refine_mma_qop_bytes(int d, Elem e);
cudaError_t launch_query_op(const float *qvec, const int64_t *qoff, int n_q, int d, Elem el,
                            unsigned char *qop, float *qop_n, float *qop_sc, cudaStream_t st);
// with qlist / qcount (device): only query sets qlist[0 .. *qcount) (the grid still spans
// n_q rows; max_mq then bounds the listed sets only)
// lists (2 n_q ints): the batch's query sets of at most 32 vectors, then the wider ones;
// counts (2 ints) their numbers
cudaError_t launch_width_lists(const int64_t *qoff, int n_q, int32_t *lists, int32_t *counts,
                               cudaStream_t st);
// stages of the refine's ring for this dimension and batch (0 if the kernel cannot run)
int refine_mma_stages(int d, int max_mq, Elem e, int qs_mode = 0);
// the ring depth a launch asking for `stages` runs with (0 if the kernel cannot run)
int refine_mma_ring(int d, int max_mq, int stages, Elem e, int qs_mode = 0);
// a kernel that waits on an mbarrier nothing completes, with a limit; sets *err on timeout
cudaError_t launch_wait_selftest(int *err, uint64_t limit_ns, cudaStream_t st);
// ---- boundary.cu: the exact top-k over the candidates (Alg. 6 line 23, Def. 4) ------
// form: the refine that ran (0 FP32, 1 BF16, 2 FP8, 3 TF32 tensor cores); stats: the
// index's rstat; pair: the MMA forms' records (value in the high word of .x); max_mq: the
// batch's largest query set; exact_band: the FP8 form's band from its rigorous bound
// (else from its 3-sigma tolerance).  Band members' cand_dist become their exact values;
// cand_dist[q][n_sel..C) is padded with +inf; out_ids / out_dist (n_q x k) = the k
// smallest (distance, id) in that order, -1 / +inf past the candidate count.
cudaError_t launch_band_topk(const float *qvec, const int64_t *qoff, int n_q, int max_mq, int d,
                             int form, const float *stats, const float *vec,
                             const int64_t *set_off, const int32_t *cand, const int32_t *thr,
                             int C, int k, const longlong2 *pair, float *cand_dist,
                             int64_t *out_ids, float *out_dist, int *err, int exact_band,
                             cudaStream_t st);
constexpr int kBandKernels = 1;
constexpr int kRoundStats = 5;   // entries of an index's rstat
// rstat of an index (x16 / x8 may be null: their entries stay 0)
cudaError_t launch_round_stats(const float *x, int64_t n, int d, const __nv_bfloat16 *x16,
                               const uint8_t *x8, const float *sc8, float *stats,
                               cudaStream_t st);

// ---- api.cu -------------------------------------------------------------------
// Records a message for bvss_last_error() on this thread and returns code.
int record_error(int code, const char *fmt, ...);

// ---- shared device helpers ---------------------------------------------------
__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace bvss
