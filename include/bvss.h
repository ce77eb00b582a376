/*
 * bvss.h -- C ABI of the GB300 BioVSS++ query path.
 *
 * Method: arXiv 2412.03301 ("Approximate Vector Set Search Inspired by Fly
 * Olfactory Neural System").  A database of vector sets is encoded with
 * FlyHash (Def. 7, Alg. 1) into sparse binary codes, summarised per set by a
 * count Bloom filter (Def. 8, Alg. 3) and a binary Bloom filter / sketch
 * (Def. 10, Alg. 5).  A query set is answered by Alg. 6: its own count
 * filter and sketch, a first-layer gate over the A most frequent code
 * positions (the inverted index of Def. 9 / Alg. 4, held here in dense
 * position-major form), a second layer keeping the C sets of smallest
 * sketch Hamming distance, then an exact Hausdorff re-rank (Def. 4) of those
 * C candidates and a top-k (Def. 5).
 *
 * Conventions for every call:
 *  - Return value: BVSS_OK (0) or a negative status; bvss_last_error()
 *    gives a message for the calling thread.  No C++ exception crosses the
 *    ABI.  A CUDA error inside a call returns BVSS_ECUDA.
 *  - "device" pointers are CUDA device (or managed) memory of the device
 *    that was current when the index was built; "host" pointers are host
 *    memory.  Where a parameter says "host or device", the library looks the
 *    pointer up (cudaPointerGetAttributes) and copies host data itself.
 *  - stream: a cudaStream_t cast to void*, or NULL for the legacy default
 *    stream.  Work is enqueued on it.  Calls that take only device pointers
 *    return without waiting; their outputs are valid once the stream has
 *    synchronised.  Calls given host outputs synchronise the stream before
 *    returning.
 *  - The caller owns every buffer it passes.  The index owns its copies.
 *  - One index must not be queried from two host threads at once (queries
 *    share index-owned scratch memory).
 *  - Inputs are assumed finite; bvss_build rejects non-finite database
 *    values, and non-finite query values give unspecified results.
 *
 * Readings of points the paper leaves open (see the oracle for the same):
 * activations are FP32 sums in the order W's row lists its dims; WTA ties
 * and P ties break by lower index; counts saturate at 255; the candidate
 * stage keeps the min(C, |F1|) smallest (Hamming, id) pairs; top-k orders
 * by (distance, id) and pads with (-1, +inf).
 */
#ifndef BVSS_H
#define BVSS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define BVSS_OK 0
#define BVSS_EINVAL (-1)   /* an argument is out of range or inconsistent */
#define BVSS_ENOMEM (-2)   /* a device or host allocation failed */
#define BVSS_ECUDA (-3)    /* a CUDA call or kernel launch failed */
#define BVSS_ETIMEOUT (-4) /* a kernel's bounded wait gave up; reported by a later
                              synchronising call (bvss_sync, or a call with host outputs) */

/* limits of this implementation */
#define BVSS_MAX_D 4096        /* vector dimension */
#define BVSS_MAX_M 32768       /* code length b (FlyHash outputs) */
#define BVSS_MAX_FANIN 32      /* nonzeros per row of the sparse projection */
#define BVSS_MAX_L 1024        /* WTA winners per code */
#define BVSS_MAX_A 64          /* inverted lists read per query */
#define BVSS_MAX_C 16384       /* candidate budget per query set */
#define BVSS_MAX_K 1024        /* results per query set */
#define BVSS_MAX_QSET 128      /* vectors per query set */

/* Build parameters (Def. 7 and Alg. 6's Theta minus the search knobs). */
/* bvss_params.flags */
#define BVSS_BUILD_FP8 2    /* also keep an FP8 E4M3 copy (1 byte per value, one FP32 scale per
                               vector: its largest magnitude maps to 448) for BVSS_SEARCH_FP8;
                               needs d % 128 == 0 */
#define BVSS_BUILD_BF16 1   /* also keep a BF16 copy of the vectors (2 bytes per value) for
                               the tensor-core refine of BVSS_SEARCH_FAST; needs d % 64 == 0 */

typedef struct bvss_params {
    int32_t d;       /* vector dimension, 4..BVSS_MAX_D, multiple of 4 */
    int32_t m;       /* code length b = Bloom filter length; multiple of 128, <= BVSS_MAX_M */
    int32_t fanin;   /* F: input dims summed by each output of W, 1..min(d, BVSS_MAX_FANIN) */
    int32_t wta_l;   /* L_wta: winners kept by WTA, 1..min(m, BVSS_MAX_L) */
    int32_t flags;   /* 0 or an OR of BVSS_BUILD_BF16 and BVSS_BUILD_FP8 */
    int32_t reserved[3];
} bvss_params;

/* Search parameters of Alg. 6 (Theta's A, M, c = T) and Def. 5's k. */
/* bvss_search.flags */
#define BVSS_SEARCH_FAST 1  /* refine on the tensor cores: squared distances in the GEMM form
                               from BF16 vectors with FP32 accumulation (tcgen05); outside the
                               boundary band the trace's cand_dist is that value (the square
                               root of the GEMM-form Hausdorff value of the BF16 copies).  The top k are exact as in
                               bvss_query; the band is wider by the copy's rounding error (zero
                               for inputs on the 2^-8 grid).  Needs an index built with
                               BVSS_BUILD_BF16; batches with a query set of more than 64 vectors
                               use the FP32 refine */

#define BVSS_SEARCH_POPC_SCAN 2  /* score sketches (Alg. 6 line 12) with CUDA-core popcounts over
                                    the sets that pass layer 1, instead of the default tensor-core
                                    form (one FP8 GEMM over all pairs, masked by layer 1); every
                                    form gives identical h */

#define BVSS_SEARCH_ALG2 4  /* the plain BioVSS search (Alg. 2) instead of Alg. 6: candidates are
                               the C sets of smallest Haus^H -- Def. 4 with the Hamming distance
                               between per-vector codes in place of the norm -- over every set, by
                               (Haus^H, id); A and M are not used and the trace's cq, sq and plist
                               are not written (its h holds Haus^H).  Query sets of at most 32
                               vectors.  Combines with BVSS_SEARCH_FAST */
#define BVSS_SEARCH_FP8 8   /* refine on the tensor cores from the FP8 copy (BVSS_BUILD_FP8): the
                               query vectors are scaled and rounded to E4M3 the same way, the
                               squared distances are |q|^2 + |v|^2 - 2 s_q s_v (q8 . v8) of the
                               scaled values (the trace's cand_dist outside the boundary band
                               is the resulting Hausdorff value).  FP8 rounding (up to 2^-4
                               relative per value) moves a distance by up to e_q + e_v, the
                               norms of the two vectors' rounding errors; a band that wide holds
                               nearly every candidate, so by default the band takes 3 standard
                               deviations of the rounding model instead (independent zero-mean
                               errors per value: sqrt(e_q^2 + e_v^2) / sqrt(d) per distance) and
                               the top k are approximate; returned distances are still exact
                               values (as in bvss_query) of the returned sets.  Query sets of up
                               to 64 vectors; batches with a larger one use the FP32 refine */
#define BVSS_SEARCH_FP8_EXACT 16  /* with BVSS_SEARCH_FP8: the band from the rigorous bound, so
                                     the top k are exact as in bvss_query */
#define BVSS_SEARCH_TF32 32  /* refine on the tensor cores from the FP32 vectors themselves
                                (no copy needed), which the tensor core reads as TF32, with
                                the query vectors rounded to TF32 (to nearest): squared
                                distances |q~|^2 + |v|^2 - 2 q~.v~ with FP32 accumulation,
                                whose error (at most 2^-10 relative per value, zero for
                                values TF32 holds, such as those on the 2^-8 grid) widens the
                                boundary band; the top k and their distances are exact as in
                                bvss_query, and outside the band the trace's cand_dist is that
                                GEMM-form value.  d % 32 == 0 and query sets of up to 64
                                vectors (batches with a larger set use the CUDA-core FP32
                                refine).  BVSS_SEARCH_FAST and BVSS_SEARCH_FP8 take
                                precedence.  Every tensor-core form streams the query set's
                                operand through its copy ring where it does not fit in shared
                                memory beside it (TF32 above d = 512 for sets of up to 32
                                vectors, above 384 for up to 64) */
#define BVSS_SEARCH_SCAN_SETS_TMEM 64  /* the tensor-core sketch scan with the set sketches
                                          expanded into tensor memory as the A operand (128
                                          sets x 128 queries per tile) instead of the query
                                          sketches as the shared-memory A operand (256 queries
                                          x 128 sets); identical h */

typedef struct bvss_search {
    int32_t k;      /* results per query set, 1..BVSS_MAX_K */
    int32_t C;      /* candidate budget (c and T of Alg. 6), k <= C <= BVSS_MAX_C */
    int32_t A;      /* inverted lists accessed, 1..min(L, BVSS_MAX_A) */
    int32_t M;      /* minimum count; 0 lets every set through the first layer */
    int32_t flags;  /* 0 or an OR of BVSS_SEARCH_FAST, BVSS_SEARCH_POPC_SCAN, BVSS_SEARCH_ALG2,
                       BVSS_SEARCH_FP8, BVSS_SEARCH_FP8_EXACT, BVSS_SEARCH_TF32,
                       BVSS_SEARCH_SCAN_SETS_TMEM */
    int32_t reserved;
} bvss_search;

typedef struct bvss_index bvss_index;   /* opaque; owns its device memory */

/* Optional intermediates of Alg. 6 for parity checks.  Every pointer is
 * device memory or NULL (skipped).  n_q = queries of the call, N = sets,
 * W = m/32, Vq = query vectors of the call. */
typedef struct bvss_trace {
    uint16_t *qpos;      /* Vq x L   FlyHash positions of the query vectors, ascending */
    int32_t *cq;         /* n_q x m  query count filter C_Q (Alg. 6 line 1) */
    uint32_t *sq;        /* n_q x W  query sketch S_Q (line 2), bit p of word p/32 */
    uint16_t *plist;     /* n_q x A  top-A positions of C_Q (lines 3-4) */
    uint16_t *h;         /* n_q x N  Hamming(S_Q, S_i) (line 12); 0xFFFF = not in F1 */
    int32_t *cand;       /* n_q x C  candidate ids (F2), ascending; -1 padded */
    int32_t *n_cand;     /* n_q      number of candidates, min(C, |F1|) */
    float *cand_dist;    /* n_q x C  Hausdorff distance of cand[j] (the exact FP32 / FP64
                            value inside the boundary band, the refine's value outside it);
                            +inf padded */
} bvss_trace;

/*
 * bvss_build -- encode every database vector (Def. 7, Alg. 1) and build the
 * per-set sketches (Def. 10, Alg. 5) and count filters (Def. 8, Alg. 3),
 * held position-major as the dense form of the inverted index (Def. 9).
 *   vectors      host or device, V x d FP32 row-major, sets stored one after
 *                another; V = set_offsets[n_sets]
 *   set_offsets  host, n_sets + 1 int64, set_offsets[0] = 0, strictly
 *                increasing (every set holds at least one vector, Def. 2)
 *   n_sets       1 .. 2^31 - 1
 *   proj         host, m x fanin uint16: row j lists the input dims whose sum
 *                is output j of the sparse binary projection W, strictly
 *                ascending, each < d
 *   params       build parameters; flags = 0
 *   stream       see conventions; bvss_build synchronises it before returning
 *   out          receives the new index (NULL on error)
 * Errors: EINVAL for any bad size, order or non-finite vector value; ENOMEM;
 * ECUDA.  The caller may free every input once the call returns.
 */
int bvss_build(const float *vectors, const int64_t *set_offsets, int64_t n_sets,
               const uint16_t *proj, const bvss_params *params, void *stream,
               bvss_index **out);

/*
 * bvss_query -- Alg. 6 for a batch of query sets: FlyHash the query vectors,
 * C_Q / S_Q / P, first-layer gate (count >= M at one of the A positions),
 * the min(C, |F1|) smallest (Hamming, id) pairs, the Hausdorff distance
 * (Def. 4) of those candidates, then the k smallest (distance, id).
 * The k results are exact for every refine form (the FP8 form: with
 * BVSS_SEARCH_FP8_EXACT): each candidate's refine value
 * comes with a rigorous error bound (rounding of the stored copy, FP32
 * accumulation); every candidate whose interval reaches the k-th smallest upper
 * bound is re-scored directly in FP32 over all pairs, and candidates that FP32
 * cannot order at the top k are re-scored in FP64 on the GPU.  The order is
 * then that of the FP64 Hausdorff distance, ties by id, and every returned
 * distance is within (36 + ceil(d / 32)) 2^-24 (relative) of it.  More than
 * max(256, 4 k) candidates within FP32 rounding of the k-th distance (many
 * identical sets) exceed the stage's room; the next bvss_sync reports it.
 *   q_vectors   host or device, Vq x d FP32, query sets stored one after
 *               another; Vq = q_offsets[n_queries]
 *   q_offsets   host, n_queries + 1 int64, q_offsets[0] = 0, strictly
 *               increasing, each set at most BVSS_MAX_QSET vectors
 *   n_queries   >= 0
 *   s           search parameters
 *   out_ids     host or device, n_queries x k int64: set ids, -1 padded
 *   out_dist    host or device, n_queries x k FP32: distances, +inf padded
 * The first call (and any call with a larger batch) allocates index-owned
 * scratch memory.  Errors: EINVAL, ENOMEM, ECUDA.
 */
int bvss_query(const bvss_index *ix, const float *q_vectors, const int64_t *q_offsets,
               int64_t n_queries, const bvss_search *s, int64_t *out_ids,
               float *out_dist, void *stream);

/* bvss_query plus the intermediates named by tr (device pointers, may be NULL). */
int bvss_query_trace(const bvss_index *ix, const float *q_vectors,
                     const int64_t *q_offsets, int64_t n_queries,
                     const bvss_search *s, int64_t *out_ids, float *out_dist,
                     const bvss_trace *tr, void *stream);

/*
 * bvss_encode -- FlyHash (Def. 7) of n vectors with the index's projection.
 *   x     device, n x d FP32
 *   pos   device, n x L uint16 winner positions, ascending (may be NULL)
 *   mask  device, n x (m/32) uint32 code bits (may be NULL)
 */
int bvss_encode(const bvss_index *ix, const float *x, int64_t n, uint16_t *pos,
                uint32_t *mask, void *stream);

/* Sizes of an index. Any output pointer may be NULL. */
int bvss_index_info(const bvss_index *ix, bvss_params *params, int64_t *n_sets,
                    int64_t *n_vectors);

/* Copy database codes (Alg. 1) of vectors [first, first + n) to pos (device, n x L). */
int bvss_get_codes(const bvss_index *ix, int64_t first, int64_t n, uint16_t *pos,
                   void *stream);

/* Gather the sketches (Def. 10) of the sets listed in ids (device, n int64)
 * into out (device, n x m/32 uint32).  Ids must lie in [0, n_sets). */
int bvss_get_sketches(const bvss_index *ix, const int64_t *ids, int64_t n,
                      uint32_t *out, void *stream);

/* Gather the count filters (Def. 8, saturated at 255) of the sets listed in
 * ids (device, n int64) into out (device, n x m uint8, set-major). */
int bvss_get_counts(const bvss_index *ix, const int64_t *ids, int64_t n,
                    uint8_t *out, void *stream);

/* Wait for `stream`, then report device-side failures of earlier work on this
 * index: BVSS_ETIMEOUT if a kernel's bounded wait gave up (the flag is then
 * cleared), BVSS_ECUDA on a CUDA error, else BVSS_OK. */
int bvss_sync(bvss_index *ix, void *stream);

/* Failure-detection self-test: launches one kernel that waits, with the given
 * limit (nanoseconds, <= 10^9), on an mbarrier that nothing completes.  The
 * wait must give up and report, so the expected result is BVSS_ETIMEOUT with
 * the CUDA context still usable.  Synchronises the device; allocates 4 bytes. */
int bvss_selftest_wait_timeout(int64_t limit_ns);

/*
 * Query plans: the batched serving form.  A plan fixes the shape of a query
 * pass -- n_queries query sets with at most max_vectors vectors in all and at
 * most max_qset per set -- and binds it to the caller's device buffers:
 *   q_vectors  max_vectors x d FP32 (query vectors, set-contiguous),
 *   q_offsets  n_queries + 1 int64, q_offsets[0] = 0 (CSR over q_vectors),
 *   out_ids    n_queries x k int64, out_dist n_queries x k FP32 (as bvss_query).
 * The whole pass (an on-device check of the offsets, the FlyHash of every
 * query vector, then Alg. 6 -- or Alg. 2 with BVSS_SEARCH_ALG2 -- for
 * batches of query sets of uneven sizes) is captured once into a CUDA graph
 * and replayed by bvss_plan_launch, one graph launch per pass, with no host
 * work, no allocation and no synchronisation.  Between launches the caller
 * may rewrite the buffers' contents (new query sets, other sizes within the
 * bounds), but not move them.  Results equal bvss_query's on the same input.
 *
 * Offsets are read on the device.  When they break the bounds (a set empty or
 * larger than max_qset, more than max_vectors vectors, q_offsets[0] != 0),
 * the pass runs on one-vector placeholder sets instead, its results are not
 * valid, and the next bvss_sync on the index returns BVSS_EINVAL.
 *
 * The plan owns its workspace (about that of a bvss_query call of the same
 * shape).  It must be freed before its index, after the streams it was
 * launched on have been synchronised.  bvss_plan_create synchronises
 * `stream` and returns EINVAL for out-of-range shapes or search parameters
 * (as bvss_query), or for host buffers.
 */
typedef struct bvss_plan bvss_plan;

int bvss_plan_create(bvss_index *ix, const bvss_search *s, int64_t n_queries,
                     int64_t max_vectors, int32_t max_qset, const float *q_vectors,
                     const int64_t *q_offsets, int64_t *out_ids, float *out_dist, void *stream,
                     bvss_plan **out);
/* One pass: one graph launch on `stream` (asynchronous). */
int bvss_plan_launch(bvss_plan *p, void *stream);
/* Autotuner: times the pass on the buffers' current contents (reps launches
 * after one warm-up per setting) while varying one choice at a time -- the
 * sketch scan (either tensor-core form, or popcounts), the tensor-core refine's candidates
 * per CTA (128, 256, 512) and the depth of its copy ring (the most stages
 * that fit, and two and four fewer), whether the widest refine instance holds or streams
 * its query operand (where both are possible), the split of a batch's query sets by width
 * (on or off) and the query sets per internal batch (1024 up to 4096) -- keeps the
 * fastest setting and re-captures the graph with it.
 * Every setting gives the same results.  Synchronises `stream` first and
 * runs on the plan's own stream; *best_ms (may be NULL) = the chosen pass's
 * time in milliseconds. */
int bvss_plan_tune(bvss_plan *p, int32_t reps, void *stream, float *best_ms);
/* knobs (host, 7 entries, may be NULL): {scan (1 tensor-core with the query sketches as
 * the A operand, 2 popcount, 3 tensor-core with the set sketches in tensor memory, 0
 * Alg. 2's own), refine candidates per CTA (0 if the FP32 refine runs),
 * refine copy-ring depth, refine query-set width (32 or 64), 1 if the query sets of at
 * most 32 vectors of a batch run on the 32-wide refine and the wider ones on the 64-wide
 * one, query sets per internal batch, 1 if the widest refine instance streams its query
 * operand through its copy ring}; *launches = kernels per pass. */
int bvss_plan_info(const bvss_plan *p, int32_t *knobs, int64_t *launches);
/* Set the choices the autotuner varies and re-capture the graph: knobs (host, 6
 * entries) = {scan (0 by the search flags, 1 tensor-core with the query sketches as the
 * A operand, 2 popcount, 3 tensor-core with the set sketches in tensor memory), refine
 * candidates per CTA (0 = 512, else 1..512), refine copy-ring depth (0 = the most
 * stages that fit; 4 up to that, else the most that fit), width split (0: the query sets
 * of at most 32 vectors on the 32-wide refine, 2: all on the widest), query sets per
 * internal batch (0: 1024 or fewer as the index's size allows; at most 4096, bounded by
 * the plan's workspace), the refine's query operand (0: streamed through the copy ring
 * where it does not fit in shared memory, or where holding it leaves a ring of five
 * stages or fewer and streaming adds two; 1: held where it fits; 2: streamed)}.
 * bvss_plan_info reports the values in effect.  Results do not depend on them. */
int bvss_plan_set_knobs(bvss_plan *p, const int32_t *knobs);
void bvss_plan_free(bvss_plan *p);

/* Stages of bvss_query timed by the profiler (CUDA events on the query
 * stream, recorded between the kernels of every batch). */
#define BVSS_STAGE_ENCODE 0   /* FlyHash of the query vectors + C_Q, S_Q, P (Alg. 6 lines 1-4) */
#define BVSS_STAGE_GATE 1     /* layer-1 words per 32 sets (lines 5-9), plus the FP8 query
                                 sketches of the tensor-core scan */
#define BVSS_STAGE_SCAN 2     /* sketch Hamming over all sets (line 12) */
#define BVSS_STAGE_SELECT 3   /* the C smallest (Hamming, id) (lines 10-18) */
#define BVSS_STAGE_REFINE 4   /* Hausdorff of the candidates (lines 19-22) */
#define BVSS_STAGE_RESCORE 5  /* empty (the boundary stage, within BVSS_STAGE_TOPK, reads the
                                 tensor-core refine's values directly); kept for the layout */
#define BVSS_STAGE_TOPK 6     /* boundary re-score and the k smallest (distance, id)
                                 (line 23; see bvss_query) */
#define BVSS_N_STAGES 7

/* Turn per-stage timing of later bvss_query calls on (on != 0) or off. */
int bvss_profile_enable(bvss_index *ix, int on);

/* Sum of the stage times (ms, host array of BVSS_N_STAGES), the number of timed
 * query batches and the number of kernels those batches launched, since the
 * last reset.  Waits for the recorded events; reset != 0 clears the sums
 * afterwards.  n_batches and n_launches may be NULL. */
int bvss_profile_read(bvss_index *ix, double *stage_ms, int64_t *n_batches, int64_t *n_launches,
                      int reset);

/*
 * bvss_select_noalloc -- the candidate select of bvss_query (the min(C, |F1|)
 * smallest (Hamming, id) pairs, listed by ascending id) for callers that
 * cannot allocate GPU memory.  The paper has no counterpart: it exists for
 * programs in which cudaMalloc is not an option, for example a host process
 * whose device memory is already reserved in full by another framework's
 * caching allocator, or a latency-bound serving loop that must not call
 * cudaMalloc / cudaFree (which can synchronise the whole device).  It calls
 * neither, nor any allocating library routine: its scratch memory is one
 * fixed array of about 5.2 MB compiled into the library, which every GPU that
 * loads the library holds until the process exits.
 *   h          device, n_queries rows of h_stride uint16 Hamming scores,
 *              16-byte aligned; the layout of bvss_trace.h with rows padded
 *              to h_stride.  A score in 0..m is a set of F1; any larger
 *              value (0xFFFF by convention) marks a set outside F1
 *   n_sets     1 .. BVSS_NOALLOC_MAX_SETS
 *   h_stride   row stride in elements, >= n_sets, multiple of 8
 *   m          code length (largest valid score), 1 .. BVSS_NOALLOC_MAX_M
 *   n_queries  0 .. BVSS_NOALLOC_MAX_QUERIES
 *   C          candidate budget, 1 .. BVSS_MAX_C
 *   cand       device, n_queries x C int32: ids ascending, -1 padded
 *   n_cand     device, n_queries int32 (may be NULL): min(C, |F1|)
 * Sizes beyond the limits return BVSS_EINVAL with a message.  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.
 * The address is kept for the life of the process: do not call it again on
 * a device after cudaDeviceReset (or any teardown of its primary context).
 * Every call shares the one array and leaves its contents behind (the call
 * clears what has to start at zero), so calls that overlap on the GPU --
 * on two streams, or from two host threads -- race and must be serialised
 * by the caller.
 */
#define BVSS_NOALLOC_MAX_QUERIES 32
#define BVSS_NOALLOC_MAX_M 8192
#define BVSS_NOALLOC_MAX_SETS 16777216LL
int bvss_select_noalloc(const uint16_t *h, int64_t n_sets, int64_t h_stride, int32_t m,
                        int32_t n_queries, int32_t C, int32_t *cand, int32_t *n_cand,
                        void *stream);

/*
 * The learned projection.  The paper's own runs use BioHash, a learned W in
 * h = WTA(W v) (Def. 7; the BioHash discussion beside it and the appendix on
 * its iteration), in place of FlyHash's random sparse binary W.  Here W is a
 * dense BF16 layer (m x d), run on the tensor cores, and is trained on
 * neighbour pairs that the exact refine itself produces; FlyHash stays the
 * fallback (bvss_build).  Readings: the layer computes a = bf16(W) bf16(x)
 * with FP32 accumulation (bf16: round to nearest even), which is exact for
 * weights and inputs on the 2^-8 grid with norms far below 2^8, so the codes
 * then equal those of an exact layer; WTA ties go to the lower index.
 */

/* bvss_build with the learned dense projection in place of FlyHash.
 *   w       host or device, m x d FP32 row-major (m = params->m, d = params->d),
 *           rounded to BF16 for the layer; the caller keeps ownership
 *   params  as bvss_build; fanin is not used (bvss_index_info reports 0); needs
 *           d % 64 == 0 and m % 128 == 0
 * Everything else (vectors, offsets, flags, errors) as bvss_build.  Queries on
 * the index (bvss_query, plans, bvss_encode) encode with the same layer. */
int bvss_build_dense(const float *vectors, const int64_t *set_offsets, int64_t n_sets,
                     const float *w, const bvss_params *params, void *stream, bvss_index **out);

/* Activations of the dense layer, a = W x, for n vectors on the tensor cores.
 *   x_bf16  device, n x d BF16 row-major (16-byte aligned)
 *   w_bf16  device, m x d BF16 row-major (16-byte aligned)
 *   act     device, n rows of ld_act FP32 (16-byte aligned): act[i][j] = w_j . x_i
 * d % 64 == 0, m % 128 == 0, ld_act >= m, ld_act % 4 == 0.  Asynchronous; a
 * bounded wait inside that gives up is reported by bvss_learn_sync.  Errors:
 * EINVAL, ECUDA. */
int bvss_dense_forward(const void *x_bf16, int64_t n, int32_t d, const void *w_bf16, int32_t m,
                       float *act, int64_t ld_act, void *stream);

/* Waits for `stream`, then reports BVSS_ETIMEOUT (and clears it) if a dense-layer
 * kernel's bounded wait gave up since the last call, BVSS_ECUDA on a CUDA error. */
int bvss_learn_sync(void *stream);

/* Training loss of n neighbour pairs and its gradient in the activations.  For pair i
 * with activations a = act_x[i], b = act_y[i] (m values each, rows ld_act apart) and
 * label y = labels[i] (1: neighbours, 0: not): thresholds t_a, t_b midway between the
 * L-th and (L+1)-th largest values; soft codes c_j = sigmoid((a_j - t) / temperature);
 * overlap o = (1/L) sum_j c_j(a) c_j(b); loss = log(1 + exp(-z)) with z = +-scale (o -
 * margin), + for y = 1.  g_x[i], g_y[i] (device, rows ld_g apart) receive d loss / d a
 * and d loss / d b with the thresholds held fixed; *loss_sum (device) is incremented by
 * the sum of the n losses.  All pointers device memory.  Errors: EINVAL, ECUDA. */
int bvss_learn_pair_grad(const float *act_x, const float *act_y, int64_t ld_act,
                         const uint8_t *labels, int64_t n, int32_t m, int32_t L,
                         float temperature, float scale, float margin, float *g_x, float *g_y,
                         int64_t ld_g, double *loss_sum, void *stream);

/* The layer's weight gradient: dw (device, m x d FP32) = (1/n) sum_i g_x[i] x_i^T +
 * g_y[i] y_i^T, with g_x, g_y as bvss_learn_pair_grad writes them and x_bf16, y_bf16
 * (device, n x d BF16) the pairs' vectors.  m and d multiples of 64. */
int bvss_learn_weight_grad(const float *g_x, const float *g_y, int64_t ld_g, const void *x_bf16,
                           const void *y_bf16, int64_t n, int32_t m, int32_t d, float *dw,
                           void *stream);

/* One normalized gradient step: w (device, m x d FP32, updated in place) <- w - eta dw /
 * max|dw| (so eta is the largest entry of the update, the update magnitude M_t of the
 * paper's BioHash iteration analysis), then every row rescaled to norm row_norm;
 * wq_bf16 (device, m x d BF16) receives the forward weights: w rounded to the nearest
 * multiple of 2^-8 (ties to even), clamped to [-1, 1].  *absmax (device) receives
 * max|dw|.  Errors: EINVAL, ECUDA. */
int bvss_learn_update(float *w, const float *dw, int32_t m, int32_t d, float eta, float row_norm,
                      float *absmax, void *wq_bf16, void *stream);

/* BF16 copy (round to nearest even) of n x d FP32 values; both device memory. */
int bvss_to_bf16(const float *x, int64_t n, int32_t d, void *out, void *stream);

/* BF16 copies of the index's database vectors rows[0..n) (device int64, global rows
 * in set order) into out (device, n x d BF16); an id outside [0, n_vectors) gives a
 * row of zeros. */
int bvss_index_rows_bf16(const bvss_index *ix, const int64_t *rows, int64_t n, void *out,
                         void *stream);

/* For mining training pairs from the refine's neighbours: rows (device, Vq x k int64)
 * [a][t] = the global row of the database vector nearest to query vector a (direct
 * FP32 distance, ties to the lower row) in set sets[q][t], q the query set holding a;
 * -1 for a set id outside [0, n_sets).  q_vectors device (Vq x d FP32), q_offsets host
 * (as bvss_query), sets device (n_queries x k int64).  Synchronises `stream`. */
int bvss_nearest_rows(const bvss_index *ix, const float *q_vectors, const int64_t *q_offsets,
                      int64_t n_queries, const int64_t *sets, int32_t k, int64_t *rows,
                      void *stream);

/* Release an index and all its device memory (NULL is a no-op).  Work that
 * uses the index must have finished. */
void bvss_free(bvss_index *ix);

/* Message of the last failed call on this thread ("" if none). */
const char *bvss_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* BVSS_H */
