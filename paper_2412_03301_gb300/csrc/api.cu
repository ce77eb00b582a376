// api.cu -- the C ABI of include/bvss.h: argument checks, index memory,
// and the order of kernels for bvss_build (Alg. 1, 3, 5 and the dense form of
// Alg. 4) and bvss_query (Alg. 6) of arXiv 2412.03301.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "bvss_internal.cuh"

using namespace bvss;

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

#define BVSS_CU(call)                                                                   \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(e_ == cudaErrorMemoryAllocation ? BVSS_ENOMEM : BVSS_ECUDA,     \
                        "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),         \
                        __FILE__, __LINE__);                                            \
    } while (0)

// device (or managed) memory, as opposed to host memory of any kind
bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <class T>
cudaError_t dalloc(T **p, size_t count) {
    *p = nullptr;
    return cudaMalloc(reinterpret_cast<void **>(p), (count ? count : 1) * sizeof(T));
}

template <class T>
void dfree(T *&p) {
    if (p) cudaFree(p);
    p = nullptr;
}

int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// device status bit of a plan whose query offsets failed the on-device check
constexpr int kErrPlanInput = 8;

// h rows are padded to 64 entries so every row starts 128-byte aligned
int64_t h_stride(const bvss_index *ix) { return round_up(ix->n_sets, 64); }

// largest query batch whose score matrix stays within 2 GiB
int64_t batch_cap(const bvss_index *ix) {
    int64_t qb = ((int64_t)1 << 30) / h_stride(ix);
    if (qb > 1024) qb = 1024;
    if (qb < 1) qb = 1;
    return qb;
}

// a plan's largest internal batch: up to 4096 query sets, score matrix within 4 GiB
int64_t plan_batch_cap(const bvss_index *ix) {
    int64_t qb = ((int64_t)1 << 31) / h_stride(ix);
    if (qb > 4096) qb = 4096;
    if (qb < 1) qb = 1;
    return qb;
}

void free_workspace(Workspace &w) {
    dfree(w.qvec);
    dfree(w.qoff);
    dfree(w.qpos);
    dfree(w.sq);
    dfree(w.plist);
    dfree(w.h);
    dfree(w.gate);
    dfree(w.q8);
    dfree(w.qpop);
    dfree(w.hist);
    dfree(w.thr);
    dfree(w.chunk);
    dfree(w.bmin);
    dfree(w.bound);
    dfree(w.cand);
    dfree(w.cand_dist);
    dfree(w.pair);
    dfree(w.wlist);
    dfree(w.qop);
    dfree(w.qop_n);
    dfree(w.qop_sc);
    dfree(w.enc_x);
    dfree(w.enc_act);
    dfree(w.out_ids);
    dfree(w.out_dist);
    w = Workspace();
}

void free_index(bvss_index *ix) {
    if (!ix) return;
    dfree(ix->vec);
    dfree(ix->vnorm);
    dfree(ix->vec16);
    dfree(ix->vnorm16);
    dfree(ix->vec8);
    dfree(ix->vscale8);
    dfree(ix->vnorm8);
    dfree(ix->rstat);
    dfree(ix->wproj16);
    dfree(ix->set_off);
    dfree(ix->proj);
    dfree(ix->codes);
    dfree(ix->sketch);
    dfree(ix->spop);
    dfree(ix->count);
    dfree(ix->flag);
    dfree(ix->err);
    for (int i = 0; i < ix->n_planes; ++i) dfree(ix->planes[i].words);
    free_workspace(ix->ws);
    for (int i = 0; i < kOffRing; ++i) {
        if (ix->off_host[i]) cudaFreeHost(ix->off_host[i]);
        if (ix->off_event[i]) cudaEventDestroy(ix->off_event[i]);
    }
    for (int64_t i = 0; i < ix->prof_cap; ++i) cudaEventDestroy(ix->prof_ev[i]);
    delete[] ix->prof_ev;
    delete ix;
}

int check_params(const bvss_params *p) {
    if (!p) return fail(BVSS_EINVAL, "params is NULL");
    if (p->d < 4 || p->d > BVSS_MAX_D || p->d % 4 != 0)
        return fail(BVSS_EINVAL, "d = %d: need 4 <= d <= %d and d %% 4 == 0", p->d, BVSS_MAX_D);
    if (p->m < 128 || p->m > BVSS_MAX_M || p->m % 128 != 0)
        return fail(BVSS_EINVAL, "m = %d: need 128 <= m <= %d and m %% 128 == 0", p->m,
                    BVSS_MAX_M);
    if (p->fanin < 1 || p->fanin > BVSS_MAX_FANIN || p->fanin > p->d)
        return fail(BVSS_EINVAL, "fanin = %d: need 1 <= fanin <= min(d, %d)", p->fanin,
                    BVSS_MAX_FANIN);
    if (p->wta_l < 1 || p->wta_l > BVSS_MAX_L || p->wta_l > p->m)
        return fail(BVSS_EINVAL, "wta_l = %d: need 1 <= L <= min(m, %d)", p->wta_l, BVSS_MAX_L);
    if (p->flags & ~(BVSS_BUILD_BF16 | BVSS_BUILD_FP8)) return fail(BVSS_EINVAL, "unknown build flags");
    if ((p->flags & BVSS_BUILD_BF16) && p->d % 64 != 0)
        return fail(BVSS_EINVAL, "BVSS_BUILD_BF16 needs d %% 64 == 0 (d = %d)", p->d);
    if ((p->flags & BVSS_BUILD_FP8) && p->d % 128 != 0)
        return fail(BVSS_EINVAL, "BVSS_BUILD_FP8 needs d %% 128 == 0 (d = %d)", p->d);
    return BVSS_OK;
}

int check_offsets(const int64_t *off, int64_t n, int64_t max_size, const char *what) {
    if (!off) return fail(BVSS_EINVAL, "%s offsets are NULL", what);
    if (off[0] != 0) return fail(BVSS_EINVAL, "%s offsets must start at 0", what);
    for (int64_t i = 0; i < n; ++i) {
        const int64_t s = off[i + 1] - off[i];
        if (s < 1) return fail(BVSS_EINVAL, "%s set %lld is empty or offsets decrease", what,
                               (long long)i);
        if (max_size > 0 && s > max_size)
            return fail(BVSS_EINVAL, "%s set %lld holds %lld vectors (limit %lld)", what,
                        (long long)i, (long long)s, (long long)max_size);
    }
    return BVSS_OK;
}

int check_device(const bvss_index *ix) {
    int dev = -1;
    BVSS_CU(cudaGetDevice(&dev));
    if (dev != ix->device)
        return fail(BVSS_EINVAL, "index lives on device %d but device %d is current", ix->device,
                    dev);
    return BVSS_OK;
}

// first-layer gate plane for minimum count M (1 <= M <= 255), built on demand
int get_plane(bvss_index *ix, int M, cudaStream_t st, const uint32_t **out) {
    for (int i = 0; i < ix->n_planes; ++i)
        if (ix->planes[i].M == M) {
            *out = ix->planes[i].words;
            return BVSS_OK;
        }
    int slot = ix->n_planes;
    if (slot == kMaxPlanes) {
        if (ix->n_plans > 0)
            return fail(BVSS_EINVAL, "%d gate planes are cached and live plans use them; free "
                                     "the plans to search with another M", kMaxPlanes);
        slot = kMaxPlanes - 1;   // replace the most recent extra plane
        BVSS_CU(cudaStreamSynchronize(st));
        dfree(ix->planes[slot].words);
    } else {
        ++ix->n_planes;
    }
    GatePlane &pl = ix->planes[slot];
    pl.M = -1;
    BVSS_CU(dalloc(&pl.words, (size_t)ix->p.m * ix->NW));
    BVSS_CU(launch_gate_plane(ix->count, ix->p.m, ix->n_sets, ix->NW, M, pl.words, st));
    pl.M = M;
    *out = pl.words;
    return BVSS_OK;
}

// allocate a workspace for batches of nq query sets with nvq vectors in all
int alloc_workspace(const bvss_index *ix, Workspace &w, int64_t nq, int64_t nvq, int C, int A,
                    int k, bool need_qvec, bool need_out) {
    const int m = ix->p.m, W = ix->W, L = ix->p.wta_l, d = ix->p.d;
    const int64_t hs = h_stride(ix);
    const int n_chunks = (int)((ix->n_sets + kSelChunk - 1) / kSelChunk);
    BVSS_CU(dalloc(&w.qoff, nq + 1));
    BVSS_CU(dalloc(&w.qpos, (size_t)nvq * L));
    BVSS_CU(dalloc(&w.sq, (size_t)nq * W));
    BVSS_CU(dalloc(&w.plist, (size_t)nq * A));
    BVSS_CU(dalloc(&w.h, (size_t)nq * hs));
    BVSS_CU(dalloc(&w.gate, (size_t)nq * ix->NW));
    BVSS_CU(dalloc(&w.q8, scan_mma_q8_bytes(nq, m)));
    BVSS_CU(dalloc(&w.qpop, (size_t)round_up(nq, 256)));
    BVSS_CU(dalloc(&w.hist, (size_t)nq * ((m > 2 * L ? m : 2 * L) + 1)));
    BVSS_CU(dalloc(&w.thr, (size_t)nq * 4));
    BVSS_CU(dalloc(&w.chunk, (size_t)nq * n_chunks * kSelRangeWords));
    BVSS_CU(dalloc(&w.bmin, (size_t)nq * ((ix->n_sets + kSelBlock - 1) / kSelBlock)));
    BVSS_CU(dalloc(&w.bound, (size_t)nq));
    BVSS_CU(dalloc(&w.cand, (size_t)nq * C));
    BVSS_CU(dalloc(&w.cand_dist, (size_t)nq * C));
    BVSS_CU(dalloc(&w.pair, (size_t)nq * C));
    BVSS_CU(dalloc(&w.wlist, (size_t)2 * nq + 2));
    // the refine's streamed query operand, for the forms this index can run that can
    // stream it (by necessity, by default or when the tuner asks)
    size_t qop = 0;
    for (int wq = 32; wq <= 64; wq += 32) {
        const Elem forms[3] = {Elem::TF32, Elem::BF16, Elem::FP8};
        const bool have[3] = {true, ix->vec16 != nullptr, ix->vec8 != nullptr};
        for (int f = 0; f < 3; ++f)
            if (have[f] && refine_mma_streams(d, wq, forms[f], 2)) {
                const size_t b = refine_mma_qop_bytes(d, forms[f]);
                if (b > qop) qop = b;
            }
    }
    if (qop) {
        BVSS_CU(dalloc(&w.qop, (size_t)nq * qop));
        BVSS_CU(dalloc(&w.qop_n, (size_t)nq * 64));
        BVSS_CU(dalloc(&w.qop_sc, (size_t)nq * 64));
    }
    if (need_qvec) BVSS_CU(dalloc(&w.qvec, (size_t)nvq * d));
    if (ix->wproj16) {
        BVSS_CU(dalloc(&w.enc_x, (size_t)kEncChunk * d));
        BVSS_CU(dalloc(&w.enc_act, (size_t)kEncChunk * m));
    }
    if (need_out) {
        BVSS_CU(dalloc(&w.out_ids, (size_t)nq * k));
        BVSS_CU(dalloc(&w.out_dist, (size_t)nq * k));
    }
    w.cap_q = nq;
    w.cap_vq = nvq;
    w.cap_C = C;
    w.cap_A = A;
    w.cap_k = k;
    return BVSS_OK;
}

int ensure_workspace(bvss_index *ix, int64_t nq, int64_t nvq, int C, int A, int k,
                     bool need_qvec, bool need_out) {
    Workspace &w = ix->ws;
    if (nq > w.cap_q || nvq > w.cap_vq || C > w.cap_C || A > w.cap_A || k > w.cap_k ||
        (need_qvec && !w.qvec) || (need_out && !w.out_ids)) {
        const int64_t cq = nq > w.cap_q ? nq : w.cap_q;
        const int64_t cvq = nvq > w.cap_vq ? nvq : w.cap_vq;
        const int cC = C > w.cap_C ? C : w.cap_C;
        const int cA = A > w.cap_A ? A : w.cap_A;
        const int ck = k > w.cap_k ? k : w.cap_k;
        const bool had_qvec = w.qvec != nullptr, had_out = w.out_ids != nullptr;
        BVSS_CU(cudaDeviceSynchronize());
        free_workspace(w);
        const int rc = alloc_workspace(ix, w, cq, cvq, cC, cA, ck, need_qvec || had_qvec,
                                       need_out || had_out);
        if (rc) {
            free_workspace(w);
            return rc;
        }
    }
    // pinned staging ring for the per-batch query offsets
    for (int i = 0; i < kOffRing; ++i) {
        if (ix->off_cap < w.cap_q + 1 || !ix->off_host[i]) {
            if (ix->off_event[i]) BVSS_CU(cudaEventSynchronize(ix->off_event[i]));
            if (ix->off_host[i]) cudaFreeHost(ix->off_host[i]);
            ix->off_host[i] = nullptr;
            BVSS_CU(cudaMallocHost(reinterpret_cast<void **>(&ix->off_host[i]),
                                   sizeof(int64_t) * (size_t)(w.cap_q + 1)));
            if (!ix->off_event[i])
                BVSS_CU(cudaEventCreateWithFlags(&ix->off_event[i], cudaEventDisableTiming));
        }
    }
    ix->off_cap = w.cap_q + 1;
    return BVSS_OK;
}

// wait for the stream, then report (and clear) the device error word
int sync_and_check(bvss_index *ix, cudaStream_t st) {
    BVSS_CU(cudaStreamSynchronize(st));
    int e = 0;
    BVSS_CU(cudaMemcpy(&e, ix->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
        BVSS_CU(cudaMemset(ix->err, 0, sizeof(int)));
        if (e == kErrPlanInput)
            return fail(BVSS_EINVAL, "a plan's query offsets were out of range; its results "
                                     "are not valid");
        if (e == kErrBandOverflow)
            return fail(BVSS_ECUDA, "more than max(256, 4 k) candidates lie within FP32 "
                                    "rounding of the k-th distance; the order among them is "
                                    "not exact");
        return fail(BVSS_ETIMEOUT, "a kernel's bounded wait gave up (device status %d)", e);
    }
    return BVSS_OK;
}

// reserve kProfEvents timing events for one batch; returns their base or null
cudaEvent_t *prof_reserve(bvss_index *ix) {
    if (ix->prof_used + kProfEvents > ix->prof_cap) {
        const int64_t cap = ix->prof_cap ? 2 * ix->prof_cap : 64 * kProfEvents;
        cudaEvent_t *ev = new (std::nothrow) cudaEvent_t[cap];
        if (!ev) return nullptr;
        for (int64_t i = 0; i < ix->prof_cap; ++i) ev[i] = ix->prof_ev[i];
        for (int64_t i = ix->prof_cap; i < cap; ++i)
            if (cudaEventCreate(&ev[i]) != cudaSuccess) {
                for (int64_t j = ix->prof_cap; j < i; ++j) cudaEventDestroy(ev[j]);
                delete[] ev;
                return nullptr;
            }
        delete[] ix->prof_ev;
        ix->prof_ev = ev;
        ix->prof_cap = cap;
    }
    cudaEvent_t *base = ix->prof_ev + ix->prof_used;
    ix->prof_used += kProfEvents;
    return base;
}

// Kernel and tile choices of one query pass.  Zero fields take the built-in
// heuristics; a plan's autotuner sets them to the fastest measured choice.
struct Knobs {
    int scan = 0;       // 1: tensor-core sketch scan, 2: popcount scan, 0: by the search flags
    int cand_cta = 0;   // tensor-core refine: candidates per CTA (0: 512)
    int stages = 0;     // tensor-core refine: depth of the copy ring (0: the most that fit)
    int bucket = 0;     // tensor-core refine of a batch holding query sets over 32 vectors:
                        // 0 the sets of at most 32 on the 32-wide instance and the others on
                        // the 64-wide one, 2 all on the 64-wide one
    int batch = 0;      // query plans: query sets per internal batch (0: the default cap)
    int qs = 0;         // tensor-core refine: 1 hold the query operand in shared memory where
                        // it fits, 2 stream it through the ring, 0 by the default rule
};

// Codes (Def. 7) of n vectors x (device FP32) with the index's projection: the sparse
// binary FlyHash W, or the learned dense layer -- blocks of kEncChunk vectors rounded to
// BF16, their activations on the tensor cores (launch_dense_gemm), then WTA.  xb / act:
// kEncChunk x d BF16 and kEncChunk x m FP32 of scratch (dense layer only).  n_dev: the
// count, read on the device (the dense layer then encodes all n rows).  Counts launches.
int encode_vectors(const bvss_index *ix, const float *x, int64_t n, uint16_t *pos,
                   uint32_t *mask, __nv_bfloat16 *xb, float *act, cudaStream_t st,
                   const int64_t *n_dev, int64_t *launches) {
    const int d = ix->p.d, m = ix->p.m, L = ix->p.wta_l;
    if (!ix->wproj16) {
        BVSS_CU(launch_encode(x, n, d, ix->proj, m, ix->p.fanin, L, pos, mask, st, n_dev));
        if (launches) ++*launches;
        return BVSS_OK;
    }
    for (int64_t v0 = 0; v0 < n; v0 += kEncChunk) {
        const int64_t nb = n - v0 < kEncChunk ? n - v0 : kEncChunk;
        BVSS_CU(launch_rows_bf16(x + v0 * d, d, nullptr, nb, xb, st));
        BVSS_CU(launch_dense_gemm(xb, nb, d, ix->wproj16, m, act, m, ix->err, st));
        BVSS_CU(launch_encode_dense(act, nb, m, m, L, pos ? pos + v0 * L : nullptr,
                                    mask ? mask + v0 * (m / 32) : nullptr, st));
        if (launches) *launches += 3;
    }
    return BVSS_OK;
}

int check_search(const bvss_index *ix, const bvss_search *s) {
    if (!s) return fail(BVSS_EINVAL, "search parameters are NULL");
    const int L = ix->p.wta_l;
    if (s->k < 1 || s->k > BVSS_MAX_K)
        return fail(BVSS_EINVAL, "k = %d: need 1 <= k <= %d", s->k, BVSS_MAX_K);
    if (s->C < s->k || s->C > BVSS_MAX_C)
        return fail(BVSS_EINVAL, "C = %d: need k <= C <= %d", s->C, BVSS_MAX_C);
    if ((s->flags & BVSS_SEARCH_ALG2) == 0 && (s->A < 1 || s->A > L || s->A > BVSS_MAX_A))
        return fail(BVSS_EINVAL, "A = %d: need 1 <= A <= min(L, %d)", s->A, BVSS_MAX_A);
    if (s->M < 0) return fail(BVSS_EINVAL, "M = %d: need M >= 0", s->M);
    if (s->flags & ~(BVSS_SEARCH_FAST | BVSS_SEARCH_POPC_SCAN | BVSS_SEARCH_ALG2 | BVSS_SEARCH_FP8 |
                     BVSS_SEARCH_FP8_EXACT | BVSS_SEARCH_TF32 | BVSS_SEARCH_SCAN_SETS_TMEM))
        return fail(BVSS_EINVAL, "unknown search flags");
    if ((s->flags & BVSS_SEARCH_FAST) && !ix->vec16)
        return fail(BVSS_EINVAL, "BVSS_SEARCH_FAST needs an index built with BVSS_BUILD_BF16");
    if ((s->flags & BVSS_SEARCH_FP8) && !ix->vec8)
        return fail(BVSS_EINVAL, "BVSS_SEARCH_FP8 needs an index built with BVSS_BUILD_FP8");
    return BVSS_OK;
}

// Refine a batch runs: 2 FP8 tensor cores, 1 BF16 tensor cores, 0 FP32.
int refine_form(const bvss_index *ix, int flags, int max_mq) {
    const int d = ix->p.d;
    if ((flags & BVSS_SEARCH_FP8) && ix->vec8 && refine_mma_supported(d, max_mq, Elem::FP8))
        return 2;
    if ((flags & (BVSS_SEARCH_FAST | BVSS_SEARCH_FP8)) && ix->vec16 &&
        refine_mma_supported(d, max_mq, Elem::BF16))
        return 1;
    if ((flags & BVSS_SEARCH_TF32) && refine_mma_supported(d, max_mq, Elem::TF32)) return 3;
    return 0;
}

// Everything a query batch needs besides the index, for enqueue_batch.
struct Batch {
    const float *qv = nullptr;       // query vectors (device)
    const int64_t *qoff = nullptr;   // nb + 1 offsets into qv and qpos (device)
    int nb = 0;                      // query sets
    int max_mq = 0;                  // bound on the vectors of one query set
    int64_t enc_n = 0;               // > 0: encode qv[0, enc_n) into w.qpos first
    const int64_t *enc_n_dev = nullptr;   // with enc_n: the count, read on the device
    const uint32_t *plane = nullptr;      // layer-1 plane for M (gate mode 1)
    int64_t *ids = nullptr;          // nb x k results (device)
    float *dist = nullptr;
    int32_t *cq_trace = nullptr;
    cudaEvent_t *ev = nullptr;       // kProfEvents stage events, or null
};

// Alg. 6 (or Alg. 2) for one batch, enqueued on st: no host synchronisation and no
// allocation, so a stream capture of it is a valid CUDA graph.  Counts the launches.
int enqueue_batch(bvss_index *ix, Workspace &w, const bvss_search *s, const Knobs &kn,
                  const Batch &b, int64_t *launches, cudaStream_t st) {
    const int L = ix->p.wta_l, m = ix->p.m, d = ix->p.d, W = ix->W;
    const int k = s->k, C = s->C, A = s->A, M = s->M, nb = b.nb;
    const bool alg2 = (s->flags & BVSS_SEARCH_ALG2) != 0;
    // the scan form: 1 tensor cores with the query blocks as the shared-memory A operand,
    // 3 tensor cores with the set sketches in tensor memory, 2 CUDA-core popcounts
    const int scan_form = kn.scan ? kn.scan
                          : (s->flags & BVSS_SEARCH_POPC_SCAN) ? 2
                          : (s->flags & BVSS_SEARCH_SCAN_SETS_TMEM) ? 3 : 1;
    const bool tensor_scan = scan_form != 2;
    const int gate_mode = M == 0 ? 0 : (M > 255 ? 2 : 1);
    const int64_t hs = h_stride(ix);
    cudaEvent_t *ev = b.ev;
    const float *qv = b.qv;
    int64_t n = 0;
    if (ev) BVSS_CU(cudaEventRecord(ev[0], st));
    // Alg. 6 lines 1-4 (Alg. 2 lines 2-5: the codes only)
    if (b.enc_n > 0) {
        const int rc = encode_vectors(ix, qv, b.enc_n, w.qpos, nullptr, w.enc_x, w.enc_act, st,
                                      b.enc_n_dev, &n);
        if (rc) return rc;
    }
    if (!alg2) {
        BVSS_CU(launch_query_prep(w.qpos, b.qoff, nb, m, L, A, w.sq, w.plist, b.cq_trace, st));
        ++n;
    }
    if (ev) BVSS_CU(cudaEventRecord(ev[1], st));
    // lines 5-9: layer-1 words per 32 sets (and the FP8 query operand)
    if (!alg2 && gate_mode == 1) {
        BVSS_CU(launch_gate(b.plane, ix->NW, w.plist, A, nb, w.gate, st));
        ++n;
    }
    if (!alg2 && tensor_scan) {
        BVSS_CU(launch_expand_q(w.sq, nb, W, w.q8, w.qpop, st));
        ++n;
    }
    if (ev) BVSS_CU(cudaEventRecord(ev[2], st));
    // line 12 (Alg. 2 lines 6-8: Haus^H against every set)
    if (alg2)
        BVSS_CU(launch_haus_h(w.qpos, b.qoff, nb, ix->codes, ix->set_off, ix->n_sets, m, L, w.h,
                              hs, st));
    else if (scan_form == 1)
        BVSS_CU(launch_scan_mma(ix->sketch, ix->spop, ix->n_sets, W, w.gate, ix->NW, gate_mode,
                                w.q8, w.qpop, nb, w.h, hs, ix->err, st, w.bmin));
    else if (scan_form == 3)
        BVSS_CU(launch_scan_tm(ix->sketch, ix->spop, ix->n_sets, W, w.gate, ix->NW, gate_mode,
                               w.q8, w.qpop, nb, w.h, hs, ix->err, st, w.bmin));
    else
        BVSS_CU(launch_scan(ix->sketch, ix->n_sets, W, w.gate, ix->NW, gate_mode, w.sq, nb, w.h,
                            hs, st));
    ++n;
    if (ev) BVSS_CU(cudaEventRecord(ev[3], st));
    // lines 10-18 (Alg. 2 line 9); scores run up to m (Hamming of sketches) or 2L (Haus^H)
    // the tensor-core scan also leaves the block minima that let the select skip blocks
    const bool bounded = !alg2 && tensor_scan;
    BVSS_CU(launch_select(w.h, ix->n_sets, hs, alg2 ? 2 * L : m, nb, C, w.hist, w.thr, w.chunk,
                          w.cand, st, bounded ? w.bmin : nullptr, bounded ? w.bound : nullptr));
    n += kSelectKernels + (bounded ? 1 : 0);
    if (ev) BVSS_CU(cudaEventRecord(ev[4], st));
    // lines 19-23
    // the FP8 copy for query sets it takes, else the BF16 one, else FP32
    const int form = refine_form(ix, s->flags, b.max_mq);
    const bool mma = form > 0;
    const Elem el = static_cast<Elem>(mma ? form : 1);
    const void *vecb = form == 2   ? (const void *)ix->vec8
                       : form == 3 ? (const void *)ix->vec
                                   : (const void *)ix->vec16;
    const float *vnb = form == 2 ? ix->vnorm8 : (form == 3 ? ix->vnorm : ix->vnorm16);
    const bool split = mma && b.max_mq > 32 && kn.bucket != 2 && refine_mma_supported(d, 32, el);
    const int qs_mode = w.qop ? kn.qs : 1;
    if (mma && (refine_mma_streams(d, b.max_mq, el, qs_mode) ||
                (split && refine_mma_streams(d, 32, el, qs_mode)))) {
        // a query operand too large for shared memory: stage it for the streamed refine
        if (!w.qop) return fail(BVSS_ECUDA, "no workspace for the streamed query operand");
        BVSS_CU(launch_query_op(qv, b.qoff, nb, d, el, w.qop, w.qop_n, w.qop_sc, st));
        ++n;
    }
    if (split) {
        // the batch's query sets by width: the narrow ones on the 32-wide instance
        BVSS_CU(launch_width_lists(b.qoff, nb, w.wlist, w.wlist + 2 * nb, st));
        BVSS_CU(launch_refine_mma(qv, b.qoff, nb, 32, vecb, ix->vscale8, vnb, el,
                                  ix->set_off, d, w.cand, w.thr, C, w.pair, ix->err, st,
                                  kn.cand_cta, kn.stages, w.wlist, w.wlist + 2 * nb, w.qop,
                                  w.qop_n, w.qop_sc, kn.qs));
        BVSS_CU(launch_refine_mma(qv, b.qoff, nb, b.max_mq, vecb, ix->vscale8, vnb, el,
                                  ix->set_off, d, w.cand, w.thr, C, w.pair, ix->err, st,
                                  kn.cand_cta, kn.stages, w.wlist + nb, w.wlist + 2 * nb + 1,
                                  w.qop, w.qop_n, w.qop_sc, kn.qs));
        n += 2;
    } else if (mma)
        BVSS_CU(launch_refine_mma(qv, b.qoff, nb, b.max_mq, vecb, ix->vscale8, vnb, el,
                                  ix->set_off, d, w.cand, w.thr, C, w.pair, ix->err, st,
                                  kn.cand_cta, kn.stages, nullptr, nullptr, w.qop, w.qop_n,
                                  w.qop_sc, kn.qs));
    else if (refine_tma_supported(d, b.max_mq))
        BVSS_CU(launch_refine_tma(qv, b.qoff, nb, b.max_mq, ix->vec, ix->vnorm, ix->set_off, d,
                                  w.cand, w.thr, C, w.cand_dist, ix->err, st));
    else
        BVSS_CU(launch_refine(qv, b.qoff, nb, b.max_mq, ix->vec, ix->vnorm, ix->set_off, d,
                              w.cand, w.thr, C, w.cand_dist, st));
    ++n;
    if (ev) BVSS_CU(cudaEventRecord(ev[5], st));
    // (the re-score stage is empty: the boundary stage reads the tensor-core refine's
    // values from its pair records)
    if (ev) BVSS_CU(cudaEventRecord(ev[6], st));
    // line 23: the k smallest (distance, id), decided exactly around the k-th
    BVSS_CU(launch_band_topk(qv, b.qoff, nb, b.max_mq, d, form, ix->rstat, ix->vec, ix->set_off,
                             w.cand, w.thr, C, k, w.pair, w.cand_dist, b.ids, b.dist, ix->err,
                             (s->flags & BVSS_SEARCH_FP8_EXACT) != 0, st));
    n += kBandKernels;
    *launches += n;
    return BVSS_OK;
}

int query_impl(bvss_index *ix, const float *q_vectors, const int64_t *q_offsets,
               int64_t n_queries, const bvss_search *s, int64_t *out_ids, float *out_dist,
               const bvss_trace *tr, void *stream) {
    if (!ix) return fail(BVSS_EINVAL, "index is NULL");
    int rc = check_search(ix, s);
    if (rc) return rc;
    const int L = ix->p.wta_l, d = ix->p.d, W = ix->W;
    const bool alg2 = (s->flags & BVSS_SEARCH_ALG2) != 0;
    if (n_queries < 0) return fail(BVSS_EINVAL, "n_queries < 0");
    if (n_queries == 0) return BVSS_OK;
    if (!q_vectors || !out_ids || !out_dist)
        return fail(BVSS_EINVAL, "query vectors or outputs are NULL");
    // Alg. 2's scoring kernel holds one bit per query vector in a 32-bit word
    rc = check_offsets(q_offsets, n_queries, alg2 ? 32 : BVSS_MAX_QSET, "query");
    if (rc) return rc;
    rc = check_device(ix);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const bool qv_dev = is_device_ptr(q_vectors);
    const bool ids_dev = is_device_ptr(out_ids), dist_dev = is_device_ptr(out_dist);
    if (tr) {
        const void *ptrs[] = {tr->qpos, tr->cq, tr->sq, tr->plist, tr->h, tr->cand, tr->n_cand,
                              tr->cand_dist};
        for (const void *p : ptrs)
            if (p && !is_device_ptr(p)) return fail(BVSS_EINVAL, "trace pointers must be device memory");
    }
    const int k = s->k, C = s->C, A = s->A, M = s->M;
    const int64_t QB = batch_cap(ix);
    int64_t max_vq = 0;
    for (int64_t b0 = 0; b0 < n_queries; b0 += QB) {
        const int64_t b1 = b0 + QB < n_queries ? b0 + QB : n_queries;
        const int64_t nv = q_offsets[b1] - q_offsets[b0];
        if (nv > max_vq) max_vq = nv;
    }
    const int64_t nq_cap = n_queries < QB ? n_queries : QB;
    rc = ensure_workspace(ix, nq_cap, max_vq, C, A, k, !qv_dev, !(ids_dev && dist_dev));
    if (rc) return rc;
    Workspace &w = ix->ws;

    const uint32_t *plane = nullptr;
    if (M >= 1 && M <= 255) {
        rc = get_plane(ix, M, st, &plane);
        if (rc) return rc;
    }
    const int64_t hs = h_stride(ix);

    for (int64_t b0 = 0; b0 < n_queries; b0 += QB) {
        const int64_t b1 = b0 + QB < n_queries ? b0 + QB : n_queries;
        const int nb = (int)(b1 - b0);
        const int64_t v0 = q_offsets[b0], v1 = q_offsets[b1], nv = v1 - v0;
        int max_mq = 0;
        // batch-relative offsets through a pinned ring slot
        const int slot = ix->off_next;
        ix->off_next = (ix->off_next + 1) % kOffRing;
        BVSS_CU(cudaEventSynchronize(ix->off_event[slot]));
        int64_t *oh = ix->off_host[slot];
        for (int j = 0; j <= nb; ++j) {
            oh[j] = q_offsets[b0 + j] - v0;
            if (j > 0 && oh[j] - oh[j - 1] > max_mq) max_mq = (int)(oh[j] - oh[j - 1]);
        }
        BVSS_CU(cudaMemcpyAsync(w.qoff, oh, sizeof(int64_t) * (size_t)(nb + 1),
                                cudaMemcpyHostToDevice, st));
        BVSS_CU(cudaEventRecord(ix->off_event[slot], st));
        cudaEvent_t *ev = ix->prof_on ? prof_reserve(ix) : nullptr;
        const float *qv = q_vectors + v0 * d;
        if (!qv_dev) {
            BVSS_CU(cudaMemcpyAsync(w.qvec, qv, sizeof(float) * (size_t)nv * d,
                                    cudaMemcpyHostToDevice, st));
            qv = w.qvec;
        }
        Batch b;
        b.qv = qv;
        b.qoff = w.qoff;
        b.nb = nb;
        b.max_mq = max_mq;
        b.enc_n = nv;
        b.plane = plane;
        b.ids = ids_dev ? out_ids + b0 * k : w.out_ids;
        b.dist = dist_dev ? out_dist + b0 * k : w.out_dist;
        b.cq_trace = tr && tr->cq ? tr->cq + b0 * ix->p.m : nullptr;
        b.ev = ev;
        int64_t launches = 0;
        rc = enqueue_batch(ix, w, s, Knobs(), b, &launches, st);
        if (rc) return rc;
        if (ev) ix->prof_launches += launches;
        if (!ids_dev)
            BVSS_CU(cudaMemcpyAsync(out_ids + b0 * k, b.ids, sizeof(int64_t) * (size_t)nb * k,
                                    cudaMemcpyDeviceToHost, st));
        if (!dist_dev)
            BVSS_CU(cudaMemcpyAsync(out_dist + b0 * k, b.dist, sizeof(float) * (size_t)nb * k,
                                    cudaMemcpyDeviceToHost, st));
        if (ev) BVSS_CU(cudaEventRecord(ev[7], st));
        if (tr) {
            const cudaMemcpyKind dd = cudaMemcpyDeviceToDevice;
            if (tr->qpos)
                BVSS_CU(cudaMemcpyAsync(tr->qpos + v0 * L, w.qpos, sizeof(uint16_t) * nv * L, dd, st));
            if (tr->sq)
                BVSS_CU(cudaMemcpyAsync(tr->sq + b0 * W, w.sq, sizeof(uint32_t) * nb * W, dd, st));
            if (tr->plist)
                BVSS_CU(cudaMemcpyAsync(tr->plist + b0 * A, w.plist, sizeof(uint16_t) * nb * A, dd, st));
            if (tr->h)
                BVSS_CU(cudaMemcpy2DAsync(tr->h + b0 * ix->n_sets, sizeof(uint16_t) * ix->n_sets,
                                          w.h, sizeof(uint16_t) * hs,
                                          sizeof(uint16_t) * ix->n_sets, nb, dd, st));
            if (tr->cand)
                BVSS_CU(cudaMemcpyAsync(tr->cand + b0 * C, w.cand, sizeof(int32_t) * nb * C, dd, st));
            if (tr->n_cand)
                BVSS_CU(cudaMemcpy2DAsync(tr->n_cand + b0, sizeof(int32_t), w.thr + 3,
                                          4 * sizeof(int32_t), sizeof(int32_t), nb, dd, st));
            if (tr->cand_dist)
                BVSS_CU(cudaMemcpyAsync(tr->cand_dist + b0 * C, w.cand_dist,
                                        sizeof(float) * nb * C, dd, st));
        }
    }
    if (!ids_dev || !dist_dev) return sync_and_check(ix, st);
    return BVSS_OK;
}

// The query offsets of a plan live on the device, so they are checked there: offsets
// from 0, every set 1..max_qset vectors, at most max_v vectors in all.  Valid offsets
// are copied into the plan's array; otherwise status bit kErrPlanInput is set and the
// array is filled with one-vector sets (j), which keeps every kernel of the pass inside
// the plan's buffers (n_q <= max_v).
__global__ void __launch_bounds__(1024)
k_plan_offsets(const int64_t *__restrict__ in, int64_t n_q, int max_qset, int64_t max_v,
               int64_t *__restrict__ out, int *__restrict__ err) {
    bool bad = false;
    for (int64_t j = threadIdx.x; j < n_q; j += blockDim.x) {
        const int64_t sz = in[j + 1] - in[j];
        bad |= sz < 1 || sz > max_qset;
    }
    if (threadIdx.x == 0) bad |= in[0] != 0 || in[n_q] > max_v;
    bad = __syncthreads_or(bad);
    for (int64_t j = threadIdx.x; j <= n_q; j += blockDim.x) out[j] = bad ? j : in[j];
    if (bad && threadIdx.x == 0) atomicOr(err, kErrPlanInput);
}

}  // namespace

// A fixed-shape query pass bound to the caller's device buffers and captured into one
// CUDA graph: the offsets check, the FlyHash of every query vector, then Alg. 6 (or
// Alg. 2) batch by batch, with its own workspace so the graph's pointers stay valid.
struct bvss_plan {
    bvss_index *ix = nullptr;
    bvss_search s{};
    int64_t n_q = 0, max_v = 0;
    int max_qset = 0;
    const float *qv = nullptr;
    const int64_t *qoff_in = nullptr;
    int64_t *ids = nullptr;
    float *dist = nullptr;
    Workspace w;
    int64_t *qoff = nullptr;   // checked offsets, n_q + 1
    const uint32_t *plane = nullptr;
    Knobs kn;
    cudaStream_t cs = nullptr;   // capture and tuning stream
    cudaGraphExec_t exec = nullptr;
    int64_t launches = 0;        // kernels per pass
};

namespace {

void free_plan(bvss_plan *p) {
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->cs) cudaStreamDestroy(p->cs);
    free_workspace(p->w);
    dfree(p->qoff);
    delete p;
}

int plan_enqueue(bvss_plan *p, cudaStream_t st, int64_t *launches) {
    bvss_index *ix = p->ix;
    const int k = p->s.k;
    k_plan_offsets<<<1, 1024, 0, st>>>(p->qoff_in, p->n_q, p->max_qset, p->max_v, p->qoff,
                                       ix->err);
    BVSS_CU(cudaGetLastError());
    *launches = 1;
    const int rc0 = encode_vectors(ix, p->qv, p->max_v, p->w.qpos, nullptr, p->w.enc_x,
                                   p->w.enc_act, st, p->qoff + p->n_q, launches);
    if (rc0) return rc0;
    // the internal batch: the tuner's choice, else the default cap, within the workspace
    int64_t QB = p->kn.batch > 0 ? p->kn.batch : batch_cap(ix);
    if (QB > p->w.cap_q) QB = p->w.cap_q;
    for (int64_t b0 = 0; b0 < p->n_q; b0 += QB) {
        Batch b;
        b.qv = p->qv;
        b.qoff = p->qoff + b0;
        b.nb = (int)(b0 + QB < p->n_q ? QB : p->n_q - b0);
        b.max_mq = p->max_qset;
        b.plane = p->plane;
        b.ids = p->ids + b0 * k;
        b.dist = p->dist + b0 * k;
        const int rc = enqueue_batch(ix, p->w, &p->s, p->kn, b, launches, st);
        if (rc) return rc;
    }
    return BVSS_OK;
}

// (re)capture the pass with the current knobs into the plan's graph
int plan_capture(bvss_plan *p) {
    BVSS_CU(cudaStreamBeginCapture(p->cs, cudaStreamCaptureModeThreadLocal));
    int64_t launches = 0;
    const int rc = plan_enqueue(p, p->cs, &launches);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(p->cs, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    BVSS_CU(e);
    cudaGraphExec_t ex = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    BVSS_CU(ei);
    if (p->exec) cudaGraphExecDestroy(p->exec);
    p->exec = ex;
    p->launches = launches;
    return BVSS_OK;
}

// mean time of one graph launch (ms) with the given knobs, after one warm-up launch
int plan_time(bvss_plan *p, const Knobs &kn, int reps, float *ms) {
    p->kn = kn;
    int rc = plan_capture(p);
    if (rc) return rc;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    BVSS_CU(cudaEventCreate(&e0));
    cudaError_t e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaGraphLaunch(p->exec, p->cs);
    if (e == cudaSuccess) e = cudaEventRecord(e0, p->cs);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = cudaGraphLaunch(p->exec, p->cs);
    if (e == cudaSuccess) e = cudaEventRecord(e1, p->cs);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    BVSS_CU(e);
    *ms /= (float)reps;
    return sync_and_check(p->ix, p->cs);
}

}  // namespace

namespace bvss {

int record_error(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

}  // namespace bvss

namespace {

// bvss_build (proj: the sparse binary FlyHash projection) and bvss_build_dense (w: the
// learned dense layer, m x d FP32, host or device, rounded to BF16)
int build_impl(const float *vectors, const int64_t *set_offsets, int64_t n_sets,
               const uint16_t *proj, const float *w, const bvss_params *params, void *stream,
               bvss_index **out) {
    if (!out) return fail(BVSS_EINVAL, "out is NULL");
    *out = nullptr;
    if (!params) return fail(BVSS_EINVAL, "params is NULL");
    bvss_params p = *params;
    if (w) p.fanin = 1;   // not used by the dense layer; checked as the smallest fan-in
    int rc = check_params(&p);
    if (rc) return rc;
    if (w && (p.d % 64 != 0 || p.m % 128 != 0))
        return fail(BVSS_EINVAL, "the dense projection needs d %% 64 == 0 and m %% 128 == 0 "
                                 "(d = %d, m = %d)", p.d, p.m);
    if (w) p.fanin = 0;
    if (n_sets < 1 || n_sets > 0x7fffffffLL)
        return fail(BVSS_EINVAL, "n_sets = %lld: need 1 <= n_sets < 2^31", (long long)n_sets);
    if (!vectors || (!proj && !w)) return fail(BVSS_EINVAL, "vectors or projection is NULL");
    rc = check_offsets(set_offsets, n_sets, 0, "database");
    if (rc) return rc;
    for (int j = 0; j < p.m && proj; ++j) {
        const uint16_t *row = proj + (int64_t)j * p.fanin;
        for (int t = 0; t < p.fanin; ++t) {
            if (row[t] >= p.d) return fail(BVSS_EINVAL, "proj[%d][%d] = %d >= d", j, t, row[t]);
            if (t > 0 && row[t] <= row[t - 1])
                return fail(BVSS_EINVAL, "proj row %d is not strictly ascending", j);
        }
    }
    bvss_index *ix = new (std::nothrow) bvss_index();
    if (!ix) return fail(BVSS_ENOMEM, "host allocation failed");
    rc = [&]() -> int {
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        BVSS_CU(cudaGetDevice(&ix->device));
        ix->p = p;
        ix->n_sets = n_sets;
        ix->n_vec = set_offsets[n_sets];
        ix->W = p.m / 32;
        ix->NW = (n_sets + 31) / 32;
        const int64_t nv = ix->n_vec;
        BVSS_CU(dalloc(&ix->vec, (size_t)nv * p.d));
        BVSS_CU(dalloc(&ix->vnorm, (size_t)nv));
        BVSS_CU(dalloc(&ix->set_off, (size_t)n_sets + 1));
        if (proj) BVSS_CU(dalloc(&ix->proj, (size_t)p.m * p.fanin));
        if (w) BVSS_CU(dalloc(&ix->wproj16, (size_t)p.m * p.d));
        BVSS_CU(dalloc(&ix->codes, (size_t)nv * p.wta_l));
        BVSS_CU(dalloc(&ix->sketch, (size_t)n_sets * ix->W));
        BVSS_CU(dalloc(&ix->spop, (size_t)n_sets));
        BVSS_CU(dalloc(&ix->count, (size_t)n_sets * p.m));
        BVSS_CU(dalloc(&ix->flag, 1));
        BVSS_CU(dalloc(&ix->err, 1));
        BVSS_CU(cudaMemsetAsync(ix->err, 0, sizeof(int), st));
        for (int64_t i = 0; i < n_sets; ++i)
            if (set_offsets[i + 1] - set_offsets[i] > ix->max_set)
                ix->max_set = set_offsets[i + 1] - set_offsets[i];
        const cudaMemcpyKind kind =
            is_device_ptr(vectors) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        BVSS_CU(cudaMemcpyAsync(ix->vec, vectors, sizeof(float) * (size_t)nv * p.d, kind, st));
        BVSS_CU(cudaMemcpyAsync(ix->set_off, set_offsets, sizeof(int64_t) * (size_t)(n_sets + 1),
                                cudaMemcpyHostToDevice, st));
        if (proj)
            BVSS_CU(cudaMemcpyAsync(ix->proj, proj, sizeof(uint16_t) * (size_t)p.m * p.fanin,
                                    cudaMemcpyHostToDevice, st));
        if (w) {
            // the layer's weights in BF16 (round to nearest even), from host or device
            float *wd = nullptr;
            const float *wsrc = w;
            if (!is_device_ptr(w)) {
                BVSS_CU(dalloc(&wd, (size_t)p.m * p.d));
                BVSS_CU(cudaMemcpyAsync(wd, w, sizeof(float) * (size_t)p.m * p.d,
                                        cudaMemcpyHostToDevice, st));
                wsrc = wd;
            }
            BVSS_CU(launch_rows_bf16(wsrc, p.d, nullptr, p.m, ix->wproj16, st));
            if (wd) {
                BVSS_CU(cudaStreamSynchronize(st));
                dfree(wd);
            }
        }
        BVSS_CU(cudaMemsetAsync(ix->flag, 0, sizeof(int), st));
        BVSS_CU(launch_check_finite(ix->vec, nv * p.d, ix->flag, st));
        int bad = 0;
        BVSS_CU(cudaMemcpyAsync(&bad, ix->flag, sizeof(int), cudaMemcpyDeviceToHost, st));
        BVSS_CU(cudaStreamSynchronize(st));
        if (bad) return fail(BVSS_EINVAL, "database vectors hold non-finite values");
        // Alg. 1 over the database, then Alg. 3 / Alg. 5 from the same codes
        BVSS_CU(launch_norms(ix->vec, nv, p.d, ix->vnorm, st));
        if (p.flags & BVSS_BUILD_BF16) {
            BVSS_CU(dalloc(&ix->vec16, (size_t)nv * p.d));
            BVSS_CU(dalloc(&ix->vnorm16, (size_t)nv));
            BVSS_CU(launch_to_bf16(ix->vec, nv, p.d, ix->vec16, ix->vnorm16, st));
        }
        if (p.flags & BVSS_BUILD_FP8) {
            BVSS_CU(dalloc(&ix->vec8, (size_t)nv * p.d));
            BVSS_CU(dalloc(&ix->vscale8, (size_t)nv));
            BVSS_CU(dalloc(&ix->vnorm8, (size_t)nv));
            BVSS_CU(launch_to_fp8(ix->vec, nv, p.d, ix->vec8, ix->vscale8, ix->vnorm8, st));
        }
        BVSS_CU(dalloc(&ix->rstat, kRoundStats));
        BVSS_CU(launch_round_stats(ix->vec, nv, p.d, ix->vec16, ix->vec8, ix->vscale8, ix->rstat,
                                   st));
        {
            // Alg. 1: codes of every database vector (the dense layer in blocks)
            __nv_bfloat16 *xb = nullptr;
            float *act = nullptr;
            if (w) {
                BVSS_CU(dalloc(&xb, (size_t)kEncChunk * p.d));
                BVSS_CU(dalloc(&act, (size_t)kEncChunk * p.m));
            }
            const int r2 = encode_vectors(ix, ix->vec, nv, ix->codes, nullptr, xb, act, st,
                                          nullptr, nullptr);
            if (w) {
                cudaStreamSynchronize(st);
                dfree(xb);
                dfree(act);
            }
            if (r2) return r2;
        }
        BVSS_CU(launch_build_filters(ix->codes, ix->set_off, n_sets, p.m, p.wta_l, ix->sketch,
                                     ix->count, st));
        BVSS_CU(launch_sketch_pop(ix->sketch, n_sets, ix->W, ix->spop, st));
        const uint32_t *pl = nullptr;
        int r = get_plane(ix, 1, st, &pl);
        if (r) return r;
        BVSS_CU(cudaStreamSynchronize(st));
        return BVSS_OK;
    }();
    if (rc) {
        cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
        free_index(ix);
        return rc;
    }
    *out = ix;
    return BVSS_OK;
}

}  // namespace

extern "C" {

int bvss_build(const float *vectors, const int64_t *set_offsets, int64_t n_sets,
               const uint16_t *proj, const bvss_params *params, void *stream,
               bvss_index **out) {
    if (!proj) return fail(BVSS_EINVAL, "proj is NULL");
    return build_impl(vectors, set_offsets, n_sets, proj, nullptr, params, stream, out);
}

int bvss_build_dense(const float *vectors, const int64_t *set_offsets, int64_t n_sets,
                     const float *w, const bvss_params *params, void *stream,
                     bvss_index **out) {
    if (!w) return fail(BVSS_EINVAL, "w is NULL");
    return build_impl(vectors, set_offsets, n_sets, nullptr, w, params, stream, out);
}

int bvss_query(const bvss_index *ix, const float *q_vectors, const int64_t *q_offsets,
               int64_t n_queries, const bvss_search *s, int64_t *out_ids, float *out_dist,
               void *stream) {
    return query_impl(const_cast<bvss_index *>(ix), q_vectors, q_offsets, n_queries, s, out_ids,
                      out_dist, nullptr, stream);
}

int bvss_query_trace(const bvss_index *ix, const float *q_vectors, const int64_t *q_offsets,
                     int64_t n_queries, const bvss_search *s, int64_t *out_ids, float *out_dist,
                     const bvss_trace *tr, void *stream) {
    return query_impl(const_cast<bvss_index *>(ix), q_vectors, q_offsets, n_queries, s, out_ids,
                      out_dist, tr, stream);
}

int bvss_encode(const bvss_index *ix, const float *x, int64_t n, uint16_t *pos, uint32_t *mask,
                void *stream) {
    if (!ix) return fail(BVSS_EINVAL, "index is NULL");
    if (n < 0) return fail(BVSS_EINVAL, "n < 0");
    if (n == 0) return BVSS_OK;
    if (!x || !is_device_ptr(x)) return fail(BVSS_EINVAL, "x must be device memory");
    if ((pos && !is_device_ptr(pos)) || (mask && !is_device_ptr(mask)))
        return fail(BVSS_EINVAL, "pos / mask must be device memory");
    int rc = check_device(ix);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    __nv_bfloat16 *xb = nullptr;
    float *act = nullptr;
    if (ix->wproj16) {   // a block of scratch for the dense layer
        BVSS_CU(dalloc(&xb, (size_t)kEncChunk * ix->p.d));
        rc = dalloc(&act, (size_t)kEncChunk * ix->p.m) == cudaSuccess
                 ? BVSS_OK : fail(BVSS_ENOMEM, "bvss_encode: scratch allocation failed");
        if (rc) {
            dfree(xb);
            return rc;
        }
    }
    rc = encode_vectors(ix, x, n, pos, mask, xb, act, st, nullptr, nullptr);
    if (ix->wproj16) {
        cudaStreamSynchronize(st);
        dfree(xb);
        dfree(act);
    }
    return rc;
}

int bvss_nearest_rows(const bvss_index *ix, const float *q_vectors, const int64_t *q_offsets,
                      int64_t n_queries, const int64_t *sets, int32_t k, int64_t *rows,
                      void *stream) {
    if (!ix) return fail(BVSS_EINVAL, "index is NULL");
    if (n_queries < 0 || n_queries > 0x7fffffffLL || k < 1)
        return fail(BVSS_EINVAL, "bvss_nearest_rows: need 0 <= n_queries < 2^31 and k >= 1");
    if (n_queries == 0) return BVSS_OK;
    if (!q_vectors || !sets || !rows || !is_device_ptr(q_vectors) || !is_device_ptr(sets) ||
        !is_device_ptr(rows))
        return fail(BVSS_EINVAL, "bvss_nearest_rows: vectors, sets and rows must be device "
                                 "memory");
    int rc = check_offsets(q_offsets, n_queries, BVSS_MAX_QSET, "query");
    if (rc) return rc;
    rc = check_device(ix);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int64_t *qoff = nullptr;
    BVSS_CU(dalloc(&qoff, (size_t)n_queries + 1));
    cudaError_t e = cudaMemcpyAsync(qoff, q_offsets, sizeof(int64_t) * (size_t)(n_queries + 1),
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = launch_nearest(q_vectors, qoff, (int)n_queries, ix->p.d, ix->vec, ix->set_off,
                           ix->n_sets, sets, k, rows, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dfree(qoff);
    if (e != cudaSuccess) return fail(BVSS_ECUDA, "bvss_nearest_rows: %s", cudaGetErrorString(e));
    return BVSS_OK;
}

int bvss_index_rows_bf16(const bvss_index *ix, const int64_t *rows, int64_t n, void *out,
                         void *stream) {
    if (!ix) return fail(BVSS_EINVAL, "index is NULL");
    if (n < 0) return fail(BVSS_EINVAL, "n < 0");
    if (n == 0) return BVSS_OK;
    if (!rows || !out || !is_device_ptr(rows) || !is_device_ptr(out))
        return fail(BVSS_EINVAL, "bvss_index_rows_bf16: rows and out must be device memory");
    int rc = check_device(ix);
    if (rc) return rc;
    BVSS_CU(launch_rows_bf16(ix->vec, ix->p.d, rows, n, static_cast<__nv_bfloat16 *>(out),
                             reinterpret_cast<cudaStream_t>(stream), ix->n_vec));
    return BVSS_OK;
}

int bvss_index_info(const bvss_index *ix, bvss_params *params, int64_t *n_sets,
                    int64_t *n_vectors) {
    if (!ix) return fail(BVSS_EINVAL, "index is NULL");
    if (params) *params = ix->p;
    if (n_sets) *n_sets = ix->n_sets;
    if (n_vectors) *n_vectors = ix->n_vec;
    return BVSS_OK;
}

int bvss_get_codes(const bvss_index *ix, int64_t first, int64_t n, uint16_t *pos, void *stream) {
    if (!ix) return fail(BVSS_EINVAL, "index is NULL");
    if (first < 0 || n < 0 || first + n > ix->n_vec)
        return fail(BVSS_EINVAL, "vector range out of bounds");
    if (n == 0) return BVSS_OK;
    if (!pos || !is_device_ptr(pos)) return fail(BVSS_EINVAL, "pos must be device memory");
    BVSS_CU(cudaMemcpyAsync(pos, ix->codes + first * ix->p.wta_l,
                            sizeof(uint16_t) * (size_t)n * ix->p.wta_l, cudaMemcpyDeviceToDevice,
                            reinterpret_cast<cudaStream_t>(stream)));
    return BVSS_OK;
}

int bvss_get_sketches(const bvss_index *ix, const int64_t *ids, int64_t n, uint32_t *out,
                      void *stream) {
    if (!ix) return fail(BVSS_EINVAL, "index is NULL");
    if (n < 0) return fail(BVSS_EINVAL, "n < 0");
    if (n == 0) return BVSS_OK;
    if (!ids || !out || !is_device_ptr(ids) || !is_device_ptr(out))
        return fail(BVSS_EINVAL, "ids and out must be device memory");
    BVSS_CU(launch_gather_sketches(ix->sketch, ix->W, ix->n_sets, ids, n, out,
                                   reinterpret_cast<cudaStream_t>(stream)));
    return BVSS_OK;
}

int bvss_get_counts(const bvss_index *ix, const int64_t *ids, int64_t n, uint8_t *out,
                    void *stream) {
    if (!ix) return fail(BVSS_EINVAL, "index is NULL");
    if (n < 0) return fail(BVSS_EINVAL, "n < 0");
    if (n == 0) return BVSS_OK;
    if (!ids || !out || !is_device_ptr(ids) || !is_device_ptr(out))
        return fail(BVSS_EINVAL, "ids and out must be device memory");
    BVSS_CU(launch_gather_counts(ix->count, ix->p.m, ix->n_sets, ids, n, out,
                                 reinterpret_cast<cudaStream_t>(stream)));
    return BVSS_OK;
}

int bvss_sync(bvss_index *ix, void *stream) {
    if (!ix) return fail(BVSS_EINVAL, "index is NULL");
    return sync_and_check(ix, reinterpret_cast<cudaStream_t>(stream));
}

int bvss_selftest_wait_timeout(int64_t limit_ns) {
    if (limit_ns < 0 || limit_ns > 1000000000LL)
        return fail(BVSS_EINVAL, "limit_ns must lie in [0, 1e9]");
    int *err = nullptr;
    BVSS_CU(dalloc(&err, 1));
    int e = 0;
    cudaError_t ce = cudaMemset(err, 0, sizeof(int));
    if (ce == cudaSuccess) ce = launch_wait_selftest(err, (uint64_t)limit_ns, 0);
    if (ce == cudaSuccess) ce = cudaDeviceSynchronize();
    if (ce == cudaSuccess) ce = cudaMemcpy(&e, err, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(err);
    if (ce != cudaSuccess) return fail(BVSS_ECUDA, "selftest: %s", cudaGetErrorString(ce));
    if (e) return fail(BVSS_ETIMEOUT, "selftest: the bounded wait gave up as intended");
    return BVSS_OK;
}

int bvss_profile_enable(bvss_index *ix, int on) {
    if (!ix) return fail(BVSS_EINVAL, "index is NULL");
    ix->prof_on = on != 0;
    return BVSS_OK;
}

int bvss_profile_read(bvss_index *ix, double *stage_ms, int64_t *n_batches, int64_t *n_launches,
                      int reset) {
    if (!ix) return fail(BVSS_EINVAL, "index is NULL");
    for (int64_t b = 0; b + kProfEvents <= ix->prof_used; b += kProfEvents) {
        BVSS_CU(cudaEventSynchronize(ix->prof_ev[b + kProfEvents - 1]));
        for (int sidx = 0; sidx < BVSS_N_STAGES; ++sidx) {
            float ms = 0.0f;
            BVSS_CU(cudaEventElapsedTime(&ms, ix->prof_ev[b + sidx], ix->prof_ev[b + sidx + 1]));
            ix->prof_ms[sidx] += ms;
        }
        ix->prof_batches += 1;
    }
    ix->prof_used = 0;
    if (stage_ms)
        for (int sidx = 0; sidx < BVSS_N_STAGES; ++sidx) stage_ms[sidx] = ix->prof_ms[sidx];
    if (n_batches) *n_batches = ix->prof_batches;
    if (n_launches) *n_launches = ix->prof_launches;
    if (reset) {
        for (int sidx = 0; sidx < BVSS_N_STAGES; ++sidx) ix->prof_ms[sidx] = 0.0;
        ix->prof_batches = 0;
        ix->prof_launches = 0;
    }
    return BVSS_OK;
}

void bvss_free(bvss_index *ix) { free_index(ix); }

const char *bvss_last_error(void) { return g_err; }

int bvss_plan_create(bvss_index *ix, const bvss_search *s, int64_t n_queries,
                     int64_t max_vectors, int32_t max_qset, const float *q_vectors,
                     const int64_t *q_offsets, int64_t *out_ids, float *out_dist, void *stream,
                     bvss_plan **out) {
    if (!out) return fail(BVSS_EINVAL, "out is NULL");
    *out = nullptr;
    if (!ix) return fail(BVSS_EINVAL, "index is NULL");
    int rc = check_search(ix, s);
    if (rc) return rc;
    const bool alg2 = (s->flags & BVSS_SEARCH_ALG2) != 0;
    const int qmax = alg2 ? 32 : BVSS_MAX_QSET;
    if (n_queries < 1) return fail(BVSS_EINVAL, "n_queries = %lld: need >= 1", (long long)n_queries);
    if (max_qset < 1 || max_qset > qmax)
        return fail(BVSS_EINVAL, "max_qset = %d: need 1 <= max_qset <= %d", max_qset, qmax);
    if (max_vectors < n_queries || max_vectors > n_queries * (int64_t)max_qset)
        return fail(BVSS_EINVAL, "max_vectors = %lld: need n_queries <= max_vectors <= "
                                 "n_queries * max_qset", (long long)max_vectors);
    if (!q_vectors || !q_offsets || !out_ids || !out_dist)
        return fail(BVSS_EINVAL, "plan buffers are NULL");
    if (!is_device_ptr(q_vectors) || !is_device_ptr(q_offsets) || !is_device_ptr(out_ids) ||
        !is_device_ptr(out_dist))
        return fail(BVSS_EINVAL, "plan buffers must be device memory");
    rc = check_device(ix);
    if (rc) return rc;
    bvss_plan *p = new (std::nothrow) bvss_plan();
    if (!p) return fail(BVSS_ENOMEM, "plan allocation failed");
    p->ix = ix;
    p->s = *s;
    p->n_q = n_queries;
    p->max_v = max_vectors;
    p->max_qset = max_qset;
    p->qv = q_vectors;
    p->qoff_in = q_offsets;
    p->ids = out_ids;
    p->dist = out_dist;
    const int64_t QB = plan_batch_cap(ix);
    rc = alloc_workspace(ix, p->w, n_queries < QB ? n_queries : QB, max_vectors, s->C, s->A,
                         s->k, false, false);
    if (!rc && dalloc(&p->qoff, n_queries + 1) != cudaSuccess)
        rc = fail(BVSS_ENOMEM, "plan offsets allocation failed");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (!rc && s->M >= 1 && s->M <= 255) rc = get_plane(ix, s->M, st, &p->plane);
    if (!rc && cudaStreamSynchronize(st) != cudaSuccess)
        rc = fail(BVSS_ECUDA, "stream synchronisation failed");
    if (!rc && cudaStreamCreateWithFlags(&p->cs, cudaStreamNonBlocking) != cudaSuccess)
        rc = fail(BVSS_ECUDA, "stream creation failed");
    if (!rc) rc = plan_capture(p);
    if (rc) {
        free_plan(p);
        return rc;
    }
    ++ix->n_plans;
    *out = p;
    return BVSS_OK;
}

int bvss_plan_launch(bvss_plan *p, void *stream) {
    if (!p || !p->exec) return fail(BVSS_EINVAL, "plan is NULL");
    BVSS_CU(cudaGraphLaunch(p->exec, reinterpret_cast<cudaStream_t>(stream)));
    return BVSS_OK;
}

int bvss_plan_tune(bvss_plan *p, int32_t reps, void *stream, float *best_ms) {
    if (!p || !p->exec) return fail(BVSS_EINVAL, "plan is NULL");
    if (reps < 1) return fail(BVSS_EINVAL, "reps = %d: need >= 1", reps);
    BVSS_CU(cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)));
    const int d = p->ix->p.d;
    const bool alg2 = (p->s.flags & BVSS_SEARCH_ALG2) != 0;
    const int form = refine_form(p->ix, p->s.flags, p->max_qset);
    const bool mma = form > 0;
    const Elem el = static_cast<Elem>(mma ? form : 1);
    Knobs best = p->kn;
    float best_t = 0.0f;
    int rc = plan_time(p, best, reps, &best_t);
    if (rc) return rc;
    // one knob at a time, each over its values, keeping the fastest pass
    auto sweep = [&](int Knobs::*field, const int *vals, int nv) -> int {
        for (int i = 0; i < nv; ++i) {
            Knobs kn = best;
            if (kn.*field == vals[i]) continue;
            kn.*field = vals[i];
            float t = 0.0f;
            const int r = plan_time(p, kn, reps, &t);
            if (r) return r;
            if (t < best_t) {
                best_t = t;
                best = kn;
            }
        }
        return BVSS_OK;
    };
    if (!alg2) {
        const int scans[] = {1, 2, 3};
        rc = sweep(&Knobs::scan, scans, 3);
    }
    if (!rc && mma) {
        const int ctas[] = {128, 256, 512};
        rc = sweep(&Knobs::cand_cta, ctas, 3);
    }
    if (!rc && mma && p->w.qop &&
        refine_mma_streams(d, p->max_qset, el, 1) != refine_mma_streams(d, p->max_qset, el, 2)) {
        // the widest instance's query operand: held in shared memory or streamed
        const int modes[] = {1, 2};
        rc = sweep(&Knobs::qs, modes, 2);
    }
    if (!rc && mma) {
        const int ns = refine_mma_stages(d, p->max_qset, el, p->w.qop ? best.qs : 1);
        int rings[4], nr = 0;
        for (int r = ns; r >= 4 && nr < 3; r -= 2) rings[nr++] = r;
        rc = sweep(&Knobs::stages, rings, nr);
    }
    if (!rc && mma && p->max_qset > 32) {
        const int buckets[] = {0, 2};
        rc = sweep(&Knobs::bucket, buckets, 2);
    }
    if (!rc && p->w.cap_q > batch_cap(p->ix)) {
        int bs[3], nb = 0;
        for (int64_t b = batch_cap(p->ix); b <= p->w.cap_q && nb < 3; b *= 2) bs[nb++] = (int)b;
        if (nb < 3 && bs[nb - 1] < p->w.cap_q) bs[nb++] = (int)p->w.cap_q;
        rc = sweep(&Knobs::batch, bs, nb);
    }
    p->kn = best;
    const int rc2 = plan_capture(p);
    if (rc) return rc;
    if (rc2) return rc2;
    if (best_ms) *best_ms = best_t;
    return BVSS_OK;
}

int bvss_plan_info(const bvss_plan *p, int32_t *knobs, int64_t *launches) {
    if (!p) return fail(BVSS_EINVAL, "plan is NULL");
    const int d = p->ix->p.d;
    const bool alg2 = (p->s.flags & BVSS_SEARCH_ALG2) != 0;
    const int form = refine_form(p->ix, p->s.flags, p->max_qset);
    const bool mma = form > 0;
    if (knobs) {
        knobs[0] = alg2 ? 0
                   : p->kn.scan ? p->kn.scan
                   : (p->s.flags & BVSS_SEARCH_POPC_SCAN) ? 2
                   : (p->s.flags & BVSS_SEARCH_SCAN_SETS_TMEM) ? 3 : 1;
        knobs[1] = mma ? (p->kn.cand_cta ? p->kn.cand_cta : 512) : 0;
        const Elem el = static_cast<Elem>(mma ? form : 1);
        const int qs_mode = p->w.qop ? p->kn.qs : 1;
        knobs[2] = mma ? refine_mma_ring(d, p->max_qset, p->kn.stages, el, qs_mode) : 0;
        knobs[3] = mma ? (p->max_qset <= 32 ? 32 : 64) : 0;
        knobs[4] = mma && p->max_qset > 32 && p->kn.bucket != 2 ? 1 : 0;
        int64_t qb = p->kn.batch > 0 ? p->kn.batch : batch_cap(p->ix);
        knobs[5] = (int32_t)(qb < p->w.cap_q ? qb : p->w.cap_q);
        knobs[6] = mma && refine_mma_streams(d, p->max_qset, el, qs_mode) ? 1 : 0;
    }
    if (launches) *launches = p->launches;
    return BVSS_OK;
}

int bvss_plan_set_knobs(bvss_plan *p, const int32_t *knobs) {
    if (!p || !p->exec) return fail(BVSS_EINVAL, "plan is NULL");
    if (!knobs) return fail(BVSS_EINVAL, "knobs are NULL");
    if (knobs[0] < 0 || knobs[0] > 3)
        return fail(BVSS_EINVAL, "scan = %d: need 0, 1, 2 or 3", knobs[0]);
    if (knobs[1] < 0 || knobs[1] > 512)
        return fail(BVSS_EINVAL, "candidates per CTA = %d: need 0..512", knobs[1]);
    if (knobs[2] < 0) return fail(BVSS_EINVAL, "stages = %d: need >= 0", knobs[2]);
    if (knobs[3] != 0 && knobs[3] != 2)
        return fail(BVSS_EINVAL, "bucket = %d: need 0 or 2", knobs[3]);
    if (knobs[4] < 0) return fail(BVSS_EINVAL, "batch = %d: need >= 0", knobs[4]);
    if (knobs[5] < 0 || knobs[5] > 2)
        return fail(BVSS_EINVAL, "query operand mode = %d: need 0, 1 or 2", knobs[5]);
    const Knobs old = p->kn;
    p->kn.scan = knobs[0];
    p->kn.cand_cta = knobs[1];
    p->kn.stages = knobs[2];
    p->kn.bucket = knobs[3];
    p->kn.batch = knobs[4];
    p->kn.qs = knobs[5];
    const int rc = plan_capture(p);
    if (rc) p->kn = old;
    return rc;
}

void bvss_plan_free(bvss_plan *p) {
    if (!p) return;
    if (p->cs) cudaStreamSynchronize(p->cs);
    --p->ix->n_plans;
    free_plan(p);
}

}  // extern "C"
