/*
 * bvss_oracle.c -- plain, slow CPU oracle for the BioVSS++ query path
 * (arXiv 2412.03301, "Approximate Vector Set Search Inspired by Fly
 * Olfactory Neural System").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header, table or constant
 * with the CUDA implementation; it includes only the C standard library.
 *
 * Every function follows one definition or algorithm of the paper, step by
 * step, with no blocking or reordering beyond what that definition states:
 *
 *   orc_encode          Def. 7 (FlyHash, h = WTA(W v)) and Alg. 1
 *   orc_build_filters   count Bloom filter (Def. 8, Alg. 3) and binary
 *                       Bloom filter / set sketch (Def. 10, Alg. 5)
 *   orc_query_filters   Alg. 6 lines 1-4 (C_Q, S_Q, P = top-A of C_Q)
 *   orc_inv_*           inverted index on count Bloom filters (Def. 9,
 *                       Alg. 4) and the list walk of Alg. 6 lines 5-9
 *   orc_gate_dense      the same first-layer predicate written directly
 *   orc_hamming         Alg. 6 line 12 (Hamming distance of sketches)
 *   orc_heap_select     Alg. 6 lines 10-18 (bounded max-heap of T entries)
 *   orc_haus*           Def. 4 (Hausdorff distance), in FP64
 *   orc_refine_topk     Alg. 6 lines 19-23 (exact re-rank, top-k)
 *   orc_haus_h          Haus^H of Alg. 2: Def. 4 with the Hamming distance
 *                       between per-vector codes in place of the norm
 *   orc_alg2_scores     Alg. 2 lines 6-8 (Haus^H against every set)
 *   orc_alg2_select     Alg. 2 line 9 (the c smallest d_H)
 *   orc_dense_encode    Def. 7 with a learned dense W (BioHash in place of
 *                       FlyHash): BF16 layer, then WTA
 *   orc_soft_pair,      the training of that W on neighbour pairs: soft-code
 *   orc_learn_step      loss and gradient, and one normalized step (the
 *                       update magnitude of the BioHash iteration analysis)
 *
 * Readings where the paper is silent (the same readings the GPU path uses):
 *   - activations a_j are FP32 sums taken in the order of W's row, starting
 *     from +0.0 (a sparse binary W row lists its F input dims ascending);
 *   - WTA keeps the L largest a_j under the strict order (a desc, j asc):
 *     values compare as numbers, so -0.0 ties with +0.0; lower index wins;
 *   - P takes positions by (C_Q desc, position asc);
 *   - counts saturate at 255 (uint8 storage);
 *   - the heap orders entries by the pair (d, i) and the sets of F1 are
 *     visited in ascending id, so it keeps the T smallest pairs (d, i);
 *   - top-k orders by (distance, id) and pads with (-1, +inf);
 *   - Alg. 2 line 9 keeps exactly c sets, the c smallest pairs (d_H, id).
 * Non-finite inputs are outside the method's domain; results are undefined.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)

/* ------------------------------------------------------------------ */
/* FlyHash: a = W x with a sparse binary W (row j lists F input dims), */
/* then winner-take-all keeps the L largest activations (Def. 7).      */
/* ------------------------------------------------------------------ */

typedef struct {
    float a;
    int32_t j;
} orc_act;

/* strict total order: larger activation first, then lower index first */
static int orc_act_cmp(const void *pa, const void *pb) {
    const orc_act *x = (const orc_act *)pa;
    const orc_act *y = (const orc_act *)pb;
    if (x->a > y->a) return -1;
    if (x->a < y->a) return 1;
    if (x->j < y->j) return -1;
    if (x->j > y->j) return 1;
    return 0;
}

static int orc_u16_cmp(const void *pa, const void *pb) {
    uint16_t x = *(const uint16_t *)pa, y = *(const uint16_t *)pb;
    return (x > y) - (x < y);
}

/* x: n x d row-major; proj: m x F (row j = the input dims summed by output j)
 * pos: n x L winner positions, ascending; mask: n x ceil(m/32) words or NULL;
 * act: n x m activations or NULL. */
int orc_encode(const float *x, int64_t n, int32_t d, const uint16_t *proj,
               int32_t m, int32_t F, int32_t L, uint16_t *pos, uint32_t *mask,
               float *act) {
    if (n < 0 || d < 1 || m < 1 || F < 1 || L < 1 || L > m) return ORC_EINVAL;
    orc_act *buf = (orc_act *)malloc(sizeof(orc_act) * (size_t)m);
    if (!buf) return ORC_ENOMEM;
    const int32_t words = (m + 31) / 32;
    for (int64_t v = 0; v < n; ++v) {
        const float *xv = x + v * (int64_t)d;
        for (int32_t j = 0; j < m; ++j) {
            float a = 0.0f;
            for (int32_t t = 0; t < F; ++t) {
                uint16_t dim = proj[(int64_t)j * F + t];
                a = a + xv[dim];
            }
            buf[j].a = a;
            buf[j].j = j;
            if (act) act[v * (int64_t)m + j] = a;
        }
        qsort(buf, (size_t)m, sizeof(orc_act), orc_act_cmp);
        uint16_t *pv = pos + v * (int64_t)L;
        for (int32_t r = 0; r < L; ++r) pv[r] = (uint16_t)buf[r].j;
        qsort(pv, (size_t)L, sizeof(uint16_t), orc_u16_cmp);
        if (mask) {
            uint32_t *mv = mask + v * (int64_t)words;
            memset(mv, 0, sizeof(uint32_t) * (size_t)words);
            for (int32_t r = 0; r < L; ++r)
                mv[pv[r] >> 5] |= 1u << (pv[r] & 31);
        }
    }
    free(buf);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Filters of every database set (Alg. 3 and Alg. 5):                  */
/*   sketch S_i = OR of the member codes, count C_i[p] = sum of codes.  */
/* pos: V_total x L code positions; set_off: n_sets+1 CSR offsets.      */
/* sketch: n_sets x ceil(m/32) words; count_pm: m x n_sets (position-major) */
/* ------------------------------------------------------------------ */
int orc_build_filters(const uint16_t *pos, int32_t L, const int64_t *set_off,
                      int64_t n_sets, int32_t m, uint32_t *sketch,
                      uint8_t *count_pm) {
    if (L < 1 || m < 1 || n_sets < 0) return ORC_EINVAL;
    const int32_t words = (m + 31) / 32;
    int32_t *c = (int32_t *)malloc(sizeof(int32_t) * (size_t)m);
    if (!c) return ORC_ENOMEM;
    for (int64_t i = 0; i < n_sets; ++i) {
        memset(c, 0, sizeof(int32_t) * (size_t)m);
        for (int64_t v = set_off[i]; v < set_off[i + 1]; ++v)
            for (int32_t r = 0; r < L; ++r) c[pos[v * L + r]] += 1;
        uint32_t *s = sketch + i * (int64_t)words;
        memset(s, 0, sizeof(uint32_t) * (size_t)words);
        for (int32_t p = 0; p < m; ++p) {
            if (c[p] > 0) s[p >> 5] |= 1u << (p & 31);
            count_pm[(int64_t)p * n_sets + i] = (uint8_t)(c[p] > 255 ? 255 : c[p]);
        }
    }
    free(c);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Query filters (Alg. 6 lines 1-4).                                   */
/* qpos: m_q x L codes of the query set.  cq: m counts (not saturated); */
/* sq: ceil(m/32) words; plist: the first A positions of C_Q sorted by  */
/* (count desc, position asc).                                          */
/* ------------------------------------------------------------------ */
typedef struct {
    int32_t c;
    int32_t p;
} orc_cpos;

static int orc_cpos_cmp(const void *pa, const void *pb) {
    const orc_cpos *x = (const orc_cpos *)pa, *y = (const orc_cpos *)pb;
    if (x->c > y->c) return -1;
    if (x->c < y->c) return 1;
    return (x->p > y->p) - (x->p < y->p);
}

int orc_query_filters(const uint16_t *qpos, int64_t m_q, int32_t L, int32_t m,
                      int32_t A, int32_t *cq, uint32_t *sq, uint16_t *plist) {
    if (m_q < 1 || L < 1 || m < 1 || A < 0 || A > m) return ORC_EINVAL;
    memset(cq, 0, sizeof(int32_t) * (size_t)m);
    for (int64_t v = 0; v < m_q; ++v)
        for (int32_t r = 0; r < L; ++r) cq[qpos[v * L + r]] += 1;
    memset(sq, 0, sizeof(uint32_t) * (size_t)((m + 31) / 32));
    for (int32_t p = 0; p < m; ++p)
        if (cq[p] > 0) sq[p >> 5] |= 1u << (p & 31);
    orc_cpos *o = (orc_cpos *)malloc(sizeof(orc_cpos) * (size_t)m);
    if (!o) return ORC_ENOMEM;
    for (int32_t p = 0; p < m; ++p) {
        o[p].c = cq[p];
        o[p].p = p;
    }
    qsort(o, (size_t)m, sizeof(orc_cpos), orc_cpos_cmp);
    for (int32_t a = 0; a < A; ++a) plist[a] = (uint16_t)o[a].p;
    free(o);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Inverted index on count Bloom filters (Def. 9, Alg. 4).             */
/* List p holds (i, C_i[p]) sorted by count descending.  Entries with   */
/* count 0 are kept implicitly: they sit at the tail of every list in   */
/* ascending id, and a walk with threshold M <= 0 reaches all of them.  */
/* ------------------------------------------------------------------ */
typedef struct {
    int32_t m;
    int64_t n_sets;
    int64_t *off;   /* m+1 */
    int32_t *ids;   /* nonzero entries, list-major */
    uint8_t *cnt;
} orc_inv;

typedef struct {
    uint8_t c;
    int32_t i;
} orc_entry;

static int orc_entry_cmp(const void *pa, const void *pb) {
    const orc_entry *x = (const orc_entry *)pa, *y = (const orc_entry *)pb;
    if (x->c > y->c) return -1;
    if (x->c < y->c) return 1;
    return (x->i > y->i) - (x->i < y->i);
}

void orc_inv_free(orc_inv *ix) {
    if (!ix) return;
    free(ix->off);
    free(ix->ids);
    free(ix->cnt);
    free(ix);
}

orc_inv *orc_inv_build(const uint8_t *count_pm, int32_t m, int64_t n_sets) {
    orc_inv *ix = (orc_inv *)calloc(1, sizeof(orc_inv));
    if (!ix) return NULL;
    ix->m = m;
    ix->n_sets = n_sets;
    ix->off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m + 1));
    if (!ix->off) { orc_inv_free(ix); return NULL; }
    int64_t total = 0;
    for (int32_t p = 0; p < m; ++p) {
        ix->off[p] = total;
        for (int64_t i = 0; i < n_sets; ++i)
            if (count_pm[(int64_t)p * n_sets + i] > 0) ++total;
    }
    ix->off[m] = total;
    ix->ids = (int32_t *)malloc(sizeof(int32_t) * (size_t)(total > 0 ? total : 1));
    ix->cnt = (uint8_t *)malloc((size_t)(total > 0 ? total : 1));
    orc_entry *tmp = (orc_entry *)malloc(sizeof(orc_entry) * (size_t)(n_sets > 0 ? n_sets : 1));
    if (!ix->ids || !ix->cnt || !tmp) { free(tmp); orc_inv_free(ix); return NULL; }
    for (int32_t p = 0; p < m; ++p) {
        int64_t k = 0;
        for (int64_t i = 0; i < n_sets; ++i) {
            uint8_t c = count_pm[(int64_t)p * n_sets + i];
            if (c > 0) { tmp[k].c = c; tmp[k].i = (int32_t)i; ++k; }
        }
        qsort(tmp, (size_t)k, sizeof(orc_entry), orc_entry_cmp);
        for (int64_t e = 0; e < k; ++e) {
            ix->ids[ix->off[p] + e] = tmp[e].i;
            ix->cnt[ix->off[p] + e] = tmp[e].c;
        }
    }
    free(tmp);
    return ix;
}

/* number of stored (nonzero) entries of list p, and a copy of them */
int64_t orc_inv_list(const orc_inv *ix, int32_t p, int32_t *ids, uint8_t *cnt) {
    int64_t n = ix->off[p + 1] - ix->off[p];
    if (ids) memcpy(ids, ix->ids + ix->off[p], sizeof(int32_t) * (size_t)n);
    if (cnt) memcpy(cnt, ix->cnt + ix->off[p], (size_t)n);
    return n;
}

/* Alg. 6 lines 5-9: F1 = union over p in P of {i : (i, c) in I[p], c >= M}.
 * gate: n_sets bytes, 1 = in F1. */
int orc_inv_gate(const orc_inv *ix, const uint16_t *plist, int32_t A,
                 int32_t M, uint8_t *gate) {
    memset(gate, 0, (size_t)ix->n_sets);
    for (int32_t a = 0; a < A; ++a) {
        int32_t p = plist[a];
        for (int64_t e = ix->off[p]; e < ix->off[p + 1]; ++e)
            if ((int32_t)ix->cnt[e] >= M) gate[ix->ids[e]] = 1;
        /* implicit zero-count entries: (i, 0) for every set not listed */
        if (M <= 0)
            for (int64_t i = 0; i < ix->n_sets; ++i) gate[i] = 1;
    }
    return ORC_OK;
}

/* the same predicate read straight off the counts: exists p in P with C_i[p] >= M */
int orc_gate_dense(const uint8_t *count_pm, int32_t m, int64_t n_sets,
                   const uint16_t *plist, int32_t A, int32_t M, uint8_t *gate) {
    (void)m;
    for (int64_t i = 0; i < n_sets; ++i) {
        uint8_t g = 0;
        for (int32_t a = 0; a < A; ++a)
            if ((int32_t)count_pm[(int64_t)plist[a] * n_sets + i] >= M) g = 1;
        gate[i] = g;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Alg. 6 line 12: Hamming distance between S_Q and every sketch,      */
/* counted bit by bit.  h[i] = -1 where gate[i] == 0 (gate may be NULL) */
/* ------------------------------------------------------------------ */
int orc_hamming(const uint32_t *sq, const uint32_t *sketch, int64_t n_sets,
                int32_t m, const uint8_t *gate, int32_t *h) {
    const int32_t words = (m + 31) / 32;
    for (int64_t i = 0; i < n_sets; ++i) {
        if (gate && !gate[i]) { h[i] = -1; continue; }
        const uint32_t *s = sketch + i * (int64_t)words;
        int32_t d = 0;
        for (int32_t p = 0; p < m; ++p) {
            uint32_t bq = (sq[p >> 5] >> (p & 31)) & 1u;
            uint32_t bi = (s[p >> 5] >> (p & 31)) & 1u;
            if (bq != bi) ++d;
        }
        h[i] = d;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Alg. 6 lines 10-18: a max-heap of capacity T over pairs (d, i),      */
/* filled by visiting F1 in ascending id.  out_ids receives the ids of */
/* the heap in ascending id order; *n_out their number.                */
/* ------------------------------------------------------------------ */
typedef struct {
    int32_t d;
    int32_t i;
} orc_hent;

static int orc_hent_gt(orc_hent x, orc_hent y) { /* (d, i) lexicographic > */
    return x.d > y.d || (x.d == y.d && x.i > y.i);
}

static void orc_heap_sift_up(orc_hent *hp, int64_t k) {
    while (k > 0) {
        int64_t par = (k - 1) / 2;
        if (!orc_hent_gt(hp[k], hp[par])) break;
        orc_hent t = hp[k]; hp[k] = hp[par]; hp[par] = t;
        k = par;
    }
}

static void orc_heap_sift_down(orc_hent *hp, int64_t n, int64_t k) {
    for (;;) {
        int64_t l = 2 * k + 1, r = l + 1, b = k;
        if (l < n && orc_hent_gt(hp[l], hp[b])) b = l;
        if (r < n && orc_hent_gt(hp[r], hp[b])) b = r;
        if (b == k) break;
        orc_hent t = hp[k]; hp[k] = hp[b]; hp[b] = t;
        k = b;
    }
}

static int orc_i32_cmp(const void *pa, const void *pb) {
    int32_t x = *(const int32_t *)pa, y = *(const int32_t *)pb;
    return (x > y) - (x < y);
}

int orc_heap_select(const int32_t *h, const uint8_t *gate, int64_t n_sets,
                    int32_t T, int32_t *out_ids, int32_t *n_out) {
    if (T < 0) return ORC_EINVAL;
    orc_hent *hp = (orc_hent *)malloc(sizeof(orc_hent) * (size_t)(T > 0 ? T : 1));
    if (!hp) return ORC_ENOMEM;
    int64_t size = 0;
    for (int64_t i = 0; i < n_sets; ++i) {
        if (gate && !gate[i]) continue;
        orc_hent e = {h[i], (int32_t)i};
        if (size < T) {                 /* |G| < T: push */
            hp[size] = e;
            orc_heap_sift_up(hp, size);
            ++size;
        } else if (T > 0 && e.d < hp[0].d) { /* d < top: pop, push */
            hp[0] = e;
            orc_heap_sift_down(hp, size, 0);
        }
    }
    for (int64_t k = 0; k < size; ++k) out_ids[k] = hp[k].i;
    qsort(out_ids, (size_t)size, sizeof(int32_t), orc_i32_cmp);
    *n_out = (int32_t)size;
    free(hp);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Def. 4: Hausdorff distance with dist = Euclidean norm, in FP64.     */
/* ------------------------------------------------------------------ */
static double orc_dist(const float *a, const float *b, int32_t d) {
    double s = 0.0;
    for (int32_t k = 0; k < d; ++k) {
        double t = (double)a[k] - (double)b[k];
        s += t * t;
    }
    return sqrt(s);
}

/* max over q in Q of min over v in V of dist(q, v) */
double orc_haus_directed(const float *Q, int64_t mq, const float *V, int64_t mv,
                         int32_t d) {
    double worst = 0.0;
    for (int64_t a = 0; a < mq; ++a) {
        double best = INFINITY;
        for (int64_t b = 0; b < mv; ++b) {
            double t = orc_dist(Q + a * d, V + b * d, d);
            if (t < best) best = t;
        }
        if (best > worst) worst = best;
    }
    return worst;
}

double orc_haus(const float *Q, int64_t mq, const float *V, int64_t mv, int32_t d) {
    double x = orc_haus_directed(Q, mq, V, mv, d);
    double y = orc_haus_directed(V, mv, Q, mq, d);
    return x > y ? x : y;
}

/* ------------------------------------------------------------------ */
/* Alg. 6 lines 19-23: exact Hausdorff of every candidate, then the k  */
/* smallest by (distance, id); padded with (-1, +inf).                  */
/* cand_dist (optional) receives the distance of every candidate.       */
/* ------------------------------------------------------------------ */
typedef struct {
    double dist;
    int64_t id;
} orc_res;

static int orc_res_cmp(const void *pa, const void *pb) {
    const orc_res *x = (const orc_res *)pa, *y = (const orc_res *)pb;
    if (x->dist < y->dist) return -1;
    if (x->dist > y->dist) return 1;
    return (x->id > y->id) - (x->id < y->id);
}

int orc_refine_topk(const float *Q, int64_t mq, const float *vectors,
                    const int64_t *set_off, int32_t d, const int32_t *cand,
                    int64_t n_cand, int32_t k, int64_t *out_ids,
                    double *out_dist, double *cand_dist) {
    if (k < 1 || n_cand < 0) return ORC_EINVAL;
    orc_res *r = (orc_res *)malloc(sizeof(orc_res) * (size_t)(n_cand > 0 ? n_cand : 1));
    if (!r) return ORC_ENOMEM;
    for (int64_t c = 0; c < n_cand; ++c) {
        int64_t i = cand[c];
        const float *V = vectors + set_off[i] * (int64_t)d;
        r[c].dist = orc_haus(Q, mq, V, set_off[i + 1] - set_off[i], d);
        r[c].id = i;
        if (cand_dist) cand_dist[c] = r[c].dist;
    }
    qsort(r, (size_t)n_cand, sizeof(orc_res), orc_res_cmp);
    for (int32_t t = 0; t < k; ++t) {
        if (t < n_cand) {
            out_ids[t] = r[t].id;
            out_dist[t] = r[t].dist;
        } else {
            out_ids[t] = -1;
            out_dist[t] = INFINITY;
        }
    }
    free(r);
    return ORC_OK;
}

/* exact top-k over all sets (Def. 5 with delta = 0): the ground truth */
int orc_bruteforce_topk(const float *Q, int64_t mq, const float *vectors,
                        const int64_t *set_off, int64_t n_sets, int32_t d,
                        int32_t k, int64_t *out_ids, double *out_dist) {
    int32_t *all = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_sets > 0 ? n_sets : 1));
    if (!all) return ORC_ENOMEM;
    for (int64_t i = 0; i < n_sets; ++i) all[i] = (int32_t)i;
    int rc = orc_refine_topk(Q, mq, vectors, set_off, d, all, n_sets, k, out_ids,
                             out_dist, NULL);
    free(all);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Alg. 2: Haus^H, the Hausdorff distance of Def. 4 with the Hamming   */
/* distance between per-vector codes (m-bit masks, counted bit by     */
/* bit) in place of the norm:                                          */
/*   max( max_a min_r ham(a, r), max_r min_a ham(a, r) )              */
/* ------------------------------------------------------------------ */
static int32_t orc_ham_codes(const uint32_t *x, const uint32_t *y, int32_t m) {
    int32_t d = 0;
    for (int32_t p = 0; p < m; ++p)
        if (((x[p >> 5] >> (p & 31)) & 1u) != ((y[p >> 5] >> (p & 31)) & 1u)) ++d;
    return d;
}

int32_t orc_haus_h(const uint32_t *qmask, int64_t mq, const uint32_t *vmask, int64_t mv,
                   int32_t m) {
    const int32_t words = (m + 31) / 32;
    int32_t fwd = 0, bwd = 0;
    for (int64_t a = 0; a < mq; ++a) {          /* max over query codes of the nearest row */
        int32_t best = INT32_MAX;
        for (int64_t r = 0; r < mv; ++r) {
            const int32_t h = orc_ham_codes(qmask + a * words, vmask + r * words, m);
            if (h < best) best = h;
        }
        if (best > fwd) fwd = best;
    }
    for (int64_t r = 0; r < mv; ++r) {          /* max over rows of the nearest query code */
        int32_t best = INT32_MAX;
        for (int64_t a = 0; a < mq; ++a) {
            const int32_t h = orc_ham_codes(qmask + a * words, vmask + r * words, m);
            if (h < best) best = h;
        }
        if (best > bwd) bwd = best;
    }
    return fwd > bwd ? fwd : bwd;
}

/* Alg. 2 lines 6-8: d_H for every set j of the database (mask holds the  */
/* codes of all database vectors, set j is rows set_off[j]..set_off[j+1]) */
int orc_alg2_scores(const uint32_t *qmask, int64_t mq, const uint32_t *mask,
                    const int64_t *set_off, int64_t n_sets, int32_t m, int32_t *score) {
    const int32_t words = (m + 31) / 32;
    for (int64_t j = 0; j < n_sets; ++j)
        score[j] = orc_haus_h(qmask, mq, mask + set_off[j] * words, set_off[j + 1] - set_off[j], m);
    return ORC_OK;
}

/* Alg. 2 line 9: the c smallest pairs (d_H, j) by a full sort; out_ids    */
/* receives them in ascending id order, *n_out = min(c, n_sets).          */
static int orc_pair_cmp(const void *pa, const void *pb) {
    const int64_t *a = (const int64_t *)pa, *b = (const int64_t *)pb;
    if (a[0] != b[0]) return a[0] < b[0] ? -1 : 1;
    return a[1] < b[1] ? -1 : (a[1] > b[1]);
}

int orc_alg2_select(const int32_t *score, int64_t n_sets, int32_t c, int32_t *out_ids,
                    int64_t *n_out) {
    int64_t *pr = (int64_t *)malloc(sizeof(int64_t) * 2 * (size_t)(n_sets > 0 ? n_sets : 1));
    if (!pr) return ORC_ENOMEM;
    for (int64_t j = 0; j < n_sets; ++j) {
        pr[2 * j] = score[j];
        pr[2 * j + 1] = j;
    }
    qsort(pr, (size_t)n_sets, 2 * sizeof(int64_t), orc_pair_cmp);
    const int64_t n = n_sets < c ? n_sets : c;
    for (int64_t t = 0; t < n; ++t) out_ids[t] = (int32_t)pr[2 * t + 1];
    qsort(out_ids, (size_t)n, sizeof(int32_t), orc_i32_cmp);
    *n_out = n;
    free(pr);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Learned projection (the paper's BioHash in place of FlyHash, Def. 7: */
/* h = WTA(W v) with W learned).  Readings, as in the GPU path:        */
/*   - the layer is BF16: a = bf16(W) bf16(x), each BF16 value the     */
/*     round-to-nearest-even of the FP32 one; here summed exactly      */
/*     in FP64 (exact for weights and inputs on the 2^-8 grid);        */
/*   - WTA keeps the L largest activations, ties to the lower index;   */
/*   - training: a logistic loss on the overlap of soft codes, the     */
/*     WTA threshold held fixed in the gradient, then a normalized     */
/*     gradient step (its largest entry is the step size, the update   */
/*     magnitude M_t of the paper's BioHash iteration analysis), rows  */
/*     rescaled to a fixed norm and the forward weights rounded to     */
/*     the 2^-8 grid.                                                  */
/* ------------------------------------------------------------------ */

/* round-to-nearest-even of an FP32 value to BF16 (8 significant bits), */
/* from the IEEE 754 binary32 layout; finite inputs                      */
float orc_bf16(float x) {
    uint32_t u;
    memcpy(&u, &x, sizeof u);
    const uint32_t lsb = (u >> 16) & 1u;
    const uint32_t rounded = u + 0x7FFFu + lsb;   /* carries into the exponent when due */
    uint32_t r = rounded & 0xFFFF0000u;
    float y;
    memcpy(&y, &r, sizeof y);
    return y;
}

typedef struct {
    double a;
    int32_t j;
} orc_dact;

static int orc_dact_cmp(const void *pa, const void *pb) {
    const orc_dact *x = (const orc_dact *)pa;
    const orc_dact *y = (const orc_dact *)pb;
    if (x->a > y->a) return -1;
    if (x->a < y->a) return 1;
    if (x->j < y->j) return -1;
    if (x->j > y->j) return 1;
    return 0;
}

/* a[j] = sum_k bf16(w[j][k]) bf16(x[k]) for n vectors (act: n x m, may be NULL), */
/* then WTA: pos (n x L, ascending) and mask (n x m/32) as orc_encode           */
int orc_dense_encode(const float *x, int64_t n, int32_t d, const float *w, int32_t m,
                     int32_t L, uint16_t *pos, uint32_t *mask, double *act) {
    if (n < 0 || d < 1 || m < 1 || L < 1 || L > m) return ORC_EINVAL;
    orc_dact *buf = (orc_dact *)malloc(sizeof(orc_dact) * (size_t)m);
    uint16_t *sel = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)L);
    if (!buf || !sel) {
        free(buf);
        free(sel);
        return ORC_ENOMEM;
    }
    const int32_t words = (m + 31) / 32;
    for (int64_t v = 0; v < n; ++v) {
        const float *xv = x + v * d;
        for (int32_t j = 0; j < m; ++j) {
            double s = 0.0;
            for (int32_t k = 0; k < d; ++k)
                s += (double)orc_bf16(w[(int64_t)j * d + k]) * (double)orc_bf16(xv[k]);
            buf[j].a = s;
            buf[j].j = j;
            if (act) act[v * m + j] = s;
        }
        qsort(buf, (size_t)m, sizeof(orc_dact), orc_dact_cmp);
        for (int32_t t = 0; t < L; ++t) sel[t] = (uint16_t)buf[t].j;
        qsort(sel, (size_t)L, sizeof(uint16_t), orc_u16_cmp);
        if (pos)
            for (int32_t t = 0; t < L; ++t) pos[v * L + t] = sel[t];
        if (mask) {
            uint32_t *mv = mask + v * words;
            for (int32_t w2 = 0; w2 < words; ++w2) mv[w2] = 0u;
            for (int32_t t = 0; t < L; ++t) mv[sel[t] >> 5] |= 1u << (sel[t] & 31);
        }
    }
    free(buf);
    free(sel);
    return ORC_OK;
}

/* the WTA threshold of one activation vector: midway between its L-th and */
/* (L+1)-th largest values (L < m)                                         */
double orc_wta_threshold(const double *a, int32_t m, int32_t L) {
    double *s = (double *)malloc(sizeof(double) * (size_t)m);
    if (!s) return 0.0;
    for (int32_t j = 0; j < m; ++j) s[j] = a[j];
    /* partial selection sort of the L + 1 largest (m is small in the tests) */
    for (int32_t t = 0; t <= L && t < m; ++t) {
        int32_t b = t;
        for (int32_t j = t + 1; j < m; ++j)
            if (s[j] > s[b]) b = j;
        const double tmp = s[t];
        s[t] = s[b];
        s[b] = tmp;
    }
    const double th = 0.5 * (s[L - 1] + s[L]);
    free(s);
    return th;
}

static double orc_sigmoid(double z) {
    return z >= 0.0 ? 1.0 / (1.0 + exp(-z)) : exp(z) / (1.0 + exp(z));
}

/* Loss of one pair and its gradient in the activations, the thresholds th_x, th_y held */
/* fixed: soft codes c_j = sigmoid((a_j - th) / T), overlap o = (1/L) sum_j c_j(x) c_j(y), */
/* logit z = s (o - mu), loss = log(1 + exp(-z)) for a positive pair (y = 1) and        */
/* log(1 + exp(z)) for a negative one.  gx, gy (m each) receive d loss / d a.            */
double orc_soft_pair(const double *ax, const double *ay, int32_t m, int32_t L, double T,
                     double s, double mu, int32_t y, double th_x, double th_y, double *gx,
                     double *gy) {
    double o = 0.0;
    for (int32_t j = 0; j < m; ++j)
        o += orc_sigmoid((ax[j] - th_x) / T) * orc_sigmoid((ay[j] - th_y) / T);
    o /= (double)L;
    const double sg = y ? 1.0 : -1.0;
    const double z = sg * s * (o - mu);
    /* log(1 + exp(-z)), evaluated without overflow */
    const double loss = z >= 0.0 ? log1p(exp(-z)) : -z + log1p(exp(z));
    const double dl_do = -sg * s * orc_sigmoid(-z);
    for (int32_t j = 0; j < m; ++j) {
        const double cx = orc_sigmoid((ax[j] - th_x) / T);
        const double cy = orc_sigmoid((ay[j] - th_y) / T);
        if (gx) gx[j] = dl_do * (cy / L) * cx * (1.0 - cx) / T;
        if (gy) gy[j] = dl_do * (cx / L) * cy * (1.0 - cy) / T;
    }
    return loss;
}

/* a weight's forward value: the nearest multiple of 2^-8 (ties to even), clamped to */
/* [-1, 1], so that BF16 holds it exactly                                            */
double orc_quant_weight(double w) {
    double q = nearbyint(w * 256.0) / 256.0;
    if (q > 1.0) q = 1.0;
    if (q < -1.0) q = -1.0;
    return q;
}

/* One training step over a batch of n pairs (x_i, y_i, label_i):                     */
/*   forward with the quantized weights wq = quant(w): a = wq bf16(x);              */
/*   d w = (1/n) sum_i g_x,i bf16(x_i)^T + g_y,i bf16(y_i)^T (orc_soft_pair);        */
/*   w' = w - eta dw / max|dw|, then every row rescaled to norm row_norm;            */
/*   wq' = quant(w').  w, w_out: m x d FP64; wq_out: m x d; loss_out: the mean loss. */
int orc_learn_step(const double *w, const float *xs, const float *ys, const uint8_t *labels,
                   int64_t n, int32_t m, int32_t d, int32_t L, double T, double s, double mu,
                   double eta, double row_norm, double *w_out, float *wq_out, double *dw_out,
                   double *loss_out) {
    if (n < 1 || m < 2 || d < 1 || L < 1 || L >= m) return ORC_EINVAL;
    const size_t md = (size_t)m * d;
    float *wq = (float *)malloc(sizeof(float) * md);
    double *dw = (double *)calloc(md, sizeof(double));
    double *ax = (double *)malloc(sizeof(double) * (size_t)m);
    double *ay = (double *)malloc(sizeof(double) * (size_t)m);
    double *gx = (double *)malloc(sizeof(double) * (size_t)m);
    double *gy = (double *)malloc(sizeof(double) * (size_t)m);
    if (!wq || !dw || !ax || !ay || !gx || !gy) {
        free(wq); free(dw); free(ax); free(ay); free(gx); free(gy);
        return ORC_ENOMEM;
    }
    for (size_t e = 0; e < md; ++e) wq[e] = (float)orc_quant_weight(w[e]);
    double loss = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        const float *x = xs + i * d, *yv = ys + i * d;
        orc_dense_encode(x, 1, d, wq, m, L, NULL, NULL, ax);
        orc_dense_encode(yv, 1, d, wq, m, L, NULL, NULL, ay);
        const double tx = orc_wta_threshold(ax, m, L), ty = orc_wta_threshold(ay, m, L);
        loss += orc_soft_pair(ax, ay, m, L, T, s, mu, labels[i], tx, ty, gx, gy);
        for (int32_t j = 0; j < m; ++j)
            for (int32_t k = 0; k < d; ++k)
                dw[(size_t)j * d + k] +=
                    (gx[j] * (double)orc_bf16(x[k]) + gy[j] * (double)orc_bf16(yv[k])) / (double)n;
    }
    double mx = 0.0;
    for (size_t e = 0; e < md; ++e) mx = fabs(dw[e]) > mx ? fabs(dw[e]) : mx;
    for (int32_t j = 0; j < m; ++j) {
        double nn = 0.0;
        for (int32_t k = 0; k < d; ++k) {
            const size_t e = (size_t)j * d + k;
            w_out[e] = w[e] - (mx > 0.0 ? eta * dw[e] / mx : 0.0);
            nn += w_out[e] * w_out[e];
        }
        nn = sqrt(nn);
        for (int32_t k = 0; k < d; ++k) {
            const size_t e = (size_t)j * d + k;
            if (nn > 0.0) w_out[e] *= row_norm / nn;
            wq_out[e] = (float)orc_quant_weight(w_out[e]);
        }
    }
    if (dw_out) memcpy(dw_out, dw, sizeof(double) * md);
    *loss_out = loss / (double)n;
    free(wq); free(dw); free(ax); free(ay); free(gx); free(gy);
    return ORC_OK;
}
