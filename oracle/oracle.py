"""CPU oracle for the BioVSS++ query path (arXiv 2412.03301).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the
benchmark's CPU-baseline leg are the only callers.  The product path never
imports this module.  It shares no code with the CUDA implementation: the
arithmetic lives in ``bvss_oracle.c`` (plain C, FP64 for the Hausdorff
distance) and this file only marshals numpy arrays into it.

Each wrapper names the passage of the paper it follows:

* ``encode``          Def. 7 (FlyHash ``h = WTA(W v)``), Alg. 1
* ``build_filters``   count Bloom filter (Def. 8, Alg. 3), binary Bloom
                      filter / set sketch (Def. 10, Alg. 5)
* ``query_filters``   Alg. 6 lines 1-4 (C_Q, S_Q, top-A positions P)
* ``InvertedIndex``   Def. 9 / Alg. 4 and the list walk of Alg. 6 lines 5-9
* ``gate_dense``      the same first-layer predicate read off the counts
* ``hamming``         Alg. 6 line 12
* ``heap_select``     Alg. 6 lines 10-18
* ``haus``            Def. 4 (FP64)
* ``refine_topk``     Alg. 6 lines 19-23
* ``bruteforce_topk`` exact top-k of Def. 5 (ground truth)
* ``query``           the whole of Alg. 6 for one query set
* ``dense_encode``    Def. 7 with a learned BF16 dense layer (BioHash)
* ``soft_pair``, ``learn_step``  training that layer on neighbour pairs

Every function is pinned by ``tests/test_oracle_*.py`` against worked
examples printed in the paper, closed forms, invariants and brute force.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bvss_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (no fast-math, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    i32, i64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "orc_encode": (ctypes.c_int, [P, i64, i32, P, i32, i32, i32, P, P, P]),
        "orc_build_filters": (ctypes.c_int, [P, i32, P, i64, i32, P, P]),
        "orc_query_filters": (ctypes.c_int, [P, i64, i32, i32, i32, P, P, P]),
        "orc_inv_build": (P, [P, i32, i64]),
        "orc_inv_free": (None, [P]),
        "orc_inv_list": (i64, [P, i32, P, P]),
        "orc_inv_gate": (ctypes.c_int, [P, P, i32, i32, P]),
        "orc_gate_dense": (ctypes.c_int, [P, i32, i64, P, i32, i32, P]),
        "orc_hamming": (ctypes.c_int, [P, P, i64, i32, P, P]),
        "orc_heap_select": (ctypes.c_int, [P, P, i64, i32, P, P]),
        "orc_haus": (dbl, [P, i64, P, i64, i32]),
        "orc_haus_directed": (dbl, [P, i64, P, i64, i32]),
        "orc_refine_topk": (ctypes.c_int, [P, i64, P, P, i32, P, i64, i32, P, P, P]),
        "orc_bruteforce_topk": (ctypes.c_int, [P, i64, P, P, i64, i32, i32, P, P]),
        "orc_haus_h": (i32, [P, i64, P, i64, i32]),
        "orc_alg2_scores": (ctypes.c_int, [P, i64, P, P, i64, i32, P]),
        "orc_alg2_select": (ctypes.c_int, [P, i64, i32, P, P]),
        "orc_bf16": (ctypes.c_float, [ctypes.c_float]),
        "orc_dense_encode": (ctypes.c_int, [P, i64, i32, P, i32, i32, P, P, P]),
        "orc_wta_threshold": (dbl, [P, i32, i32]),
        "orc_soft_pair": (dbl, [P, P, i32, i32, dbl, dbl, dbl, i32, dbl, dbl, P, P]),
        "orc_quant_weight": (dbl, [dbl]),
        "orc_learn_step": (ctypes.c_int, [P, P, P, P, i64, i32, i32, i32, dbl, dbl, dbl, dbl,
                                          dbl, P, P, P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _check(rc, what):
    if rc != 0:
        raise ValueError("oracle %s failed with status %d" % (what, rc))


def encode(x, proj, L, return_act=False):
    """FlyHash codes (Def. 7): positions (n, L) ascending and masks (n, m/32)."""
    lib = _load()
    x = _c(x, np.float32)
    proj = _c(proj, np.uint16)
    n, d = x.shape
    m, F = proj.shape
    pos = np.zeros((n, L), np.uint16)
    mask = np.zeros((n, (m + 31) // 32), np.uint32)
    act = np.zeros((n, m), np.float32) if return_act else None
    _check(lib.orc_encode(_p(x), n, d, _p(proj), m, F, L, _p(pos), _p(mask),
                          _p(act)), "encode")
    return (pos, mask, act) if return_act else (pos, mask)


def build_filters(pos, set_off, m):
    """Sketches (n_sets, m/32) uint32 and counts (m, n_sets) uint8 (Alg. 3, 5)."""
    lib = _load()
    pos = _c(pos, np.uint16)
    set_off = _c(set_off, np.int64)
    n_sets = set_off.shape[0] - 1
    L = pos.shape[1]
    sketch = np.zeros((n_sets, (m + 31) // 32), np.uint32)
    count = np.zeros((m, n_sets), np.uint8)
    _check(lib.orc_build_filters(_p(pos), L, _p(set_off), n_sets, m, _p(sketch),
                                 _p(count)), "build_filters")
    return sketch, count


def query_filters(qpos, m, A):
    """C_Q (m,) int32, S_Q (m/32,) uint32, P (A,) uint16 (Alg. 6 lines 1-4)."""
    lib = _load()
    qpos = _c(qpos, np.uint16)
    mq, L = qpos.shape
    cq = np.zeros(m, np.int32)
    sq = np.zeros((m + 31) // 32, np.uint32)
    plist = np.zeros(max(A, 1), np.uint16)
    _check(lib.orc_query_filters(_p(qpos), mq, L, m, A, _p(cq), _p(sq), _p(plist)),
           "query_filters")
    return cq, sq, plist[:A]


class InvertedIndex:
    """Count-sorted inverted lists (Def. 9, Alg. 4) with the Alg. 6 walk."""

    def __init__(self, count_pm):
        self._lib = _load()
        self.count = _c(count_pm, np.uint8)
        self.m, self.n_sets = self.count.shape
        self._h = self._lib.orc_inv_build(_p(self.count), self.m, self.n_sets)
        if not self._h:
            raise MemoryError("oracle inverted index")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_inv_free(h)
            self._h = None

    def list(self, p):
        n = self._lib.orc_inv_list(self._h, p, None, None)
        ids = np.zeros(max(n, 1), np.int32)
        cnt = np.zeros(max(n, 1), np.uint8)
        self._lib.orc_inv_list(self._h, p, _p(ids), _p(cnt))
        return ids[:n], cnt[:n]

    def gate(self, plist, M):
        plist = _c(plist, np.uint16)
        g = np.zeros(self.n_sets, np.uint8)
        _check(self._lib.orc_inv_gate(self._h, _p(plist) if plist.size else None,
                                      plist.shape[0], M, _p(g)), "inv_gate")
        return g


def gate_dense(count_pm, plist, M):
    lib = _load()
    count_pm = _c(count_pm, np.uint8)
    plist = _c(plist, np.uint16)
    m, n_sets = count_pm.shape
    g = np.zeros(n_sets, np.uint8)
    _check(lib.orc_gate_dense(_p(count_pm), m, n_sets,
                              _p(plist) if plist.size else None, plist.shape[0],
                              M, _p(g)), "gate_dense")
    return g


def hamming(sq, sketch, gate=None, m=None):
    """h[i] = Hamming(S_Q, S_i), -1 where the gate is closed (Alg. 6 line 12)."""
    lib = _load()
    sq = _c(sq, np.uint32)
    sketch = _c(sketch, np.uint32)
    n_sets, words = sketch.shape
    m = words * 32 if m is None else m
    g = None if gate is None else _c(gate, np.uint8)
    h = np.zeros(n_sets, np.int32)
    _check(lib.orc_hamming(_p(sq), _p(sketch), n_sets, m, _p(g), _p(h)),
           "hamming")
    return h


def heap_select(h, gate, T):
    """Ids kept by the capacity-T max-heap of Alg. 6 lines 10-18, ascending."""
    lib = _load()
    h = _c(h, np.int32)
    g = None if gate is None else _c(gate, np.uint8)
    out = np.zeros(max(T, 1), np.int32)
    n = ctypes.c_int32(0)
    _check(lib.orc_heap_select(_p(h), _p(g), h.shape[0], T, _p(out),
                               ctypes.byref(n)), "heap_select")
    return out[:n.value]


def haus(Q, V):
    """Hausdorff distance of Def. 4 in FP64."""
    lib = _load()
    Q = _c(Q, np.float32)
    V = _c(V, np.float32)
    return lib.orc_haus(_p(Q), Q.shape[0], _p(V), V.shape[0], Q.shape[1])


def haus_directed(Q, V):
    """max over q in Q of min over v in V of ||q - v|| (one term of Def. 4)."""
    lib = _load()
    Q = _c(Q, np.float32)
    V = _c(V, np.float32)
    return lib.orc_haus_directed(_p(Q), Q.shape[0], _p(V), V.shape[0], Q.shape[1])


def refine_topk(Q, vectors, set_off, cand, k):
    """(ids (k,), dists (k,), per-candidate dists) of Alg. 6 lines 19-23."""
    lib = _load()
    Q = _c(Q, np.float32)
    vectors = _c(vectors, np.float32)
    set_off = _c(set_off, np.int64)
    cand = _c(cand, np.int32)
    ids = np.zeros(k, np.int64)
    dist = np.zeros(k, np.float64)
    cd = np.zeros(max(cand.shape[0], 1), np.float64)
    _check(lib.orc_refine_topk(_p(Q), Q.shape[0], _p(vectors), _p(set_off),
                               vectors.shape[1], _p(cand) if cand.size else None,
                               cand.shape[0], k, _p(ids), _p(dist), _p(cd)),
           "refine_topk")
    return ids, dist, cd[:cand.shape[0]]


def bruteforce_topk(Q, vectors, set_off, k):
    lib = _load()
    Q = _c(Q, np.float32)
    vectors = _c(vectors, np.float32)
    set_off = _c(set_off, np.int64)
    ids = np.zeros(k, np.int64)
    dist = np.zeros(k, np.float64)
    _check(lib.orc_bruteforce_topk(_p(Q), Q.shape[0], _p(vectors), _p(set_off),
                                   set_off.shape[0] - 1, vectors.shape[1], k,
                                   _p(ids), _p(dist)), "bruteforce_topk")
    return ids, dist


class Index:
    """The oracle's index: codes, sketches, counts and inverted lists."""

    def __init__(self, vectors, set_off, proj, L, threads=1, dense_w=None):
        self.vectors = _c(vectors, np.float32)
        self.set_off = _c(set_off, np.int64)
        self.dense_w = None if dense_w is None else _c(dense_w, np.float32)
        self.proj = None if proj is None else _c(proj, np.uint16)
        self.m = (self.proj if self.dense_w is None else self.dense_w).shape[0]
        self.L = L
        if self.dense_w is not None:
            # the learned dense projection in place of FlyHash
            self.pos, self.mask = dense_encode(self.vectors, self.dense_w, L)
        elif threads > 1:
            # the vectors are encoded independently (Alg. 1 line 4): chunks on host
            # threads (the C calls release the GIL), the same codes as one call
            from concurrent.futures import ThreadPoolExecutor
            n = self.vectors.shape[0]
            step = max(1, -(-n // (4 * threads)))
            with ThreadPoolExecutor(threads) as ex:
                parts = list(ex.map(lambda v0: encode(self.vectors[v0:v0 + step], self.proj, L),
                                    range(0, n, step)))
            self.pos = np.concatenate([p[0] for p in parts]) if parts else \
                np.zeros((0, L), np.uint16)
            self.mask = np.concatenate([p[1] for p in parts]) if parts else \
                np.zeros((0, (self.m + 31) // 32), np.uint32)
        else:
            self.pos, self.mask = encode(self.vectors, self.proj, L)
        self.sketch, self.count = build_filters(self.pos, self.set_off, self.m)
        self.inv = InvertedIndex(self.count)

    @property
    def n_sets(self):
        return self.set_off.shape[0] - 1


def _codes(index: Index, Q):
    if index.dense_w is not None:
        return dense_encode(Q, index.dense_w, index.L)
    return encode(Q, index.proj, index.L)


def query(index: Index, Q, k, C, A, M):
    """Alg. 6 for one query set; returns every intermediate as a dict."""
    qpos, qmask = _codes(index, Q)
    cq, sq, plist = query_filters(qpos, index.m, A)
    gate = index.inv.gate(plist, M)
    h = hamming(sq, index.sketch, gate, m=index.m)
    cand = heap_select(h, gate, C)
    ids, dist, cand_dist = refine_topk(Q, index.vectors, index.set_off, cand, k)
    return dict(qpos=qpos, qmask=qmask, cq=cq, sq=sq, plist=plist, gate=gate,
                h=h, cand=cand, cand_dist=cand_dist, ids=ids, dist=dist)


def haus_h(qmask, vmask, m):
    """Haus^H (Alg. 2) between two sets of m-bit codes, rows of uint32 words."""
    qmask = _c(qmask, np.uint32)
    vmask = _c(vmask, np.uint32)
    return int(_load().orc_haus_h(_p(qmask), qmask.shape[0], _p(vmask), vmask.shape[0], m))


def alg2_scores(qmask, mask, set_off, m):
    qmask = _c(qmask, np.uint32)
    mask = _c(mask, np.uint32)
    set_off = _c(set_off, np.int64)
    n = set_off.shape[0] - 1
    score = np.empty(n, np.int32)
    _check(_load().orc_alg2_scores(_p(qmask), qmask.shape[0], _p(mask), _p(set_off), n, m,
                                   _p(score)), "alg2_scores")
    return score


def alg2_select(score, c):
    score = _c(score, np.int32)
    out = np.empty(max(1, min(c, score.shape[0])), np.int32)
    n = ctypes.c_int64()
    _check(_load().orc_alg2_select(_p(score), score.shape[0], c, _p(out), ctypes.byref(n)),
           "alg2_select")
    return out[:n.value]


def query_alg2(index: Index, Q, k, C):
    """Alg. 2 (plain BioVSS) for one query set; returns every intermediate."""
    qpos, qmask = _codes(index, Q)
    score = alg2_scores(qmask, index.mask, index.set_off, index.m)
    cand = alg2_select(score, C)
    ids, dist, cand_dist = refine_topk(Q, index.vectors, index.set_off, cand, k)
    return dict(qpos=qpos, qmask=qmask, score=score, cand=cand, cand_dist=cand_dist, ids=ids,
                dist=dist)


# ---- learned projection (BioHash in place of FlyHash, Def. 7) ----------------------
def bf16(x):
    """Round-to-nearest-even BF16 value of each FP32 value."""
    f = _load().orc_bf16
    return np.array([f(float(v)) for v in np.asarray(x, np.float32).ravel()],
                    np.float32).reshape(np.shape(x))


def dense_encode(x, w, L, return_act=False):
    """Codes of a BF16 dense layer: a = bf16(w) bf16(x) exactly, then WTA top-L."""
    lib = _load()
    x = _c(x, np.float32)
    w = _c(w, np.float32)
    n, d = x.shape
    m = w.shape[0]
    pos = np.zeros((n, L), np.uint16)
    mask = np.zeros((n, (m + 31) // 32), np.uint32)
    act = np.zeros((n, m), np.float64) if return_act else None
    _check(lib.orc_dense_encode(_p(x), n, d, _p(w), m, L, _p(pos), _p(mask), _p(act)),
           "dense_encode")
    return (pos, mask, act) if return_act else (pos, mask)


def wta_threshold(a, L):
    a = _c(a, np.float64)
    return float(_load().orc_wta_threshold(_p(a), a.shape[0], L))


def soft_pair(ax, ay, L, T, s, mu, y, th_x, th_y):
    """(loss, d loss / d ax, d loss / d ay) of one pair, thresholds fixed."""
    ax = _c(ax, np.float64)
    ay = _c(ay, np.float64)
    gx = np.zeros_like(ax)
    gy = np.zeros_like(ay)
    loss = _load().orc_soft_pair(_p(ax), _p(ay), ax.shape[0], L, T, s, mu, int(y), th_x, th_y,
                                 _p(gx), _p(gy))
    return loss, gx, gy


def quant_weight(w):
    f = _load().orc_quant_weight
    return np.vectorize(lambda v: f(float(v)))(np.asarray(w, np.float64))


def learn_step(w, xs, ys, labels, L, T, s, mu, eta, row_norm):
    """One training step; returns (w', wq', dw, mean loss)."""
    lib = _load()
    w = _c(w, np.float64)
    xs = _c(xs, np.float32)
    ys = _c(ys, np.float32)
    labels = _c(labels, np.uint8)
    m, d = w.shape
    w_out = np.zeros_like(w)
    wq = np.zeros((m, d), np.float32)
    dw = np.zeros_like(w)
    loss = ctypes.c_double()
    _check(lib.orc_learn_step(_p(w), _p(xs), _p(ys), _p(labels), xs.shape[0], m, d, L, T, s,
                              mu, eta, row_norm, _p(w_out), _p(wq), _p(dw),
                              ctypes.byref(loss)), "learn_step")
    return w_out, wq, dw, loss.value


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
