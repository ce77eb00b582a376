"""Thin Python binding of the C ABI in include/bvss.h (same names).

Argument marshalling only: torch tensors supply device memory and streams,
numpy arrays supply host offsets and the projection table, and every step of
the search runs in the CUDA kernels of ``libbvss.so``.  There is no CPU
fallback: loading fails loudly when the library is missing.
"""
from __future__ import annotations

import ctypes
import os
import weakref

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libbvss.so")

BVSS_OK, BVSS_EINVAL, BVSS_ENOMEM, BVSS_ECUDA, BVSS_ETIMEOUT = 0, -1, -2, -3, -4
GATED_OUT = 0xFFFF

_c_i32, _c_i64, _vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p


class bvss_params(ctypes.Structure):
    _fields_ = [("d", _c_i32), ("m", _c_i32), ("fanin", _c_i32), ("wta_l", _c_i32),
                ("flags", _c_i32), ("reserved", _c_i32 * 3)]


class bvss_search(ctypes.Structure):
    _fields_ = [("k", _c_i32), ("C", _c_i32), ("A", _c_i32), ("M", _c_i32), ("flags", _c_i32),
                ("reserved", _c_i32)]


BVSS_BUILD_BF16 = 1
BVSS_BUILD_FP8 = 2
BVSS_SEARCH_FAST = 1
BVSS_SEARCH_POPC_SCAN = 2
BVSS_SEARCH_ALG2 = 4
BVSS_SEARCH_FP8 = 8
BVSS_SEARCH_FP8_EXACT = 16
BVSS_SEARCH_TF32 = 32
BVSS_SEARCH_SCAN_SETS_TMEM = 64


class bvss_trace(ctypes.Structure):
    _fields_ = [("qpos", _vp), ("cq", _vp), ("sq", _vp), ("plist", _vp), ("h", _vp),
                ("cand", _vp), ("n_cand", _vp), ("cand_dist", _vp)]


class BvssError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("bvss status %d: %s" % (code, msg))
        self.code = code


SYMBOLS = {
    "bvss_build": (ctypes.c_int, [_vp, _vp, _c_i64, _vp, ctypes.POINTER(bvss_params), _vp,
                                  ctypes.POINTER(_vp)]),
    "bvss_query": (ctypes.c_int, [_vp, _vp, _vp, _c_i64, ctypes.POINTER(bvss_search), _vp,
                                  _vp, _vp]),
    "bvss_query_trace": (ctypes.c_int, [_vp, _vp, _vp, _c_i64, ctypes.POINTER(bvss_search),
                                        _vp, _vp, ctypes.POINTER(bvss_trace), _vp]),
    "bvss_encode": (ctypes.c_int, [_vp, _vp, _c_i64, _vp, _vp, _vp]),
    "bvss_index_info": (ctypes.c_int, [_vp, ctypes.POINTER(bvss_params),
                                       ctypes.POINTER(_c_i64), ctypes.POINTER(_c_i64)]),
    "bvss_get_codes": (ctypes.c_int, [_vp, _c_i64, _c_i64, _vp, _vp]),
    "bvss_get_sketches": (ctypes.c_int, [_vp, _vp, _c_i64, _vp, _vp]),
    "bvss_get_counts": (ctypes.c_int, [_vp, _vp, _c_i64, _vp, _vp]),
    "bvss_profile_enable": (ctypes.c_int, [_vp, ctypes.c_int]),
    "bvss_profile_read": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(_c_i64), ctypes.POINTER(_c_i64),
                                         ctypes.c_int]),
    "bvss_select_noalloc": (ctypes.c_int, [_vp, _c_i64, _c_i64, _c_i32, _c_i32, _c_i32, _vp,
                                           _vp, _vp]),
    "bvss_sync": (ctypes.c_int, [_vp, _vp]),
    "bvss_selftest_wait_timeout": (ctypes.c_int, [_c_i64]),
    "bvss_plan_create": (ctypes.c_int, [_vp, ctypes.POINTER(bvss_search), _c_i64, _c_i64,
                                        _c_i32, _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(_vp)]),
    "bvss_plan_launch": (ctypes.c_int, [_vp, _vp]),
    "bvss_plan_tune": (ctypes.c_int, [_vp, _c_i32, _vp, ctypes.POINTER(ctypes.c_float)]),
    "bvss_plan_info": (ctypes.c_int, [_vp, ctypes.POINTER(_c_i32), ctypes.POINTER(_c_i64)]),
    "bvss_plan_set_knobs": (ctypes.c_int, [_vp, ctypes.POINTER(_c_i32)]),
    "bvss_plan_free": (None, [_vp]),
    "bvss_free": (None, [_vp]),
    "bvss_last_error": (ctypes.c_char_p, []),
    "bvss_build_dense": (ctypes.c_int, [_vp, _vp, _c_i64, _vp, ctypes.POINTER(bvss_params),
                                        _vp, ctypes.POINTER(_vp)]),
    "bvss_dense_forward": (ctypes.c_int, [_vp, _c_i64, _c_i32, _vp, _c_i32, _vp, _c_i64, _vp]),
    "bvss_learn_sync": (ctypes.c_int, [_vp]),
    "bvss_learn_pair_grad": (ctypes.c_int, [_vp, _vp, _c_i64, _vp, _c_i64, _c_i32, _c_i32,
                                            ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                            _vp, _vp, _c_i64, _vp, _vp]),
    "bvss_learn_weight_grad": (ctypes.c_int, [_vp, _vp, _c_i64, _vp, _vp, _c_i64, _c_i32,
                                              _c_i32, _vp, _vp]),
    "bvss_learn_update": (ctypes.c_int, [_vp, _vp, _c_i32, _c_i32, ctypes.c_float,
                                         ctypes.c_float, _vp, _vp, _vp]),
    "bvss_to_bf16": (ctypes.c_int, [_vp, _c_i64, _c_i32, _vp, _vp]),
    "bvss_index_rows_bf16": (ctypes.c_int, [_vp, _vp, _c_i64, _vp, _vp]),
    "bvss_nearest_rows": (ctypes.c_int, [_vp, _vp, _vp, _c_i64, _vp, _c_i32, _vp, _vp]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libbvss.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libbvss.so not found at %s: build it with "
                           "`python -m paper_2412_03301_gb300.build`" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in SYMBOLS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def bvss_last_error() -> str:
    return load().bvss_last_error().decode()


def _check(rc):
    if rc != BVSS_OK:
        raise BvssError(rc, bvss_last_error())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _host_i64(a):
    a = np.ascontiguousarray(np.asarray(a), dtype=np.int64)
    return a, ctypes.c_void_p(a.ctypes.data)


class Index:
    """Owns a bvss_index handle; freed with bvss_free."""

    def __init__(self, handle, params: bvss_params, n_sets: int, n_vectors: int, device):
        self.handle = handle
        self.params = params
        self.n_sets = n_sets
        self.n_vectors = n_vectors
        self.device = device
        self._plans = weakref.WeakSet()   # plans are freed before their index

    @property
    def d(self):
        return self.params.d

    @property
    def m(self):
        return self.params.m

    @property
    def L(self):
        return self.params.wta_l

    def close(self):
        if self.handle:
            for p in list(self._plans):
                p.close()
            torch.cuda.synchronize(self.device)
            load().bvss_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bvss_build(vectors: torch.Tensor, set_offsets, proj, *, fanin=None, wta_l: int,
               bf16: bool = False, fp8: bool = False, stream=None) -> Index:
    """Build an index (Alg. 1, 3, 4, 5). vectors: (V, d) float32, host or CUDA."""
    lib = load()
    assert vectors.dtype == torch.float32 and vectors.is_contiguous()
    off, off_p = _host_i64(set_offsets)
    proj = np.ascontiguousarray(proj, dtype=np.uint16)
    p = bvss_params(d=vectors.shape[1], m=proj.shape[0],
                    fanin=proj.shape[1] if fanin is None else fanin, wta_l=wta_l,
                    flags=(BVSS_BUILD_BF16 if bf16 else 0) | (BVSS_BUILD_FP8 if fp8 else 0))
    h = ctypes.c_void_p()
    dev = vectors.device if vectors.is_cuda else torch.device("cuda", torch.cuda.current_device())
    with torch.cuda.device(dev):
        _check(lib.bvss_build(_dptr(vectors), off_p, off.shape[0] - 1,
                              ctypes.c_void_p(proj.ctypes.data), ctypes.byref(p),
                              _stream(stream), ctypes.byref(h)))
    return Index(h, p, off.shape[0] - 1, int(off[-1]), dev)


def _search_flags(fast, popc_scan, alg2=False, fp8=False, fp8_exact=False, tf32=False,
                  scan_sets_tmem=False):
    return ((BVSS_SEARCH_FAST if fast else 0) | (BVSS_SEARCH_POPC_SCAN if popc_scan else 0)
            | (BVSS_SEARCH_ALG2 if alg2 else 0) | (BVSS_SEARCH_FP8 if fp8 else 0)
            | (BVSS_SEARCH_FP8_EXACT if fp8_exact else 0) | (BVSS_SEARCH_TF32 if tf32 else 0)
            | (BVSS_SEARCH_SCAN_SETS_TMEM if scan_sets_tmem else 0))


def bvss_query(ix: Index, q_vectors: torch.Tensor, q_offsets, *, k: int, C: int, A: int = 3,
               M: int = 1, fast: bool = False, popc_scan: bool = False, alg2: bool = False,
               fp8: bool = False, fp8_exact: bool = False, tf32: bool = False,
               scan_sets_tmem: bool = False, out_ids=None, out_dist=None, stream=None):
    """Alg. 6 for a batch of query sets -> (ids (n_q, k) int64, dist (n_q, k) float32).

    q_vectors and the outputs may live on the host or on the index's GPU."""
    lib = load()
    off, off_p = _host_i64(q_offsets)
    nq = off.shape[0] - 1
    dev = ix.device
    if out_ids is None:
        out_ids = torch.empty((nq, k), dtype=torch.int64, device=dev)
    if out_dist is None:
        out_dist = torch.empty((nq, k), dtype=torch.float32, device=dev)
    s = bvss_search(k=k, C=C, A=A, M=M,
                    flags=_search_flags(fast, popc_scan, alg2, fp8, fp8_exact, tf32, scan_sets_tmem))
    _check(lib.bvss_query(ix.handle, _dptr(q_vectors), off_p, nq, ctypes.byref(s),
                          _dptr(out_ids), _dptr(out_dist), _stream(stream)))
    return out_ids, out_dist


class Plan:
    """A graph-captured query pass over fixed device buffers (bvss_plan_*).

    The plan allocates its buffers: ``q_vectors`` (max_vectors, d) float32,
    ``q_offsets`` (n_queries + 1,) int64, ``ids`` (n_queries, k) int64 and
    ``dist`` (n_queries, k) float32, all on the index's GPU.  Write a batch
    into the first two (``set_queries``), call ``launch`` and read the last two.
    """

    def __init__(self, ix: Index, n_queries: int, max_vectors: int, max_qset: int, *, k: int,
                 C: int, A: int = 3, M: int = 1, fast: bool = False, popc_scan: bool = False,
                 alg2: bool = False, fp8: bool = False, fp8_exact: bool = False,
                 tf32: bool = False, scan_sets_tmem: bool = False, stream=None):
        lib = load()
        dev = ix.device
        self.ix = ix
        self.n_queries, self.max_vectors, self.max_qset = n_queries, max_vectors, max_qset
        self.q_vectors = torch.zeros((max_vectors, ix.d), dtype=torch.float32, device=dev)
        self.q_offsets = torch.arange(n_queries + 1, dtype=torch.int64, device=dev)
        self.ids = torch.empty((n_queries, k), dtype=torch.int64, device=dev)
        self.dist = torch.empty((n_queries, k), dtype=torch.float32, device=dev)
        s = bvss_search(k=k, C=C, A=A, M=M,
                    flags=_search_flags(fast, popc_scan, alg2, fp8, fp8_exact, tf32, scan_sets_tmem))
        h = ctypes.c_void_p()
        with torch.cuda.device(dev):
            _check(lib.bvss_plan_create(ix.handle, ctypes.byref(s), n_queries, max_vectors,
                                        max_qset, _dptr(self.q_vectors), _dptr(self.q_offsets),
                                        _dptr(self.ids), _dptr(self.dist), _stream(stream),
                                        ctypes.byref(h)))
        self.handle = h
        ix._plans.add(self)

    def set_queries(self, q_vectors: torch.Tensor, q_offsets, stream=None):
        """Copy a batch (vectors on any device, offsets host or device) into the buffers."""
        n = q_vectors.shape[0]
        if n > self.max_vectors:
            raise ValueError("batch has %d vectors, the plan holds %d" % (n, self.max_vectors))
        off = torch.as_tensor(np.asarray(q_offsets) if not torch.is_tensor(q_offsets)
                              else q_offsets, dtype=torch.int64)
        if off.shape[0] != self.n_queries + 1:
            raise ValueError("the plan takes %d query sets" % self.n_queries)
        st = torch.cuda.current_stream(self.ix.device) if stream is None else stream
        with torch.cuda.stream(st):
            self.q_vectors[:n].copy_(q_vectors, non_blocking=True)
            self.q_offsets.copy_(off, non_blocking=True)

    def launch(self, stream=None):
        _check(load().bvss_plan_launch(self.handle, _stream(stream)))
        return self.ids, self.dist

    def tune(self, reps: int = 3, stream=None) -> float:
        ms = ctypes.c_float()
        _check(load().bvss_plan_tune(self.handle, reps, _stream(stream), ctypes.byref(ms)))
        return ms.value

    def info(self):
        kn = (_c_i32 * 7)()
        nl = _c_i64()
        _check(load().bvss_plan_info(self.handle, kn, ctypes.byref(nl)))
        return dict(scan={1: "tensor", 2: "popcount", 3: "tensor_sets_tmem", 0: "alg2"}[kn[0]],
                    cand_cta=kn[1], stages=kn[2], mq=kn[3], width_split=kn[4], batch=kn[5],
                    streams_query=kn[6], launches=nl.value)

    def set_knobs(self, scan=0, cand_cta=0, stages=0, bucket=0, batch=0, query_operand=0):
        """Pin the tuner's choices (0 = default); scan 1 = tensor-core (query sketches as the
        A operand), 2 = popcount, 3 = tensor-core (set sketches in tensor memory);
        bucket 2 = no width split; batch = query sets per internal batch; query_operand
        1 = held in shared memory where it fits, 2 = streamed through the copy ring."""
        kn = (_c_i32 * 6)(scan, cand_cta, stages, bucket, batch, query_operand)
        _check(load().bvss_plan_set_knobs(self.handle, kn))

    def close(self):
        if getattr(self, "handle", None):
            torch.cuda.synchronize(self.ix.device)
            load().bvss_plan_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bvss_query_trace(ix: Index, q_vectors: torch.Tensor, q_offsets, *, k: int, C: int,
                     A: int = 3, M: int = 1, fast: bool = False, popc_scan: bool = False,
                     alg2: bool = False, fp8: bool = False, fp8_exact: bool = False,
                     tf32: bool = False, scan_sets_tmem: bool = False, stream=None):
    """bvss_query plus every intermediate of Alg. 6, as a dict of CUDA tensors.

    Unsigned 16- and 32-bit outputs are returned in int16 / int32 tensors
    holding the same bits (view them as uint16 / uint32 in numpy)."""
    lib = load()
    off, off_p = _host_i64(q_offsets)
    nq = off.shape[0] - 1
    dev = ix.device
    vq = int(off[-1])
    t = dict(
        qpos=torch.empty((vq, ix.L), dtype=torch.int16, device=dev),
        cq=torch.empty((nq, ix.m), dtype=torch.int32, device=dev),
        sq=torch.empty((nq, ix.m // 32), dtype=torch.int32, device=dev),
        plist=torch.empty((nq, A), dtype=torch.int16, device=dev),
        h=torch.empty((nq, ix.n_sets), dtype=torch.int16, device=dev),
        cand=torch.empty((nq, C), dtype=torch.int32, device=dev),
        n_cand=torch.empty((nq,), dtype=torch.int32, device=dev),
        cand_dist=torch.empty((nq, C), dtype=torch.float32, device=dev),
    )
    tr = bvss_trace(**{name: t[name].data_ptr() for name in t})
    ids = torch.empty((nq, k), dtype=torch.int64, device=dev)
    dist = torch.empty((nq, k), dtype=torch.float32, device=dev)
    s = bvss_search(k=k, C=C, A=A, M=M,
                    flags=_search_flags(fast, popc_scan, alg2, fp8, fp8_exact, tf32, scan_sets_tmem))
    _check(lib.bvss_query_trace(ix.handle, _dptr(q_vectors), off_p, nq, ctypes.byref(s),
                                _dptr(ids), _dptr(dist), ctypes.byref(tr), _stream(stream)))
    t["ids"] = ids
    t["dist"] = dist
    return t


def bvss_encode(ix: Index, x: torch.Tensor, stream=None):
    """FlyHash codes (Def. 7) of x (n, d) on the GPU -> (pos (n, L), mask (n, m/32)).

    pos holds uint16 bits in an int16 tensor, mask uint32 bits in an int32 tensor."""
    lib = load()
    n = x.shape[0]
    pos = torch.empty((n, ix.L), dtype=torch.int16, device=x.device)
    mask = torch.empty((n, ix.m // 32), dtype=torch.int32, device=x.device)
    _check(lib.bvss_encode(ix.handle, _dptr(x), n, _dptr(pos), _dptr(mask), _stream(stream)))
    return pos, mask


def bvss_index_info(ix: Index):
    lib = load()
    p = bvss_params()
    n_sets, n_vec = _c_i64(), _c_i64()
    _check(lib.bvss_index_info(ix.handle, ctypes.byref(p), ctypes.byref(n_sets),
                               ctypes.byref(n_vec)))
    return dict(d=p.d, m=p.m, fanin=p.fanin, wta_l=p.wta_l, n_sets=n_sets.value,
                n_vectors=n_vec.value)


def bvss_get_codes(ix: Index, first: int, n: int, stream=None):
    lib = load()
    out = torch.empty((n, ix.L), dtype=torch.int16, device=ix.device)   # uint16 bits
    _check(lib.bvss_get_codes(ix.handle, first, n, _dptr(out), _stream(stream)))
    return out


def bvss_get_sketches(ix: Index, ids: torch.Tensor, stream=None):
    lib = load()
    ids = ids.to(device=ix.device, dtype=torch.int64).contiguous()
    out = torch.empty((ids.shape[0], ix.m // 32), dtype=torch.int32, device=ix.device)  # uint32 bits
    _check(lib.bvss_get_sketches(ix.handle, _dptr(ids), ids.shape[0], _dptr(out),
                                 _stream(stream)))
    return out


def bvss_get_counts(ix: Index, ids: torch.Tensor, stream=None):
    lib = load()
    ids = ids.to(device=ix.device, dtype=torch.int64).contiguous()
    out = torch.empty((ids.shape[0], ix.m), dtype=torch.uint8, device=ix.device)
    _check(lib.bvss_get_counts(ix.handle, _dptr(ids), ids.shape[0], _dptr(out),
                               _stream(stream)))
    return out


def bvss_select_noalloc(h: torch.Tensor, n_sets: int, m: int, C: int, cand=None,
                        n_cand=None, stream=None):
    """Candidate select without any GPU allocation inside the library.

    For callers that cannot call cudaMalloc (device memory fully reserved by
    another allocator, or a loop that must not synchronise the device).
    h: (n_q, h_stride) int16 CUDA tensor holding uint16 scores, 0xFFFF for
    sets outside F1.  Returns (cand (n_q, C) int32, n_cand (n_q,) int32);
    pass preallocated tensors to keep the call allocation-free end to end."""
    nq, hs = h.shape
    if cand is None:
        cand = torch.empty((nq, C), dtype=torch.int32, device=h.device)
    if n_cand is None:
        n_cand = torch.empty((nq,), dtype=torch.int32, device=h.device)
    _check(load().bvss_select_noalloc(_dptr(h), n_sets, hs, m, nq, C, _dptr(cand),
                                      _dptr(n_cand), _stream(stream)))
    return cand, n_cand


def bvss_sync(ix: Index, stream=None):
    """Wait for the stream; raise BvssError if a kernel's bounded wait gave up."""
    _check(load().bvss_sync(ix.handle, _stream(stream)))


def bvss_selftest_wait_timeout(limit_ns: int = 10_000_000) -> int:
    """Run the bounded-wait self-test; returns the status (BVSS_ETIMEOUT expected)."""
    return load().bvss_selftest_wait_timeout(limit_ns)


STAGES = ("encode", "gate", "scan", "select", "refine", "rescore", "topk")


def bvss_profile_enable(ix: Index, on: bool = True):
    _check(load().bvss_profile_enable(ix.handle, 1 if on else 0))


def bvss_profile_read(ix: Index, reset: bool = True):
    """({stage: summed ms}, timed batches, kernels they launched) since the last reset."""
    ms = (ctypes.c_double * len(STAGES))()
    nb, nl = _c_i64(), _c_i64()
    _check(load().bvss_profile_read(ix.handle, ms, ctypes.byref(nb), ctypes.byref(nl),
                                    1 if reset else 0))
    return dict(zip(STAGES, list(ms))), nb.value, nl.value


# ---- the learned projection (BioHash in place of FlyHash, Def. 7) --------------------
def bvss_build_dense(vectors: torch.Tensor, set_offsets, w: torch.Tensor, *, wta_l: int,
                     bf16: bool = False, fp8: bool = False, stream=None) -> Index:
    """Build an index whose codes come from the dense layer w (m, d) float32 (any device)."""
    lib = load()
    assert vectors.dtype == torch.float32 and vectors.is_contiguous()
    assert w.dtype == torch.float32 and w.is_contiguous()
    off, off_p = _host_i64(set_offsets)
    p = bvss_params(d=vectors.shape[1], m=w.shape[0], fanin=0, wta_l=wta_l,
                    flags=(BVSS_BUILD_BF16 if bf16 else 0) | (BVSS_BUILD_FP8 if fp8 else 0))
    h = ctypes.c_void_p()
    dev = vectors.device if vectors.is_cuda else torch.device("cuda", torch.cuda.current_device())
    with torch.cuda.device(dev):
        _check(lib.bvss_build_dense(_dptr(vectors), off_p, off.shape[0] - 1, _dptr(w),
                                    ctypes.byref(p), _stream(stream), ctypes.byref(h)))
    return Index(h, p, off.shape[0] - 1, int(off[-1]), dev)


def bvss_to_bf16(x: torch.Tensor, stream=None) -> torch.Tensor:
    out = torch.empty(x.shape, dtype=torch.bfloat16, device=x.device)
    _check(load().bvss_to_bf16(_dptr(x), x.shape[0], x.shape[1], _dptr(out), _stream(stream)))
    return out


def bvss_dense_forward(x_bf16: torch.Tensor, w_bf16: torch.Tensor, out=None, stream=None):
    """Activations (n, m) float32 of the BF16 layer on the tensor cores."""
    n, d = x_bf16.shape
    m = w_bf16.shape[0]
    if out is None:
        out = torch.empty((n, m), dtype=torch.float32, device=x_bf16.device)
    _check(load().bvss_dense_forward(_dptr(x_bf16), n, d, _dptr(w_bf16), m, _dptr(out),
                                     out.stride(0), _stream(stream)))
    return out


def bvss_learn_sync(stream=None):
    _check(load().bvss_learn_sync(_stream(stream)))


def bvss_learn_pair_grad(act_x, act_y, labels, L, temperature, scale, margin, g_x=None,
                         g_y=None, loss_sum=None, stream=None):
    """(g_x, g_y, loss_sum): the pairs' loss gradients in their activations."""
    n, m = act_x.shape
    g_x = torch.empty_like(act_x) if g_x is None else g_x
    g_y = torch.empty_like(act_y) if g_y is None else g_y
    if loss_sum is None:
        loss_sum = torch.zeros(1, dtype=torch.float64, device=act_x.device)
    _check(load().bvss_learn_pair_grad(_dptr(act_x), _dptr(act_y), act_x.stride(0),
                                       _dptr(labels), n, m, L, temperature, scale, margin,
                                       _dptr(g_x), _dptr(g_y), g_x.stride(0), _dptr(loss_sum),
                                       _stream(stream)))
    return g_x, g_y, loss_sum


def bvss_learn_weight_grad(g_x, g_y, x_bf16, y_bf16, out=None, stream=None):
    n, m = g_x.shape
    d = x_bf16.shape[1]
    out = torch.empty((m, d), dtype=torch.float32, device=g_x.device) if out is None else out
    _check(load().bvss_learn_weight_grad(_dptr(g_x), _dptr(g_y), g_x.stride(0), _dptr(x_bf16),
                                         _dptr(y_bf16), n, m, d, _dptr(out), _stream(stream)))
    return out


def bvss_learn_update(w, dw, eta, row_norm, wq_bf16=None, absmax=None, stream=None):
    """In place: w <- rows rescaled to row_norm of w - eta dw / max|dw|; returns
    (wq_bf16, absmax)."""
    m, d = w.shape
    wq_bf16 = torch.empty((m, d), dtype=torch.bfloat16, device=w.device) if wq_bf16 is None \
        else wq_bf16
    absmax = torch.empty(1, dtype=torch.float32, device=w.device) if absmax is None else absmax
    _check(load().bvss_learn_update(_dptr(w), _dptr(dw), m, d, eta, row_norm, _dptr(absmax),
                                    _dptr(wq_bf16), _stream(stream)))
    return wq_bf16, absmax


def bvss_index_rows_bf16(ix: Index, rows: torch.Tensor, out=None, stream=None):
    n = rows.shape[0]
    out = torch.empty((n, ix.d), dtype=torch.bfloat16, device=ix.device) if out is None else out
    _check(load().bvss_index_rows_bf16(ix.handle, _dptr(rows), n, _dptr(out), _stream(stream)))
    return out


def bvss_nearest_rows(ix: Index, q_vectors: torch.Tensor, q_offsets, sets: torch.Tensor,
                      stream=None):
    """(Vq, k) int64 global rows: each query vector's nearest vector in each of its query
    set's k neighbour sets."""
    off, off_p = _host_i64(q_offsets)
    nq, k = sets.shape
    rows = torch.empty((int(off[-1]), k), dtype=torch.int64, device=ix.device)
    _check(load().bvss_nearest_rows(ix.handle, _dptr(q_vectors), off_p, nq, _dptr(sets), k,
                                    _dptr(rows), _stream(stream)))
    return rows


def bvss_free(ix: Index):
    ix.close()
