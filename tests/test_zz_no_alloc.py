"""bvss_select_noalloc: the candidate select for callers that cannot allocate.

Some programs cannot let a library call cudaMalloc: their GPU memory is
already reserved in full by another framework's caching allocator, or they
run a serving loop that must never hit cudaMalloc / cudaFree and the device
synchronisation those can cause.  bvss_select_noalloc serves them with a
fixed scratch array compiled into the library.  This test calls it through
the C ABI, twice in a row on different inputs (and once more on the first
input), and checks each result against the candidate lists the regular query
path (bvss_query_trace) produced for the same Hamming scores: ids and counts
must match exactly, as for every other integer output of the path.

The file name makes pytest collect it last; it builds everything it needs,
so it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2412_03301_gb300 import datagen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    from paper_2412_03301_gb300 import build, bvss
    build.build()
    lib = bvss.load()
    s = datagen.SMALL
    w = datagen.workload(n_sets=s["n_sets"], size_lo=s["size_lo"], size_hi=s["size_hi"],
                         d=s["d"], n_components=s["n_components"], n_queries=s["n_queries"],
                         q_lo=s["q_lo"], q_hi=s["q_hi"], m=s["m"], fanin=s["fanin"], seed=0)
    ix = bvss.bvss_build(w["vectors"].cuda(), w["offsets"], w["proj"], wta_l=s["L"])
    yield bvss, lib, ix, w
    ix.close()


def _trace(bvss, ix, w, q0, nq, C, M):
    qo = w["q_offsets"][q0:q0 + nq + 1] - w["q_offsets"][q0]
    qv = w["q_vectors"][w["q_offsets"][q0]:w["q_offsets"][q0 + nq]].cuda()
    return bvss.bvss_query_trace(ix, qv, qo, k=10, C=C, A=3, M=M)


def _padded(h, stride):
    out = torch.full((h.shape[0], stride), -1, dtype=torch.int16, device=h.device)
    out[:, :h.shape[1]] = h
    return out


def _call(lib, h, n_sets, m, C, cand, n_cand):
    rc = lib.bvss_select_noalloc(ctypes.c_void_p(h.data_ptr()), n_sets, h.shape[1], m,
                                 h.shape[0], C, ctypes.c_void_p(cand.data_ptr()),
                                 ctypes.c_void_p(n_cand.data_ptr()),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return rc


def test_two_calls_in_a_row_match_the_query_path(setup):
    bvss, lib, ix, w = setup
    n, m = ix.n_sets, ix.m
    t1 = _trace(bvss, ix, w, 0, 20, C=200, M=1)
    t2 = _trace(bvss, ix, w, 40, 32, C=150, M=0)
    torch.cuda.synchronize()
    h1, h2 = _padded(t1["h"], 2048), _padded(t2["h"], 2056)
    cand1 = torch.full((20, 200), 7, dtype=torch.int32, device="cuda")
    cnt1 = torch.zeros(20, dtype=torch.int32, device="cuda")
    cand2 = torch.full((32, 150), 7, dtype=torch.int32, device="cuda")
    cnt2 = torch.zeros(32, dtype=torch.int32, device="cuda")
    assert _call(lib, h1, n, m, 200, cand1, cnt1) == 0, bvss.bvss_last_error()
    assert torch.equal(cand1, t1["cand"]) and torch.equal(cnt1, t1["n_cand"])
    assert _call(lib, h2, n, m, 150, cand2, cnt2) == 0, bvss.bvss_last_error()
    assert torch.equal(cand2, t2["cand"]) and torch.equal(cnt2, t2["n_cand"])
    # the array keeps the previous call's contents; a repeat must not see them
    cand1.fill_(7)
    assert _call(lib, h1, n, m, 200, cand1, cnt1) == 0, bvss.bvss_last_error()
    assert torch.equal(cand1, t1["cand"]) and torch.equal(cnt1, t1["n_cand"])


def test_sizes_beyond_the_limits_are_rejected(setup):
    bvss, lib, ix, w = setup
    h = torch.zeros((33, 2048), dtype=torch.int16, device="cuda")
    cand = torch.zeros((33, 10), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(33, dtype=torch.int32, device="cuda")
    assert _call(lib, h, 2000, 2048, 10, cand, cnt) == bvss.BVSS_EINVAL
    assert b"n_queries" in lib.bvss_last_error()
    h = h[:4]
    assert _call(lib, h, 2000, 16384, 10, cand, cnt) == bvss.BVSS_EINVAL
    assert b"m = 16384" in lib.bvss_last_error()


def _synthetic_h(rng, n_q, n_sets, stride, m, p_out, p_above):
    """Seeded scores in 0..m with many ties, some 0xFFFF (outside F1) and some
    values in (m, 0xFFFE] (also outside F1 by the entry point's contract)."""
    h = rng.integers(0, m + 1, size=(n_q, n_sets)).astype(np.int64)
    u = rng.random((n_q, n_sets))
    h[u < p_out] = 0xFFFF
    above = (u >= p_out) & (u < p_out + p_above)
    h[above] = rng.integers(m + 1, 0xFFFF, size=int(above.sum()))
    full = np.full((n_q, stride), 0xFFFF, np.int64)
    full[:, :n_sets] = h
    return h, torch.from_numpy(full.astype(np.uint16).view(np.int16)).cuda()


def test_several_chunks_match_the_oracle_heap(setup, orc):
    """50,000 sets span four of the select's 16,384-set chunks, so the fixed
    array's per-range records, the cross-chunk tie ranks and the output slots
    of later chunks are all used; the oracle's literal bounded heap (Alg. 6
    lines 10-18) over the same scores decides the expected lists."""
    bvss, lib, ix, w = setup
    rng = np.random.default_rng(11)
    n_sets, stride = 50_000, 50_008
    for m, n_q, C in ((64, 5, 1000), (4096, 3, 16384)):
        h, dh = _synthetic_h(rng, n_q, n_sets, stride, m, 0.1, 0.02)
        cand = torch.full((n_q, C), 7, dtype=torch.int32, device="cuda")
        cnt = torch.zeros(n_q, dtype=torch.int32, device="cuda")
        for _ in range(2):   # two calls in a row on the same array
            cand.fill_(7)
            assert _call(lib, dh, n_sets, m, C, cand, cnt) == 0, bvss.bvss_last_error()
            got, got_n = cand.cpu().numpy(), cnt.cpu().numpy()
            for q in range(n_q):
                gate = (h[q] <= m).astype(np.uint8)
                ref = orc.heap_select(h[q].astype(np.int32), gate, C)
                assert got_n[q] == ref.shape[0]
                assert np.array_equal(got[q, :ref.shape[0]], ref)
                assert np.all(got[q, ref.shape[0]:] == -1)


def test_bad_layouts_are_rejected(setup):
    bvss, lib, ix, w = setup
    cand = torch.zeros((2, 10), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(2, dtype=torch.int32, device="cuda")
    h = torch.zeros((2, 2056), dtype=torch.int16, device="cuda")
    # more sets than the array's per-chunk records cover
    rc = lib.bvss_select_noalloc(ctypes.c_void_p(h.data_ptr()), 16777217, 16777224, 64, 2, 10,
                                 ctypes.c_void_p(cand.data_ptr()),
                                 ctypes.c_void_p(cnt.data_ptr()), None)
    assert rc == bvss.BVSS_EINVAL and b"n_sets" in lib.bvss_last_error()
    # a row stride that is not a multiple of 8 scores
    rc = lib.bvss_select_noalloc(ctypes.c_void_p(h.data_ptr()), 2000, 2052, 64, 2, 10,
                                 ctypes.c_void_p(cand.data_ptr()),
                                 ctypes.c_void_p(cnt.data_ptr()), None)
    assert rc == bvss.BVSS_EINVAL and b"h_stride" in lib.bvss_last_error()
    # h not on a 16-byte boundary
    rc = lib.bvss_select_noalloc(ctypes.c_void_p(h.data_ptr() + 2), 2000, 2048, 64, 2, 10,
                                 ctypes.c_void_p(cand.data_ptr()),
                                 ctypes.c_void_p(cnt.data_ptr()), None)
    assert rc == bvss.BVSS_EINVAL and b"aligned" in lib.bvss_last_error()
    torch.cuda.synchronize()
