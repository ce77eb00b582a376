"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Codes, filters, query filters, gate, Hamming scores and candidate lists are
compared bit for bit; Hausdorff distances within 1e-5 relative of the FP64
oracle (on these grid-valued inputs the FP32 sums are exact, so the only
difference is the final square root's rounding); result ids exactly.
"""
import numpy as np
import pytest
import torch

from paper_2412_03301_gb300 import datagen

pytestmark = pytest.mark.gpu

RTOL = 1e-5


def _np(t, dtype=None):
    a = t.detach().cpu().numpy()
    return a.view(dtype) if dtype is not None else a


@pytest.fixture(scope="module")
def bv():
    from paper_2412_03301_gb300 import build, bvss
    build.build()
    bvss.load()
    return bvss


def _workload(n_sets, lo, hi, d, K, nq, qlo, qhi, m, F, seed):
    return datagen.workload(n_sets=n_sets, size_lo=lo, size_hi=hi, d=d, n_components=K,
                            n_queries=nq, q_lo=qlo, q_hi=qhi, m=m, fanin=F, seed=seed)


class Case:
    """A database built both ways: the CUDA index and the oracle index."""

    def __init__(self, bv, orc, w, L, bf16=False):
        self.w = w
        self.L = L
        self.vec = w["vectors"].numpy()
        self.qvec = w["q_vectors"].numpy()
        self.ix = bv.bvss_build(w["vectors"].cuda(), w["offsets"], w["proj"], wta_l=L, bf16=bf16)
        self.orc_ix = orc.Index(self.vec, w["offsets"], w["proj"], L)
        self.qv_cuda = w["q_vectors"].cuda()


@pytest.fixture(scope="module")
def small(bv, orc):
    s = datagen.SMALL
    w = _workload(s["n_sets"], s["size_lo"], s["size_hi"], s["d"], s["n_components"],
                  s["n_queries"], s["q_lo"], s["q_hi"], s["m"], s["fanin"], seed=0)
    return Case(bv, orc, w, s["L"])


def test_database_codes(bv, small):
    got = _np(bv.bvss_get_codes(small.ix, 0, small.ix.n_vectors), np.uint16)
    assert np.array_equal(got, small.orc_ix.pos)
    pos, mask = bv.bvss_encode(small.ix, torch.from_numpy(small.vec[:3000]).cuda())
    assert np.array_equal(_np(pos, np.uint16), small.orc_ix.pos[:3000])
    assert np.array_equal(_np(mask, np.uint32), small.orc_ix.mask[:3000])


def test_database_filters(bv, small):
    ids = torch.arange(small.ix.n_sets)
    sk = _np(bv.bvss_get_sketches(small.ix, ids), np.uint32)
    assert np.array_equal(sk, small.orc_ix.sketch)
    cnt = _np(bv.bvss_get_counts(small.ix, ids))
    assert np.array_equal(cnt, small.orc_ix.count.T)


def _check_query(bv, orc, case, k, C, A, M, nq=None, fast=False, popc_scan=False, tf32=False):
    w = case.w
    qo = w["q_offsets"] if nq is None else w["q_offsets"][:nq + 1]
    nq = qo.shape[0] - 1
    t = bv.bvss_query_trace(case.ix, case.qv_cuda, qo, k=k, C=C, A=A, M=M, fast=fast,
                            popc_scan=popc_scan, tf32=tf32)
    torch.cuda.synchronize()
    qpos = _np(t["qpos"], np.uint16)
    h = _np(t["h"], np.uint16)
    cand = _np(t["cand"])
    ncand = _np(t["n_cand"])
    cdist = _np(t["cand_dist"])
    ids, dist = _np(t["ids"]), _np(t["dist"])
    for q in range(nq):
        Q = case.qvec[qo[q]:qo[q + 1]]
        r = orc.query(case.orc_ix, Q, k=k, C=C, A=A, M=M)
        assert np.array_equal(qpos[qo[q]:qo[q + 1]], r["qpos"]), q
        assert np.array_equal(_np(t["cq"])[q], r["cq"]), q
        assert np.array_equal(_np(t["sq"], np.uint32)[q], r["sq"]), q
        assert np.array_equal(_np(t["plist"], np.uint16)[q], r["plist"]), q
        want_h = np.where(r["gate"] == 1, r["h"], 0xFFFF)
        assert np.array_equal(h[q].astype(np.int64), want_h.astype(np.int64)), q
        n = int(ncand[q])
        assert n == r["cand"].shape[0], q
        assert np.array_equal(cand[q, :n], r["cand"]), q
        assert np.all(cand[q, n:] == -1)
        np.testing.assert_allclose(cdist[q, :n], r["cand_dist"], rtol=RTOL, atol=0)
        assert np.all(np.isinf(cdist[q, n:]))
        assert ids[q].tolist() == r["ids"].tolist(), q
        fin = np.isfinite(r["dist"])
        np.testing.assert_allclose(dist[q][fin], r["dist"][fin], rtol=RTOL, atol=0)
        assert np.all(np.isinf(dist[q][~fin]))


def test_query_parity_default(bv, orc, small):
    s = datagen.SMALL
    _check_query(bv, orc, small, k=s["k"], C=s["C"], A=3, M=1)


def test_query_parity_popcount_scan(bv, orc, small):
    """The CUDA-core popcount scan (gated sets only) against the oracle."""
    s = datagen.SMALL
    _check_query(bv, orc, small, k=s["k"], C=s["C"], A=3, M=1, popc_scan=True)
    _check_query(bv, orc, small, k=10, C=50, A=2, M=0, nq=20, popc_scan=True)


@pytest.mark.parametrize("n_sets,nq,m,L,A,M", [
    (1000, 300, 4096, 64, 3, 1),     # ragged set tiles, three query blocks (last ragged)
    (257, 129, 128, 8, 2, 1),        # one K-block, one set past a tile, one query past a block
    (600, 40, 8192, 100, 5, 0),      # every set passes layer 1
    (600, 40, 2048, 32, 3, 300),     # no set passes layer 1
    (300, 1, 1024, 16, 1, 2),        # a single query
])
def test_scan_forms_agree(bv, orc, n_sets, nq, m, L, A, M):
    """Both tensor-core scans (all pairs, masked by layer 1) and the popcount scan give
    the same h bit for bit; the default form also matches the oracle on a sample."""
    w = _workload(n_sets, 3, 12, 32, 16, nq, 2, 9, m, 4, seed=n_sets + nq)
    ix = bv.bvss_build(w["vectors"].cuda(), w["offsets"], w["proj"], wta_l=L)
    qv = w["q_vectors"].cuda()
    C = min(50, n_sets)
    a = bv.bvss_query_trace(ix, qv, w["q_offsets"], k=5, C=C, A=A, M=M)
    b = bv.bvss_query_trace(ix, qv, w["q_offsets"], k=5, C=C, A=A, M=M, popc_scan=True)
    c = bv.bvss_query_trace(ix, qv, w["q_offsets"], k=5, C=C, A=A, M=M, scan_sets_tmem=True)
    torch.cuda.synchronize()
    ha, hb = _np(a["h"], np.uint16), _np(b["h"], np.uint16)
    assert np.array_equal(ha, hb)
    assert np.array_equal(ha, _np(c["h"], np.uint16))
    assert torch.equal(a["ids"], b["ids"]) and torch.equal(a["dist"], b["dist"])
    assert torch.equal(a["ids"], c["ids"]) and torch.equal(a["dist"], c["dist"])
    oix = orc.Index(w["vectors"].numpy(), w["offsets"], w["proj"], L)
    qo = w["q_offsets"]
    for q in sorted({0, nq // 2, nq - 1}):
        r = orc.query(oix, w["q_vectors"].numpy()[qo[q]:qo[q + 1]], k=5, C=C, A=A, M=M)
        want = np.where(r["gate"] == 1, r["h"], 0xFFFF)
        assert np.array_equal(ha[q].astype(np.int64), want.astype(np.int64)), q


def test_profile_stages_and_launch_count(bv, small):
    """The profiler sees every stage and counts the kernels each form launches:
    encode, prep, gate, [FP8 query operand], scan, [select bound], 5 select kernels,
    refine, [re-score], and the boundary stage (exact re-score near the k-th, top-k)."""
    w = small.w
    qv = small.qv_cuda
    for popc, want in ((False, 13), (True, 11)):
        bv.bvss_profile_enable(small.ix, True)
        bv.bvss_profile_read(small.ix, reset=True)
        bv.bvss_query(small.ix, qv, w["q_offsets"], k=10, C=200, A=3, M=1, popc_scan=popc)
        ms, nb, nl = bv.bvss_profile_read(small.ix, reset=True)
        bv.bvss_profile_enable(small.ix, False)
        assert nb == 1 and nl == want
        assert set(ms) == set(bv.STAGES) and ms["scan"] > 0 and ms["refine"] > 0
        assert ms["rescore"] == pytest.approx(0.0, abs=0.05)


def test_query_results_without_trace_match(bv, small):
    s = datagen.SMALL
    w = small.w
    t = bv.bvss_query_trace(small.ix, small.qv_cuda, w["q_offsets"], k=10, C=s["C"], A=3, M=1)
    ids, dist = bv.bvss_query(small.ix, small.qv_cuda, w["q_offsets"], k=10, C=s["C"], A=3, M=1)
    assert torch.equal(ids, t["ids"]) and torch.equal(dist, t["dist"])
    # host buffers in and out give the same answer
    hq = w["q_vectors"].pin_memory()
    hi = torch.empty_like(ids, device="cpu").pin_memory()
    hd = torch.empty_like(dist, device="cpu").pin_memory()
    bv.bvss_query(small.ix, hq, w["q_offsets"], k=10, C=s["C"], A=3, M=1, out_ids=hi,
                  out_dist=hd)
    assert torch.equal(hi, ids.cpu()) and torch.equal(hd, dist.cpu())


@pytest.mark.parametrize("C,A,M", [(1, 3, 1), (10, 3, 1), (100, 3, 0), (157, 3, 1), (158, 3, 0),
                                   (500, 1, 1), (40, 2, 2)])
def test_select_skips_blocks_exactly(bv, orc, C, A, M):
    # 20,000 sets = 157 blocks of 128: with C below the number of blocks in F1 the select
    # reads only blocks whose minimum score can reach the threshold; the candidate lists
    # must still equal the oracle's (ties at the threshold broken by id), and the
    # popcount scan (no block minima, every block read) must agree
    w = _workload(20000, 2, 6, 64, 16, 6, 2, 8, 512, 8, seed=27)
    case = Case(bv, orc, w, 8)
    _check_query(bv, orc, case, k=1, C=C, A=A, M=M)
    ta = bv.bvss_query_trace(case.ix, case.qv_cuda, w["q_offsets"], k=1, C=C, A=A, M=M)
    tb = bv.bvss_query_trace(case.ix, case.qv_cuda, w["q_offsets"], k=1, C=C, A=A, M=M,
                             popc_scan=True)
    assert torch.equal(ta["cand"], tb["cand"]) and torch.equal(ta["n_cand"], tb["n_cand"])


@pytest.mark.parametrize("A,M,C", [(1, 1, 200), (3, 0, 200), (3, 2, 50), (32, 1, 200),
                                   (3, 300, 200), (3, 1, 2000), (2, 1, 10)])
def test_query_parity_knobs(bv, orc, small, A, M, C):
    _check_query(bv, orc, small, k=10, C=C, A=A, M=M, nq=25)


def test_edge_shapes(bv, orc):
    """Single-vector sets and queries, duplicate sets, a ragged set count, m = 128."""
    w = _workload(77, 1, 3, 16, 8, 9, 1, 4, 128, 3, seed=4)
    # set 5 duplicates set 2 exactly, so their distances tie and ids decide
    off = w["offsets"]
    vec = w["vectors"].clone()
    n2 = off[3] - off[2]
    sizes = np.diff(off)
    sizes[5] = n2
    off2 = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    parts = [vec[off[i]:off[i + 1]] if i != 5 else vec[off[2]:off[3]] for i in range(77)]
    w["vectors"] = torch.cat(parts).contiguous()
    w["offsets"] = off2
    case = Case(bv, orc, w, 5)
    for A, M, C, k in ((3, 1, 20, 5), (5, 0, 77, 10), (1, 2, 8, 8), (2, 1, 100, 3)):
        _check_query(bv, orc, case, k=k, C=C, A=A, M=M)


def test_large_code_length(bv, orc):
    """m = 8192 (two sketch chunks per lane) and L = 200 with fan-in 1."""
    w = _workload(300, 2, 6, 64, 16, 6, 2, 5, 8192, 1, seed=6)
    case = Case(bv, orc, w, 200)
    got = _np(bv.bvss_get_codes(case.ix, 0, case.ix.n_vectors), np.uint16)
    assert np.array_equal(got, case.orc_ix.pos)
    _check_query(bv, orc, case, k=7, C=40, A=4, M=1)


def test_invalid_query_arguments(bv, small):
    w = small.w
    for kw in (dict(k=0, C=10), dict(k=20, C=10), dict(k=5, C=10, A=0),
               dict(k=5, C=10, A=33), dict(k=5, C=10, M=-1), dict(k=5, C=20000)):
        with pytest.raises(bv.BvssError) as e:
            bv.bvss_query(small.ix, small.qv_cuda, w["q_offsets"], **kw)
        assert e.value.code == bv.BVSS_EINVAL
    bad = w["q_offsets"].copy()
    bad[3] = bad[2]
    with pytest.raises(bv.BvssError):
        bv.bvss_query(small.ix, small.qv_cuda, bad, k=5, C=10)


def test_nonfinite_database_rejected(bv):
    x = torch.zeros(8, 8, device="cuda")
    x[3, 2] = float("nan")
    proj = datagen.projection(8, 128, 2, seed=1)
    with pytest.raises(bv.BvssError) as e:
        bv.bvss_build(x, np.array([0, 4, 8]), proj, wta_l=4)
    assert e.value.code == bv.BVSS_EINVAL


@pytest.mark.parametrize("qlo,qhi,d", [(33, 64, 64), (65, 100, 32), (3, 9, 1024), (1, 40, 516)])
def test_refine_paths(bv, orc, qlo, qhi, d):
    """Query sets over one and two tiles of 32 query vectors in the TMA-staged
    refine, and the general refine it falls back to (more than 64 query
    vectors, or rows too wide for its shared-memory stages)."""
    w = _workload(120, 2, 40, d, 16, 6, qlo, qhi, 256, 4, seed=9)
    case = Case(bv, orc, w, 8)
    _check_query(bv, orc, case, k=6, C=90, A=3, M=1)


def test_bounded_wait_reports_timeout(bv, small):
    """A kernel waits on an mbarrier nothing completes; its 10 ms limit must
    run out, the status must say so, and the context must stay usable."""
    assert bv.bvss_selftest_wait_timeout(10_000_000) == bv.BVSS_ETIMEOUT
    assert "gave up" in bv.bvss_last_error()
    w = small.w
    ids, _ = bv.bvss_query(small.ix, small.qv_cuda, w["q_offsets"], k=5, C=50)
    bv.bvss_sync(small.ix)
    assert ids.shape == (w["q_offsets"].shape[0] - 1, 5)


@pytest.mark.parametrize("m", [16384, 32768])
def test_longest_codes(bv, orc, m):
    """Sketches long enough that the scan stages 64- or 32-set tiles."""
    w = _workload(70, 1, 4, 32, 8, 4, 1, 4, m, 8, seed=12)
    case = Case(bv, orc, w, 40)
    _check_query(bv, orc, case, k=5, C=30, A=3, M=1)


# ---- fast form: tensor-core refine from BF16 vectors --------------------------------
# On grid-valued inputs BF16 holds every value exactly and the FP32 tensor-core
# accumulation is exact, so the fast form must match the oracle like the plain one.

@pytest.mark.parametrize("n_sets,lo,hi,d,qlo,qhi,C,seed", [
    (2000, 4, 16, 128, 4, 16, 200, 0),     # the small workload's shapes
    (3000, 8, 32, 384, 8, 32, 1000, 13),   # the large workload's shapes, 8 CTAs per query
    (300, 1, 3, 64, 1, 5, 300, 14),        # one 64-dim block, tiny sets, C > |F1|
    (500, 20, 140, 192, 2, 32, 150, 15),   # sets longer than one 128-row tile
    (3000, 1, 1, 64, 1, 3, 1500, 21),      # one-row sets: 128 candidates finish per tile
    (400, 2, 6, 1024, 2, 8, 300, 22),      # d = 1024: the shallowest stage ring
    (600, 1, 128, 768, 1, 64, 400, 23),    # the serving load's d and sizes: 64-wide refine
    (500, 8, 32, 384, 33, 64, 700, 24),    # every query set wider than 32
    (300, 20, 140, 192, 60, 64, 150, 25),  # long sets and wide query sets together
    (200, 2, 20, 1024, 33, 64, 200, 26),   # d = 1024, 64 wide: the query operand streamed
    (300, 1, 40, 1024, 1, 64, 250, 27),    # streamed, split by width (32- and 64-wide)
])
def test_fast_refine_parity(bv, orc, n_sets, lo, hi, d, qlo, qhi, C, seed):
    w = _workload(n_sets, lo, hi, d, 32, 12, qlo, qhi, 1024, 8, seed=seed)
    case = Case(bv, orc, w, 24, bf16=True)
    _check_query(bv, orc, case, k=10, C=C, A=3, M=1, fast=True)
    _check_query(bv, orc, case, k=10, C=C, A=2, M=0, nq=4, fast=True)


# ---- TF32 form: tensor-core refine from the FP32 vectors read as TF32 ----------------
# TF32 holds every value on the 2^-8 grid (at most 9 significant bits here), so this form
# too is exact on grid inputs and must match the oracle like the plain one.

@pytest.mark.parametrize("n_sets,lo,hi,d,qlo,qhi,C,seed", [
    (2000, 4, 16, 128, 4, 16, 200, 0),     # the small workload's shapes
    (3000, 8, 32, 384, 8, 32, 1000, 13),   # the large workload's shapes, 8 CTAs per query
    (300, 1, 3, 32, 1, 5, 300, 14),        # one 32-dim block, tiny sets, C > |F1|
    (500, 20, 140, 160, 2, 32, 150, 15),   # sets longer than one 128-row tile, odd K-blocks
    (3000, 1, 1, 64, 1, 3, 1500, 21),      # one-row sets: 128 candidates finish per tile
    (400, 2, 6, 512, 2, 8, 300, 22),       # the widest rows the 32-wide ring takes
    (500, 8, 32, 384, 1, 64, 700, 24),     # mixed widths: the 32- and 64-wide instances
    (300, 20, 140, 192, 60, 64, 150, 25),  # long sets and wide query sets together
    (300, 2, 12, 768, 2, 16, 200, 28),     # d = 768: the query operand streamed (32-wide)
    (200, 1, 40, 1024, 1, 64, 250, 29),    # d = 1024, streamed, split by width
])
def test_tf32_refine_parity(bv, orc, n_sets, lo, hi, d, qlo, qhi, C, seed):
    w = _workload(n_sets, lo, hi, d, 32, 12, qlo, qhi, 1024, 8, seed=seed)
    case = Case(bv, orc, w, 24)
    _check_query(bv, orc, case, k=10, C=C, A=3, M=1, tf32=True)
    _check_query(bv, orc, case, k=10, C=C, A=2, M=0, nq=4, tf32=True)


def test_tf32_form_falls_back(bv, orc):
    # shapes the TF32 refine does not take run the CUDA-core FP32 refine: d % 32 != 0,
    # query sets over 64 vectors
    for n_sets, d, qlo, qhi, seed in ((100, 48, 2, 6, 26), (100, 64, 65, 80, 28)):
        w = _workload(n_sets, 2, 8, d, 16, 4, qlo, qhi, 256, 4, seed=seed)
        case = Case(bv, orc, w, 8)
        _check_query(bv, orc, case, k=5, C=40, A=3, M=1, tf32=True)


def test_fast_form_falls_back_and_validates(bv, orc):
    # query sets of 33-64 vectors take the 64-wide tensor-core refine, larger ones the
    # CUDA-core FP32 refine
    for qlo, qhi, seed in ((33, 50, 16), (40, 64, 18), (65, 90, 19)):
        w = _workload(150, 2, 10, 128, 16, 5, qlo, qhi, 512, 8, seed=seed)
        case = Case(bv, orc, w, 16, bf16=True)
        _check_query(bv, orc, case, k=5, C=60, A=3, M=1, fast=True)
    # the fast form needs the BF16 copy, which needs d % 64 == 0
    w2 = _workload(50, 2, 4, 48, 8, 3, 2, 4, 256, 4, seed=17)
    ix = bv.bvss_build(w2["vectors"].cuda(), w2["offsets"], w2["proj"], wta_l=8)
    with pytest.raises(bv.BvssError) as e:
        bv.bvss_query(ix, w2["q_vectors"].cuda(), w2["q_offsets"], k=3, C=10, fast=True)
    assert e.value.code == bv.BVSS_EINVAL
    with pytest.raises(bv.BvssError) as e:
        bv.bvss_build(w2["vectors"].cuda(), w2["offsets"], w2["proj"], wta_l=8, bf16=True)
    assert e.value.code == bv.BVSS_EINVAL


def _check_alg2(bv, orc, case, k, C, nq=None, fast=False):
    """The plain BioVSS search (Alg. 2) against the oracle: Haus^H of every
    set bit for bit, the candidates, their distances and the top-k."""
    w = case.w
    qo = w["q_offsets"] if nq is None else w["q_offsets"][:nq + 1]
    nq = qo.shape[0] - 1
    t = bv.bvss_query_trace(case.ix, case.qv_cuda, qo, k=k, C=C, fast=fast, alg2=True)
    torch.cuda.synchronize()
    qpos = _np(t["qpos"], np.uint16)
    h = _np(t["h"], np.uint16)
    cand, ncand, cdist = _np(t["cand"]), _np(t["n_cand"]), _np(t["cand_dist"])
    ids, dist = _np(t["ids"]), _np(t["dist"])
    for q in range(nq):
        Q = case.qvec[qo[q]:qo[q + 1]]
        r = orc.query_alg2(case.orc_ix, Q, k=k, C=C)
        assert np.array_equal(qpos[qo[q]:qo[q + 1]], r["qpos"]), q
        assert np.array_equal(h[q].astype(np.int64), r["score"].astype(np.int64)), q
        n = int(ncand[q])
        assert n == r["cand"].shape[0], q
        assert np.array_equal(cand[q, :n], r["cand"]), q
        np.testing.assert_allclose(cdist[q, :n], r["cand_dist"], rtol=RTOL, atol=0)
        assert ids[q].tolist() == r["ids"].tolist(), q
        fin = np.isfinite(r["dist"])
        np.testing.assert_allclose(dist[q][fin], r["dist"][fin], rtol=RTOL, atol=0)


def test_alg2_parity(bv, orc, small):
    s = datagen.SMALL
    _check_alg2(bv, orc, small, k=s["k"], C=s["C"], nq=40)
    _check_alg2(bv, orc, small, k=10, C=small.ix.n_sets, nq=5)   # every set refined


def test_alg2_edges_and_long_codes(bv, orc):
    # one-vector sets and queries, m = 128, L = 5 (the smallest counter)
    w = _workload(90, 1, 3, 16, 8, 7, 1, 4, 128, 3, seed=31)
    case = Case(bv, orc, w, 5)
    _check_alg2(bv, orc, case, k=5, C=30)
    # L = 200 on m = 8192: eight counter planes
    w = _workload(120, 2, 6, 64, 16, 5, 2, 9, 8192, 1, seed=32)
    case = Case(bv, orc, w, 200)
    _check_alg2(bv, orc, case, k=7, C=40)
    # L = 64 (four carry-save groups, seven planes), sets of more than 32 rows (several
    # row chunks per set) and query sets of up to 32 vectors
    w = _workload(300, 20, 45, 64, 16, 6, 20, 32, 2048, 8, seed=35)
    case = Case(bv, orc, w, 64)
    _check_alg2(bv, orc, case, k=6, C=50)


def test_alg2_with_fast_refine_and_limits(bv, orc):
    w = _workload(800, 4, 20, 128, 32, 8, 3, 32, 1024, 8, seed=33)
    case = Case(bv, orc, w, 24, bf16=True)
    _check_alg2(bv, orc, case, k=10, C=300, fast=True)
    # Alg. 2 scoring holds one bit per query vector: sets of 33 vectors are refused
    w2 = _workload(50, 2, 4, 32, 8, 2, 33, 34, 256, 4, seed=34)
    ix = bv.bvss_build(w2["vectors"].cuda(), w2["offsets"], w2["proj"], wta_l=8)
    with pytest.raises(bv.BvssError) as e:
        bv.bvss_query(ix, w2["q_vectors"].cuda(), w2["q_offsets"], k=3, C=10, alg2=True)
    assert e.value.code == bv.BVSS_EINVAL
