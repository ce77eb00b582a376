"""The FP8 refine (BVSS_SEARCH_FP8): approximate, with a stated bound.

The FP8 form rounds every database vector and query vector to E4M3 over a
per-vector scale.  Round to nearest keeps each value within 2^-4 of itself
(relative) or, below the smallest normal, within 2^-10 of the scale, so a
vector x moves by at most e(x) = 2^-4 |x| + 2^-10 s_x sqrt(d).  Every
pairwise distance then moves by at most e(q) + e(v) (triangle inequality),
and the Hausdorff value of Def. 4 by at most the largest of those over the
pairs (max and min are 1-Lipschitz).  The kernel keeps the pair that attains
the rounded Hausdorff value and reports that pair's FP32 distance, so a
candidate's value is within 2 eps of its true Hausdorff distance, eps = max
e(q) + max e(v) plus the FP32 rounding of the GEMM form.  The boundary stage
then re-scores exactly the candidates within its band of the k-th value (by
default a 3-sigma tolerance, with BVSS_SEARCH_FP8_EXACT the rigorous bound),
so a returned distance is the exact value of its set and a returned set's true
distance is within 4 eps of the true k-th smallest among the same candidates
(the candidates themselves are exact: scan and select do not depend on the
refine).  The tests check those statements against the FP64 oracle, that the
exact band returns the oracle's ids, and that batches the FP8 copy does not
take fall back to the exact forms.
"""
import numpy as np
import pytest
import torch

from paper_2412_03301_gb300 import datagen

pytestmark = pytest.mark.gpu

GEMM_SLACK = 0.01   # distance units: sqrt of the FP32 GEMM-form rounding of d^2 (<= 4)


@pytest.fixture(scope="module")
def bv():
    from paper_2412_03301_gb300 import build, bvss
    build.build()
    bvss.load()
    return bvss


def _qerr(x):
    """Upper bound of |round_e4m3(x / s) s - x| per vector (rows of x)."""
    x = np.asarray(x, np.float64)
    s = np.abs(x).max(axis=1) / 448.0
    s[s == 0] = 1.0
    return 2.0 ** -4 * np.linalg.norm(x, axis=1) + 2.0 ** -10 * s * np.sqrt(x.shape[1])


@pytest.fixture(scope="module")
def case(bv, orc):
    w = datagen.workload(n_sets=1500, size_lo=2, size_hi=24, d=128, n_components=32,
                         n_queries=16, q_lo=1, q_hi=32, m=1024, fanin=8, seed=61)
    vec = w["vectors"].numpy()
    ix = bv.bvss_build(w["vectors"].cuda(), w["offsets"], w["proj"], wta_l=16, bf16=True, fp8=True)
    oix = orc.Index(vec, w["offsets"], w["proj"], 16)
    return w, ix, oix, _qerr(vec)


def test_fp8_distances_and_ranks_within_the_bound(bv, orc, case):
    w, ix, oix, ev = case
    k, C = 10, 300
    qv, qo = w["q_vectors"], w["q_offsets"]
    ids, dist = bv.bvss_query(ix, qv.cuda(), qo, k=k, C=C, fp8=True)
    ids, dist = ids.cpu().numpy(), dist.cpu().numpy()
    off = w["offsets"]
    for q in range(qo.shape[0] - 1):
        Q = qv[qo[q]:qo[q + 1]].numpy()
        r = orc.query(oix, Q, k=k, C=C, A=3, M=1)
        n = int((r["ids"] >= 0).sum())
        assert int((ids[q] >= 0).sum()) == n
        got = ids[q][:n].astype(np.int32)
        assert set(got.tolist()) <= set(r["cand"].tolist())        # candidates are exact
        _, _, true_d = orc.refine_topk(Q, oix.vectors, oix.set_off, got, n)
        eq = _qerr(Q).max()
        for j, sid in enumerate(got):
            rows = slice(int(off[sid]), int(off[sid + 1]))
            eps = eq + ev[rows].max() + GEMM_SLACK
            assert abs(dist[q][j] - true_d[j]) <= 2 * eps + 1e-5 * true_d[j], (q, j)
            # the boundary stage returns the set's exact value
            assert abs(dist[q][j] - true_d[j]) <= (40 + 4) * 2.0 ** -24 * true_d[j], (q, j)
            # near-optimal: within 4 eps of the true k-th smallest over the same candidates
            assert true_d[j] <= r["dist"][n - 1] + 4 * eps + 1e-5, (q, j)
        assert np.all(np.diff(dist[q][:n]) >= 0)


def test_fp8_exact_band_returns_the_oracle_top_k(bv, orc, case):
    w, ix, oix, _ = case
    qv, qo = w["q_vectors"], w["q_offsets"]
    ids, dist = bv.bvss_query(ix, qv.cuda(), qo, k=10, C=300, fp8=True, fp8_exact=True)
    for q in range(qo.shape[0] - 1):
        r = orc.query(oix, qv[qo[q]:qo[q + 1]].numpy(), k=10, C=300, A=3, M=1)
        assert ids[q].tolist() == r["ids"].tolist(), q
        fin = np.isfinite(r["dist"])
        np.testing.assert_allclose(dist[q].cpu().numpy()[fin], r["dist"][fin], rtol=3e-6)


def test_fp8_64_wide_with_the_exact_band(bv, orc, case):
    # query sets of 33-64 vectors take the 64-wide FP8 instance; with the rigorous band
    # the ids are the oracle's
    w, ix, oix, _ = case
    sizes = datagen.set_sizes(6, 33, 64, 73)
    qv = datagen.Mixture(128, 32, 61).draw_sets(sizes, 74)
    qo = datagen.offsets_from_sizes(sizes)
    ids, dist = bv.bvss_query(ix, qv.cuda(), qo, k=8, C=200, fp8=True, fp8_exact=True)
    ids8, _ = bv.bvss_query(ix, qv.cuda(), qo, k=8, C=200, fp8=True)
    for q in range(6):
        r = orc.query(oix, qv[qo[q]:qo[q + 1]].numpy(), k=8, C=200, A=3, M=1)
        assert ids[q].tolist() == r["ids"].tolist()
        np.testing.assert_allclose(dist[q].cpu().numpy(), r["dist"], rtol=3e-6)
        # the default band: approximate, but every returned set is among the candidates
        assert set(ids8[q].tolist()) <= set(r["cand"].tolist())


def test_every_tensor_core_form_at_d_2048(bv, orc):
    """At d = 2048 no form holds a 64-wide query operand in shared memory beside its ring,
    and BF16 and TF32 not even a 32-wide one: every launch streams the operand (and the
    64-wide ones run the split epilogue).  On these grid values BF16, TF32 and FP8 with
    its rigorous band must return the oracle's ids and distances; query sets of 1-64
    vectors exercise both widths."""
    w = datagen.workload(n_sets=250, size_lo=1, size_hi=12, d=2048, n_components=16,
                         n_queries=8, q_lo=1, q_hi=64, m=1024, fanin=8, seed=75)
    ix = bv.bvss_build(w["vectors"].cuda(), w["offsets"], w["proj"], wta_l=16, bf16=True,
                       fp8=True)
    oix = orc.Index(w["vectors"].numpy(), w["offsets"], w["proj"], 16)
    qv, qo = w["q_vectors"], w["q_offsets"]
    want = [orc.query(oix, qv[qo[q]:qo[q + 1]].numpy(), k=6, C=120, A=3, M=1)
            for q in range(8)]
    for kw in (dict(fast=True), dict(tf32=True), dict(fp8=True, fp8_exact=True)):
        ids, dist = bv.bvss_query(ix, qv.cuda(), qo, k=6, C=120, **kw)
        bv.bvss_sync(ix)
        for q, r in enumerate(want):
            assert ids[q].tolist() == r["ids"].tolist(), (kw, q)
            np.testing.assert_allclose(dist[q].cpu().numpy(), r["dist"], rtol=3e-6)
    ix.close()


def test_fp8_falls_back_for_wide_query_sets(bv, orc, case):
    # query sets of more than 64 vectors take the FP32 refine: exact again
    w, ix, oix, _ = case
    sizes = datagen.set_sizes(5, 65, 80, 71)
    qv = datagen.Mixture(128, 32, 61).draw_sets(sizes, 72)
    qo = datagen.offsets_from_sizes(sizes)
    ids, dist = bv.bvss_query(ix, qv.cuda(), qo, k=5, C=100, fp8=True)
    for q in range(5):
        r = orc.query(oix, qv[qo[q]:qo[q + 1]].numpy(), k=5, C=100, A=3, M=1)
        assert ids[q].tolist() == r["ids"].tolist()
        np.testing.assert_allclose(dist[q].cpu().numpy(), r["dist"], rtol=1e-5)


def test_fp8_plan_matches_query(bv, case):
    w, ix, _, _ = case
    qv, qo = w["q_vectors"], w["q_offsets"]
    nq = qo.shape[0] - 1
    plan = bv.Plan(ix, nq, int(qo[-1]), 32, k=10, C=300, fp8=True)
    plan.set_queries(qv.cuda(), qo)
    ids, dist = plan.launch()
    bv.bvss_sync(ix)
    ids_q, dist_q = bv.bvss_query(ix, qv.cuda(), qo, k=10, C=300, fp8=True)
    assert torch.equal(ids, ids_q) and torch.equal(dist, dist_q)
    plan.close()


def test_fp8_argument_checks(bv):
    w = datagen.workload(n_sets=40, size_lo=2, size_hi=4, d=64, n_components=8, n_queries=2,
                         q_lo=2, q_hi=3, m=256, fanin=4, seed=62)
    with pytest.raises(bv.BvssError) as e:   # the FP8 copy needs d % 128 == 0
        bv.bvss_build(w["vectors"].cuda(), w["offsets"], w["proj"], wta_l=8, fp8=True)
    assert e.value.code == bv.BVSS_EINVAL
    ix = bv.bvss_build(w["vectors"].cuda(), w["offsets"], w["proj"], wta_l=8, bf16=True)
    with pytest.raises(bv.BvssError) as e:   # FP8 search on an index without the copy
        bv.bvss_query(ix, w["q_vectors"].cuda(), w["q_offsets"], k=2, C=5, fp8=True)
    assert e.value.code == bv.BVSS_EINVAL
