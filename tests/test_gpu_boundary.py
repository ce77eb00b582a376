"""The exact top-k (Alg. 6 line 23 over Def. 4) for every refine form.

Off the 2^-8 grid the BF16 and FP8 copies round the vectors, the TF32 form's tensor
cores round them as they read them, and FP32 GEMM-form sums round too, so each form's
candidate values are approximate.  The
boundary stage re-scores, directly in FP32 over all pairs, every candidate
whose error interval reaches the k-th smallest upper bound, and in FP64 the
candidates that FP32 cannot order at the top k.  So every form (the FP8 form
with its rigorous band, BVSS_SEARCH_FP8_EXACT) must return
the oracle's ids (FP64 Hausdorff, ties by id) exactly, with distances within
the stated (36 + ceil(d / 32)) 2^-24 relative bound of the oracle's FP64 values.
"""
import numpy as np
import pytest
import torch

from paper_2412_03301_gb300 import datagen

pytestmark = pytest.mark.gpu

FORMS = (dict(), dict(fast=True), dict(fp8=True, fp8_exact=True), dict(tf32=True))


@pytest.fixture(scope="module")
def bv():
    from paper_2412_03301_gb300 import build, bvss
    build.build()
    bvss.load()
    return bvss


def _eta(d):
    return (36 + -(-d // 32)) * 2.0 ** -24


def _check(bv, orc, w, L, k, C, A, M, forms=FORMS):
    d = w["vectors"].shape[1]
    ix = bv.bvss_build(w["vectors"].cuda(), w["offsets"], w["proj"], wta_l=L, bf16=True,
                       fp8=True)
    oix = orc.Index(w["vectors"].numpy(), w["offsets"], w["proj"], L)
    qv, qo = w["q_vectors"], w["q_offsets"]
    want = [orc.query(oix, qv.numpy()[qo[q]:qo[q + 1]], k=k, C=C, A=A, M=M)
            for q in range(qo.shape[0] - 1)]
    for kw in forms:
        ids, dist = bv.bvss_query(ix, qv.cuda(), qo, k=k, C=C, A=A, M=M, **kw)
        bv.bvss_sync(ix)
        ids, dist = ids.cpu().numpy(), dist.cpu().numpy().astype(np.float64)
        for q, r in enumerate(want):
            assert ids[q].tolist() == r["ids"].tolist(), (kw, q, ids[q], r["ids"])
            fin = np.isfinite(r["dist"])
            err = np.abs(dist[q][fin] - r["dist"][fin])
            assert np.all(err <= _eta(d) * r["dist"][fin] + 1e-30), (kw, q, err.max())
            assert np.all(np.isinf(dist[q][~fin]))
    ix.close()


@pytest.mark.parametrize("n_sets,lo,hi,d,qlo,qhi,C,k", [
    (3000, 4, 16, 128, 4, 16, 300, 10),
    (1500, 8, 40, 256, 8, 32, 400, 25),    # rows over one 32-row pair tile, wider k
    (600, 1, 3, 128, 1, 4, 600, 7),        # tiny sets, every set a candidate
    (800, 8, 32, 384, 1, 64, 200, 10),     # the large workload's d, 32- and 64-wide sets
])
def test_every_form_returns_the_fp64_top_k_off_the_grid(bv, orc, n_sets, lo, hi, d, qlo, qhi,
                                                        C, k):
    w = datagen.workload(n_sets=n_sets, size_lo=lo, size_hi=hi, d=d, n_components=32,
                         n_queries=12, q_lo=qlo, q_hi=qhi, m=1024, fanin=8, seed=n_sets + d,
                         grid=False)
    _check(bv, orc, w, 16, k, C, 3, 1)
    _check(bv, orc, w, 16, k, min(C, 60), 2, 0)


def test_fp64_orders_what_fp32_cannot(bv, orc):
    """Single-vector sets: set 1 holds v, set 2 an exact copy of v, set 0 holds v moved
    one FP32 ulp away from the query in one coordinate (its distance larger by about
    1e-9, below FP32's resolution).  FP64 must put 1 and 2 (tied, by id) before 0."""
    rng = np.random.default_rng(81)
    d, n = 128, 400
    vec = rng.standard_normal((n, d)).astype(np.float32)
    vec /= np.linalg.norm(vec, axis=1, keepdims=True)
    qv = vec[:1].copy()
    u = rng.standard_normal(d).astype(np.float32)
    v = (qv[0] + 0.05 * u / np.linalg.norm(u)).astype(np.float32)
    c = int(np.argmax(np.abs(v - qv[0])))
    far = v.copy()
    far[c] = np.nextafter(v[c], np.float32(np.sign(v[c] - qv[0, c]) * np.inf))
    vec[0], vec[1], vec[2] = far, v, v
    w = dict(vectors=torch.from_numpy(vec), offsets=np.arange(n + 1, dtype=np.int64),
             q_vectors=torch.from_numpy(qv), q_offsets=np.array([0, 1], np.int64),
             proj=datagen.projection(d, 512, 8, seed=82))
    d_far = np.linalg.norm(far.astype(np.float64) - qv[0])
    d_v = np.linalg.norm(v.astype(np.float64) - qv[0])
    assert d_far > d_v
    r = orc.query(orc.Index(vec, w["offsets"], w["proj"], 8), qv, k=3, C=n, A=3, M=0)
    assert r["ids"].tolist() == [1, 2, 0]
    _check(bv, orc, w, 8, 3, n, 3, 0)


@pytest.mark.parametrize("bits,scale", [(8, 1.0), (10, 0.9), (8, 8.0), (6, 12.0)])
def test_grid_certificate_and_its_limits(bv, orc, bits, scale):
    """Values on a 2^-bits grid: where (N_Q + N_V)^2 < 2^(22 - 2 bits) the stage certifies
    the refine's arithmetic exact and only selects; beyond it (norms of 8 on the 2^-8 grid,
    12 on 2^-6) it re-scores the band.  Every case must give the oracle's top k."""
    w = datagen.workload(n_sets=1200, size_lo=2, size_hi=14, d=128, n_components=32,
                         n_queries=10, q_lo=2, q_hi=14, m=1024, fanin=8, seed=90 + bits,
                         grid=False)
    g = 2.0 ** bits
    for key in ("vectors", "q_vectors"):
        w[key] = (torch.round(w[key].double() * scale * g) / g).float()
    _check(bv, orc, w, 16, 10, 200, 3, 1)
