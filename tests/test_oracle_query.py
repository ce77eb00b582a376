"""Pins for the oracle's whole Alg. 6 query.

With M = 0 (every set passes the first layer) and C = N the candidate
stage keeps every set, so the result must equal exact brute-force top-k.
On tiny inputs every intermediate is re-derived with numpy.
"""
import numpy as np
import pytest
from scipy.spatial.distance import directed_hausdorff

from paper_2412_03301_gb300 import datagen


@pytest.fixture(scope="module")
def small(orc):
    w = datagen.workload(n_sets=150, size_lo=1, size_hi=8, d=24, n_components=32,
                         n_queries=6, q_lo=1, q_hi=6, m=256, fanin=6, seed=3)
    ix = orc.Index(w["vectors"].numpy(), w["offsets"], w["proj"], 12)
    return w, ix


def _haus64(Q, V):
    Q, V = Q.astype(np.float64), V.astype(np.float64)
    return max(directed_hausdorff(Q, V)[0], directed_hausdorff(V, Q)[0])


def test_full_candidate_budget_is_exact(orc, small):
    w, ix = small
    qv, qo = w["q_vectors"].numpy(), w["q_offsets"]
    for q in range(qo.shape[0] - 1):
        Q = qv[qo[q]:qo[q + 1]]
        r = orc.query(ix, Q, k=10, C=ix.n_sets, A=3, M=0)
        ids, dist = orc.bruteforce_topk(Q, ix.vectors, ix.set_off, 10)
        assert r["ids"].tolist() == ids.tolist()
        np.testing.assert_array_equal(r["dist"], dist)


def test_intermediates_by_numpy(orc, small):
    w, ix = small
    qv, qo = w["q_vectors"].numpy(), w["q_offsets"]
    m = ix.m
    for q in range(qo.shape[0] - 1):
        Q = qv[qo[q]:qo[q + 1]]
        for A, M, C in ((3, 1, 20), (1, 2, 7), (2, 1, 1000)):
            r = orc.query(ix, Q, k=5, C=C, A=A, M=M)
            cq = np.bincount(r["qpos"].astype(np.int64).ravel(), minlength=m)
            assert np.array_equal(r["cq"], cq)
            plist = np.lexsort((np.arange(m), -cq))[:A]
            assert r["plist"].tolist() == plist.tolist()
            gate = (ix.count[plist] >= M).any(axis=0)
            assert np.array_equal(r["gate"].astype(bool), gate)
            h = np.bitwise_count(ix.sketch ^ r["sq"][None]).sum(axis=1)
            assert np.array_equal(r["h"][gate], h[gate])
            idx = np.flatnonzero(gate)
            order = idx[np.lexsort((idx, h[idx]))][:C]
            assert r["cand"].tolist() == sorted(order.tolist())
            d = np.array([_haus64(Q, ix.vectors[ix.set_off[i]:ix.set_off[i + 1]])
                          for i in r["cand"]])
            np.testing.assert_allclose(r["cand_dist"], d, rtol=1e-12, atol=0)
            o = np.lexsort((r["cand"], d))[:5]
            want = [int(r["cand"][j]) for j in o] + [-1] * (5 - len(o))
            assert r["ids"].tolist() == want


def test_threaded_index_build_is_identical(orc):
    """Encoding the database in chunks on host threads gives the same index."""
    from paper_2412_03301_gb300 import datagen
    w = datagen.workload(n_sets=300, size_lo=1, size_hi=9, d=32, n_components=16,
                         n_queries=1, q_lo=1, q_hi=2, m=512, fanin=4, seed=71)
    a = orc.Index(w["vectors"].numpy(), w["offsets"], w["proj"], 12)
    b = orc.Index(w["vectors"].numpy(), w["offsets"], w["proj"], 12, threads=4)
    for name in ("pos", "mask", "sketch", "count"):
        assert np.array_equal(getattr(a, name), getattr(b, name)), name
