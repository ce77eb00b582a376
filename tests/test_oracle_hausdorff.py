"""Pins for the oracle's Hausdorff distance (Def. 4) and exact top-k.

The expected values come from the paper's printed examples (tests/golden),
from scipy's independent directed-Hausdorff routine, from the unit-vector
similarity form stated in the paper's assumptions, and from the metric
axioms.
"""
import json
import os

import numpy as np
import pytest
from scipy.spatial.distance import directed_hausdorff

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hausdorff_paper_examples.json")


def _realise(rows):
    """2-D points X (one per row) and Q = {Q1, Q2} with |X_r - Q_c| = rows[r][c].

    Q1 = (0, 0), Q2 = (s, 0) with s inside every row's triangle interval.
    """
    rows = np.asarray(rows, np.float64)
    lo = np.max(np.abs(rows[:, 0] - rows[:, 1]))
    hi = np.min(rows[:, 0] + rows[:, 1])
    assert lo <= hi
    s = 0.5 * (lo + hi)
    X = []
    for d0, d1 in rows:
        x = (d0 * d0 - d1 * d1 + s * s) / (2 * s)
        X.append((x, np.sqrt(max(d0 * d0 - x * x, 0.0))))
    return np.array(X), np.array([(0.0, 0.0), (s, 0.0)])


def test_paper_distance_matrices(orc):
    g = json.load(open(GOLDEN))
    for case in g["matrix_cases"]:
        X, Q = _realise(case["rows"])
        Xf, Qf = X.astype(np.float32), Q.astype(np.float32)
        # the realisation reproduces the printed matrix
        D = np.linalg.norm(Xf[:, None, :].astype(np.float64) - Qf[None].astype(np.float64), axis=2)
        np.testing.assert_allclose(D, case["rows"], rtol=1e-6, atol=1e-6)
        # the printed Min / MeanMin values fix the orientation of the matrix
        pr = case["printed"]
        assert abs(D.min() - pr["min"]) < 1e-5
        assert abs(D.min(axis=0).mean() - pr["meanmin_Q_to_set"]) < 1e-5
        if "meanmin_set_to_Q" in pr:
            assert abs(D.min(axis=1).mean() - pr["meanmin_set_to_Q"]) < 5e-3
        h = orc.haus(Qf, Xf)
        assert abs(h - case["haus"]) < 1e-5, (case["name"], h)
        assert abs(orc.haus(Xf, Qf) - case["haus"]) < 1e-5
        if "erratum" not in case:
            assert case["haus"] == pr["haus"]


def test_example_2_directed_terms(orc):
    g = json.load(open(GOLDEN))["directed_case"]
    Q = np.array(g["realisation_1d"]["Q"], np.float32)[:, None]
    V = np.array(g["realisation_1d"]["V"], np.float32)[:, None]
    assert orc.haus_directed(V, Q) == g["printed"]["v_to_q"]
    assert orc.haus_directed(Q, V) == g["printed"]["q_to_v"]
    assert orc.haus(Q, V) == g["printed"]["haus"]


def test_against_scipy_directed_hausdorff(orc):
    rng = np.random.default_rng(5)
    for _ in range(40):
        d = int(rng.integers(1, 40))
        Q = rng.standard_normal((int(rng.integers(1, 12)), d)).astype(np.float32)
        V = rng.standard_normal((int(rng.integers(1, 12)), d)).astype(np.float32)
        Q64, V64 = Q.astype(np.float64), V.astype(np.float64)
        ref = max(directed_hausdorff(Q64, V64)[0], directed_hausdorff(V64, Q64)[0])
        assert abs(orc.haus(Q, V) - ref) <= 1e-12 * max(1.0, ref)
        assert abs(orc.haus_directed(Q, V) - directed_hausdorff(Q64, V64)[0]) <= 1e-12 * max(1.0, ref)


def _exact_unit_vectors(rng, n, d=16):
    """Vectors with exactly unit norm in float32: 4 entries of +-1/2 or 16 of +-1/4."""
    out = np.zeros((n, d), np.float32)
    for r in range(n):
        if rng.random() < 0.5:
            idx = rng.choice(d, 4, replace=False)
            out[r, idx] = rng.choice([-0.5, 0.5], 4)
        else:
            out[r] = rng.choice([-0.25, 0.25], d)
    return out


def test_unit_vector_similarity_form(orc):
    """For unit vectors Haus = sqrt(2 - 2 Sim_Haus) with Sim_Haus the min-max
    similarity of the paper's assumptions (sigma of Lemma 1 on S = Q V^T)."""
    rng = np.random.default_rng(11)
    for _ in range(60):
        Q = _exact_unit_vectors(rng, int(rng.integers(1, 8)))
        V = _exact_unit_vectors(rng, int(rng.integers(1, 8)))
        S = Q.astype(np.float64) @ V.astype(np.float64).T
        sigma = min(S.max(axis=1).min(), S.max(axis=0).min())
        # Lemma 1: min S <= sigma <= max S
        assert S.min() <= sigma <= S.max()
        want = np.sqrt(max(2.0 - 2.0 * sigma, 0.0))
        assert abs(orc.haus(Q, V) - want) < 1e-12


def test_axioms(orc):
    rng = np.random.default_rng(3)
    d = 7
    for _ in range(30):
        A = rng.standard_normal((int(rng.integers(1, 6)), d)).astype(np.float32)
        B = rng.standard_normal((int(rng.integers(1, 6)), d)).astype(np.float32)
        C = rng.standard_normal((int(rng.integers(1, 6)), d)).astype(np.float32)
        assert orc.haus(A, A) == 0.0
        assert orc.haus(A, B) == orc.haus(B, A)
        assert orc.haus(A, C) <= orc.haus(A, B) + orc.haus(B, C) + 1e-12
        # order and duplicates of members do not matter
        assert orc.haus(A[::-1].copy(), B) == orc.haus(A, B)
        assert orc.haus(np.concatenate([A, A[:1]]), B) == orc.haus(A, B)
        # the value is one of the pairwise distances, between their min and max
        D = np.linalg.norm(A[:, None].astype(np.float64) - B[None].astype(np.float64), axis=2)
        h = orc.haus(A, B)
        assert D.min() - 1e-12 <= h <= D.max() + 1e-12
        assert np.min(np.abs(D - h)) <= 1e-12 * max(1.0, h)


def test_single_vector_sets_reduce_to_euclidean(orc):
    rng = np.random.default_rng(8)
    for _ in range(20):
        q = rng.standard_normal((1, 9)).astype(np.float32)
        v = rng.standard_normal((1, 9)).astype(np.float32)
        want = np.linalg.norm(q.astype(np.float64) - v.astype(np.float64))
        assert abs(orc.haus(q, v) - want) <= 1e-12 * want


def _brute_ids(Q, vectors, off, k):
    dist = []
    for i in range(off.shape[0] - 1):
        V = vectors[off[i]:off[i + 1]].astype(np.float64)
        Qd = Q.astype(np.float64)
        dist.append(max(directed_hausdorff(Qd, V)[0], directed_hausdorff(V, Qd)[0]))
    dist = np.array(dist)
    order = np.lexsort((np.arange(dist.shape[0]), dist))
    return order[:k], dist[order[:k]]


def test_refine_topk_and_bruteforce(orc):
    rng = np.random.default_rng(21)
    sizes = rng.integers(1, 6, 40)
    # sets 3 and 7 hold one identical vector, so an exact tie must break by id
    sizes[7] = 1
    sizes[3] = 1
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    vectors = rng.standard_normal((off[-1], 5)).astype(np.float32)
    vectors[off[7]] = vectors[off[3]]
    Q = vectors[off[3]:off[4]].copy()
    ids, dist = orc.bruteforce_topk(Q, vectors, off, 6)
    want_ids, want_dist = _brute_ids(Q, vectors, off, 6)
    assert list(ids) == list(want_ids)
    np.testing.assert_allclose(dist, want_dist, rtol=1e-12)
    assert ids[0] == 3 and ids[1] == 7 and dist[0] == 0.0 and dist[1] == 0.0
    # refine over a candidate subset, with padding when k > |candidates|
    cand = np.array([1, 5, 9], np.int32)
    rid, rdist, cdist = orc.refine_topk(Q, vectors, off, cand, 5)
    assert list(rid[3:]) == [-1, -1] and np.all(np.isinf(rdist[3:]))
    assert sorted(rid[:3]) == [1, 5, 9]
    assert np.all(np.diff(rdist[:3]) >= 0)
    for c, dv in zip(cand, cdist):
        assert abs(dv - orc.haus(Q, vectors[off[c]:off[c + 1]])) == 0.0
