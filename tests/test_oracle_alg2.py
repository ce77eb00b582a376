"""Pins for the oracle's plain BioVSS search (Alg. 2).

Haus^H is Def. 4 with the Hamming distance between per-vector codes in place
of the Euclidean one.  It is pinned against scipy's Hamming distance matrix
(``cdist`` with the 'hamming' metric returns the fraction of differing
positions; times m it is the count), against hand examples, and against the
identities the codes fix: WTA codes have exactly L ones, so every Hamming
distance is even and at most 2L.  Line 9 keeps the c smallest (d_H, id) pairs,
checked against a numpy lexicographic sort; with c = N the whole search must
equal exact brute-force Hausdorff top-k.
"""
import numpy as np
import pytest
from scipy.spatial.distance import cdist

from paper_2412_03301_gb300 import datagen


def _bits(mask, m):
    """uint32 code words -> 0/1 matrix of m columns (bit p of word p // 32)."""
    mask = np.asarray(mask, np.uint32)
    out = np.zeros((mask.shape[0], m), np.uint8)
    for p in range(m):
        out[:, p] = (mask[:, p // 32] >> np.uint32(p % 32)) & 1
    return out


def _haus_h_scipy(qmask, vmask, m):
    D = np.rint(cdist(_bits(qmask, m), _bits(vmask, m), "hamming") * m).astype(np.int64)
    return int(max(D.min(axis=1).max(), D.min(axis=0).max()))


def test_hand_example(orc):
    m = 64
    # query codes {0,1}, {2,3}; set codes {0,1} and {4,5}
    q = np.zeros((2, 2), np.uint32)
    q[0, 0] = 0b11
    q[1, 0] = 0b1100
    v = np.zeros((2, 2), np.uint32)
    v[0, 0] = 0b11
    v[1, 0] = 0b110000
    # ham: q0-v0 0, q0-v1 4, q1-v0 4, q1-v1 4 -> directed Q->V max(0, 4) = 4,
    # V->Q max(0, 4) = 4
    assert orc.haus_h(q, v, m) == 4
    assert orc.haus_h(q[:1], v[:1], m) == 0
    # one set inside the other: Q -> V is 0, V -> Q is 4
    assert orc.haus_h(v[:1], v, m) == 4


@pytest.fixture(scope="module")
def codes(orc):
    w = datagen.workload(n_sets=60, size_lo=1, size_hi=7, d=24, n_components=16,
                         n_queries=8, q_lo=1, q_hi=6, m=256, fanin=6, seed=9)
    ix = orc.Index(w["vectors"].numpy(), w["offsets"], w["proj"], 10)
    return w, ix


def test_matches_scipy_hamming_and_code_identities(orc, codes):
    w, ix = codes
    qv, qo = w["q_vectors"].numpy(), w["q_offsets"]
    for q in range(qo.shape[0] - 1):
        _, qmask = orc.encode(qv[qo[q]:qo[q + 1]], ix.proj, ix.L)
        score = orc.alg2_scores(qmask, ix.mask, ix.set_off, ix.m)
        for j in range(ix.n_sets):
            vm = ix.mask[ix.set_off[j]:ix.set_off[j + 1]]
            want = _haus_h_scipy(qmask, vm, ix.m)
            assert score[j] == want, (q, j)
            assert score[j] % 2 == 0 and 0 <= score[j] <= 2 * ix.L
            assert orc.haus_h(vm, qmask, ix.m) == score[j]   # symmetric
        assert orc.haus_h(qmask, qmask, ix.m) == 0


def test_single_vector_sets_reduce_to_hamming(orc, codes):
    _, ix = codes
    a, b = ix.mask[:1], ix.mask[5:6]
    ham = int(np.bitwise_count(a ^ b).sum())
    assert orc.haus_h(a, b, ix.m) == ham


def test_select_keeps_the_c_smallest_pairs(orc):
    rng = np.random.default_rng(5)
    score = rng.integers(0, 12, size=400).astype(np.int32)    # many ties
    for c in (0, 1, 7, 50, 399, 400, 1000):
        got = orc.alg2_select(score, c)
        order = np.lexsort((np.arange(score.size), score))
        assert got.tolist() == sorted(order[:min(c, score.size)].tolist())


def test_full_budget_equals_brute_force(orc, codes):
    w, ix = codes
    qv, qo = w["q_vectors"].numpy(), w["q_offsets"]
    for q in range(qo.shape[0] - 1):
        Q = qv[qo[q]:qo[q + 1]]
        r = orc.query_alg2(ix, Q, k=8, C=ix.n_sets)
        ids, dist = orc.bruteforce_topk(Q, ix.vectors, ix.set_off, 8)
        assert r["ids"].tolist() == ids.tolist()
        np.testing.assert_array_equal(r["dist"], dist)
