"""Pins for the oracle's filters and candidate stage.

Count and binary Bloom filters (Defs. 8 and 10, Algs. 3 and 5), the query
side of Alg. 6 (lines 1-4), the inverted-index walk (Def. 9, Alg. 4, Alg. 6
lines 5-9) against the dense predicate, the Hamming score (line 12) against
numpy's popcount, and the bounded heap (lines 10-18) against a full sort.
"""
import numpy as np
import pytest

from paper_2412_03301_gb300 import datagen


def _bits(words, m):
    return np.unpackbits(np.ascontiguousarray(words).view(np.uint8),
                         bitorder="little")[:m]


def test_hand_filters(orc):
    # two sets over m = 8 with L = 3: {2,5,7} + {1,2,5}; {0,1,7}
    pos = np.array([[2, 5, 7], [1, 2, 5], [0, 1, 7]], np.uint16)
    off = np.array([0, 2, 3], np.int64)
    sk, cnt = orc.build_filters(pos, off, 8)
    assert _bits(sk[0], 8).tolist() == [0, 1, 1, 0, 0, 1, 0, 1]
    assert _bits(sk[1], 8).tolist() == [1, 1, 0, 0, 0, 0, 0, 1]
    assert cnt[:, 0].tolist() == [0, 1, 2, 0, 0, 2, 0, 1]
    assert cnt[:, 1].tolist() == [1, 1, 0, 0, 0, 0, 0, 1]


def test_hand_query_filters(orc):
    qpos = np.array([[2, 5, 7], [1, 2, 5], [0, 1, 7]], np.uint16)
    cq, sq, plist = orc.query_filters(qpos, 8, 3)
    assert cq.tolist() == [1, 2, 2, 0, 0, 2, 0, 2]
    assert _bits(sq, 8).tolist() == [1, 1, 1, 0, 0, 1, 0, 1]
    # four positions tie at count 2: the lowest three are taken
    assert plist.tolist() == [1, 2, 5]
    _, _, p5 = orc.query_filters(qpos, 8, 5)
    assert p5.tolist() == [1, 2, 5, 7, 0]


def _random_codes(rng, n, m, L):
    pos = np.zeros((n, L), np.uint16)
    for v in range(n):
        pos[v] = np.sort(rng.choice(m, L, replace=False))
    return pos


def test_filter_invariants(orc):
    rng = np.random.default_rng(1)
    m, L = 256, 12
    sizes = rng.integers(1, 20, 60)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    pos = _random_codes(rng, off[-1], m, L)
    # set 5: every member carries the same code
    pos[off[5]:off[6]] = pos[off[5]]
    sk, cnt = orc.build_filters(pos, off, m)
    for i in range(60):
        members = pos[off[i]:off[i + 1]].astype(np.int64)
        sb = _bits(sk[i], m)
        assert np.all(sb[members.ravel()] == 1)                 # members' bits set
        assert sb.sum() <= min(m, L * sizes[i])
        assert int(cnt[:, i].sum()) == L * sizes[i]              # counts = multiplicities
        assert np.array_equal(cnt[:, i] > 0, sb == 1)
        want = np.bincount(members.ravel(), minlength=m)
        assert np.array_equal(cnt[:, i], want)
    c5 = np.zeros(m, np.int64)
    c5[pos[off[5]].astype(np.int64)] = sizes[5]
    assert np.array_equal(cnt[:, 5], c5)


def test_counts_saturate(orc):
    pos = np.tile(np.array([[0, 3]], np.uint16), (300, 1))
    off = np.array([0, 300], np.int64)
    _, cnt = orc.build_filters(pos, off, 32)
    assert cnt[0, 0] == 255 and cnt[3, 0] == 255 and cnt[1, 0] == 0


def test_inverted_lists_sorted(orc):
    rng = np.random.default_rng(2)
    cnt = rng.integers(0, 4, (16, 50)).astype(np.uint8)
    inv = orc.InvertedIndex(cnt)
    for p in range(16):
        ids, c = inv.list(p)
        nz = np.flatnonzero(cnt[p])
        assert sorted(ids.tolist()) == nz.tolist()
        assert np.array_equal(c, cnt[p, ids])
        key = list(zip((-c.astype(int)).tolist(), ids.tolist()))
        assert key == sorted(key)                 # count desc, then id asc


@pytest.mark.parametrize("M", [0, 1, 2, 3, 300])
def test_gate_literal_equals_dense(orc, M):
    rng = np.random.default_rng(M)
    m, L = 128, 10
    sizes = rng.integers(1, 25, 200)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    pos = _random_codes(rng, off[-1], m, L)
    _, cnt = orc.build_filters(pos, off, m)
    inv = orc.InvertedIndex(cnt)
    for A in (1, 2, 3, 7):
        plist = rng.choice(m, A, replace=False).astype(np.uint16)
        g_lit = inv.gate(plist, M)
        g_den = orc.gate_dense(cnt, plist, M)
        assert np.array_equal(g_lit, g_den)
        want = (cnt[plist.astype(np.int64)] >= M).any(axis=0)
        assert np.array_equal(g_den.astype(bool), want)
        if M == 0:
            assert g_lit.all()
        if M > 255:
            assert not g_lit.any()


def test_hamming_against_popcount(orc):
    rng = np.random.default_rng(4)
    m = 512
    sk = rng.integers(0, 2**32, (300, m // 32), dtype=np.uint64).astype(np.uint32)
    sq = rng.integers(0, 2**32, m // 32, dtype=np.uint64).astype(np.uint32)
    h = orc.hamming(sq, sk)
    want = np.bitwise_count(sk ^ sq[None]).sum(axis=1)
    assert np.array_equal(h, want)
    gate = (rng.random(300) < 0.5).astype(np.uint8)
    hg = orc.hamming(sq, sk, gate)
    assert np.array_equal(hg[gate == 1], want[gate == 1])
    assert np.all(hg[gate == 0] == -1)


@pytest.mark.parametrize("T", [0, 1, 5, 40, 150, 1000])
def test_heap_equals_sort_rule(orc, T):
    rng = np.random.default_rng(T + 7)
    n = 500
    h = rng.integers(0, 12, n).astype(np.int32)       # many ties
    gate = (rng.random(n) < 0.6).astype(np.uint8)
    got = orc.heap_select(h, gate, T)
    idx = np.flatnonzero(gate)
    order = idx[np.lexsort((idx, h[idx]))]            # (h, id) ascending
    assert got.tolist() == sorted(order[:T].tolist())
    got_all = orc.heap_select(h, None, T)
    order_all = np.lexsort((np.arange(n), h))
    assert got_all.tolist() == sorted(order_all[:T].tolist())


def test_end_to_end_filters_on_mixture(orc):
    """Sketch / count invariants on a small database of the real workload shape."""
    w = datagen.workload(n_sets=60, size_lo=2, size_hi=9, d=32, n_components=16,
                         n_queries=3, q_lo=2, q_hi=5, m=256, fanin=4, seed=5)
    vec = w["vectors"].numpy()
    pos, mask = orc.encode(vec, w["proj"], 8)
    sk, cnt = orc.build_filters(pos, w["offsets"], 256)
    off = w["offsets"]
    for i in range(60):
        ored = np.bitwise_or.reduce(mask[off[i]:off[i + 1]], axis=0)
        assert np.array_equal(ored, sk[i])
