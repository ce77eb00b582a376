"""Pins for the oracle's FlyHash encoder (Def. 7, Alg. 1).

Hand-derived codes on a tiny projection, a brute-force full sort of the
activations, and the invariants every code must satisfy.
"""
import numpy as np

from paper_2412_03301_gb300 import datagen

# d = 4, m = 8, F = 2: row j lists the two input dims output j sums.
PROJ = np.array([[0, 1], [0, 2], [0, 3], [1, 2], [1, 3], [2, 3], [0, 1], [2, 3]],
                np.uint16)
X = np.array([[0.5, -0.25, 0.125, 0.75]], np.float32)
# a = (0.25, 0.625, 1.25, -0.125, 0.5, 0.875, 0.25, 0.875)
ACT = [0.25, 0.625, 1.25, -0.125, 0.5, 0.875, 0.25, 0.875]
# winners by (a desc, j asc): 2, 5, 7, 1, 4, 0, 6, 3
HAND = {1: [2], 2: [2, 5], 3: [2, 5, 7], 4: [1, 2, 5, 7], 5: [1, 2, 4, 5, 7],
        6: [0, 1, 2, 4, 5, 7], 7: [0, 1, 2, 4, 5, 6, 7], 8: list(range(8))}


def test_hand_computed_codes(orc):
    for L, want in HAND.items():
        pos, mask, act = orc.encode(X, PROJ, L, return_act=True)
        assert act[0].tolist() == ACT
        assert pos[0].tolist() == want, L
        assert int(mask[0, 0]) == sum(1 << p for p in want)


def test_ties_break_by_lower_index(orc):
    # every activation equal (the zero vector): positions 0..L-1
    z = np.zeros((1, 4), np.float32)
    for L in (1, 3, 8):
        pos, _ = orc.encode(z, PROJ, L)
        assert pos[0].tolist() == list(range(L))
    # -0.0 and +0.0 are the same value: with F = 1 the winner among equal
    # zeros is the lowest index, whatever the sign bit
    proj1 = np.array([[0], [1], [2], [3]], np.uint16)
    x = np.array([[-0.0, 0.0, -1.0, -0.0]], np.float32)
    pos, _ = orc.encode(x, proj1, 2)
    assert pos[0].tolist() == [0, 1]
    x = np.array([[-1.0, -0.0, -1.0, 0.0]], np.float32)
    pos, _ = orc.encode(x, proj1, 1)
    assert pos[0].tolist() == [1]


def test_against_full_sort(orc):
    rng = np.random.default_rng(0)
    d, m, F, L = 32, 256, 4, 16
    proj = datagen.projection(d, m, F, seed=4)
    # grid values (multiples of 2^-8) make every activation exact and tie often
    x = (np.round(rng.standard_normal((50, d)) * 8) / 256).astype(np.float32)
    pos, mask, act = orc.encode(x, proj, L, return_act=True)
    want_act = x[:, proj.astype(np.int64)].astype(np.float64).sum(axis=2)
    np.testing.assert_array_equal(act.astype(np.float64), want_act)
    for v in range(x.shape[0]):
        order = np.lexsort((np.arange(m), -want_act[v]))
        assert pos[v].tolist() == sorted(order[:L].tolist())
        bits = np.unpackbits(mask[v].view(np.uint8), bitorder="little")
        assert np.flatnonzero(bits).tolist() == pos[v].tolist()
        assert bits.sum() == L


def test_projection_rows_distinct_sorted():
    proj = datagen.projection(128, 2048, 8, seed=2)
    assert proj.shape == (2048, 8) and proj.dtype == np.uint16
    assert np.all(np.diff(proj.astype(np.int64), axis=1) > 0)
    assert proj.max() < 128
    # seeded: the same seed gives the same table, another seed another one
    assert np.array_equal(proj, datagen.projection(128, 2048, 8, seed=2))
    assert not np.array_equal(proj, datagen.projection(128, 2048, 8, seed=3))
