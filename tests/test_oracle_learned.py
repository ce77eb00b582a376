"""Pins of the learned-projection oracle (BioHash in place of FlyHash, Def. 7).

The oracle's dense layer, its soft-code training loss and its update step are
checked against things other than themselves: torch's BF16 conversion, the
FlyHash oracle (a dense W holding FlyHash's 0/1 rows must give FlyHash's
codes), hand-derived codes, central finite differences of the loss, the
zero-temperature limit of the soft overlap (the WTA codes' intersection,
counted by numpy), identities of the logistic loss, and invariants of the
normalized step.
"""
import numpy as np
import pytest
import torch

from paper_2412_03301_gb300 import datagen


def test_bf16_rounding_matches_torch(orc):
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.standard_normal(2000).astype(np.float32) * 10.0 ** rng.integers(
        -6, 6, 2000), np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 0.0,
                                65504.0, 2 ** -126], np.float32)]).astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(orc.bf16(x), want)


def test_dense_encode_hand_example(orc):
    # d = 2, m = 4: a = (0.5, 0.25, 0.75, -0.25) for x = (0.5, 0.25)
    w = np.array([[1, 0], [0, 1], [1, 1], [-1, 1]], np.float32)
    x = np.array([[0.5, 0.25]], np.float32)
    pos, mask, act = orc.dense_encode(x, w, 2, return_act=True)
    assert np.array_equal(act[0], [0.5, 0.25, 0.75, -0.25])
    assert pos[0].tolist() == [0, 2] and int(mask[0, 0]) == 0b0101
    # ties go to the lower index: rows 1 and 3 tie at 0.25 once row 3 is (0, 1)
    w[3] = [0, 1]
    pos, _ = orc.dense_encode(x, w, 3)
    assert pos[0].tolist() == [0, 1, 2]


def test_dense_encode_of_flyhash_rows_is_flyhash(orc):
    """A dense W with FlyHash's sparse 0/1 rows gives exactly FlyHash's codes."""
    w = datagen.workload(n_sets=60, size_lo=1, size_hi=5, d=64, n_components=8, n_queries=1,
                         q_lo=1, q_hi=2, m=512, fanin=8, seed=5)
    x = w["vectors"].numpy()
    dense = np.zeros((512, 64), np.float32)
    for j, row in enumerate(w["proj"]):
        dense[j, row] = 1.0
    pos_d, mask_d = orc.dense_encode(x, dense, 16)
    pos_f, mask_f = orc.encode(x, w["proj"], 16)
    assert np.array_equal(pos_d, pos_f) and np.array_equal(mask_d, mask_f)


def test_wta_threshold_separates_the_winners(orc):
    rng = np.random.default_rng(4)
    a = rng.standard_normal(300)
    t = orc.wta_threshold(a, 20)
    srt = np.sort(a)[::-1]
    assert srt[19] > t > srt[20] and t == pytest.approx(0.5 * (srt[19] + srt[20]), abs=0)


@pytest.mark.parametrize("y", [0, 1])
def test_soft_pair_gradient_matches_finite_differences(orc, y):
    rng = np.random.default_rng(10 + y)
    m, L, T, s, mu = 64, 8, 0.3, 6.0, 0.3
    ax, ay = rng.standard_normal(m), rng.standard_normal(m)
    tx, ty = orc.wta_threshold(ax, L), orc.wta_threshold(ay, L)
    loss, gx, gy = orc.soft_pair(ax, ay, L, T, s, mu, y, tx, ty)
    h = 1e-6
    for j in range(0, m, 7):
        e = np.zeros(m)
        e[j] = h
        fx = (orc.soft_pair(ax + e, ay, L, T, s, mu, y, tx, ty)[0] -
              orc.soft_pair(ax - e, ay, L, T, s, mu, y, tx, ty)[0]) / (2 * h)
        fy = (orc.soft_pair(ax, ay + e, L, T, s, mu, y, tx, ty)[0] -
              orc.soft_pair(ax, ay - e, L, T, s, mu, y, tx, ty)[0]) / (2 * h)
        assert gx[j] == pytest.approx(fx, rel=1e-5, abs=1e-9)
        assert gy[j] == pytest.approx(fy, rel=1e-5, abs=1e-9)
    assert loss > 0


def test_soft_overlap_limit_and_loss_identities(orc):
    """At a tiny temperature the soft codes are the WTA codes: the overlap o is the
    codes' intersection over L, and then loss(y=1) - loss(y=0) = -s (o - mu)."""
    rng = np.random.default_rng(12)
    m, L, s, mu = 256, 16, 5.0, 0.25
    ax = rng.standard_normal(m)
    ay = ax + 0.6 * rng.standard_normal(m)
    tx, ty = orc.wta_threshold(ax, L), orc.wta_threshold(ay, L)
    inter = len(set(np.argsort(-ax)[:L]) & set(np.argsort(-ay)[:L]))
    l1, _, _ = orc.soft_pair(ax, ay, L, 1e-9, s, mu, 1, tx, ty)
    l0, _, _ = orc.soft_pair(ax, ay, L, 1e-9, s, mu, 0, tx, ty)
    assert l1 - l0 == pytest.approx(-s * (inter / L - mu), abs=1e-9)
    # at o = mu both labels cost log 2
    same = np.concatenate([np.full(4, 5.0), np.full(m - 4, -5.0)])
    th = orc.wta_threshold(same, 4)
    la, _, _ = orc.soft_pair(same, same, 4, 1e-9, s, 1.0, 1, th, th)
    assert la == pytest.approx(np.log(2.0), abs=1e-9)


def test_quant_weight_rounds_to_even_and_clamps(orc):
    q = orc.quant_weight([0.5 / 256, 1.5 / 256, -0.5 / 256, 1.2, -7.0, 0.3])
    assert q.tolist() == [0.0, 2 / 256, 0.0, 1.0, -1.0, round(0.3 * 256) / 256]


def test_learn_step_aggregates_its_pinned_parts(orc):
    """dw is the batch mean of g_x bf16(x)^T + g_y bf16(y)^T with g from soft_pair on
    the dense_encode activations of the quantized weights; the step moves w by eta
    at its largest entry, then rescales every row to row_norm; wq is on the grid."""
    rng = np.random.default_rng(13)
    m, d, L, n = 48, 16, 6, 9
    T, s, mu, eta, rn = 0.05, 6.0, 0.3, 0.01, 1.5
    w = rng.standard_normal((m, d)) * 0.3
    xs = (np.round(rng.standard_normal((n, d)) * 64) / 256).astype(np.float32)
    ys = (np.round(rng.standard_normal((n, d)) * 64) / 256).astype(np.float32)
    lab = (rng.random(n) < 0.5).astype(np.uint8)
    w2, wq2, dw, loss = orc.learn_step(w, xs, ys, lab, L, T, s, mu, eta, rn)
    wq = orc.quant_weight(w).astype(np.float32)
    _, _, ax = orc.dense_encode(xs, wq, L, return_act=True)
    _, _, ay = orc.dense_encode(ys, wq, L, return_act=True)
    want, tot = np.zeros((m, d)), 0.0
    for i in range(n):
        li, gx, gy = orc.soft_pair(ax[i], ay[i], L, T, s, mu, int(lab[i]),
                                   orc.wta_threshold(ax[i], L), orc.wta_threshold(ay[i], L))
        tot += li
        want += (np.outer(gx, orc.bf16(xs[i])) + np.outer(gy, orc.bf16(ys[i]))) / n
    np.testing.assert_allclose(dw, want, rtol=1e-12, atol=1e-15)
    assert loss == pytest.approx(tot / n, rel=1e-12)
    step = w - eta * dw / np.abs(dw).max()
    assert np.abs(step - w).max() == pytest.approx(eta, rel=1e-12)
    np.testing.assert_allclose(np.linalg.norm(w2, axis=1), rn, rtol=1e-12)
    np.testing.assert_allclose(w2, step * (rn / np.linalg.norm(step, axis=1))[:, None],
                               rtol=1e-12)
    assert np.array_equal(wq2, orc.quant_weight(w2).astype(np.float32))
    assert np.all(wq2 * 256 == np.round(wq2 * 256)) and np.abs(wq2).max() <= 1.0
