"""The learned projection on the GPU against its oracle (BioHash in place of FlyHash).

The BF16 dense layer runs on the tensor cores with FP32 accumulation.  With
weights and inputs on the 2^-8 grid every partial sum is exact, so its
activations, codes, filters, candidates and results must equal the oracle's
bit for bit (and FlyHash's own 0/1 rows given as a dense layer must give
FlyHash's codes).  The training kernels compute in FP32 against the oracle's
FP64, so they are compared within stated tolerances: the loss and gradients
to 2e-4 relative (FP32 sigmoid and sums of a few thousand terms), the weight
gradient to 1e-4, and the step's weights to 1e-5, its grid-rounded forward
weights exactly except where the FP32 and FP64 values straddle a rounding
boundary.
"""
import numpy as np
import pytest
import torch

from paper_2412_03301_gb300 import datagen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bv():
    from paper_2412_03301_gb300 import build, bvss
    build.build()
    bvss.load()
    return bvss


def _grid_weights(m, d, seed, norm=8 ** 0.5):
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((m, d))
    w *= norm / np.linalg.norm(w, axis=1, keepdims=True)
    return np.clip(np.round(w * 256) / 256, -1, 1).astype(np.float32)


@pytest.mark.parametrize("n,d,m", [(300, 128, 256), (130, 384, 4096), (1, 64, 128)])
def test_dense_forward_is_exact_on_the_grid(bv, orc, n, d, m):
    x = datagen.Mixture(d, 16, n + d).draw_sets(np.full(n, 1), n + 1).numpy()
    w = _grid_weights(m, d, m + d)
    act = bv.bvss_dense_forward(torch.from_numpy(x).cuda().to(torch.bfloat16),
                                torch.from_numpy(w).cuda().to(torch.bfloat16))
    bv.bvss_learn_sync()
    _, _, want = orc.dense_encode(x, w, min(8, m - 1), return_act=True)
    assert np.array_equal(act.cpu().numpy().astype(np.float64), want)


def test_dense_forward_off_the_grid_within_fp32_rounding(bv, orc):
    rng = np.random.default_rng(1)
    n, d, m = 200, 192, 384
    x = rng.standard_normal((n, d)).astype(np.float32)
    w = rng.standard_normal((m, d)).astype(np.float32)
    act = bv.bvss_dense_forward(torch.from_numpy(x).cuda().to(torch.bfloat16),
                                torch.from_numpy(w).cuda().to(torch.bfloat16)).cpu().numpy()
    _, _, want = orc.dense_encode(x, w, 8, return_act=True)
    scale = np.abs(orc.bf16(x)) @ np.abs(orc.bf16(w)).T     # sum_k |x_k w_k|
    assert np.all(np.abs(act - want) <= (d + 2) * 2.0 ** -23 * scale)


class _Case:
    def __init__(self, bv, orc, w, L, dense):
        self.w, self.L = w, L
        self.vec = w["vectors"].numpy()
        self.qvec = w["q_vectors"].numpy()
        self.ix = bv.bvss_build_dense(w["vectors"].cuda(), w["offsets"],
                                      torch.from_numpy(dense).cuda(), wta_l=L, bf16=True)
        self.orc_ix = orc.Index(self.vec, w["offsets"], None, L, dense_w=dense)
        self.qv_cuda = w["q_vectors"].cuda()


def test_dense_index_matches_the_oracle(bv, orc):
    from tests.test_gpu_parity import _check_query
    s = datagen.SMALL
    w = datagen.workload(n_sets=1500, size_lo=4, size_hi=16, d=128, n_components=64,
                         n_queries=30, q_lo=4, q_hi=16, m=2048, fanin=8, seed=3)
    case = _Case(bv, orc, w, s["L"], _grid_weights(2048, 128, 7))
    got = bv.bvss_get_codes(case.ix, 0, case.ix.n_vectors).cpu().numpy().view(np.uint16)
    assert np.array_equal(got, case.orc_ix.pos)
    assert bv.bvss_index_info(case.ix)["fanin"] == 0
    _check_query(bv, orc, case, k=10, C=200, A=3, M=1)
    _check_query(bv, orc, case, k=10, C=150, A=2, M=0, nq=8, fast=True)


def test_flyhash_rows_as_a_dense_layer_give_flyhash_codes(bv):
    w = datagen.workload(n_sets=400, size_lo=2, size_hi=8, d=64, n_components=16,
                         n_queries=10, q_lo=2, q_hi=6, m=512, fanin=8, seed=8)
    dense = np.zeros((512, 64), np.float32)
    for j, row in enumerate(w["proj"]):
        dense[j, row] = 1.0
    a = bv.bvss_build(w["vectors"].cuda(), w["offsets"], w["proj"], wta_l=16)
    b = bv.bvss_build_dense(w["vectors"].cuda(), w["offsets"], torch.from_numpy(dense).cuda(),
                            wta_l=16)
    n = a.n_vectors
    assert torch.equal(bv.bvss_get_codes(a, 0, n), bv.bvss_get_codes(b, 0, n))
    ta = bv.bvss_query_trace(a, w["q_vectors"].cuda(), w["q_offsets"], k=5, C=40)
    tb = bv.bvss_query_trace(b, w["q_vectors"].cuda(), w["q_offsets"], k=5, C=40)
    for key in ("qpos", "h", "cand", "ids", "dist"):
        assert torch.equal(ta[key], tb[key]), key


def test_pair_gradient_matches_the_oracle(bv, orc):
    rng = np.random.default_rng(5)
    n, m, L, T, s, mu = 37, 512, 16, 0.05, 8.0, 0.3
    ax = (rng.standard_normal((n, m)) * 0.2).astype(np.float32)
    ay = (ax + rng.standard_normal((n, m)) * 0.1).astype(np.float32)
    lab = (rng.random(n) < 0.5).astype(np.uint8)
    gx, gy, loss = bv.bvss_learn_pair_grad(torch.from_numpy(ax).cuda(),
                                           torch.from_numpy(ay).cuda(),
                                           torch.from_numpy(lab).cuda(), L, T, s, mu)
    gx, gy = gx.cpu().numpy(), gy.cpu().numpy()
    tot = 0.0
    for i in range(n):
        a64, b64 = ax[i].astype(np.float64), ay[i].astype(np.float64)
        li, wx, wy = orc.soft_pair(a64, b64, L, T, s, mu, int(lab[i]),
                                   orc.wta_threshold(a64, L), orc.wta_threshold(b64, L))
        tot += li
        for g, want in ((gx[i], wx), (gy[i], wy)):
            np.testing.assert_allclose(g, want, rtol=2e-4, atol=2e-4 * np.abs(want).max())
    assert float(loss.item()) == pytest.approx(tot, rel=2e-4)


def test_weight_gradient_matches_a_float64_sum(bv):
    rng = np.random.default_rng(6)
    n, m, d = 101, 128, 64
    gx = rng.standard_normal((n, m)).astype(np.float32)
    gy = rng.standard_normal((n, m)).astype(np.float32)
    x = torch.from_numpy(rng.standard_normal((n, d)).astype(np.float32)).to(torch.bfloat16)
    y = torch.from_numpy(rng.standard_normal((n, d)).astype(np.float32)).to(torch.bfloat16)
    dw = bv.bvss_learn_weight_grad(torch.from_numpy(gx).cuda(), torch.from_numpy(gy).cuda(),
                                   x.cuda(), y.cuda()).cpu().numpy()
    want = (gx.astype(np.float64).T @ x.float().numpy().astype(np.float64) +
            gy.astype(np.float64).T @ y.float().numpy().astype(np.float64)) / n
    np.testing.assert_allclose(dw, want, rtol=1e-4, atol=1e-4 * np.abs(want).max())


def test_training_step_matches_the_oracle(bv, orc):
    """Forward on the tensor cores, pair gradient, weight gradient and the update, on one
    batch, against the oracle's FP64 step."""
    rng = np.random.default_rng(7)
    m, d, L, n = 256, 64, 8, 50
    T, s, mu, eta, rn = 0.05, 6.0, 0.3, 0.01, 8 ** 0.5
    w = rng.standard_normal((m, d))
    w *= rn / np.linalg.norm(w, axis=1, keepdims=True)
    xs = (np.round(rng.standard_normal((n, d)) * 256 / 8) / 256).astype(np.float32)
    ys = (xs + np.round(rng.standard_normal((n, d)) * 256 / 32) / 256).astype(np.float32)
    lab = (rng.random(n) < 0.5).astype(np.uint8)
    w2, wq2, dw, loss = orc.learn_step(w, xs, ys, lab, L, T, s, mu, eta, rn)

    wg = torch.from_numpy(w.astype(np.float32)).cuda()
    wq = torch.from_numpy(orc.quant_weight(w).astype(np.float32)).cuda().to(torch.bfloat16)
    xb = torch.from_numpy(xs).cuda().to(torch.bfloat16)
    yb = torch.from_numpy(ys).cuda().to(torch.bfloat16)
    ax = bv.bvss_dense_forward(xb, wq)
    ay = bv.bvss_dense_forward(yb, wq)
    gx, gy, lsum = bv.bvss_learn_pair_grad(ax, ay, torch.from_numpy(lab).cuda(), L, T, s, mu)
    dwg = bv.bvss_learn_weight_grad(gx, gy, xb, yb)
    np.testing.assert_allclose(dwg.cpu().numpy(), dw, rtol=2e-3, atol=2e-3 * np.abs(dw).max())
    assert float(lsum.item()) / n == pytest.approx(loss, rel=2e-4)
    # the update from the oracle's own gradient, so only the step itself is compared
    wq_new, absmax = bv.bvss_learn_update(wg, torch.from_numpy(dw.astype(np.float32)).cuda(),
                                          eta, rn)
    bv.bvss_learn_sync()
    assert float(absmax.item()) == pytest.approx(np.abs(dw).max(), rel=1e-6)
    np.testing.assert_allclose(wg.cpu().numpy(), w2, rtol=1e-5, atol=1e-6)
    got_q = wq_new.float().cpu().numpy()
    frac = np.abs(w2 * 256 - np.floor(w2 * 256) - 0.5)       # distance from a rounding tie
    near = frac < 1e-3
    assert np.array_equal(got_q[~near], wq2[~near])


def test_nearest_rows_match_brute_force(bv):
    w = datagen.workload(n_sets=300, size_lo=1, size_hi=9, d=64, n_components=16,
                         n_queries=12, q_lo=1, q_hi=7, m=256, fanin=4, seed=9)
    ix = bv.bvss_build(w["vectors"].cuda(), w["offsets"], w["proj"], wta_l=8)
    rng = np.random.default_rng(10)
    sets = rng.integers(0, 300, size=(12, 5)).astype(np.int64)
    sets[3, 2] = -1
    sets[4, 0] = 300
    rows = bv.bvss_nearest_rows(ix, w["q_vectors"].cuda(), w["q_offsets"],
                                torch.from_numpy(sets).cuda()).cpu().numpy()
    vec, off = w["vectors"].numpy().astype(np.float64), w["offsets"]
    qv, qo = w["q_vectors"].numpy().astype(np.float64), w["q_offsets"]
    for q in range(12):
        for a in range(qo[q], qo[q + 1]):
            for t in range(5):
                sid = sets[q, t]
                if sid < 0 or sid >= 300:
                    assert rows[a, t] == -1
                    continue
                dd = np.linalg.norm(vec[off[sid]:off[sid + 1]] - qv[a], axis=1)
                assert rows[a, t] == off[sid] + int(np.argmin(dd))


def test_index_rows_in_bf16(bv):
    w = datagen.workload(n_sets=50, size_lo=1, size_hi=4, d=64, n_components=8, n_queries=1,
                         q_lo=1, q_hi=2, m=256, fanin=4, seed=11)
    ix = bv.bvss_build(w["vectors"].cuda(), w["offsets"], w["proj"], wta_l=8)
    rows = torch.tensor([0, 5, ix.n_vectors - 1, -1, ix.n_vectors], device="cuda")
    out = bv.bvss_index_rows_bf16(ix, rows).cpu()
    want = w["vectors"][[0, 5, ix.n_vectors - 1]].to(torch.bfloat16)
    assert torch.equal(out[:3], want) and torch.all(out[3:] == 0)


def test_training_pipeline_small(bv, orc):
    """Mine pairs with the library's refine, train two epochs, build the learned index:
    the loss falls, the first step's update magnitude is eta0, the forward weights stay
    on the 2^-8 grid, and the trained layer's codes equal the oracle's."""
    from paper_2412_03301_gb300 import learn
    w = datagen.workload(n_sets=2000, size_lo=2, size_hi=10, d=128, n_components=32,
                         n_queries=4, q_lo=2, q_hi=8, m=1024, fanin=8, seed=21)
    ix = bv.bvss_build(w["vectors"].cuda(), w["offsets"], w["proj"], wta_l=16, bf16=True)
    ts = datagen.set_sizes(300, 2, 8, 22)
    tq = datagen.Mixture(128, 32, 21).draw_sets(ts, 23).cuda()
    pairs = learn.mine_pairs(ix, tq, datagen.offsets_from_sizes(ts), k=5, C=200, n_pos=3000,
                             n_neg=3000, seed=24, hard=20)
    assert int(pairs[2].sum()) == 3000 and pairs[0].shape[0] == 6000
    wl, wq, hist = learn.train(ix, tq, pairs, learn.flyhash_dense(w["proj"], 128), L=16,
                               epochs=2, batch=1000, eta0=0.002)
    assert len(hist) == 12 and hist[0][1] == pytest.approx(0.002)
    assert np.mean([h[0] for h in hist[-3:]]) < np.mean([h[0] for h in hist[:3]])
    q = wq.float().cpu().numpy()
    assert np.all(q * 256 == np.round(q * 256)) and np.abs(q).max() <= 1.0
    np.testing.assert_allclose(wl.norm(dim=1).cpu().numpy(), 8 ** 0.5, rtol=1e-5)
    lix = bv.bvss_build_dense(w["vectors"].cuda(), w["offsets"], wq.float().contiguous(),
                              wta_l=16)
    got = bv.bvss_get_codes(lix, 0, lix.n_vectors).cpu().numpy().view(np.uint16)
    want, _ = orc.dense_encode(w["vectors"].numpy(), q, 16)
    assert np.array_equal(got, want)
