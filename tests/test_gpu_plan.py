"""The batched serving form: query plans captured into one CUDA graph.

A plan's results must equal the oracle's (ids exactly, distances within 1e-5
relative of the FP64 Hausdorff value) and bvss_query's on the same batch:
across re-written batches of uneven sizes, after the autotuner (every setting
it tries computes the same thing), over several internal batches, with query
sets of up to 64 vectors (the 64-wide tensor-core refine).  The on-device
offset check must turn an out-of-range batch into an error reported by
bvss_sync, and the plan must work again afterwards.
"""
import numpy as np
import pytest
import torch

from paper_2412_03301_gb300 import datagen

pytestmark = pytest.mark.gpu

RTOL = 1e-5
D, K_MIX, SEED = 128, 32, 41


@pytest.fixture(scope="module")
def bv():
    from paper_2412_03301_gb300 import build, bvss
    build.build()
    bvss.load()
    return bvss


@pytest.fixture(scope="module")
def serving(bv, orc):
    # the serving load's shapes, scaled down: Zipf set sizes in 1..128, query sets of 1..64
    w = datagen.workload(n_sets=1500, size_lo=1, size_hi=128, d=D, n_components=K_MIX,
                         n_queries=24, q_lo=1, q_hi=64, m=1024, fanin=8, seed=SEED,
                         size_dist="zipf")
    ix = bv.bvss_build(w["vectors"].cuda(), w["offsets"], w["proj"], wta_l=16, bf16=True)
    orc_ix = orc.Index(w["vectors"].numpy(), w["offsets"], w["proj"], 16)
    return w, ix, orc_ix


def _queries(nq, lo, hi, seed):
    sizes = datagen.set_sizes(nq, lo, hi, seed)
    mix = datagen.Mixture(D, K_MIX, SEED)
    return mix.draw_sets(sizes, seed + 1), datagen.offsets_from_sizes(sizes)


def _check_oracle(orc, orc_ix, qv, qo, ids, dist, k, C, sample):
    ids, dist = ids.cpu().numpy(), dist.cpu().numpy()
    for q in sample:
        r = orc.query(orc_ix, qv[qo[q]:qo[q + 1]].numpy(), k=k, C=C, A=3, M=1)
        assert ids[q].tolist() == r["ids"].tolist(), q
        fin = np.isfinite(r["dist"])
        np.testing.assert_allclose(dist[q][fin], r["dist"][fin], rtol=RTOL, atol=0)
        assert np.all(np.isinf(dist[q][~fin]))


def test_plan_matches_oracle_and_query(bv, orc, serving):
    w, ix, orc_ix = serving
    k, C, nq = 10, 300, 24
    plan = bv.Plan(ix, nq, nq * 64, 64, k=k, C=C, fast=True)
    assert plan.info()["mq"] == 64
    for seed in (5, 6):
        qv, qo = _queries(nq, 1, 64, seed)
        plan.set_queries(qv.cuda(), qo)
        ids, dist = plan.launch()
        bv.bvss_sync(ix)
        _check_oracle(orc, orc_ix, qv, qo, ids, dist, k, C, range(nq))
        ids_q, dist_q = bv.bvss_query(ix, qv.cuda(), qo, k=k, C=C, fast=True)
        assert torch.equal(ids, ids_q)
        assert torch.equal(dist, dist_q)
    plan.close()


def test_plan_small_sets_and_plain_refine(bv, orc, serving):
    # query sets of at most 32 vectors take the 32-wide refine; without the fast flag
    # the FP32 refine runs inside the graph
    w, ix, orc_ix = serving
    qv, qo = _queries(16, 1, 32, 9)
    for fast in (True, False):
        plan = bv.Plan(ix, 16, int(qo[-1]) + 5, 32, k=5, C=120, fast=fast)
        assert plan.info()["mq"] == (32 if fast else 0)
        plan.set_queries(qv.cuda(), qo)
        ids, dist = plan.launch()
        bv.bvss_sync(ix)
        _check_oracle(orc, orc_ix, qv, qo, ids, dist, 5, 120, range(16))
        plan.close()


def test_tuned_plan_gives_the_same_results(bv, orc, serving):
    w, ix, orc_ix = serving
    qv, qo = _queries(24, 1, 64, 12)
    plan = bv.Plan(ix, 24, int(qo[-1]), 64, k=10, C=300, fast=True)
    plan.set_queries(qv.cuda(), qo)
    ids0, dist0 = [t.clone() for t in plan.launch()]
    ms = plan.tune(reps=2)
    assert ms > 0
    kn = plan.info()
    assert kn["scan"] in ("tensor", "popcount") and kn["cand_cta"] in (128, 256, 512)
    assert 4 <= kn["stages"] <= 10 and kn["launches"] >= 8
    assert kn["width_split"] in (0, 1) and kn["batch"] >= 24
    ids1, dist1 = plan.launch()
    bv.bvss_sync(ix)
    assert torch.equal(ids0, ids1) and torch.equal(dist0, dist1)
    _check_oracle(orc, orc_ix, qv, qo, ids1, dist1, 10, 300, [0, 7, 23])
    plan.close()


def test_width_split_and_batch_knobs_give_the_same_results(bv, orc, serving):
    # query sets of 1-64 vectors: by default the ones of at most 32 run on the 32-wide
    # refine and the rest on the 64-wide one (two launches over device lists); without the
    # split every set runs 64 wide.  A smaller internal batch splits the pass in several.
    w, ix, orc_ix = serving
    nq = 40
    qv, qo = _queries(nq, 1, 64, 21)
    assert (np.diff(qo) <= 32).any() and (np.diff(qo) > 32).any()
    plan = bv.Plan(ix, nq, int(qo[-1]), 64, k=10, C=300, fast=True)
    plan.set_queries(qv.cuda(), qo)
    kn = plan.info()
    assert kn["width_split"] == 1 and kn["mq"] == 64
    ids0, dist0 = [t.clone() for t in plan.launch()]
    bv.bvss_sync(ix)
    _check_oracle(orc, orc_ix, qv, qo, ids0, dist0, 10, 300, range(nq))
    n_split = kn["launches"]
    for bucket, batch in ((2, 0), (0, 7), (2, 13), (0, 1)):
        plan.set_knobs(bucket=bucket, batch=batch)
        kn = plan.info()
        assert kn["width_split"] == (0 if bucket == 2 else 1)
        assert kn["batch"] == (batch if batch else nq)
        ids1, dist1 = plan.launch()
        bv.bvss_sync(ix)
        assert torch.equal(ids0, ids1) and torch.equal(dist0, dist1), (bucket, batch)
        if batch == 0:
            assert kn["launches"] == n_split - 2
    # the query operand held in shared memory or streamed through the copy ring
    for mode, streams in ((2, 1), (1, 0)):
        plan.set_knobs(query_operand=mode)
        assert plan.info()["streams_query"] == streams
        ids1, dist1 = plan.launch()
        bv.bvss_sync(ix)
        assert torch.equal(ids0, ids1) and torch.equal(dist0, dist1), mode
    with pytest.raises(bv.BvssError):
        plan.set_knobs(query_operand=3)
    with pytest.raises(bv.BvssError):
        plan.set_knobs(bucket=1)
    with pytest.raises(bv.BvssError):
        plan.set_knobs(batch=-1)
    plan.close()


def test_plan_streams_the_query_operand(bv, orc):
    """At d = 1024 the BF16 refine's 64-wide query operand does not fit in shared memory:
    the graph holds the operand pre-pass and the streamed refine (split by width), and
    the plan must still equal the oracle and bvss_query."""
    w = datagen.workload(n_sets=400, size_lo=1, size_hi=24, d=1024, n_components=16,
                         n_queries=10, q_lo=1, q_hi=64, m=1024, fanin=8, seed=SEED + 3)
    ix = bv.bvss_build(w["vectors"].cuda(), w["offsets"], w["proj"], wta_l=16, bf16=True)
    orc_ix = orc.Index(w["vectors"].numpy(), w["offsets"], w["proj"], 16)
    qv, qo = w["q_vectors"], w["q_offsets"]
    for kw in (dict(fast=True), dict(tf32=True)):
        plan = bv.Plan(ix, 10, int(qo[-1]), 64, k=8, C=150, **kw)
        plan.set_queries(qv.cuda(), qo)
        ids, dist = plan.launch()
        bv.bvss_sync(ix)
        _check_oracle(orc, orc_ix, qv, qo, ids, dist, 8, 150, range(10))
        ids_q, dist_q = bv.bvss_query(ix, qv.cuda(), qo, k=8, C=150, **kw)
        assert torch.equal(ids, ids_q) and torch.equal(dist, dist_q), kw
        assert plan.info()["launches"] >= 14   # the operand pre-pass is in the graph
        plan.close()
    ix.close()


def test_plan_spans_several_batches(bv, orc, serving):
    # more query sets than one internal batch holds (1024 at this index size)
    w, ix, orc_ix = serving
    nq = 1100
    qv, qo = _queries(nq, 1, 4, 13)
    plan = bv.Plan(ix, nq, int(qo[-1]), 4, k=3, C=40, fast=True)
    plan.set_queries(qv.cuda(), qo)
    ids, dist = plan.launch()
    bv.bvss_sync(ix)
    ids_q, dist_q = bv.bvss_query(ix, qv.cuda(), qo, k=3, C=40, fast=True)
    assert torch.equal(ids, ids_q) and torch.equal(dist, dist_q)
    _check_oracle(orc, orc_ix, qv, qo, ids, dist, 3, 40, [0, 1023, 1024, nq - 1])
    plan.close()


def test_plan_rejects_bad_offsets_on_device(bv, orc, serving):
    w, ix, orc_ix = serving
    qv, qo = _queries(8, 1, 16, 14)
    plan = bv.Plan(ix, 8, 8 * 16, 16, k=3, C=50, fast=True)
    bad = qo.copy()
    bad[3:] += 20                      # set 2 holds more than max_qset vectors
    plan.set_queries(qv.cuda(), qo)
    plan.q_offsets.copy_(torch.from_numpy(bad))
    plan.launch()
    with pytest.raises(bv.BvssError) as e:
        bv.bvss_sync(ix)
    assert e.value.code == bv.BVSS_EINVAL
    plan.set_queries(qv.cuda(), qo)
    ids, dist = plan.launch()
    bv.bvss_sync(ix)
    _check_oracle(orc, orc_ix, qv, qo, ids, dist, 3, 50, range(8))
    plan.close()


def test_plan_argument_checks(bv, serving):
    w, ix, _ = serving
    with pytest.raises(bv.BvssError) as e:
        bv.Plan(ix, 4, 3, 8, k=3, C=10)          # fewer vectors than query sets
    assert e.value.code == bv.BVSS_EINVAL
    with pytest.raises(bv.BvssError) as e:
        bv.Plan(ix, 4, 8, 200, k=3, C=10)        # max_qset above the limit
    assert e.value.code == bv.BVSS_EINVAL
    with pytest.raises(bv.BvssError) as e:
        bv.Plan(ix, 4, 8, 33, k=3, C=10, alg2=True)   # Alg. 2 takes query sets of <= 32
    assert e.value.code == bv.BVSS_EINVAL
