"""The set-sharded search, run through the library on one GPU.

A database split into contiguous id ranges is searched shard by shard:
each shard is an index of its own, whose candidate stage (Alg. 6 lines
10-18) keeps its local C smallest (Hamming, id) pairs.  Offsetting the ids
by the shard's base and merging the local lists with ``shard.merge_candidates``
must give exactly the candidate list of one index over the whole database;
each shard's refine (Def. 4) of its own members of that list, merged with
``shard.merge_topk``, must give exactly the same top-k.  This is the
exchange of the multi-GPU design with the library as the per-rank scorer
(the gloo test covers the collective itself).
"""
import numpy as np
import pytest
import torch

from paper_2412_03301_gb300 import datagen, shard

pytestmark = pytest.mark.gpu


def _np(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("world,fast", [(2, False), (3, True)])
def test_sharded_search_equals_one_index(world, fast):
    from paper_2412_03301_gb300 import build, bvss
    build.build()
    bvss.load()
    n_sets, L, k, C = 4000, 16, 10, 300
    w = datagen.workload(n_sets=n_sets, size_lo=2, size_hi=12, d=64, n_components=32,
                         n_queries=20, q_lo=2, q_hi=12, m=1024, fanin=8, seed=61)
    off = w["offsets"]
    vec = w["vectors"].cuda()
    qv, qo = w["q_vectors"].cuda(), w["q_offsets"]
    nq = qo.shape[0] - 1
    full = bvss.bvss_build(vec, off, w["proj"], wta_l=L, bf16=fast)
    t = bvss.bvss_query_trace(full, qv, qo, k=k, C=C, A=3, M=1, fast=fast)
    torch.cuda.synchronize()
    want_cand, want_n = _np(t["cand"]), _np(t["n_cand"])
    want_ids, want_dist = _np(t["ids"]), _np(t["dist"])
    full.close()

    parts = []
    for r in range(world):
        lo, hi = shard.shard_range(n_sets, world, r)
        ix = bvss.bvss_build(vec[off[lo]:off[hi]].contiguous(), off[lo:hi + 1] - off[lo],
                             w["proj"], wta_l=L, bf16=fast)
        tr = bvss.bvss_query_trace(ix, qv, qo, k=k, C=C, A=3, M=1, fast=fast)
        torch.cuda.synchronize()
        parts.append((lo, _np(tr["h"]).view(np.uint16), _np(tr["cand"]), _np(tr["n_cand"]),
                      _np(tr["cand_dist"])))
        ix.close()

    for q in range(nq):
        local = []
        for lo, h, cand, ncand, _ in parts:
            c = cand[q, :ncand[q]].astype(np.int64)
            local.append((h[q, c].astype(np.int64), c + lo))
        merged = shard.merge_candidates(local, C)
        assert merged.shape[0] == want_n[q], q
        assert np.array_equal(merged, want_cand[q, :want_n[q]]), q
        # each shard refines its own members of the global list
        members = set(merged.tolist())
        topk_parts = []
        for lo, _, cand, ncand, cdist in parts:
            c = cand[q, :ncand[q]].astype(np.int64) + lo
            keep = np.array([i in members for i in c.tolist()], bool)
            topk_parts.append((cdist[q, :ncand[q]][keep], c[keep]))
        d, ids = shard.merge_topk(topk_parts, k)
        assert ids.tolist() == want_ids[q].tolist(), q
        fin = np.isfinite(want_dist[q])
        np.testing.assert_array_equal(d[fin].astype(np.float32), want_dist[q][fin])
