"""Multi-rank host logic on CPU (gloo, world size 2).

The database is split into two contiguous id ranges; each rank scores its
range with the oracle (layer-1 gate and sketch Hamming of Alg. 6), keeps its
local C smallest (h, id), and the ranks exchange their lists with an
all-gather.  The merged list must equal the single-process candidate list,
and merging the ranks' refined top-k lists must give the single-process
top-k.  The bench's max-over-ranks timing is checked the same way.
"""
import os
import socket

import numpy as np
import torch
import torch.multiprocessing as mp

from paper_2412_03301_gb300 import datagen, shard

WORLD = 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _workload():
    return datagen.workload(n_sets=301, size_lo=2, size_hi=9, d=32, n_components=16,
                            n_queries=6, q_lo=2, q_hi=7, m=512, fanin=4, seed=12)


def _rank_main(rank, port, results):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.distributed.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        from oracle import oracle as orc
        w = _workload()
        ix = orc.Index(w["vectors"].numpy(), w["offsets"], w["proj"], 16)
        lo, hi = shard.shard_range(ix.n_sets, WORLD, rank)
        qv, qo = w["q_vectors"].numpy(), w["q_offsets"]
        C, k, A, M = 40, 5, 3, 1
        merged, topk = [], []
        for q in range(qo.shape[0] - 1):
            Q = qv[qo[q]:qo[q + 1]]
            qpos, _ = orc.encode(Q, ix.proj, ix.L)
            _, sq, plist = orc.query_filters(qpos, ix.m, A)
            gate = orc.gate_dense(ix.count, plist, M)[lo:hi]
            h = orc.hamming(sq, ix.sketch[lo:hi], None, m=ix.m)
            lh, lid = shard.local_candidates(h, gate, lo, C)
            cand = shard.exchange(lh, lid, C)
            merged.append(cand.tolist())
            # each rank refines its own members of the global list
            mine = cand[(cand >= lo) & (cand < hi)].astype(np.int32)
            ids, dist, _ = orc.refine_topk(Q, ix.vectors, ix.set_off, mine, k)
            d_all = [torch.zeros(k, dtype=torch.float64) for _ in range(WORLD)]
            i_all = [torch.zeros(k, dtype=torch.int64) for _ in range(WORLD)]
            torch.distributed.all_gather(d_all, torch.as_tensor(dist, dtype=torch.float64))
            torch.distributed.all_gather(i_all, torch.as_tensor(ids, dtype=torch.int64))
            gd, gi = shard.merge_topk([(d.numpy(), i.numpy()) for d, i in zip(d_all, i_all)], k)
            topk.append((gi.tolist(), gd.tolist()))
        slowest = shard.max_over_ranks(10.0 + rank)
        # replica form: the same database everywhere, query sets of each rank's own
        c = dict(n_queries=6, q_lo=2, q_hi=7, d=32, n_components=16)
        rq, ro = shard.replica_queries(w, c, 12, rank)
        replica = (float(w["vectors"].double().sum()), rq.double().sum().item(),
                   rq.shape, np.asarray(ro).tolist())
        results[rank] = (merged, topk, slowest, replica)
    finally:
        torch.distributed.destroy_process_group()


def test_sharded_candidates_and_topk_match_one_process(orc):
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    results = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, port, results)) for r in range(WORLD)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
        assert p.exitcode == 0
    w = _workload()
    ix = orc.Index(w["vectors"].numpy(), w["offsets"], w["proj"], 16)
    qv, qo = w["q_vectors"].numpy(), w["q_offsets"]
    for q in range(qo.shape[0] - 1):
        r = orc.query(ix, qv[qo[q]:qo[q + 1]], k=5, C=40, A=3, M=1)
        for rank in range(WORLD):
            merged, topk, slowest, _ = results[rank]
            assert merged[q] == r["cand"].tolist(), (rank, q)
            assert topk[q][0] == r["ids"].tolist(), (rank, q)
            np.testing.assert_array_equal(np.array(topk[q][1]), r["dist"])
            assert slowest == 10.0 + WORLD - 1
    # replicas: one database, rank 0 answers the workload's query sets, the
    # others sets of their own (same dimension, sizes in range)
    db = [results[r][3][0] for r in range(WORLD)]
    assert db[0] == db[1] == float(w["vectors"].double().sum())
    r0, r1 = results[0][3], results[1][3]
    assert r0[1] == w["q_vectors"].double().sum().item()
    assert r0[3] == np.asarray(w["q_offsets"]).tolist()
    assert r1[1] != r0[1] and r1[2][1] == 32
    sizes = np.diff(r1[3])
    assert sizes.shape[0] == 6 and sizes.min() >= 2 and sizes.max() <= 7


def test_shard_ranges_cover_every_set():
    for n in (0, 1, 5, 301, 1000):
        for world in (1, 2, 3, 8):
            parts = [shard.shard_range(n, world, r) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(parts[i][1] == parts[i + 1][0] for i in range(world - 1))
            sizes = [b - a for a, b in parts]
            assert max(sizes) - min(sizes) <= 1


def test_merge_keeps_the_global_smallest_pairs():
    rng = np.random.default_rng(3)
    h = rng.integers(0, 20, size=500)
    gate = rng.random(500) < 0.7
    C = 37
    ids_all = np.arange(500)[gate]
    order = np.lexsort((ids_all, h[gate]))[:C]
    want = np.sort(ids_all[order])
    for world in (1, 2, 5):
        parts = []
        for r in range(world):
            lo, hi = shard.shard_range(500, world, r)
            parts.append(shard.local_candidates(h[lo:hi], gate[lo:hi], lo, C))
        assert shard.merge_candidates(parts, C).tolist() == want.tolist()
