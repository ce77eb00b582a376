"""Host logic for searching a database split across ranks (one GPU each).

The sets are independent units of Alg. 6: layer 1 and layer 2 score every
set on its own, and the candidate stage keeps the C smallest pairs
(h_i, i) over all sets.  With the sets split into contiguous id ranges, each
rank scores its own range and keeps its local C smallest pairs; the global C
smallest are among the union of the local lists (any pair in the global top
C is in the top C of its own range), so one exchange of at most C pairs per
rank and query gives exactly the single-GPU candidate list.  The refine
(Def. 4) is again per set: each rank refines its own members of the global
list, and the final k smallest (distance, id) are merged the same way.

Only merging and the exchange live here; the per-rank search is the library's
own.  On one GPU per machine this runs as replicas instead (each rank answers
its own query sets against a full copy of the index), which needs no
exchange at all.
"""
from __future__ import annotations

import numpy as np
import torch


def shard_range(n_sets: int, world: int, rank: int):
    """Contiguous set-id range [lo, hi) of `rank` when n_sets sets are split
    over `world` ranks (the first n_sets % world ranks take one more)."""
    base, extra = divmod(n_sets, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def local_candidates(h, gate, lo, C):
    """The C smallest (h, id) of one rank's range.  h, gate: scores and layer-1
    flags of the range's sets (global ids lo, lo + 1, ...).  Returns
    (h, ids) int64 arrays, at most C pairs, ascending by (h, id)."""
    h = np.asarray(h, np.int64)
    ids = np.arange(lo, lo + h.shape[0], dtype=np.int64)
    keep = np.asarray(gate, bool)
    h, ids = h[keep], ids[keep]
    order = np.lexsort((ids, h))[:C]
    return h[order], ids[order]


def merge_candidates(parts, C):
    """Global candidate list from the ranks' local lists [(h, ids), ...]: the C
    smallest (h, id) pairs, returned in ascending id order (the order of the
    single-GPU list)."""
    h = np.concatenate([np.asarray(p[0], np.int64) for p in parts])
    ids = np.concatenate([np.asarray(p[1], np.int64) for p in parts])
    order = np.lexsort((ids, h))[:C]
    return np.sort(ids[order])


def merge_topk(parts, k):
    """Global top-k from the ranks' local top-k lists [(dist, ids), ...]: the k
    smallest (distance, id), padded with (-1, +inf)."""
    d = np.concatenate([np.asarray(p[0], np.float64) for p in parts])
    ids = np.concatenate([np.asarray(p[1], np.int64) for p in parts])
    keep = ids >= 0
    d, ids = d[keep], ids[keep]
    order = np.lexsort((ids, d))[:k]
    out_d = np.full(k, np.inf)
    out_i = np.full(k, -1, np.int64)
    out_d[:order.shape[0]] = d[order]
    out_i[:order.shape[0]] = ids[order]
    return out_d, out_i


def exchange(local_h, local_ids, C, group=None):
    """All-gather of one query's local candidate lists (at most C pairs per
    rank, padded to C with id -1) over torch.distributed; returns the merged
    global list (ascending ids).  Works with any backend whose tensors live on
    the device of the inputs (gloo on the host, nccl on the GPU)."""
    world = torch.distributed.get_world_size(group)
    buf = torch.full((2, C), -1, dtype=torch.int64)
    n = len(local_ids)
    buf[0, :n] = torch.as_tensor(np.asarray(local_h, np.int64))
    buf[1, :n] = torch.as_tensor(np.asarray(local_ids, np.int64))
    out = [torch.empty_like(buf) for _ in range(world)]
    torch.distributed.all_gather(out, buf, group=group)
    parts = []
    for t in out:
        valid = t[1] >= 0
        parts.append((t[0][valid].numpy(), t[1][valid].numpy()))
    return merge_candidates(parts, C)


def max_over_ranks(value: float, device=None, group=None) -> float:
    """The largest of every rank's value (the bench takes the slowest rank's
    time); on one rank the value itself."""
    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX, group=group)
    return float(t.item())


def replica_queries(w, c, seed, rank, device="cpu"):
    """Query sets of one replica rank.  Every rank holds the same database
    (drawn from `seed`); rank 0 answers the workload's own query sets and
    rank r > 0 draws its own from the same mixture with a seed of its own, so
    the ranks' work is disjoint and the whole job answers world x n_queries
    sets.  Returns (q_vectors, q_offsets)."""
    from . import datagen
    if rank == 0:
        return w["q_vectors"], w["q_offsets"]
    qs = datagen.set_sizes(c["n_queries"], c["q_lo"], c["q_hi"], 1000 * (seed + rank) + 12)
    mix = datagen.Mixture(c["d"], c["n_components"], seed, device=device)
    return mix.draw_sets(qs, 1000 * (seed + rank) + 22), datagen.offsets_from_sizes(qs)
