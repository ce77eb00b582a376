"""Training the learned projection (BioHash in place of FlyHash in Def. 7).

The paper's runs use BioHash: h = WTA(W v) with W learned from the data by a
normalized gradient method, whose per-batch update magnitude max |dW| the
appendix on BioHash iterations follows.  Here W is a dense BF16 layer trained
on neighbour pairs that the exact Hausdorff refine itself produces:

* pairs: for training query sets drawn from the workload's mixture, the
  library's exact top sets; a positive pair is a query vector and its
  nearest vector in one of the k nearest sets (bvss_nearest_rows), a
  negative pair either a query vector and a random database vector or (hard
  negatives, which the candidate stage needs: random pairs are too easy to
  teach the layer anything the sketch ranking uses) its nearest vector in a
  set ranked just below the k nearest;
* each step: the layer's activations of both sides on the tensor cores
  (bvss_dense_forward), the pairs' soft-code loss and its gradient
  (bvss_learn_pair_grad), the weight gradient (bvss_learn_weight_grad) and
  the normalized update (bvss_learn_update), whose largest entry is the
  step size eta_t, decaying linearly to zero;
* W starts as FlyHash's own 0/1 rows (as a dense layer they give exactly
  FlyHash's codes), so the random FlyHash is the fallback and the starting
  point at once.

This module only orders the calls and moves data: every arithmetic step runs
in the library's kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import bvss


def flyhash_dense(proj: np.ndarray, d: int) -> torch.Tensor:
    """FlyHash's sparse binary projection (m x F dims) as a dense m x d 0/1 matrix."""
    w = torch.zeros((proj.shape[0], d), dtype=torch.float32)
    w.scatter_(1, torch.from_numpy(proj.astype(np.int64)), 1.0)
    return w


def mine_pairs(ix: bvss.Index, q_vectors: torch.Tensor, q_offsets: np.ndarray, *, k: int,
               C: int, n_pos: int, n_neg: int, seed: int, fast: bool = True,
               batch: int = 1000, hard: int = 0):
    """(x_idx, y_rows, labels): x_idx indexes q_vectors, y_rows the index's rows.

    The top sets of every training query set come from the library's query path
    (candidate filter, then the exact refine); positives are (query vector, its nearest
    vector in one of the k nearest sets).  Negatives are (query vector, a random database
    vector), or with hard = K > k (query vector, its nearest vector in one of the sets
    ranked k+1..K): near misses, the sets that compete for the candidate slots."""
    dev = ix.device
    nq = q_offsets.shape[0] - 1
    kk = max(k, hard)
    rows = []
    for q0 in range(0, nq, batch):
        q1 = min(nq, q0 + batch)
        off = q_offsets[q0:q1 + 1] - q_offsets[q0]
        qv = q_vectors[int(q_offsets[q0]):int(q_offsets[q1])]
        ids, _ = bvss.bvss_query(ix, qv, off, k=kk, C=C, fast=fast)
        rows.append(bvss.bvss_nearest_rows(ix, qv, off, ids))
    rows = torch.cat(rows)                                   # (Vq, kk)
    vq = rows.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)

    def sample(cols, count):
        a = torch.arange(vq, device=dev).repeat_interleave(cols.stop - cols.start)
        f = rows[:, cols].reshape(-1)
        keep = f >= 0
        a, f = a[keep], f[keep]
        pick = torch.randperm(a.shape[0], generator=g)[:count].to(dev)
        return a[pick], f[pick]

    pos_x, pos_y = sample(slice(0, k), n_pos)
    if hard > k:
        neg_x, neg_y = sample(slice(k, kk), n_neg)
    else:
        neg_x = torch.randint(0, vq, (n_neg,), generator=g).to(dev)
        neg_y = torch.randint(0, ix.n_vectors, (n_neg,), generator=g).to(dev)
    x = torch.cat([pos_x, neg_x])
    y = torch.cat([pos_y, neg_y])
    lab = torch.cat([torch.ones(pos_x.shape[0], dtype=torch.uint8, device=dev),
                     torch.zeros(neg_x.shape[0], dtype=torch.uint8, device=dev)])
    return x, y, lab


def train(ix: bvss.Index, q_vectors: torch.Tensor, pairs, w0: torch.Tensor, *, L: int,
          epochs: int = 5, batch: int = 10_000, temperature: float = 0.01,
          scale: float = 10.0, margin: float = 0.3, eta0: float = 0.0005,
          row_norm: float | None = None, seed: int = 0):
    """Train the layer from w0 (m x d FP32).  Returns (w, wq_bf16, history) with
    history = per-step (mean loss, eta_t, max |dW|)."""
    x_idx, y_rows, lab = pairs
    dev = ix.device
    w = w0.to(dev).contiguous().clone()
    m, d = w.shape
    if row_norm is None:
        row_norm = float(w.norm(dim=1).mean())
    n = x_idx.shape[0]
    steps = epochs * ((n + batch - 1) // batch)
    g = torch.Generator(device="cpu").manual_seed(seed)
    act_x = torch.empty((batch, m), dtype=torch.float32, device=dev)
    act_y = torch.empty_like(act_x)
    gx = torch.empty_like(act_x)
    gy = torch.empty_like(act_x)
    dw = torch.empty((m, d), dtype=torch.float32, device=dev)
    losses = torch.zeros(steps, dtype=torch.float64, device=dev)     # per step: summed loss
    absmax = torch.zeros(steps + 1, dtype=torch.float32, device=dev)  # per step: max |dW|
    wq = torch.empty((m, d), dtype=torch.bfloat16, device=dev)
    # the starting forward weights: w on the 2^-8 grid (a zero step)
    bvss.bvss_learn_update(w, torch.zeros_like(dw), 0.0, row_norm, wq, absmax[steps:])
    sizes, etas = [], []
    t = 0
    for _ in range(epochs):
        order = torch.randperm(n, generator=g).to(dev)
        for b0 in range(0, n, batch):
            sel = order[b0:b0 + batch]
            nb = sel.shape[0]
            xb = bvss.bvss_to_bf16(q_vectors[x_idx[sel]])
            yb = bvss.bvss_index_rows_bf16(ix, y_rows[sel])
            bvss.bvss_dense_forward(xb, wq, out=act_x[:nb])
            bvss.bvss_dense_forward(yb, wq, out=act_y[:nb])
            bvss.bvss_learn_pair_grad(act_x[:nb], act_y[:nb], lab[sel], L, temperature, scale,
                                      margin, gx[:nb], gy[:nb], losses[t:t + 1])
            bvss.bvss_learn_weight_grad(gx[:nb], gy[:nb], xb, yb, out=dw)
            eta = eta0 * (1.0 - t / steps)
            bvss.bvss_learn_update(w, dw, eta, row_norm, wq, absmax[t:t + 1])
            sizes.append(nb)
            etas.append(eta)
            t += 1
    bvss.bvss_learn_sync()
    lo, am = losses.cpu().numpy(), absmax.cpu().numpy()
    history = [(float(lo[i]) / sizes[i], etas[i], float(am[i])) for i in range(t)]
    return w, wq, history
