"""The bench's recall ground truth is pinned to the oracle's brute force.

Recall@10 (Sec. 7.1's metric) is measured against the exact Hausdorff
top-10 over every set (Def. 5).  The bench computes that top-10 with a
torch GEMM-form brute force (``bench.exact_topk``); here it must equal the
oracle's direct FP64 brute force (``oracle.bruteforce_topk``) on a few
thousand sets: the same ids, and squared distances equal to the oracle's
distances squared.  On values that are multiples of 2^-8 every FP32 sum of
the GEMM form is exact, so the comparison is exact up to the oracle's own
FP64 square root.

The GPU case uses values on a 2^-12 grid with norms of at most 1/2: FP32
still holds every sum exactly, but TF32 (11 significant bits) would round
the inputs, so the tool must stay exact with TF32 switched on globally,
and must leave that setting as it found it.
"""
import numpy as np
import pytest
import torch

import bench
from paper_2412_03301_gb300 import datagen


def _ground_truth(w, device):
    vec = w["vectors"].to(device)
    off = w["offsets"]
    n_sets = off.shape[0] - 1
    vnorm = (vec * vec).sum(1)
    sizes = torch.from_numpy(np.diff(off)).to(device)
    set_of_row = torch.repeat_interleave(torch.arange(n_sets, device=device), sizes)
    qv, qo = w["q_vectors"].to(device), w["q_offsets"]
    qids = list(range(qo.shape[0] - 1))
    ids, d2 = bench.exact_topk(vec, vnorm, set_of_row, n_sets, qv, qo, qids, 10,
                               chunk=4096)
    return ids.cpu().numpy(), d2.cpu().numpy().astype(np.float64)


def _check_against_oracle(orc, w, ids, d2):
    vec = w["vectors"].numpy()
    qv, qo = w["q_vectors"].numpy(), w["q_offsets"]
    for q in range(qo.shape[0] - 1):
        r_ids, r_dist = orc.bruteforce_topk(qv[qo[q]:qo[q + 1]], vec, w["offsets"], 10)
        assert ids[q].tolist() == r_ids.tolist(), q
        np.testing.assert_allclose(d2[q], r_dist ** 2, rtol=1e-12, atol=0)


def test_exact_topk_equals_oracle_bruteforce(orc):
    w = datagen.workload(n_sets=3000, size_lo=2, size_hi=12, d=64, n_components=32,
                         n_queries=12, q_lo=2, q_hi=12, m=256, fanin=4, seed=51)
    # set 6 := a copy of set 5 and query set 0 := set 5 as well, so sets 5 and 6 tie
    # at distance 0 and the lower id must come first on both sides
    off, vec = w["offsets"], w["vectors"]
    parts = [vec[off[i]:off[i + 1]] if i != 6 else vec[off[5]:off[6]] for i in range(3000)]
    sizes = np.array([p.shape[0] for p in parts])
    w["vectors"] = torch.cat(parts).contiguous()
    w["offsets"] = datagen.offsets_from_sizes(sizes)
    qo, qv = w["q_offsets"], w["q_vectors"]
    qparts = [vec[off[5]:off[6]]] + [qv[qo[q]:qo[q + 1]] for q in range(1, qo.shape[0] - 1)]
    w["q_vectors"] = torch.cat(qparts).contiguous()
    w["q_offsets"] = datagen.offsets_from_sizes(np.array([p.shape[0] for p in qparts]))
    ids, d2 = _ground_truth(w, "cpu")
    assert ids[0, :2].tolist() == [5, 6] and d2[0, 0] == 0 and d2[0, 1] == 0
    _check_against_oracle(orc, w, ids, d2)


@pytest.mark.gpu
def test_exact_topk_on_gpu_is_exact_even_with_tf32_enabled(orc):
    w = datagen.workload(n_sets=3000, size_lo=2, size_hi=12, d=64, n_components=32,
                         n_queries=12, q_lo=2, q_hi=12, m=256, fanin=4, seed=52, grid=False)
    # norms of at most 1/2 on the 2^-12 grid: exact in FP32, not in TF32
    for key in ("vectors", "q_vectors"):
        x = w[key].to(torch.float64)
        w[key] = (torch.round(x * 0.5 * 4096) / 4096).to(torch.float32)
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        ids, d2 = _ground_truth(w, "cuda")
        assert torch.backends.cuda.matmul.allow_tf32 is True
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    _check_against_oracle(orc, w, ids, d2)
