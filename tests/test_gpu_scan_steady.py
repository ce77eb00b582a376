"""The tensor-core sketch scans and the bounded select in their steady state.

Both tensor-core scans (Alg. 6 line 12 as an FP8 GEMM) are persistent kernels:
one CTA per SM walks tiles, alternating two TMEM accumulators whose full/empty
barrier phases flip every second tile.  The default form (query sketches as
the A operand) takes tiles of 256 query sets x 128 sets: here 60,000 sets (469
set tiles) x 600 query sets (3 query-block pairs) give 1,407 tiles, about 9 per
CTA on 152 SMs.  The form with the set sketches expanded into tensor memory
takes 128 sets x 128 query sets: 2,345 tiles, about 15 per CTA, and its
8-stage ring turns over 15 times.  The other GPU tests
reach at most two tiles per CTA, so here every phase of every barrier runs
many times.  The popcount scan (CUDA cores,
no persistence, no block minima) must give the same Hamming scores for
every query set bit for bit, and the select that skips blocks by their
minima must give the same candidate lists as the one that reads every
block; sampled query sets are checked against the oracle's literal
Alg. 6 on every intermediate.
"""
import numpy as np
import pytest
import torch

from paper_2412_03301_gb300 import datagen

pytestmark = pytest.mark.gpu

N_SETS, N_Q, M_CODE, L, D = 60_000, 600, 1024, 16, 32


@pytest.fixture(scope="module")
def steady(orc):
    from paper_2412_03301_gb300 import build, bvss
    build.build()
    bvss.load()
    w = datagen.workload(n_sets=N_SETS, size_lo=1, size_hi=3, d=D, n_components=64,
                         n_queries=N_Q, q_lo=1, q_hi=6, m=M_CODE, fanin=4, seed=41)
    ix = bvss.bvss_build(w["vectors"].cuda(), w["offsets"], w["proj"], wta_l=L)
    oix = orc.Index(w["vectors"].numpy(), w["offsets"], w["proj"], L)
    yield bvss, w, ix, oix
    ix.close()


def _np(t, dtype=None):
    a = t.detach().cpu().numpy()
    return a.view(dtype) if dtype is not None else a


@pytest.mark.parametrize("A,M,C", [(3, 1, 300), (2, 0, 1000), (3, 2, 40)])
def test_scan_steady_state_against_popcount_and_oracle(steady, orc, A, M, C):
    bvss, w, ix, oix = steady
    qv, qo = w["q_vectors"].cuda(), w["q_offsets"]
    a = bvss.bvss_query_trace(ix, qv, qo, k=5, C=C, A=A, M=M)
    b = bvss.bvss_query_trace(ix, qv, qo, k=5, C=C, A=A, M=M, popc_scan=True)
    c = bvss.bvss_query_trace(ix, qv, qo, k=5, C=C, A=A, M=M, scan_sets_tmem=True)
    torch.cuda.synchronize()
    bvss.bvss_sync(ix)
    ha, hb, hc = _np(a["h"], np.uint16), _np(b["h"], np.uint16), _np(c["h"], np.uint16)
    assert ha.shape == (N_Q, N_SETS)
    for other, name in ((hb, "popcount"), (hc, "sets-in-tensor-memory")):
        rows = np.nonzero((ha != other).any(axis=1))[0]
        assert rows.size == 0, "h differs from the %s form for query sets %s" % (
            name, rows[:10].tolist())
    for t in (b, c):
        assert torch.equal(a["cand"], t["cand"]) and torch.equal(a["n_cand"], t["n_cand"])
        assert torch.equal(a["ids"], t["ids"]) and torch.equal(a["dist"], t["dist"])
    cand, ncand = _np(a["cand"]), _np(a["n_cand"])
    qvec = w["q_vectors"].numpy()
    # query sets of the first, a middle and the last query-block pair, and the last query
    for q in (0, 255, 256, 300, 511, 512, N_Q - 1):
        r = orc.query(oix, qvec[qo[q]:qo[q + 1]], k=5, C=C, A=A, M=M)
        assert np.array_equal(_np(a["sq"], np.uint32)[q], r["sq"]), q
        assert np.array_equal(_np(a["plist"], np.uint16)[q], r["plist"]), q
        want = np.where(r["gate"] == 1, r["h"], 0xFFFF)
        assert np.array_equal(ha[q].astype(np.int64), want.astype(np.int64)), q
        n = int(ncand[q])
        assert n == r["cand"].shape[0], q
        assert np.array_equal(cand[q, :n], r["cand"]), q
        assert np.all(cand[q, n:] == -1), q
        assert _np(a["ids"])[q].tolist() == r["ids"].tolist(), q
