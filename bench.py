#!/usr/bin/env python
"""Throughput of the BioVSS++ query path (arXiv 2412.03301) on GB300.

One step = one bvss_query call over a batch of 1000 query sets against an
index of 1,000,000 synthetic vector sets (d = 384, FlyHash m = 4096, F = 8,
L = 64, C = 2000, k = 10, A = 3, M = 1): FlyHash of the queries, both filter
layers over every set, the candidate select, the exact FP32 Hausdorff
re-rank and the top-k -- all in the library's CUDA kernels.

Prints one JSON line (rank 0).  Under torchrun every rank holds its own copy
of the index and answers its own query batch (query sets are independent),
so the work per GPU is fixed ("weak" scaling) and no collective touches the
data path; ranks only meet at the barriers around the timed region.

--impl reference times the CPU oracle instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "query sets/s at recall@10≥0.95 (1M sets); fast vs plain form, same GB300"
UNIT = "query sets/s"
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
POPC_PER_CLK_PER_SM = 16   # 32-bit population count throughput per SM per clock
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["large", "small", "profile"], default="large",
                    help="large: the 1M-set workload; small: the 2000-set test case; "
                         "profile: large-case shapes at 120k sets and 100 query sets, a few GB "
                         "on the device, for profiler captures")
    ap.add_argument("--queries", type=int, default=0,
                    help="override the number of query sets of the workload (profiling)")
    ap.add_argument("--recall-queries", type=int, default=200)
    ap.add_argument("--alg2-queries", type=int, default=100,
                    help="query sets for the plain BioVSS search (Alg. 2) line; 0 skips it")
    ap.add_argument("--learned", type=int, default=1,
                    help="1: also train the learned projection and compare it with FlyHash")
    ap.add_argument("--learned-train-queries", type=int, default=20000)
    ap.add_argument("--learned-pairs", type=int, default=2_000_000)
    ap.add_argument("--offgrid", type=int, default=1,
                    help="1: also time the three refine forms on the large workload off the "
                         "2^-8 grid and check them against the FP64 oracle")
    ap.add_argument("--offgrid-recall-queries", type=int, default=100)
    ap.add_argument("--fp8-high-d", type=int, default=1,
                    help="1: also run every refine form at the FP8 load (500k sets, d = 1024)")
    ap.add_argument("--fp8-recall-queries", type=int, default=100)
    ap.add_argument("--serving-queries", type=int, default=4096,
                    help="query sets per pass of the batched serving line (200k Zipf-sized "
                         "sets, d=768, one graph launch per pass); 0 skips it")
    ap.add_argument("--serving-recall-queries", type=int, default=500)
    ap.add_argument("--cpu-sample-sets", type=int, default=10000)
    ap.add_argument("--cpu-sample-queries", type=int, default=32,
                    help="query sets of the all-core oracle sample (a quarter of them, at "
                         "least 4, for the one-core figure)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--seed", type=int, default=0)
    return ap.parse_args()


def workload_cfg(name, n_queries=0):
    from paper_2412_03301_gb300 import datagen
    c = dict(datagen.SMALL if name == "small" else datagen.LARGE)
    if name == "profile":
        c["n_sets"], c["n_queries"] = 120_000, 100
    if n_queries > 0:
        c["n_queries"] = n_queries
    c["A"], c["M"] = 3, 1
    return c


def workload_name(c):
    return ("vector-set search, N=%d sets of %d-%d vectors, d=%d FP32 (grid 2^-8), "
            "%d-component mixture; FlyHash m=%d F=%d L=%d; %d query sets of %d-%d; "
            "A=%d M=%d C=%d k=%d" % (c["n_sets"], c["size_lo"], c["size_hi"], c["d"],
                                     c["n_components"], c["m"], c["fanin"], c["L"],
                                     c["n_queries"], c["q_lo"], c["q_hi"], c["A"], c["M"],
                                     c["C"], c["k"]))


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.proc = None
        self.uuid = None
        try:
            u = str(torch.cuda.get_device_properties(device).uuid)
            self.uuid = u if u.startswith("GPU-") else "GPU-" + u
        except Exception:
            pass

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=10)
        except Exception:
            self.proc.kill()
            out = ""
        sm, smax, power, reasons = [], [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            if self.uuid and f[0] != self.uuid:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# --------------------------------------------------------------------------
# exact ground truth (recall measurement only; plain torch GEMM + reductions)
# --------------------------------------------------------------------------
def exact_topk(vec, vnorm, set_of_row, n_sets, qvec, qoff, qids, k, chunk=1 << 21):
    """Exact Hausdorff top-k over every set for the listed query sets.

    Squared distances |q|^2 + |v|^2 - 2 q.v in FP32 (exact for values on the
    2^-8 grid).  Ties go to the lower id.  Returns (ids (len(qids), k), their
    squared distances, ascending)."""
    # TF32 would round the GEMM's inputs to 11 significant bits: the tool must stay FP32
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        return _exact_topk(vec, vnorm, set_of_row, n_sets, qvec, qoff, qids, k, chunk)
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


def _exact_topk(vec, vnorm, set_of_row, n_sets, qvec, qoff, qids, k, chunk):
    V = vec.shape[0]
    out_ids, out_d2 = [], []
    for q in qids:
        Q = qvec[qoff[q]:qoff[q + 1]]
        mq = Q.shape[0]
        qn = (Q * Q).sum(1)
        rowpart = torch.full((mq, n_sets), float("inf"), device=vec.device)
        colpart = torch.zeros(n_sets, device=vec.device)
        for r0 in range(0, V, chunk):
            r1 = min(V, r0 + chunk)
            D = torch.addmm(qn[:, None] + vnorm[None, r0:r1], Q, vec[r0:r1].T, beta=1, alpha=-2)
            D.clamp_(min=0)
            sid = set_of_row[r0:r1]
            rowpart.scatter_reduce_(1, sid.expand(mq, -1), D, "amin")
            colpart.scatter_reduce_(0, sid, D.min(0).values, "amax")
        h2 = torch.maximum(rowpart.max(0).values, colpart)
        srt, idx = torch.sort(h2, stable=True)
        out_ids.append(idx[:k])
        out_d2.append(srt[:k])
    return torch.stack(out_ids), torch.stack(out_d2)


def recall_at_k(got_ids, gt_ids, gt_d2, got_true_d2, k):
    """(strict, tie-aware) recall@k averaged over queries (Sec. 7.1.3 metric)."""
    strict, ties = [], []
    for q in range(gt_ids.shape[0]):
        g = set(gt_ids[q].tolist())
        r = [i for i in got_ids[q].tolist() if i >= 0]
        strict.append(len(g.intersection(r)) / len(g))
        kth = gt_d2[q, k - 1]
        ties.append(min(k, int((got_true_d2[q] <= kth).sum())) / k)
    return float(np.mean(strict)), float(np.mean(ties))


def true_d2_of(vec, vnorm, qvec, qoff, offsets, qids, ids):
    """Squared Hausdorff (same FP32 GEMM form as exact_topk) of given (query, set) pairs."""
    out = np.full(ids.shape, np.inf)
    for j, q in enumerate(qids):
        Q = qvec[qoff[q]:qoff[q + 1]]
        qn = (Q * Q).sum(1)
        for c, i in enumerate(ids[j].tolist()):
            if i < 0:
                continue
            r0, r1 = int(offsets[i]), int(offsets[i + 1])
            D = qn[:, None] + vnorm[None, r0:r1] - 2 * Q @ vec[r0:r1].T
            D.clamp_(min=0)
            out[j, c] = float(torch.maximum(D.min(1).values.max(), D.min(0).values.max()))
    return out


# --------------------------------------------------------------------------
# the learned projection (BioHash in place of FlyHash): trained on mined pairs
# --------------------------------------------------------------------------
def learned_line(args, dev, stream, ix, w, c, qids, gt_ids, gt_d2, vec, vnorm):
    """Train the dense layer on pairs mined from the exact refine's neighbours of
    20,000 training query sets (1M positives, 1M hard negatives, 5 epochs of 10k-pair
    batches), build the learned index, and compare recall@10 and query sets/s with the
    random FlyHash index at several candidate budgets C (BF16 fast form both)."""
    from paper_2412_03301_gb300 import bvss, datagen, learn
    off, qv, qo = w["offsets"], w["q_vectors"], w["q_offsets"]
    nq = qo.shape[0] - 1
    ts = datagen.set_sizes(args.learned_train_queries, c["q_lo"], c["q_hi"], 777 + args.seed)
    mix = datagen.Mixture(c["d"], c["n_components"], args.seed, device=dev)
    tq = mix.draw_sets(ts, 778 + args.seed)
    to = datagen.offsets_from_sizes(ts)
    t0 = time.perf_counter()
    pairs = learn.mine_pairs(ix, tq, to, k=c["k"], C=c["C"], n_pos=args.learned_pairs // 2,
                             n_neg=args.learned_pairs // 2, seed=5 + args.seed, hard=50)
    torch.cuda.synchronize(dev)
    t1 = time.perf_counter()
    w0 = learn.flyhash_dense(w["proj"], c["d"])
    wl, wq, hist = learn.train(ix, tq, pairs, w0, L=c["L"], epochs=5, batch=10_000,
                               seed=args.seed)
    torch.cuda.synchronize(dev)
    t2 = time.perf_counter()
    lix = bvss.bvss_build_dense(w["vectors"], off, wq.float().contiguous(), wta_l=c["L"],
                                bf16=True)
    torch.cuda.synchronize(dev)
    t3 = time.perf_counter()
    out_ids = torch.empty((nq, c["k"]), dtype=torch.int64, device=dev)
    out_dist = torch.empty((nq, c["k"]), dtype=torch.float32, device=dev)
    nr = len(qids)

    def measure(index, C):
        kw = dict(k=c["k"], C=C, A=c["A"], M=c["M"], fast=True)
        for _ in range(max(1, args.warmup)):
            bvss.bvss_query(index, qv, qo, out_ids=out_ids, out_dist=out_dist, stream=stream,
                            **kw)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = max(2, min(args.steps, 5))
        e0.record(stream)
        for _ in range(reps):
            bvss.bvss_query(index, qv, qo, out_ids=out_ids, out_dist=out_dist, stream=stream,
                            **kw)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / reps
        got = out_ids[:nr].cpu().numpy()
        d2 = true_d2_of(vec, vnorm, qv, qo, off, qids, got)
        r = recall_at_k(got, gt_ids, gt_d2, d2, c["k"])
        return {"C": C, "value": nq / (ms / 1e3), "ms_per_step": ms, "recall_at_10": r[0],
                "recall_at_10_ties": r[1]}

    budgets = (500, 750, 1000, 1250, 1500, 1750, 2000)
    learned = [measure(lix, C) for C in budgets]
    flyhash = [measure(ix, C) for C in budgets]
    lix.close()
    return {"train_query_sets": int(ts.shape[0]), "pairs": int(pairs[0].shape[0]),
            "hard_negatives": "nearest vector in a set ranked 11-50 by the exact refine",
            "epochs": 5, "batch": 10_000, "steps": len(hist), "mine_s": t1 - t0,
            "train_s": t2 - t1, "build_s": t3 - t2,
            "loss_first": hist[0][0], "loss_last": hist[-1][0],
            "update_magnitude_first": hist[0][1], "update_magnitude_last": hist[-1][1],
            "grad_absmax_first": hist[0][2], "grad_absmax_last": hist[-1][2],
            "recall_queries": nr, "learned": learned, "flyhash": flyhash,
            "form": "BF16 dense 384->4096 layer on the tensor cores (tcgen05), WTA top-64; "
                    "BF16 fast refine"}


# --------------------------------------------------------------------------
# the large workload off the 2^-8 grid: every form against the FP64 oracle
# --------------------------------------------------------------------------
def fp64_recall(ids, gt_ids, qvec, qoff, vec_of, k):
    """Recall@k decided in FP64: the true top k of each query set are the k smallest
    oracle Hausdorff distances (Def. 4, FP64) among the ground truth's list (which holds
    them: its FP32 errors are far below the spacing it leaves beyond k) and the returned
    ids, ties by id.  vec_of(i) -> set i's vectors (numpy).  Returns (recall, the FP64
    distances of the returned ids)."""
    from oracle import oracle
    rec, dist = [], np.full(ids.shape, np.inf)
    for j in range(ids.shape[0]):
        Q = qvec[qoff[j]:qoff[j + 1]]
        pool = sorted(set(int(i) for i in gt_ids[j]) | set(int(i) for i in ids[j] if i >= 0))
        hd = {i: oracle.haus(Q, vec_of(i)) for i in pool}
        true = sorted(pool, key=lambda i: (hd[i], i))[:k]
        rec.append(len(set(true) & set(int(i) for i in ids[j])) / k)
        for c_, i in enumerate(ids[j]):
            if i >= 0:
                dist[j, c_] = hd[int(i)]
    return float(np.mean(rec)), dist


def offgrid_line(args, dev, stream):
    """The large workload (1M sets, d = 384) drawn with the same seed but not rounded to
    the 2^-8 grid, so BF16 / FP8 copies and FP32 sums all round: the three refine forms
    timed on it, their ids compared, recall@10 decided in FP64 and every returned distance
    compared with the oracle's FP64 Hausdorff value on sampled query sets."""
    from paper_2412_03301_gb300 import bvss, datagen
    c = dict(datagen.LARGE)
    c["A"], c["M"] = 3, 1
    w = datagen.workload(n_sets=c["n_sets"], size_lo=c["size_lo"], size_hi=c["size_hi"],
                         d=c["d"], n_components=c["n_components"], n_queries=c["n_queries"],
                         q_lo=c["q_lo"], q_hi=c["q_hi"], m=c["m"], fanin=c["fanin"],
                         seed=args.seed, device=dev, grid=False)
    off, qv, qo = w["offsets"], w["q_vectors"], w["q_offsets"]
    nq = qo.shape[0] - 1
    ix = bvss.bvss_build(w["vectors"], off, w["proj"], wta_l=c["L"], bf16=True, fp8=True)
    kw = dict(k=c["k"], C=c["C"], A=c["A"], M=c["M"])
    out_ids = torch.empty((nq, c["k"]), dtype=torch.int64, device=dev)
    out_dist = torch.empty((nq, c["k"]), dtype=torch.float32, device=dev)
    forms, res = {}, {}
    steps = max(1, min(args.steps, 5))
    for name, f in (("plain", {}), ("tf32", {"tf32": True}), ("fast", {"fast": True}),
                    ("fp8", {"fp8": True})):
        for _ in range(args.warmup):
            bvss.bvss_query(ix, qv, qo, out_ids=out_ids, out_dist=out_dist, stream=stream,
                            **kw, **f)
        torch.cuda.synchronize(dev)
        bvss.bvss_profile_enable(ix, True)
        bvss.bvss_profile_read(ix, reset=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            bvss.bvss_query(ix, qv, qo, out_ids=out_ids, out_dist=out_dist, stream=stream,
                            **kw, **f)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        st, _, nl = bvss.bvss_profile_read(ix, reset=True)
        bvss.bvss_profile_enable(ix, False)
        bvss.bvss_sync(ix, stream)
        ms = e0.elapsed_time(e1) / steps
        res[name] = (out_ids.cpu().numpy().copy(), out_dist.cpu().numpy().astype(np.float64))
        forms[name] = {"value": nq / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
                       "stages_ms_per_step": {k_: v / steps for k_, v in st.items()},
                       "gpu_launches_per_step": nl // steps}
    ids_p = res["plain"][0]
    same = {name: int((res[name][0] == ids_p).all(axis=1).sum())
            for name in ("tf32", "fast", "fp8")}
    # recall and distance errors against the FP64 oracle on the first query sets
    nr = min(args.offgrid_recall_queries, nq)
    vec = w["vectors"]
    vnorm = (vec * vec).sum(1)
    set_of_row = torch.repeat_interleave(torch.arange(c["n_sets"], device=dev),
                                         torch.from_numpy(np.diff(off)).to(dev))
    gt_ids, _ = exact_topk(vec, vnorm, set_of_row, c["n_sets"], qv, qo, list(range(nr)),
                           c["k"] + 5)
    gt_ids = gt_ids.cpu().numpy()
    del vnorm, set_of_row
    qvec_h = qv[:int(qo[nr])].cpu().numpy()
    cache = {}

    def vec_of(i):
        if i not in cache:
            cache[i] = vec[int(off[i]):int(off[i + 1])].cpu().numpy()
        return cache[i]

    for name in ("plain", "tf32", "fast", "fp8"):
        ids, dist = res[name][0][:nr], res[name][1][:nr]
        r, d64 = fp64_recall(ids, gt_ids, qvec_h, qo, vec_of, c["k"])
        ok = np.isfinite(d64)
        rel = np.abs(dist[ok] - d64[ok]) / np.maximum(d64[ok], 1e-30)
        forms[name].update({"recall_at_10_fp64": r, "queries": nr,
                            "dist_rel_err_max": float(rel.max()) if rel.size else 0.0,
                            "dist_rel_err_mean": float(rel.mean()) if rel.size else 0.0,
                            "dist_rel_err_bound": (36 + -(-c["d"] // 32)) * 2.0 ** -24})
    ix.close()
    del w
    torch.cuda.empty_cache()
    return {"workload": "N=%d sets of %d-%d vectors, d=%d FP32 unit vectors NOT rounded to the "
                        "2^-8 grid, %d-component mixture; FlyHash m=%d F=%d L=%d; %d query sets; "
                        "A=%d M=%d C=%d k=%d" % (c["n_sets"], c["size_lo"], c["size_hi"], c["d"],
                                                c["n_components"], c["m"], c["fanin"], c["L"],
                                                nq, c["A"], c["M"], c["C"], c["k"]),
            "forms": forms, "same_ids_as_plain": same, "query_sets": nq}


# --------------------------------------------------------------------------
# the FP8 refine at its own load: 500k Zipf-sized sets at d = 1024, C = 4000
# --------------------------------------------------------------------------
def fp8_high_d_line(args, dev, stream):
    """datagen.FP8_HIGH_D: every refine form on the same 2000 query sets (C = 4000):
    query sets/s, the FP8 refine's HBM fraction, ids against the exact FP32 form, recall@10
    decided in FP64 and every returned distance against the oracle's FP64 value on the
    first query sets."""
    from paper_2412_03301_gb300 import bvss, datagen
    c = dict(datagen.FP8_HIGH_D)
    c["A"], c["M"] = 3, 1
    w = datagen.workload(n_sets=c["n_sets"], size_lo=c["size_lo"], size_hi=c["size_hi"],
                         d=c["d"], n_components=c["n_components"], n_queries=c["n_queries"],
                         q_lo=c["q_lo"], q_hi=c["q_hi"], m=c["m"], fanin=c["fanin"],
                         seed=args.seed + 11, device=dev, size_dist="zipf", q_dist="zipf")
    off, qv, qo = w["offsets"], w["q_vectors"], w["q_offsets"]
    nq = qo.shape[0] - 1
    t0 = time.perf_counter()
    ix = bvss.bvss_build(w["vectors"], off, w["proj"], wta_l=c["L"], bf16=True, fp8=True)
    torch.cuda.synchronize(dev)
    build_s = time.perf_counter() - t0
    kw = dict(k=c["k"], C=c["C"], A=c["A"], M=c["M"])
    tr = bvss.bvss_query_trace(ix, qv, qo, **kw)
    torch.cuda.synchronize(dev)
    sizes = torch.from_numpy(np.diff(off)).to(dev)
    cand = tr["cand"]
    cand_rows = int(sizes[cand.clamp(min=0).to(torch.int64)].masked_fill(cand < 0, 0).sum())
    del tr, cand
    out_ids = torch.empty((nq, c["k"]), dtype=torch.int64, device=dev)
    out_dist = torch.empty((nq, c["k"]), dtype=torch.float32, device=dev)
    hbm, basis = measured_peaks()
    forms, res = {}, {}
    for name, f in (("plain", {}), ("tf32", {"tf32": True}), ("fast", {"fast": True}),
                    ("fp8", {"fp8": True}), ("fp8_exact", {"fp8": True, "fp8_exact": True})):
        bvss.bvss_query(ix, qv, qo, out_ids=out_ids, out_dist=out_dist, stream=stream, **kw, **f)
        torch.cuda.synchronize(dev)
        bvss.bvss_profile_enable(ix, True)
        bvss.bvss_profile_read(ix, reset=True)
        reps = 2
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            bvss.bvss_query(ix, qv, qo, out_ids=out_ids, out_dist=out_dist, stream=stream,
                            **kw, **f)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        st, _, nl = bvss.bvss_profile_read(ix, reset=True)
        bvss.bvss_profile_enable(ix, False)
        bvss.bvss_sync(ix, stream)
        ms = e0.elapsed_time(e1) / reps
        stages = {k_: v / reps for k_, v in st.items()}
        res[name] = (out_ids.cpu().numpy().copy(), out_dist.cpu().numpy().astype(np.float64))
        forms[name] = {"value": nq / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
                       "stages_ms_per_step": stages, "gpu_launches_per_step": nl // reps}
        row_bytes = {"plain": 4, "tf32": 4, "fast": 2, "fp8": 1, "fp8_exact": 1}[name] * c["d"]
        ach = cand_rows * row_bytes / (stages["refine"] / 1e3) / 1e9
        forms[name]["refine_roofline"] = {"bound": "hbm", "achieved": ach, "peak": hbm,
                                          "unit": "GB/s", "frac": ach / hbm,
                                          "peak_basis": basis,
                                          "algorithmic_bytes": cand_rows * row_bytes}
    ids_p = res["plain"][0]
    same = {n_: int((res[n_][0] == ids_p).all(axis=1).sum()) for n_ in res if n_ != "plain"}
    nr = min(args.fp8_recall_queries, nq)
    vec = w["vectors"]
    vnorm = (vec * vec).sum(1)
    sor = torch.repeat_interleave(torch.arange(c["n_sets"], device=dev), sizes)
    gt_ids, _ = exact_topk(vec, vnorm, sor, c["n_sets"], qv, qo, list(range(nr)), c["k"] + 5)
    gt_ids = gt_ids.cpu().numpy()
    del vnorm, sor
    qvec_h = qv[:int(qo[nr])].cpu().numpy()
    cache = {}

    def vec_of(i):
        if i not in cache:
            cache[i] = vec[int(off[i]):int(off[i + 1])].cpu().numpy()
        return cache[i]

    for name in res:
        ids, dist = res[name][0][:nr], res[name][1][:nr]
        r, d64 = fp64_recall(ids, gt_ids, qvec_h, qo, vec_of, c["k"])
        ok = np.isfinite(d64)
        rel = np.abs(dist[ok] - d64[ok]) / np.maximum(d64[ok], 1e-30)
        forms[name].update({"recall_at_10_fp64": r, "dist_rel_err_max": float(rel.max()),
                            "dist_rel_err_mean": float(rel.mean())})
    ix.close()
    del w
    torch.cuda.empty_cache()
    return {"workload": "N=%d sets of Zipf 4-64 vectors (%d vectors), d=%d FP32 (grid 2^-8), "
                        "%d-component mixture; FlyHash m=%d F=%d L=%d; %d query sets of Zipf "
                        "4-64; A=%d M=%d C=%d k=%d" % (c["n_sets"], int(off[-1]), c["d"],
                                                      c["n_components"], c["m"], c["fanin"],
                                                      c["L"], nq, c["A"], c["M"], c["C"],
                                                      c["k"]),
            "build_s": build_s, "candidate_rows_per_step": cand_rows, "forms": forms,
            "same_ids_as_plain": same, "query_sets": nq, "recall_queries": nr,
            "dist_rel_err_bound_exact": (36 + -(-c["d"] // 32)) * 2.0 ** -24}


# --------------------------------------------------------------------------
# batched serving line: a query plan (one CUDA graph launch per pass)
# --------------------------------------------------------------------------
def serving_line(args, dev, stream):
    """The serving load (datagen.SERVING): 200k sets of Zipf sizes 1-128, d = 768, a pass of
    uneven query sets of 1-64 vectors run as one graph launch of a tuned plan."""
    from paper_2412_03301_gb300 import bvss, datagen
    c = dict(datagen.SERVING)
    c["A"], c["M"] = 3, 1
    nq = args.serving_queries
    w = datagen.workload(n_sets=c["n_sets"], size_lo=c["size_lo"], size_hi=c["size_hi"],
                         d=c["d"], n_components=c["n_components"], n_queries=nq,
                         q_lo=c["q_lo"], q_hi=c["q_hi"], m=c["m"], fanin=c["fanin"],
                         seed=args.seed + 7, device=dev, size_dist="zipf")
    off, qv, qo = w["offsets"], w["q_vectors"], w["q_offsets"]
    ix = bvss.bvss_build(w["vectors"], off, w["proj"], wta_l=c["L"], bf16=True)
    kw = dict(k=c["k"], C=c["C"], A=c["A"], M=c["M"], fast=True)
    plan = bvss.Plan(ix, nq, int(qo[-1]), c["q_hi"], stream=stream, **kw)
    plan.set_queries(qv, qo, stream=stream)

    def time_plan(steps):
        for _ in range(args.warmup):
            plan.launch(stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            plan.launch(stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / steps

    ms_default = time_plan(max(2, args.steps // 4))
    knobs_default = plan.info()
    t0 = time.perf_counter()
    plan.tune(reps=2, stream=stream)
    tune_s = time.perf_counter() - t0
    ms = time_plan(args.steps)
    bvss.bvss_sync(ix, stream)
    ids_plan = plan.ids.clone()
    # the same pass through bvss_query (host offsets, no graph), for comparison and parity
    ids_q, _ = bvss.bvss_query(ix, qv, qo, stream=stream, **kw)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(max(2, args.steps // 4)):
        bvss.bvss_query(ix, qv, qo, out_ids=ids_q, stream=stream, **kw)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_query = e0.elapsed_time(e1) / max(2, args.steps // 4)
    rec = None
    if args.serving_recall_queries > 0:
        vec = w["vectors"]
        vnorm = (vec * vec).sum(1)
        set_of_row = torch.repeat_interleave(torch.arange(c["n_sets"], device=dev),
                                             torch.from_numpy(np.diff(off)).to(dev))
        qids = list(range(min(args.serving_recall_queries, nq)))
        gt_ids, gt_d2 = exact_topk(vec, vnorm, set_of_row, c["n_sets"], qv, qo, qids, c["k"])
        got = ids_plan[qids].cpu().numpy()
        got_d2 = true_d2_of(vec, vnorm, qv, qo, off, qids, got)
        rs, rt = recall_at_k(got, gt_ids.cpu().numpy(), gt_d2.cpu().numpy(), got_d2, c["k"])
        rec = {"recall_at_10": rs, "recall_at_10_ties": rt, "queries": len(qids)}
    nv = int(off[-1])
    out = {"value": nq / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "query_sets": nq,
           "query_vectors": int(qo[-1]),
           "workload": "N=%d sets, Zipf sizes %d-%d (%d vectors), d=%d (BF16-exact grid values), "
                       "%d-component mixture; FlyHash m=%d F=%d L=%d; %d query sets of %d-%d "
                       "vectors; A=%d M=%d C=%d k=%d"
                       % (c["n_sets"], c["size_lo"], c["size_hi"], nv, c["d"],
                          c["n_components"], c["m"], c["fanin"], c["L"], nq, c["q_lo"],
                          c["q_hi"], c["A"], c["M"], c["C"], c["k"]),
           "form": "one CUDA graph launch per pass (bvss_plan), tensor-core scan and BF16 "
                   "tensor-core refine (query sets of <= 32 vectors on the 32-wide instance, "
                   "the wider ones on the 64-wide one, unless the tuner drops the split), "
                   "boundary re-score for the exact top-k",
           "tuned": plan.info(), "untuned": dict(knobs_default, ms_per_step=ms_default),
           "tune_s": tune_s,
           "bvss_query_ms_per_step": ms_query, "same_ids_as_bvss_query": bool(torch.equal(ids_plan, ids_q)),
           "recall": rec,
           "l2": "vectors %.1f GB BF16 + %.1f GB FP32; the %.0f MB sketch matrix is evicted by "
                 "each pass's refine traffic" % (nv * c["d"] * 2 / 1e9, nv * c["d"] * 4 / 1e9,
                                                 c["n_sets"] * c["m"] / 8 / 1e6)}
    plan.close()
    ix.close()
    return out


# --------------------------------------------------------------------------
# CPU oracle timing (bounded sample)
# --------------------------------------------------------------------------
def host_cores():
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_sample_index(vec_host, offsets, proj, c, n_sets_s, threads=1):
    from oracle import oracle
    off_s = offsets[:n_sets_s + 1].copy()
    return oracle.Index(vec_host[:off_s[-1]], off_s, proj, c["L"], threads=threads)


def oracle_throughput(ix, qvec_host, qoff, qids, c, n_sets_s, threads):
    """Query sets/s of the oracle's Alg. 6 run on `threads` host threads, one query set
    per thread at a time (parallel over query sets only; each query set's arithmetic
    is the oracle's own, and its C calls release the GIL).  Every query set's
    full-size time is estimated from its own stage times (oracle_query_estimate),
    measured while the other threads run beside it, so throughput = threads / the
    mean estimated time.  Returns (query sets/s, mean seconds, mean stage parts)."""
    from concurrent.futures import ThreadPoolExecutor

    def one(q):
        return oracle_query_estimate(ix, qvec_host[qoff[q]:qoff[q + 1]], c, n_sets_s)

    if threads == 1:
        ests = [one(q) for q in qids]
    else:
        with ThreadPoolExecutor(threads) as ex:
            ests = list(ex.map(one, qids))
    per_q = float(np.mean([e[0] for e in ests]))
    parts = np.mean([e[1] for e in ests], axis=0)
    return threads / per_q, per_q, parts


def oracle_query_estimate(ix, Q, c, n_sets_s):
    """Seconds the oracle's Alg. 6 would take for one query set at full size.

    Measured on the sample index: the fixed part (query FlyHash and filters),
    the per-set part (gate walk, Hamming scan, heap) scaled by N / n_sets_s,
    and the refine time per candidate scaled to C candidates."""
    from oracle import oracle
    C_s = min(n_sets_s, 10 * max(c["k"], int(round(c["C"] * n_sets_s / c["n_sets"]))))
    t0 = time.perf_counter()
    qpos, _ = oracle.encode(Q, ix.proj, ix.L)
    cq, sq, plist = oracle.query_filters(qpos, ix.m, c["A"])
    t1 = time.perf_counter()
    gate = ix.inv.gate(plist, c["M"])
    h = oracle.hamming(sq, ix.sketch, gate, m=ix.m)
    cand = oracle.heap_select(h, gate, C_s)
    t2 = time.perf_counter()
    oracle.refine_topk(Q, ix.vectors, ix.set_off, cand, c["k"])
    t3 = time.perf_counter()
    parts = ((t1 - t0), (t2 - t1) * c["n_sets"] / n_sets_s,
             (t3 - t2) / max(1, len(cand)) * c["C"])
    return sum(parts), parts


def oracle_description(c, n_sets_s, n_q, threads):
    return ("oracle Alg. 6 (literal inverted lists, bit-loop Hamming, heap, FP64 refine) on "
            "%d host thread(s), one query set per thread; index of the first %d of %d sets, "
            "%d query sets; per query set, extrapolated to the full size: query "
            "FlyHash+filters + (gate walk, Hamming, heap) x %d/%d + refine time per candidate "
            "x C=%d" % (threads, n_sets_s, c["n_sets"], n_q, c["n_sets"], n_sets_s, c["C"]))


# --------------------------------------------------------------------------
# roofline
# --------------------------------------------------------------------------
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "of measured"
    except Exception:
        return 6800.0, "of fallback"


# DRAM bytes per unit of work (dram__bytes_read.sum + dram__bytes_write.sum of one ncu
# capture, divided by the units the captured launch processed), with the SHA-256 of the
# kernel's source file at capture time; the summaries are in profiles/.
TRAFFIC = {
    "k_refine_mma": dict(source="paper_2412_03301_gb300/csrc/refine_mma.cu",
                         sha256="08f24612e7c8e6fe02bcbe03b794d093c156c7e1e35c967f91493a26279fd9e3",
                         bytes_per_unit=779.5, unit="candidate row"),
    "k_refine_mma_tf32": dict(source="paper_2412_03301_gb300/csrc/refine_mma.cu",
                              sha256="08f24612e7c8e6fe02bcbe03b794d093c156c7e1e35c967f91493a26279fd9e3",
                              bytes_per_unit=1548.6, unit="candidate row"),
    "k_scan_mma": dict(source="paper_2412_03301_gb300/csrc/scan_mma.cu",
                       sha256="829de8659085867ca25179631a803c06e3b812b050ed20c942c0d3eb881e94b8",
                       bytes_per_unit=2.607505, unit="(query set, set) pair"),
    "k_refine": dict(source="paper_2412_03301_gb300/csrc/refine.cu",
                     sha256="6c5ad74bce97e56f0ef9f81aa61baf4f5f2a700f738ffa6bc0c9eadcc846e9ca",
                     bytes_per_unit=1367.8, unit="candidate row"),
}


def traffic_per_unit(kernel):
    """DRAM bytes per unit of work of `kernel` from TRAFFIC, if its source file still
    has the SHA-256 the capture was taken with (else None: the counters are stale)."""
    import hashlib
    t = TRAFFIC.get(kernel)
    if t is None:
        return None
    try:
        sha = hashlib.sha256(open(os.path.join(ROOT, t["source"]), "rb").read()).hexdigest()
    except OSError:
        return None
    return float(t["bytes_per_unit"]) if sha == t["sha256"] else None


def roofline(c, stage_ms, nbatch, nq, gated_pairs, pair_elems, cand_rows, fast=False, steps=1):
    """Roofline of the dominant kernel (scan or refine) of the timed region.

    Each kernel has a compute roof and an HBM roof; the one with the longer time
    at peak binds.  Times are the kernel's own CUDA-event stage (the gate words
    and the FP8 query operand are a stage of their own, so is the re-score).

    k_scan_mma (tensor cores, FP8): FLOPs = 2 x query sets x N x m (every pair,
    the algorithmic GEMM) against the FP8 peak (measured sustained BF16 x 2, the
    nominal FP8/BF16 ratio); bytes = sketch matrix once + gate words read + h
    written.  k_scan (CUDA cores): 32-bit popcounts = gated pairs x m/32 at
    152 SMs x 16/clk x 2070 MHz.  k_refine_mma: bytes = candidate rows x d x 2
    (BF16 gather); tensor FLOPs = 2 x (query vector, candidate vector) pairs x d
    against sustained BF16.  k_refine_tma / k_refine: the same pairs on FP32
    lanes (152 x 128 x 2 x 2070 MHz), bytes = rows x d x 4."""
    hbm, hbm_basis = measured_peaks()
    per = {k: v / max(1, nbatch) for k, v in stage_ms.items()}     # ms per launch
    # work per launch: stage_ms and nbatch cover `steps` steps, the work counts one step,
    # and each kernel launches once per internal batch
    per_launch = steps / max(1, nbatch)
    nq, gated_pairs, pair_elems, cand_rows = (x * per_launch for x in
                                              (nq, gated_pairs, pair_elems, cand_rows))
    clock = SM_MAX_MHZ * 1e6
    try:
        mp = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        bf16_peak, bf16_basis = float(mp["bf16_tflops_sustained"]) * 1e12, "of measured"
    except Exception:
        bf16_peak, bf16_basis = 1.7e15, "of fallback"
    nw = (c["n_sets"] + 31) // 32
    scan_bytes = c["n_sets"] * c["m"] / 8 + nq * nw * 4 + nq * c["n_sets"] * 2
    tensor_scan = True          # the library default (BVSS_SEARCH_POPC_SCAN off)
    if tensor_scan:
        scan = dict(name="k_scan_mma", t=per["scan"],
                    alu=(2.0 * nq * c["n_sets"] * c["m"], 2 * bf16_peak, "TFLOP/s",
                         bf16_basis + " sustained bf16 x 2 (FP8 nominal ratio)", "tensor"),
                    hbm_bytes=scan_bytes, units=nq * c["n_sets"])
    else:
        scan = dict(name="k_scan", t=per["scan"],
                    alu=(gated_pairs * (c["m"] // 32), SM_COUNT * POPC_PER_CLK_PER_SM * clock,
                         "Tpopc/s", "152 SMs x 16 popc/clk x 2070 MHz (nominal, measured 15.1)",
                         "alu"),
                    hbm_bytes=scan_bytes, units=None)
    if fast and c["d"] % 64 == 0 and c["q_hi"] <= 64:
        refine = dict(name="k_refine_mma", t=per["refine"],
                      alu=(2.0 * pair_elems * c["d"], bf16_peak, "TFLOP/s",
                           bf16_basis + " sustained bf16", "tensor"),
                      hbm_bytes=cand_rows * c["d"] * 2.0, units=cand_rows)
    else:
        refine = dict(name="k_refine_tma" if c["d"] % 4 == 0 and c["q_hi"] <= 64 else "k_refine",
                      t=per["refine"],
                      alu=(2.0 * pair_elems * c["d"], SM_COUNT * FP32_LANES_PER_SM * 2 * clock,
                           "TFLOP/s", "152 SMs x 128 FP32 lanes x 2 x 2070 MHz (nominal FMA)",
                           "alu"),
                      hbm_bytes=cand_rows * c["d"] * 4.0, units=cand_rows)
    kern = {"scan": scan, "refine": refine}

    def entry(k):
        t = k["t"] / 1e3
        ops, peak_ops, unit, basis, alu_bound = k["alu"]
        t_alu, t_hbm = ops / peak_ops, k["hbm_bytes"] / (hbm * 1e9)
        tpu = traffic_per_unit(k["name"])
        traffic = tpu * k["units"] if (tpu is not None and k["units"]) else None
        if t_hbm >= t_alu:
            ach = k["hbm_bytes"] / t / 1e9
            return {"kernel": k["name"], "bound": "hbm", "achieved": ach, "peak": hbm,
                    "unit": "GB/s", "frac": ach / hbm, "traffic": traffic,
                    "algorithmic_bytes": k["hbm_bytes"], "launch_ms": k["t"],
                    "peak_basis": hbm_basis + " (MEASURED_PEAKS.json hbm_gbs)" if hbm_basis ==
                    "of measured" else hbm_basis,
                    "compute_roof": {"achieved": ops / t / 1e12, "peak": peak_ops / 1e12,
                                     "unit": unit, "basis": basis}}
        ach = ops / t / 1e12
        return {"kernel": k["name"], "bound": alu_bound, "achieved": ach, "peak": peak_ops / 1e12,
                "unit": unit, "frac": ach / (peak_ops / 1e12), "traffic": traffic,
                "peak_basis": basis, "algorithmic_bytes": k["hbm_bytes"], "launch_ms": k["t"],
                "hbm_roof": {"achieved": k["hbm_bytes"] / t / 1e9, "peak": hbm, "unit": "GB/s"}}

    # the dominant kernel's roofline, with the other large kernel's beside it
    dom = max(kern, key=lambda k: kern[k]["t"])
    out = entry(kern[dom])
    out["other_kernels"] = [entry(kern[k]) for k in kern if k != dom]
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    from paper_2412_03301_gb300 import datagen
    from oracle import oracle
    oracle.build()
    c = workload_cfg(args.workload, args.queries)
    n_s = min(args.cpu_sample_sets, c["n_sets"])
    gen_dev = "cuda" if torch.cuda.is_available() else "cpu"
    w = datagen.workload(n_sets=c["n_sets"], size_lo=c["size_lo"], size_hi=c["size_hi"],
                         d=c["d"], n_components=c["n_components"], n_queries=c["n_queries"],
                         q_lo=c["q_lo"], q_hi=c["q_hi"], m=c["m"], fanin=c["fanin"],
                         seed=args.seed, device=gen_dev)
    off, qoff = w["offsets"], w["q_offsets"]
    vec_host = w["vectors"][:int(off[n_s])].cpu().numpy()
    qvec_host = w["q_vectors"].cpu().numpy()
    del w["vectors"]
    P = host_cores()
    ix = oracle_sample_index(vec_host, off, w["proj"], c, n_s, threads=P)
    # each step: P query sets at once, one per host thread
    times, nq_done = [], 0
    for s in range(args.warmup + args.steps):
        qids = [(s * P + j) % c["n_queries"] for j in range(P)]
        v, per_q, _ = oracle_throughput(ix, qvec_host, qoff, qids, c, n_s, P)
        if s >= args.warmup:
            times.append(per_q / P)
            nq_done += P
    value = 1.0 / float(np.mean(times))
    desc = oracle_description(c, n_s, nq_done, P) + "; %d query sets per step" % P
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.mean(times)) * P, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(c)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": P, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, rank, world, local_rank):
    from paper_2412_03301_gb300 import build as libbuild
    libbuild.build()
    from paper_2412_03301_gb300 import bvss, datagen, shard
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    c = workload_cfg(args.workload, args.queries)
    stream = torch.cuda.current_stream(dev)
    w = datagen.workload(n_sets=c["n_sets"], size_lo=c["size_lo"], size_hi=c["size_hi"],
                         d=c["d"], n_components=c["n_components"], n_queries=c["n_queries"],
                         q_lo=c["q_lo"], q_hi=c["q_hi"], m=c["m"], fanin=c["fanin"],
                         seed=args.seed, device=dev)
    # each rank answers its own query sets against the same database
    w["q_vectors"], w["q_offsets"] = shard.replica_queries(w, c, args.seed, rank, device=dev)
    off = w["offsets"]
    t0 = time.perf_counter()
    fp8_ok = c["d"] % 128 == 0 and c["q_hi"] <= 64
    ix = bvss.bvss_build(w["vectors"], off, w["proj"], wta_l=c["L"], bf16=c["d"] % 64 == 0,
                         fp8=fp8_ok)
    fast_ok = c["d"] % 64 == 0
    torch.cuda.synchronize(dev)
    build_s = time.perf_counter() - t0
    qv, qoff = w["q_vectors"], w["q_offsets"]
    nq = qoff.shape[0] - 1
    kw = dict(k=c["k"], C=c["C"], A=c["A"], M=c["M"])

    kw_fast = dict(kw, fast=fast_ok)
    # the plain form: FP32 vectors, exact FP32 results; its refine on the tensor cores
    # reading the FP32 rows as TF32 where the kernel takes the shape (the boundary stage
    # re-scores the band in FP32), the CUDA-core FP32 refine timed beside it
    kw_plain = dict(kw, tf32=c["d"] % 32 == 0)
    # one traced pass (outside the timed region): |F1| per query for the roofline
    tr = bvss.bvss_query_trace(ix, qv, qoff, **kw)
    torch.cuda.synchronize(dev)
    h = tr["h"]
    gated_pairs = int((h != -1).sum().item())        # 0xFFFF as int16 is -1
    n_cand = tr["n_cand"].to(torch.int64)
    sum_cand = int(n_cand.sum().item())
    cand = tr["cand"]
    sizes = torch.from_numpy(np.diff(off)).to(dev)
    cand_rows = int(sizes[cand.clamp(min=0).to(torch.int64)].masked_fill(cand < 0, 0).sum().item())
    qsz = torch.from_numpy(np.diff(qoff)).to(dev)
    pair_elems = int((sizes[cand.clamp(min=0).to(torch.int64)].masked_fill(cand < 0, 0)
                      * qsz[:, None]).sum().item())
    ids_ref = tr["ids"].clone()
    del tr, h, cand
    ids_fast, _ = bvss.bvss_query(ix, qv, qoff, **kw_fast)
    torch.cuda.synchronize(dev)
    fast_same = bool(torch.equal(ids_fast, ids_ref))

    # recall@10 against exact brute force (rank 0, subset of the query sets)
    rec = None
    if rank == 0 and args.recall_queries > 0:
        vec = w["vectors"]
        vnorm = (vec * vec).sum(1)
        set_of_row = torch.repeat_interleave(torch.arange(c["n_sets"], device=dev),
                                             torch.from_numpy(np.diff(off)).to(dev))
        qids = list(range(min(args.recall_queries, nq)))
        gt_ids, gt_d2 = exact_topk(vec, vnorm, set_of_row, c["n_sets"], qv, qoff, qids, c["k"])
        got = ids_fast[qids].cpu().numpy()
        got_d2 = true_d2_of(vec, vnorm, qv, qoff, off, qids, got)
        rs, rt = recall_at_k(got, gt_ids.cpu().numpy(), gt_d2.cpu().numpy(), got_d2, c["k"])
        rec = {"recall_at_10": rs, "recall_at_10_ties": rt, "queries": len(qids)}
        if c["d"] % 128 == 0 and c["q_hi"] <= 64:
            # FP8 refine: recall and the error of each returned distance against the
            # exact (FP32 GEMM-form on grid values) Hausdorff distance of the same set
            nr = len(qids)
            ids8, dist8 = bvss.bvss_query(ix, qv[:int(qoff[nr])], qoff[:nr + 1], fp8=True, **kw)
            got8 = ids8.cpu().numpy()
            d2_8 = true_d2_of(vec, vnorm, qv, qoff, off, qids, got8)
            r8 = recall_at_k(got8, gt_ids.cpu().numpy(), gt_d2.cpu().numpy(), d2_8, c["k"])
            dd = dist8.cpu().numpy().astype(np.float64)
            ok = np.isfinite(d2_8) & (got8 >= 0)
            err = np.abs(dd[ok] - np.sqrt(d2_8[ok]))
            rel = err / np.maximum(np.sqrt(d2_8[ok]), 1e-30)
            rec["fp8"] = {"recall_at_10": r8[0], "recall_at_10_ties": r8[1],
                          "dist_abs_err_max": float(err.max()) if err.size else 0.0,
                          "dist_rel_err_max": float(rel.max()) if rel.size else 0.0,
                          "dist_rel_err_mean": float(rel.mean()) if rel.size else 0.0}
        if args.alg2_queries > 0 and c["q_hi"] <= 32:
            # the same query sets through the plain BioVSS search (Alg. 2)
            nr = len(qids)
            ids2, _ = bvss.bvss_query(ix, qv[:int(qoff[nr])], qoff[:nr + 1], alg2=True, **kw_fast)
            got2 = ids2.cpu().numpy()
            d2_2 = true_d2_of(vec, vnorm, qv, qoff, off, qids, got2)
            rec["alg2"] = dict(zip(("recall_at_10", "recall_at_10_ties"),
                                   recall_at_k(got2, gt_ids.cpu().numpy(), gt_d2.cpu().numpy(),
                                               d2_2, c["k"])))
        if args.learned and args.workload == "large":
            rec["learned_projection"] = learned_line(args, dev, stream, ix, w, c, qids,
                                                     gt_ids.cpu().numpy(), gt_d2.cpu().numpy(),
                                                     vec, vnorm)
        del vnorm, set_of_row

    # CPU baseline sample (rank 0): copy the sample before freeing the database
    cpu = None
    if rank == 0 and not args.no_cpu:
        n_s = min(args.cpu_sample_sets, c["n_sets"])
        vec_host = w["vectors"][:int(off[n_s])].cpu().numpy()
        qvec_host = qv.cpu().numpy()
    del w["vectors"]
    torch.cuda.empty_cache()

    # device-resident inputs: the timed regions, plain form then fast form
    out_ids = torch.empty((nq, c["k"]), dtype=torch.int64, device=dev)
    out_dist = torch.empty((nq, c["k"]), dtype=torch.float32, device=dev)

    def timed(kwq, sample_clocks, exact=True):
        for _ in range(args.warmup):
            bvss.bvss_query(ix, qv, qoff, out_ids=out_ids, out_dist=out_dist, stream=stream, **kwq)
        torch.cuda.synchronize(dev)
        if exact:
            assert torch.equal(out_ids, ids_ref)
        bvss.bvss_profile_enable(ix, True)
        bvss.bvss_profile_read(ix, reset=True)
        clocks = ClockSampler(dev) if sample_clocks else None
        if clocks:
            clocks.start()
            time.sleep(0.3)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            bvss.bvss_query(ix, qv, qoff, out_ids=out_ids, out_dist=out_dist, stream=stream,
                            **kwq)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        clk = clocks.stop() if clocks else None
        t_ms = e0.elapsed_time(e1) / args.steps
        st_ms, nb, nl = bvss.bvss_profile_read(ix, reset=True)
        bvss.bvss_profile_enable(ix, False)
        bvss.bvss_sync(ix, stream)
        t_ms = shard.max_over_ranks(t_ms, device=dev)
        return t_ms, st_ms, nb, nl, clk

    ms_plain, stage_plain, _, _, _ = timed(kw_plain, False)
    ms_simt, stage_simt, _, _, _ = timed(kw, False)
    ms, stage_ms, nbatch, launches, clk = timed(kw_fast, True)
    value = world * nq / (ms / 1e3)
    # the FP8 refine on the same index (approximate: recall and distance error below)
    fp8 = None
    if fp8_ok:
        ms8, stage8, _, nl8, _ = timed(dict(kw, fp8=True), False, exact=False)
        fp8 = {"value": world * nq / (ms8 / 1e3), "unit": UNIT, "ms_per_step": ms8,
               "stages_ms_per_step": {k: v / args.steps for k, v in stage8.items()},
               "gpu_launches_per_step": nl8 // args.steps,
               "refine_bytes_per_step": cand_rows * c["d"],
               "refine_roofline": {
                   "bound": "hbm", "unit": "GB/s", "peak": measured_peaks()[0],
                   "achieved": cand_rows * c["d"] / (stage8["refine"] / args.steps / 1e3) / 1e9,
                   "frac": cand_rows * c["d"] / (stage8["refine"] / args.steps / 1e3) / 1e9
                   / measured_peaks()[0]},
               "accuracy": rec.get("fp8") if rec else None,
               "form": "FP8 E4M3 copies with per-vector scales on the tensor cores "
                       "(tcgen05 kind::f8f6f4), 3-sigma boundary band re-scored in FP32"}

    # the plain BioVSS search (Alg. 2) on the same index: every set is scored with Haus^H over
    # codes, so it is timed on the first --alg2-queries query sets only
    alg2 = None
    if rank == 0 and args.alg2_queries > 0 and c["q_hi"] <= 32:
        na = min(args.alg2_queries, nq)
        qo2, qv2 = qoff[:na + 1], qv[:int(qoff[na])]
        oi2 = torch.empty((na, c["k"]), dtype=torch.int64, device=dev)
        od2 = torch.empty((na, c["k"]), dtype=torch.float32, device=dev)
        kw2 = dict(kw_fast, alg2=True)
        bvss.bvss_query(ix, qv2, qo2, out_ids=oi2, out_dist=od2, stream=stream, **kw2)
        torch.cuda.synchronize(dev)
        bvss.bvss_profile_enable(ix, True)
        bvss.bvss_profile_read(ix, reset=True)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n_rep = 3
        a0.record(stream)
        for _ in range(n_rep):
            bvss.bvss_query(ix, qv2, qo2, out_ids=oi2, out_dist=od2, stream=stream, **kw2)
        a1.record(stream)
        torch.cuda.synchronize(dev)
        st2, _, nl2 = bvss.bvss_profile_read(ix, reset=True)
        bvss.bvss_profile_enable(ix, False)
        t2 = a0.elapsed_time(a1) / n_rep
        alg2 = {"value": na / (t2 / 1e3), "unit": UNIT, "query_sets": na, "ms_per_step": t2,
                "stages_ms_per_step": {k: v / n_rep for k, v in st2.items()},
                "gpu_launches_per_step": nl2 // n_rep,
                "recall": rec.get("alg2") if rec else None,
                "form": "plain BioVSS (Alg. 2): Haus^H over per-vector codes against every set, "
                        "C smallest, BF16 tensor-core refine" if fast_ok else
                        "plain BioVSS (Alg. 2), FP32 refine"}

    # end to end through the same API: pinned host query vectors in, host results out
    hq = qv.cpu().pin_memory()
    hi = torch.empty((nq, c["k"]), dtype=torch.int64).pin_memory()
    hd = torch.empty((nq, c["k"]), dtype=torch.float32).pin_memory()
    for _ in range(max(1, args.warmup)):
        bvss.bvss_query(ix, hq, qoff, out_ids=hi, out_dist=hd, stream=stream, **kw_fast)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        bvss.bvss_query(ix, hq, qoff, out_ids=hi, out_dist=hd, stream=stream, **kw_fast)
    torch.cuda.synchronize(dev)
    e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps
    e2e_ms = shard.max_over_ranks(e2e_ms, device=dev)
    assert torch.equal(hi, ids_ref.cpu())
    h2d = hq.numel() * 4 + (nq + 1) * 8
    d2h = hi.numel() * 8 + hd.numel() * 4

    if rank != 0:
        return 0
    if not args.no_cpu:
        P = host_cores()
        oix = oracle_sample_index(vec_host, off, w["proj"], c, n_s, threads=P)
        nqs = min(max(args.cpu_sample_queries, P), nq)
        v_all, per_all, parts = oracle_throughput(oix, qvec_host, qoff, list(range(nqs)), c,
                                                  n_s, P)
        n1 = min(nqs, max(4, args.cpu_sample_queries // 4))
        v_one, per_one, _ = oracle_throughput(oix, qvec_host, qoff, list(range(n1)), c, n_s, 1)
        cpu = {"value": v_all, "unit": UNIT, "cores": P, "kind": "oracle",
               "sample": oracle_description(c, n_s, nqs, P),
               "one_core": {"value": v_one, "unit": UNIT, "cores": 1,
                            "sample": oracle_description(c, n_s, n1, 1)},
               "parts_s": {"query_filters": float(parts[0]), "scan_scaled": float(parts[1]),
                           "refine_scaled": float(parts[2])}}

    # the learned projection against the plain FP32 random-FlyHash form at equal recall:
    # the smallest budget at which the learned fast form reaches the recall the FlyHash
    # indexes reach at the workload's own C
    learned = rec.pop("learned_projection", None) if rec else None
    if learned:
        target = max(r["recall_at_10_ties"] for r in learned["flyhash"] if r["C"] == c["C"])
        ok = [r for r in learned["learned"] if r["recall_at_10_ties"] >= target]
        best = min(ok, key=lambda r: r["C"]) if ok else None
        learned["equal_recall"] = {
            "target_recall_at_10_ties": target, "target": "FlyHash at C=%d" % c["C"],
            "learned_C": best["C"] if best else None,
            "learned_value": best["value"] if best else None,
            "plain_fp32_flyhash_value": world * nq / (ms_plain / 1e3),
            "learned_over_plain": best["value"] / (world * nq / (ms_plain / 1e3)) if best
            else None}
        # the metric's own operating point: the fastest budget with recall@10 >= 0.95
        for name in ("learned", "flyhash"):
            ok95 = [r for r in learned[name] if r["recall_at_10_ties"] >= 0.95]
            b95 = max(ok95, key=lambda r: r["value"]) if ok95 else None
            learned[name + "_at_0.95"] = ({"C": b95["C"], "value": b95["value"],
                                          "recall_at_10_ties": b95["recall_at_10_ties"]}
                                         if b95 else None)

    # roofline of the dominant kernel, from the per-stage CUDA events of the timed region
    roof = roofline(c, stage_ms, nbatch, nq, gated_pairs, pair_elems, cand_rows, fast_ok,
                    steps=args.steps)
    ix.close()
    torch.cuda.empty_cache()
    offgrid = (offgrid_line(args, dev, stream)
               if args.offgrid and args.workload == "large" and rank == 0 else None)
    serving = (serving_line(args, dev, stream)
               if args.serving_queries > 0 and args.workload == "large" else None)
    fp8_high_d = (fp8_high_d_line(args, dev, stream)
                  if args.fp8_high_d and args.workload == "large" and rank == 0 else None)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16" if fast_ok else "f32", "data": "synthetic",
        "config": {"workload": workload_name(c),
                   "form": ("fast: BF16 tensor-core refine (tcgen05), boundary band "
                            "re-scored in FP32 for the exact top-k; random FlyHash" if fast_ok else
                            "plain: FP32 refine, random FlyHash"),
                   "query_sets_per_step_per_gpu": nq,
                   "l2": "inputs larger than L2 (sketch matrix %.0f MB, vectors %.1f GB)"
                         % (c["n_sets"] * c["m"] / 8 / 1e6, off[-1] * c["d"] * 4 / 1e9),
                   "parallelism": "replicated index, query sets split over ranks"},
        "recall": rec,
        "plain_form": {"value": world * nq / (ms_plain / 1e3), "ms_per_step": ms_plain,
                       "stages_ms_per_step": {k: v / args.steps for k, v in stage_plain.items()},
                       "dtype": "f32", "same_ids_as_fast": fast_same,
                       "form": "FP32 vectors, random FlyHash; refine on the tensor cores "
                               "reading the FP32 rows as TF32 (tcgen05 kind::tf32), boundary "
                               "band re-scored in FP32: the same ids and distances as the "
                               "CUDA-core FP32 refine" if kw_plain["tf32"] else
                               "FP32 CUDA-core refine",
                       "refine_roofline": {
                           "bound": "hbm", "unit": "GB/s", "peak": measured_peaks()[0],
                           "achieved": cand_rows * c["d"] * 4
                           / (stage_plain["refine"] / args.steps / 1e3) / 1e9,
                           "frac": cand_rows * c["d"] * 4
                           / (stage_plain["refine"] / args.steps / 1e3) / 1e9
                           / measured_peaks()[0],
                           "traffic": (traffic_per_unit("k_refine_mma_tf32") * cand_rows
                                       if kw_plain["tf32"] and
                                       traffic_per_unit("k_refine_mma_tf32") else None)},
                       "cuda_core_refine": {
                           "value": world * nq / (ms_simt / 1e3), "ms_per_step": ms_simt,
                           "stages_ms_per_step": {k: v / args.steps
                                                  for k, v in stage_simt.items()}}},
        "roofline": roof,
        "stages_ms_per_step": {k: v / args.steps for k, v in stage_ms.items()},
        "cpu_baseline": cpu,
        "e2e": {"value": world * nq / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "alg2": alg2,
        "fp8": fp8,
        "learned": learned,
        "offgrid": offgrid,
        "serving": serving,
        "fp8_high_d": fp8_high_d,
        "clocks": clk,
        "build_s": build_s,
        "work": {"gated_pairs_per_step": gated_pairs, "candidates_per_step": sum_cand,
                 "candidate_rows_per_step": cand_rows},
    }
    print(json.dumps(line), flush=True)
    ix.close()
    return 0


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if world > 1:
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        return run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
