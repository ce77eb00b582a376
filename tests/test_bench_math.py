"""The benchmark's own arithmetic (CPU): recall with and without ties, the roofline
of the dominant kernel and its neighbour, and traffic that only counts while the
kernel's source is the one the counters were taken on."""
import importlib.util
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        spec = importlib.util.spec_from_file_location("bench_under_test",
                                                      os.path.join(ROOT, "bench.py"))
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
    finally:
        sys.argv = argv
    return mod


def test_recall_strict_and_with_ties(bench):
    gt_ids = np.array([[1, 2, 3], [4, 5, 6]])
    gt_d2 = np.array([[0.1, 0.2, 0.3], [0.1, 0.2, 0.3]])
    got = np.array([[3, 2, 9], [4, 5, 6]])
    # query 0: ids 3 and 2 are in the truth; 9 ties the third distance exactly
    got_d2 = np.array([[0.3, 0.2, 0.3], [0.1, 0.2, 0.3]])
    strict, ties = bench.recall_at_k(got, gt_ids, gt_d2, got_d2, 3)
    assert strict == pytest.approx((2 / 3 + 1) / 2)
    assert ties == pytest.approx(1.0)
    # a padded (-1) slot counts as a miss
    got[1, 2] = -1
    got_d2[1, 2] = np.inf
    strict, ties = bench.recall_at_k(got, gt_ids, gt_d2, got_d2, 3)
    assert strict == pytest.approx((2 / 3 + 2 / 3) / 2)
    assert ties == pytest.approx((1 + 2 / 3) / 2)


def test_roofline_picks_the_slower_kernel_and_reports_both(bench):
    from paper_2412_03301_gb300 import datagen
    c = dict(datagen.LARGE)
    c["A"], c["M"] = 3, 1
    hbm, _ = bench.measured_peaks()
    rows = 33_483_707
    per = {"encode": 0.5, "gate": 0.2, "scan": 4.0, "select": 1.0, "refine": 5.0,
           "rescore": 0.6, "topk": 0.1}
    # stage times summed over two steps of one batch each; work counted per step
    r = bench.roofline(c, {k: 2 * v for k, v in per.items()}, 2, 1000, 1, rows * 20, rows, True,
                       steps=2)
    assert r["kernel"] == "k_refine_mma" and r["bound"] == "hbm"
    assert r["achieved"] == pytest.approx(rows * 384 * 2 / 5e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / hbm)
    other = r["other_kernels"][0]
    assert other["kernel"] == "k_scan_mma" and other["bound"] == "tensor"
    assert other["achieved"] == pytest.approx(2.0 * 1000 * c["n_sets"] * c["m"] / 4e-3 / 1e12)
    # one step split into two internal batches: each launch does half the step's work
    r = bench.roofline(c, per, 2, 1000, 1, rows * 20, rows, True, steps=1)
    assert r["achieved"] == pytest.approx(rows / 2 * 384 * 2 / 2.5e-3 / 1e9)
    assert r["algorithmic_bytes"] == pytest.approx(rows / 2 * 384 * 2)
    # the scan dominates when it is the slower one
    per["scan"], per["refine"] = 6.0, 5.0
    r = bench.roofline(c, per, 1, 1000, 1, rows * 20, rows, True)
    assert r["kernel"] == "k_scan_mma" and r["other_kernels"][0]["kernel"] == "k_refine_mma"


def test_traffic_only_for_the_profiled_source(bench, tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("kernel v1\n")
    import hashlib
    sha = hashlib.sha256(src.read_bytes()).hexdigest()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "TRAFFIC", {"k_x": dict(source="k.cu", sha256=sha,
                                                       bytes_per_unit=123.5, unit="row")})
    assert bench.traffic_per_unit("k_x") == pytest.approx(123.5)
    assert bench.traffic_per_unit("k_y") is None
    src.write_text("kernel v2\n")                      # the kernel changed: no traffic
    assert bench.traffic_per_unit("k_x") is None


def test_committed_traffic_entries_name_existing_sources(bench):
    import os
    for name, t in bench.TRAFFIC.items():
        assert os.path.exists(os.path.join(bench.ROOT, t["source"])), name
        assert len(t["sha256"]) == 64 and t["bytes_per_unit"] > 0


def test_fp64_recall_decides_with_the_oracle(bench, orc):
    """Recall against the k smallest FP64 Hausdorff distances of the pooled lists."""
    rng = np.random.default_rng(5)
    sets = [rng.standard_normal((3, 8)).astype(np.float32) for _ in range(30)]
    Q = rng.standard_normal((2, 8)).astype(np.float32)
    truth = sorted(range(30), key=lambda i: (orc.haus(Q, sets[i]), i))
    qoff = np.array([0, 2])
    gt = np.array([truth[:6]])            # the ground truth's longer list
    r, dist = bench.fp64_recall(np.array([truth[:4]]), gt, Q, qoff, lambda i: sets[i], 4)
    assert r == 1.0
    assert np.allclose(dist[0], [orc.haus(Q, sets[i]) for i in truth[:4]])
    got = np.array([[truth[0], truth[1], truth[5], -1]])
    r, dist = bench.fp64_recall(got, gt, Q, qoff, lambda i: sets[i], 4)
    assert r == 0.5 and np.isinf(dist[0, 3])
