"""Host logic of bench.py: the nvidia-smi clock record read back into the
line's `clocks` object (which decides whether a timed run is kept), the
ground truth and recall that the quoted recall@10 comes from, and the
algorithmic bytes and profiled traffic of the roofline object."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _summary(tmp_path, lines):
    p = tmp_path / "clocks.csv"
    p.write_text("".join(line + "\n" for line in lines))
    c = bench.ClockSampler(0)
    c.path = str(p)
    return c.summary()


def test_clock_summary_median_max_and_reasons(tmp_path):
    s = _summary(tmp_path, [
        "0, 2032, 2032, 812.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2032, 1099.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2010, 2032, 950.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
    ])
    assert s["sm_mhz"] == 2010.0 and s["sm_max_mhz"] == 2032.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    assert s["power_w_max"] == 1099.0
    assert not os.path.exists(tmp_path / "clocks.csv")  # the record is removed once read


def test_clock_summary_reports_throttle_reasons_by_name(tmp_path):
    s = _summary(tmp_path, [
        "0, 1500, 2032, 900.0, 0x0000000000000048, Active, Active, Not Active, Not Active",
        "0, 1400, 2032, 900.0, 0x0000000000000020, Not Active, Not Active, Active, Not Active",
    ])
    assert s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_summary_without_samples_or_power(tmp_path):
    s = _summary(tmp_path, ["No devices were found", ""])
    assert s["samples"] == 0 and s["reasons"] == ["unsampled"] and s["sm_mhz"] is None
    s = _summary(tmp_path, ["0, 2032, 2032, [N/A], 0x0, Not Active, Not Active, Not Active, Not Active"])
    assert s["samples"] == 1 and s["power_w_max"] is None


def _brute(X, Q, k, keep=None):
    """FP64 brute force, ties by id, -1 where fewer than k rows qualify."""
    import numpy as np

    out = np.full((len(Q), k), -1, dtype=np.int64)
    for qi, q in enumerate(Q.astype(np.float64)):
        d = ((X.astype(np.float64) - q) ** 2).sum(1)
        ids = np.arange(len(X)) if keep is None else np.nonzero(keep[qi])[0]
        order = ids[np.lexsort((ids, d[ids]))][:k]
        out[qi, :len(order)] = order
    return out


def test_ground_truth_matches_brute_force_across_chunks_and_ties():
    import numpy as np
    import torch

    rng = np.random.default_rng(5)
    X = rng.standard_normal((3000, 16)).astype(np.float32)
    X[2500:2510] = X[100]  # ten exact duplicates of row 100: ties broken by id
    Q = rng.standard_normal((40, 16)).astype(np.float32)
    Q[0] = X[100]
    got = bench.exact_topk(torch.from_numpy(X), torch.from_numpy(Q), 10, qblock=16, chunk=512).numpy()
    np.testing.assert_array_equal(got, _brute(X, Q, 10))
    assert got[0].tolist() == [100] + list(range(2500, 2509))


def test_ground_truth_with_range_filters_and_short_rows():
    import numpy as np
    import torch

    rng = np.random.default_rng(6)
    X = rng.standard_normal((2000, 8)).astype(np.float32)
    Q = rng.standard_normal((30, 8)).astype(np.float32)
    attr = rng.integers(0, 1000, 2000)
    lo = rng.integers(0, 900, 30)
    hi = lo + rng.integers(0, 120, 30)
    lo[0], hi[0] = 5000, 6000  # no row qualifies
    hi[1] = lo[1]  # about two rows qualify
    R = np.stack([lo, hi], 1)
    keep = (attr[None] >= lo[:, None]) & (attr[None] <= hi[:, None])
    got = bench.exact_topk(torch.from_numpy(X), torch.from_numpy(Q), 10, chunk=700, attr=torch.from_numpy(attr),
                           ranges=torch.from_numpy(R)).numpy()
    np.testing.assert_array_equal(got, _brute(X, Q, 10, keep))
    assert (got[0] == -1).all()


def test_recall_counts_only_true_neighbours_in_the_first_k():
    import numpy as np

    truth = np.array([[1, 2, 3, 4], [5, 6, -1, -1], [-1, -1, -1, -1]])
    found = np.array([[4, 3, 9, 8, 1], [6, 7, 5, 0, 0], [0, 1, 2, 3, 4]])
    # query 0: {4, 3} of 4 in its first 4; query 1: {6, 5} of 2; query 2 has no neighbours
    assert bench.recall_at_k(found, truth) == (0.5 + 1.0) / 2


def test_stage_bytes_by_hand():
    """Grains of 10, 20, 30, 40 rows; queries probing {0, 1} and {1, 3}: the
    union of probed grains (70 rows, 3 bases) is read once per batch."""
    import numpy as np

    rows_g = np.array([10, 20, 30, 40])
    probe = np.array([[0, 1], [1, 3]])
    w = {"r": 8, "d": 16, "G": 4, "C": 5}
    assert bench.stage_bytes(None, rows_g, probe, w, 2) == {
        "scan": 70 * (4 * 8 + 4), "project": 3 * 9 * 16 * 4, "rerank": 2 * 5 * 16 * 4, "route": 4 * 16 * 4 + 2 * 16 * 4}
    w["precision"] = "bf16-fp8"
    assert bench.stage_bytes(None, rows_g, probe, w, 2) == {
        "scan": 70 * (8 + 4), "project": 3 * 9 * 16 * 2, "rerank": 2 * 5 * 16 * 2, "route": 4 * 16 * 2 + 2 * 16 * 4}


def test_profile_traffic_is_dropped_once_its_kernel_source_changes(tmp_path, monkeypatch):
    """A committed DRAM-traffic figure is used only while the kernel source it
    was captured on is unchanged; captured on a smaller case it is scaled by
    the launch's queries (traffic in proportion to them) or by a fixed factor
    valid for the batch it names."""
    import hashlib
    import json

    csrc = tmp_path / "paper_2606_08813_b300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    src = b"// kernel source\n"
    (csrc / "k.cuh").write_bytes(src)
    sha = hashlib.sha256(src).hexdigest()[:16]
    rec = {"w": {"scan": {"source_sha": {"k.cuh": sha}, "dram_bytes_per_launch": 1000, "scale_to_full_launch": 4.0,
                          "captured_batch": 64},
                 "rerank": {"source_sha": {"k.cuh": sha}, "dram_bytes_per_launch": 3000, "captured_queries": 16}}}
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_from_profiles("w", "scan", 64) == 4000
    assert bench.traffic_from_profiles("w", "scan", 128) is None  # another batch: the factor does not hold
    assert bench.traffic_from_profiles("w", "rerank", 64) == 12000  # 3000 bytes for 16 queries, 64 queries
    assert bench.traffic_from_profiles("w", "route", 64) is None
    (csrc / "k.cuh").write_bytes(src + b"// changed\n")
    assert bench.traffic_from_profiles("w", "scan", 64) is None
    assert bench.traffic_from_profiles("w", "rerank", 64) is None
