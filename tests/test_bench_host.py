"""Host-side arithmetic of bench.py's roofline and rate reporting (no GPU)."""
import numpy as np

import bench


def test_union_rows_merges_overlapping_and_adjacent_ranges():
    ts = np.array([20, 0, 5, 3, 11])
    te = np.array([25, 4, 10, 6, 11])
    # [0..11] (0-4, 3-6, 5-10 overlap; 11 is adjacent) and [20..25]
    assert bench.union_rows(ts, te) == 12 + 6
    assert bench.union_rows(np.array([7]), np.array([7])) == 1


def test_union_rows_matches_brute_force():
    rng = np.random.default_rng(3)
    for _ in range(20):
        ts = rng.integers(0, 500, size=30)
        te = ts + rng.integers(0, 60, size=30)
        covered = np.zeros(600, dtype=bool)
        for a, z in zip(ts, te):
            covered[a:z + 1] = True
        assert bench.union_rows(ts, te) == int(covered.sum())


def test_lift_model_counts_writes_and_distinct_reads():
    import synthetic
    w = synthetic.WORKLOADS["compress_f32"]
    bound, units = bench.kernel_model("lift", w, 1, 1000, 400)
    assert bound == "hbm" and units == (1000 + 400) * w.k * 4


def test_kernel_text_hash_covers_only_the_kernel(tmp_path, monkeypatch):
    src = tmp_path / "k.cuh"
    src.write_text("head\n// BEGIN k\nbody 1\n// END\ntail\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h1 = bench.kernel_text_sha256("k.cuh", "// BEGIN k", "// END")
    src.write_text("other head\n// BEGIN k\nbody 1\n// END\nother tail\n")
    assert bench.kernel_text_sha256("k.cuh", "// BEGIN k", "// END") == h1
    src.write_text("head\n// BEGIN k\nbody 2\n// END\ntail\n")
    assert bench.kernel_text_sha256("k.cuh", "// BEGIN k", "// END") != h1


def test_measured_traffic_only_for_the_captured_kernel():
    assert bench.measured_traffic("sketch", 1000) is None
    t1 = bench.measured_traffic("lift", 1000)
    if t1 is not None:               # the capture matches the current kernel source
        assert abs(bench.measured_traffic("lift", 2000) - 2 * t1) < 1e-6 * t1


def test_sweep_batch_size_bounds_the_stacked_bytes():
    budget = 2 << 30
    for b in bench.SWEEP_B:
        for L in bench.SWEEP_LEN:
            nq = bench.sweep_batch_size(L, b, 16, 256, budget=budget)
            assert 1 <= nq <= 256
            assert nq == 1 or nq * (L // b + 2) * 16 * 256 * 4 <= budget
    assert bench.sweep_batch_size(100_000, 64, 16, 256) < 256
