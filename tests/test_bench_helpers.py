"""Host-side helpers of bench.py (no GPU): the union of kernel intervals used for
the X-matvec roofline when frequency groups overlap, the Lanczos step's algorithmic
bytes, and the traffic record lookup."""
import json
import os

import bench


def test_union_of_intervals():
    assert bench.union_ms([], []) == 0.0
    assert bench.union_ms([0.0], [2.0]) == 2.0
    assert bench.union_ms([0.0, 1.0, 5.0], [2.0, 3.0, 6.0]) == 4.0          # overlap, then a gap
    assert bench.union_ms([5.0, 0.0, 1.0], [6.0, 2.0, 1.5]) == 3.0          # unsorted, nested
    assert bench.union_ms([0.0, 2.0], [2.0, 4.0]) == 4.0                    # touching


def test_recorded_traffic_needs_matching_source():
    path = os.path.join(bench.ROOT, "profiles", "traffic.json")
    with open(path) as f:
        rec = json.load(f)
    for kernel, per_workload in rec.items():
        for workload, e in per_workload.items():
            assert e["dram_bytes_per_step"] > 0
            got = bench.recorded_traffic(kernel, workload)
            # a record applies only while the kernels are the ones it was taken from
            assert got is None or got == e["dram_bytes_per_step"]
            assert (got is not None) == (e["source_hash"] == bench.kernel_source_hash())
    assert bench.recorded_traffic("k_xmatvec<float>", "no such workload") is None


def test_lanczos_algorithmic_bytes_counts_each_step():
    N = 1000
    for reads in (2, 3):
        brute = sum(sum((reads * j + 6) * N * 16 for j in range(1, n + 1)) for n in (5, 1, 64))
        assert bench.lanczos_algorithmic_bytes([5, 1, 64], N, reads) == brute
    assert bench.lanczos_algorithmic_bytes([], N, 2) == 0.0
