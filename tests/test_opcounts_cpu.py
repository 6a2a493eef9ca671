"""CPU: the frozen algorithmic op counts the benchmark's roofline reads (profiles/opcounts.json)
are those the binary32 replica counts now; regenerate with `python -m oracle.freeze_opcounts`."""
import json
import os

from oracle import freeze_opcounts


def test_frozen_opcounts_are_current():
    with open(freeze_opcounts.OUT) as f:
        table = json.load(f)
    for w in freeze_opcounts.workloads():
        assert w.name in table, w.name
        now = freeze_opcounts.count(w)
        assert table[w.name]["ops_per_frame"] == now["ops_per_frame"], w.name
        assert table[w.name]["counts_per_frame"] == now["counts_per_frame"], w.name


def test_bench_reads_the_frozen_counts():
    import bench
    import scenegen
    ops, counts = bench.algorithmic_ops_per_frame(scenegen.workload_4k())
    assert ops is not None and 58 < ops / bench.samples_per_frame(scenegen.workload_4k()) < 61
    w = bench.make_workload("1080p", 32, radius=0.8)  # an override the table does not hold
    assert bench.algorithmic_ops_per_frame(w) == (None, None)
