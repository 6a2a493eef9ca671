"""Freeze the algorithmic operation counts of the benchmark workloads.

TEST INFRASTRUCTURE: runs only the binary32 replica of this package (its op counter) on the
seeded inputs of `scenegen`, and writes `profiles/opcounts.json`, which the benchmark reads as
the numerator of its ALU roofline.  The count is one op per IEEE add/sub/mul/fma/div/sqrt,
compare, select, min/max, conversion, shift, logic op and popcount the replica performs (loads
and stores are not ops), on a uniform sample of 24,576 pixels (seed 123) scaled to the frame.
A CPU test recomputes the counts and checks the file is current.

    python -m oracle.freeze_opcounts
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import scenegen  # noqa: E402

OUT = os.path.join(ROOT, "profiles", "opcounts.json")
N_PIX, SEED = 24576, 123


def workloads():
    """The single-frame benchmark workloads whose roofline the bench reports."""
    return [scenegen.workload_4k(sector_count=32), scenegen.workload_4k(sector_count=64),
            scenegen.workload_4k(sector_count=128), scenegen.workload_1080p(), scenegen.workload_256()]


def count(w):
    H, W = w.gbuf.depth.shape
    rng = np.random.default_rng(SEED)
    idx = rng.choice(H * W, size=min(N_PIX, H * W), replace=False)
    xy = np.stack([idx % W, idx // W], 1).astype(np.int32)
    _, _, _, c = oracle.fp32(oracle.Problem(w.gbuf, w.params, w.noise, w.sh), xy, counts=True)
    scale = (H * W) / len(idx)
    spf = H * W * 2 * w.params.num_slices * w.params.steps_per_side
    return {"ops_per_frame": c["ops"] * scale, "ops_per_nominal_sample": c["ops"] * scale / spf,
            "pixels_sampled": int(len(idx)), "counts_per_frame": {k: v * scale for k, v in c.items()}}


def main():
    table = {w.name: count(w) for w in workloads()}
    with open(OUT, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
        f.write("\n")
    for k, v in table.items():
        print(f"{k}: {v['ops_per_nominal_sample']:.2f} ops per nominal sample")


if __name__ == "__main__":
    main()
