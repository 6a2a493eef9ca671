"""Host-side multi-rank path of bench.py on CPU: two gloo ranks on 127.0.0.1.  The gather is
replicas only (frames are independent), so the only cross-rank steps are the barrier, the
max-over-ranks time and rank 0 printing; the reference arm runs on rank 0 only."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    w, r, _ = bench.dist_init()
    assert (w, r) == (world, rank) and dist.get_backend() == "gloo"
    t_max = bench.max_over_ranks(w, 0.5 + rank)  # per-rank timed seconds
    bench.barrier(w)
    # replicas: every rank gathers its own frames; value = all ranks' samples / the slowest rank's time
    value = w * 10 * 1e9 / t_max / 1e9
    q.put((rank, t_max, value))
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_max_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=90) for _ in procs)
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [1.5, 1.5]
    assert all(abs(o[2] - 2 * 10 / 1.5) < 1e-9 for o in out)


def test_reference_arm_rank_nonzero_does_no_work():
    import argparse

    import bench
    args = argparse.Namespace(workload="256", nb=32, warmup=1, steps=1, gpus=2)
    assert bench.run_reference(args, 2, 1) is None


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` (the CPU oracle on the host cores) prints one JSON line with the
    fields the benchmark contract asks of the reference arm."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=root, check=True)
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1
    assert d["value"] > 0 and d["unit"] == "Gsamples/s" and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["sampled"]["pixels_per_step"] < d["sampled"]["pixels_per_frame"]  # extrapolated, and says so
    assert d["sampled"]["ms_per_frame_extrapolated"] > d["ms_per_step"]  # ms_per_step is the measured step
    import bench
    assert d["config"] == bench.line_config(bench.make_workload("4k", 32), 1)  # the main arm's config
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "3840x2160" in d["config"]["workload"]
