"""Multi-process host logic of bench.py on CPU (gloo, world size 2).

The matvec does not shard: N GPUs run N independent replicas (each rank its own
seeded instance), and ranks meet only to combine the timing: units summed over
ranks, time taken as the slowest rank's. The reference arm runs on rank 0 only.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench

    dist = bench.init_group(world, "gloo")
    units, secs = bench.aggregate(1000.0 * (rank + 1), 0.5 + rank, dist)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out, f"r{rank}.json"), "w") as f:
        json.dump({"units": units, "secs": secs}, f)


def test_aggregate_sums_units_and_takes_slowest_rank(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        got = json.load(open(tmp_path / f"r{r}.json"))
        assert got["units"] == 3000.0
        assert got["secs"] == 1.5


def test_single_process_aggregate_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.aggregate(123.0, 4.5, None) == (123.0, 4.5)


def test_replicas_get_independent_instances_of_equal_size():
    sys.path.insert(0, ROOT)
    import argparse

    import bench

    args = argparse.Namespace(n=4096, seed=0, nrhs=1)
    w0, w1 = bench.workload(args, 0), bench.workload(args, 1)
    assert w0.points.shape == w1.points.shape == (4096, 3)
    assert not np.array_equal(w0.points, w1.points)
    assert np.array_equal(w0.points, bench.workload(args, 0).points)


def _reference(env_extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                           "--warmup", "0", "--n", "8192", "--cpu-sample-n", "2048"],
                          capture_output=True, text=True, env=env, timeout=600)


def test_reference_arm_runs_on_rank_zero_only():
    r1 = _reference({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r1.returncode == 0 and r1.stdout.strip() == ""
    r0 = _reference({"RANK": "0", "WORLD_SIZE": "2", "LOCAL_RANK": "0"})
    assert r0.returncode == 0, r0.stderr
    line = json.loads(r0.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["value"] > 0


def test_secondary_bench_lines_record_their_failure():
    sys.path.insert(0, ROOT)
    import bench

    def boom():
        raise RuntimeError("no device")

    assert bench.optional_line(boom) == {"error": "RuntimeError: no device"}
    assert bench.optional_line(lambda a, b: a + b, 2, 3) == 5


def test_traffic_is_scaled_only_for_the_captured_source_and_storage():
    sys.path.insert(0, ROOT)
    import bench

    cap = bench.TRAFFIC_CAPTURE
    saved = cap["apply_sha256"]
    try:
        cap["apply_sha256"] = bench.apply_source_sha256()
        r = cap["ratio"]["fp32+fp16"]["vapply"]
        assert bench.scaled_traffic("vapply", 1e9, "fp32+fp16", 1, 33) == r * 1e9
        assert bench.scaled_traffic("vapply", 1e9, "bf16", 1, 33) is None      # no capture for that storage
        assert bench.scaled_traffic("vapply", 1e9, "fp32+fp16", 4, 33) is None  # nor for other chunk widths
        # captured with the near field on SMs of its own: not for the shared setting's kernels
        assert bench.scaled_traffic("vapply", 1e9, "fp32+fp16", 1, 0) is None
        cap["apply_sha256"] = "0" * 64  # the apply source changed since the capture
        assert bench.scaled_traffic("vapply", 1e9, "fp32+fp16", 1, 33) is None
    finally:
        cap["apply_sha256"] = saved


def test_near_roofline_takes_the_share_of_its_sms():
    sys.path.insert(0, ROOT)
    import bench

    peaks = {"fp32_tflops": 78.0, "mufu_rsqrt_gops": 5000.0}
    s = {"dense_pairs": 1e9}
    whole = bench.near_roofline(s, 3, 1, 1e-3, peaks)
    part = bench.near_roofline(s, 3, 1, 1e-3, peaks, near_sms=38, sms=152)
    assert whole["achieved"] == part["achieved"]
    assert abs(part["peak"] - whole["peak"] / 4) < 1e-9 * whole["peak"]
    assert abs(part["frac"] - 4 * whole["frac"]) < 1e-12
    assert "38 of 152" in part["kernel"] and bench.near_roofline({"dense_pairs": 0}, 3, 1, 1e-3, peaks) is None
