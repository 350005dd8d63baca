#!/usr/bin/env python3
"""HODLRdD matvec throughput on one GB300 (or N independent replicas).

Workload (default): d=3, N=262144 points uniform in [-1,1]^3, F = 1/r with zero
diagonal, leaf 64, ACA tol 1e-7, one right-hand side ~ N(0,1). One step = one
HODLRdD matrix-vector product y = K x (gather, low-rank applies over all
levels, on-the-fly near field, scatter) with x already in HBM. The build
(tree, lists, ACA, packing) runs once before timing and is reported separately,
as the paper reports initialisation and product times separately.

Reported: throughput in N*nrhs per second of the headline precision form and of
the plain FP64 form, the headline form's relative error against the FP64 form,
the dominant kernel's roofline, end-to-end throughput through the C ABI with
host buffers, and the CPU oracle timed on the host cores on a bounded sample.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "HODLRdD matvec N·nrhs/s vs plain FP64 @rel err≤1e-6; serving p50/p99 ms"
UNIT = "N·nrhs/s"
ERR_BAR = 1e-6


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="native", choices=["native", "reference"])
    p.add_argument("--precision", default="fp32+fp16", choices=["fp64", "fp32", "fp16", "bf16", "fp32+fp16"])
    p.add_argument("--near-coords", default="hi", choices=["hi", "hilo"],
                   help="near-field tile coordinates of the headline product: hi only (default; distances carry "
                        "2^-24 h absolute error) or hi + lo pairs (exact distances)")
    p.add_argument("--near-sms", default="auto",
                   help="SMs given to the headline product's near field: auto (default; the build times the "
                        "settings and keeps the fastest), 0 (shared with the applies on every SM) or a count")
    p.add_argument("--n", type=int, default=262144)
    p.add_argument("--nrhs", type=int, default=1)
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--cpu-sample-n", type=int, default=32768)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--no-many-rhs", action="store_true", help="skip the many-right-hand-side (d=4, nrhs 64) line")
    p.add_argument("--no-solve", action="store_true", help="skip the integral-equation solve line")
    p.add_argument("--no-batch", action="store_true", help="skip the batched uneven-trees line")
    p.add_argument("--no-skeleton", action="store_true", help="skip the skeleton-form line")
    p.add_argument("--no-serve", action="store_true", help="skip the request-loop (serving) line")
    p.add_argument("--no-admissibility", action="store_true", help="skip the admissibility comparison line")
    p.add_argument("--only", default=None, choices=["many_rhs", "batch", "solve", "serve", "admissibility"],
                   help="run only this workload's products (--steps of them after --warmup) and print its line; "
                        "for profiling")
    p.add_argument("--many-n", type=int, default=65536, help="points of the many-right-hand-side workload")
    p.add_argument("--solve-n", type=int, default=262144, help="points of the integral-equation solve")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def init_group(world, backend):
    if world <= 1:
        return None
    import torch.distributed as dist

    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group(backend=backend)
    return dist


def aggregate(units: float, seconds: float, dist, device=None):
    """Whole-job throughput: units summed over ranks / slowest rank's time."""
    if dist is None:
        return units, seconds
    import torch

    t = torch.tensor([units, seconds], dtype=torch.float64, device=device)
    u = t[:1].clone()
    s = t[1:].clone()
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(s, op=dist.ReduceOp.MAX)
    return float(u.item()), float(s.item())


def workload(args, rank):
    import workloads as W

    w = W.precision_3d(N=args.n, seed=args.seed + rank)
    if args.nrhs != 1:
        rng = np.random.default_rng(args.seed + rank + 7)
        w.x = rng.standard_normal((w.N, args.nrhs))
        w.nrhs = args.nrhs
    return w


def workload_name(w):
    return (f"d={w.d} N={w.N} uniform [-1,1]^{w.d}, F=1/r (zero diagonal), leaf {w.leaf}, "
            f"tol {w.tol:g}, nrhs {w.nrhs}")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# DRAM traffic of each apply stage (its panel and combine launches) per
# algorithmic byte, from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum per launch) of the d=3 N=65536 case of this workload
# with one right-hand side, per storage precision, with the near field on SMs
# of its own (near_sms 32: the apply kernels' four-slot ring on 120 CTAs);
# scaled to a full launch by the bytes processed (traffic grows with the factor
# bytes). It is reported only while the apply source is the one that was
# captured and the product ran in that configuration (near_sms > 0).
TRAFFIC_CAPTURE = {
    "apply_sha256": "e7170237b287aade596668c107215e67a821197b5eed3005fd1d810d2e8595ff",
    "nrhs": 1,
    "near_sms_split": True,
    "ratio": {"fp32+fp16": {"vapply": 1.0046, "uapply": 1.0014}},  # mean over the two captured matvecs
}


def apply_source_sha256():
    import hashlib

    with open(os.path.join(ROOT, "paper_2209_05819_gb300", "csrc", "apply.cu"), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def scaled_traffic(kernel, algo_bytes, precision, nrhs, near_sms):
    c = TRAFFIC_CAPTURE
    r = c["ratio"].get(precision, {})
    if (c["apply_sha256"] is None or kernel not in r or nrhs != c["nrhs"] or (near_sms > 0) != c["near_sms_split"]
            or apply_source_sha256() != c["apply_sha256"]):
        return None
    return r[kernel] * algo_bytes


# Algorithmic arithmetic of one kernel evaluation with its accumulation, for
# F = 1/r in d dimensions: d subtractions and d multiply-adds form |x_i - x_j|^2,
# one rsqrt evaluates F (a MUFU operation in FP32), and one FMA per right-hand
# side adds F x_j. FP32 pipe operations per pair: 2d + nrhs; MUFU: 1. As FP64
# flops (for the FP64 form): d + 2d - 1 for the distance, 1 for F, 2 nrhs.
def near_roofline(s, d, nrhs, seconds, peaks, near_sms=0, sms=None):
    """near_sms > 0: the near field ran on near_sms of the sms SMs (k_tile_split), so its peak is that share."""
    pairs = int(s["dense_pairs"])
    if seconds <= 0 or pairs == 0:
        return None
    ops = 2 * d + nrhs
    share = near_sms / sms if near_sms and sms else 1.0
    fp32_ops_peak = peaks["fp32_tflops"] * 1e12 / 2 * share  # FMA lane-operations per second
    mufu_peak = peaks["mufu_rsqrt_gops"] * 1e9 * share
    achieved = pairs * ops / seconds
    kernel = (f"near field (k_tile_split on {near_sms} of {sms} SMs, second stream)" if near_sms
              else "near field (k_tile, second stream, sharing the SMs with the applies)")
    return {"kernel": kernel, "bound": "alu", "unit": "G FP32 ops/s",
            "pairs": pairs, "ops_per_pair": ops, "achieved": achieved / 1e9, "peak": fp32_ops_peak / 1e9,
            "frac": achieved / fp32_ops_peak, "mufu_frac": pairs / seconds / mufu_peak,
            "stage_ms": 1e3 * seconds, "peak_source": "measured (hodlrdd_probe_peaks)", "traffic": None}


def fp64_roofline(s, d, nrhs, seconds, peaks):
    """The FP64 form against the measured FP64 FMA rate: every factor element in
    one FMA per right-hand side, every near-field pair as counted above."""
    flops = 2.0 * int(s["factor_elems"]) * nrhs + int(s["dense_pairs"]) * (3 * d + 2 * nrhs)
    achieved = flops / seconds
    peak = peaks["fp64_tflops"] * 1e12
    return {"kernel": "whole FP64 matvec", "bound": "fp64", "unit": "TFLOP/s", "flops": flops,
            "achieved": achieved / 1e12, "peak": peak / 1e12, "frac": achieved / peak,
            "peak_source": "measured (hodlrdd_probe_peaks)", "traffic": None}


def factor_bytes(h, precision):
    """Algorithmic bytes of the packed U and V streams (incl. alignment pads) and scales."""
    s = h.stats()
    tr = int(s["total_rank"])
    scales = 8 * tr if precision in ("fp16", "bf16") else 8 * int(s["tail_cols"]) if precision == "fp32+fp16" else 0
    return int(s["factor_bytes_u"]), int(s["factor_bytes_v"]), tr, scales


def time_steps(fn, steps, warmup, torch, stream):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def cpu_baseline(args, rank_w):
    """The oracle (FP64 C++), as it stands, on the host cores: HODLRdD build and
    matvec on a smaller draw of the same point distribution."""
    import oracle
    import workloads as W

    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    ws = W.subsample(rank_w, args.cpu_sample_n, seed=args.seed + 12345)
    t0 = time.perf_counter()
    T = oracle.Tree(ws.points, ws.kernel, ws.params, ws.leaf, ws.tol, dense_if_cheaper=True)
    t_build = time.perf_counter() - t0
    times = []
    t_end = time.perf_counter() + 8.0
    while len(times) < 3 or (time.perf_counter() < t_end and len(times) < 20):
        t0 = time.perf_counter()
        T.matvec(ws.x)
        times.append(time.perf_counter() - t0)
    t = statistics.median(times)
    # the same oracle on one core, and its direct O(N^2) sum on a row sample
    oracle.set_threads(1)
    t0 = time.perf_counter()
    T.matvec(ws.x)
    t1 = time.perf_counter() - t0
    oracle.set_threads(cores)
    nrow = min(ws.N, 1024)
    t0 = time.perf_counter()
    oracle.direct(ws.points, ws.kernel, ws.params, ws.x, (0, nrow))
    t_dir = (time.perf_counter() - t0) * ws.N / nrow
    # the plain FP64 configuration (d=2, N=4096, log r) in full on the oracle
    c1 = W.plain_fp64_2d()
    T1 = oracle.Tree(c1.points, c1.kernel, c1.params, c1.leaf, c1.tol, dense_if_cheaper=True)
    t0 = time.perf_counter()
    for _ in range(5):
        T1.matvec(c1.x)
    t_c1 = (time.perf_counter() - t0) / 5
    extra = {"single_core_value": ws.N * ws.nrhs / t1, "direct_value": ws.N * ws.nrhs / t_dir,
             "plain_fp64_c1_value": c1.N / t_c1, "machine": f"{os.uname().machine}, {cores} threads"}
    return {"value": ws.N * ws.nrhs / t, "unit": UNIT, "cores": cores, "kind": "oracle", "sample_n": ws.N, **extra,
            "sample": f"oracle FP64 HODLRdD on a {ws.N}-point draw of the same distribution (d={ws.d}, 1/r, "
                      f"leaf {ws.leaf}, tol {ws.tol:g}); matvec median of {len(times)} runs; build {t_build:.1f} s; "
                      f"single_core_value: one matvec on one thread; direct_value: the oracle's direct sum on "
                      f"{nrow} rows scaled to all rows"}


def plain_fp64_line(args, torch, stream, hd, peaks):
    """The plain FP64 configuration (d=2, N=4096 uniform [-1,1]^2, log r with a
    zero diagonal, leaf 64, tol 1e-8, one right-hand side): product time and its
    fraction of the measured FP64 rate."""
    import workloads as W

    w = W.plain_fp64_2d()
    h = hd.Handle(torch.from_numpy(w.points).cuda(), w.kernel, w.params, w.leaf, w.tol, precision="fp64")
    x = torch.from_numpy(np.ascontiguousarray(w.x)).cuda()
    y = torch.empty_like(x)
    n = 200
    t = time_steps(lambda: h.matvec(x, y), n, 10, torch, stream) / n
    s = h.stats()
    h.close()
    out = {"workload": f"d=2 N={w.N} uniform [-1,1]^2, F=log r (zero diagonal), leaf {w.leaf}, tol {w.tol:g}, nrhs 1",
           "precision": "fp64", "ms_per_matvec": 1e3 * t, "value": w.N / t, "unit": UNIT,
           "roofline": fp64_roofline(s, w.d, 1, t, peaks)}
    out["note"] = ("a 4096-point tree is latency-bound: " + str(s["kappa"]) + " levels, "
                   + str(s["n_blocks"]) + " blocks, about a dozen dependent launches per product")
    return out


def many_rhs_line(args, torch, stream, hd, peaks=None):
    """The many-right-hand-side workload (d=4, N=65536, Matern-3/2, 64 columns):
    the tensor-core form (factors as FP16 high / scaled-low pairs, tcgen05 MMAs
    for the low-rank applies and the near field's 64-wide accumulation), the
    FP32 CUDA-core form and the plain FP64 form; errors against FP64, stage
    times and the applies' HBM roofline."""
    import workloads as W

    w = W.many_rhs_4d(seed=args.seed)
    pts = torch.from_numpy(w.points).cuda()
    out = {"workload": f"d=4 N={w.N} uniform [0,1]^4, Matern-3/2 l=0.2, leaf {w.leaf}, tol {w.tol:g}, "
                       f"nrhs {w.nrhs}", "precision": "fp16x2"}
    res = {}
    for prec in ("fp16x2", "fp32", "fp64"):
        # the tensor-core form streams the coarse full-rank blocks as factors
        # (dense-if-cheaper at the leaf level only); the others keep the default rule
        h = hd.Handle(pts, w.kernel, w.params, w.leaf, w.tol, precision=prec, max_nrhs=w.nrhs,
                      dense_if_cheaper="leaf" if prec == "fp16x2" else True)
        io = torch.float64 if prec == "fp64" else torch.float32
        x = torch.from_numpy(np.ascontiguousarray(w.x)).to(io).cuda()
        y = torch.empty_like(x)
        n = 10 if prec == "fp16x2" else 3 if prec == "fp32" else 1
        t = time_steps(lambda: h.matvec(x, y), n, 2, torch, stream)
        entry = {"ms": 1e3 * t / n, "y": y.double()}
        if prec == "fp16x2":
            h.set_profiling(True)
            for _ in range(3):
                h.matvec(x, y)
            torch.cuda.synchronize()
            pr = h.profile()
            h.set_profiling(False)
            h.sync()
            entry["prof"] = {k: pr[k] / max(pr["chunks"], 1) for k in ("gather_ms", "vapply_ms", "uapply_ms", "near_ms")}
            entry["stats"] = h.stats()
        res[prec] = entry
        h.close()
    y64 = res["fp64"]["y"]

    def err(y):
        return float((torch.linalg.norm(y - y64, dim=0) / torch.linalg.norm(y64, dim=0)).max().item())

    tc = res["fp16x2"]
    s = tc["stats"]
    units = w.N * w.nrhs
    R = 64
    hbm, _ = measured_peaks()
    vbytes = s["factor_bytes_v"] + s["total_rank"] * R * 4 + w.N * R * 4      # V planes, t written, x_t read
    ubytes = s["factor_bytes_u"] + s["total_rank"] * R * 4 + s["kappa"] * w.N * R * 4  # U planes, t read, y_l written
    pr = tc["prof"]
    out.update({"ms_per_matvec": tc["ms"], "value": units / (tc["ms"] / 1e3), "unit": UNIT,
                "rel_err_vs_fp64": err(tc["y"]), "fp64_ms_per_matvec": res["fp64"]["ms"],
                "speedup_vs_fp64": res["fp64"]["ms"] / tc["ms"],
                "fp32_cuda_cores": {"ms_per_matvec": res["fp32"]["ms"], "value": units / (res["fp32"]["ms"] / 1e3),
                                    "rel_err_vs_fp64": err(res["fp32"]["y"])},
                "speedup_vs_fp32_cuda_cores": res["fp32"]["ms"] / tc["ms"],
                "stage_ms": {k: round(v, 4) for k, v in pr.items()},
                "factor_gb": (s["factor_bytes_u"] + s["factor_bytes_v"]) / 1e9, "dense_pairs": s["dense_pairs"]})
    roof = {}
    for name, byt, ms in (("vapply", vbytes, pr["vapply_ms"]), ("uapply", ubytes, pr["uapply_ms"])):
        if ms > 0:
            roof[name] = {"bound": "hbm", "algorithmic_bytes": byt, "achieved": byt / (ms / 1e3) / 1e9, "peak": hbm,
                          "unit": "GB/s", "frac": byt / (ms / 1e3) / 1e9 / hbm}
    if peaks and pr["near_ms"] > 0:
        pairs = s["dense_pairs"]
        ops = 2 * w.d + 4  # d subtractions, d multiply-adds, the scale, 1 + a and the product (sqrt, exp on MUFU)
        tsec = pr["near_ms"] / 1e3
        roof["near"] = {"bound": "alu", "pairs": pairs, "ops_per_pair": ops, "unit": "G FP32 ops/s",
                        "achieved": pairs * ops / tsec / 1e9, "peak": peaks["fp32_tflops"] * 1e3 / 2,
                        "frac": pairs * ops / tsec / (peaks["fp32_tflops"] * 1e12 / 2),
                        "tensor_tflops": pairs * R * 2 * 3 / tsec / 1e12}
    out["roofline"] = roof
    return out


def skeleton_line(args, torch, stream, hd, w, pts, x, y64):
    """The memory-efficient skeleton form (pivots + LU of K(sigma, tau), entries
    evaluated on the fly) on the headline workload: FP32 form against the FP64
    stored-factor product, and the FP64 skeleton form; time, error and memory."""
    out = {"workload": "the headline workload, low-rank blocks in the skeleton form"}
    hs = hd.Handle(pts, w.kernel, w.params, w.leaf, w.tol, precision="fp32", lowrank_form="skeleton")
    y = torch.empty_like(x)
    n = max(5, min(args.steps // 20, 50))
    t = time_steps(lambda: hs.matvec(x, y), n, 3, torch, stream)
    hs.set_profiling(True)
    hs.matvec(x, y)
    torch.cuda.synchronize()
    prof = hs.profile()
    hs.set_profiling(False)
    s = hs.stats()
    err = None
    if y64 is not None:
        err = float((torch.linalg.norm(y.double() - y64, dim=0) / torch.linalg.norm(y64, dim=0)).max().item())
    out["fp32"] = {"ms_per_step": 1e3 * t / n, "value": w.N * w.nrhs * n / t, "unit": UNIT, "steps": n,
                   "rel_err_vs_fp64": err, "device_gb": s["device_bytes"] / 1e9,
                   "skeleton_gb": s["skeleton_bytes"] / 1e9, "skeleton_terms": s["skeleton_terms"],
                   "total_rank": s["total_rank"], "kernel_evals_lowrank": s["skeleton_pairs"],
                   "lowrank_evals_per_s": s["skeleton_pairs"] * n / t,
                   "stage_ms": {"rows_and_solve": prof["vapply_ms"], "cols": prof["uapply_ms"],
                                "near": prof["near_ms"]}}
    hs.close()
    if not args.no_fp64:
        h6 = hd.Handle(pts, w.kernel, w.params, w.leaf, w.tol, precision="fp64", lowrank_form="skeleton")
        x64 = x.double()
        y6 = torch.empty_like(x64)
        t6 = time_steps(lambda: h6.matvec(x64, y6), 3, 1, torch, stream)
        e6 = None
        if y64 is not None:
            e6 = float((torch.linalg.norm(y6 - y64, dim=0) / torch.linalg.norm(y64, dim=0)).max().item())
        out["fp64"] = {"ms_per_step": 1e3 * t6 / 3, "rel_err_vs_stored_fp64": e6,
                       "device_gb": h6.stats()["device_bytes"] / 1e9}
        h6.close()
    return out


def serving_line(args, torch, hd, rates=(200.0, 50.0), seconds=3.0, n_models=6, budget_gb=40.0, workers=4):
    """Requests arriving over time against models resident under an HBM budget:
    Poisson arrivals, 70% products / 30% solves of second-kind systems
    (I + K/N) u = b, d in {2, 3, 4}, N log-uniform in [4096, 262144], four
    kernels; latency from submission to completion, per kind."""
    import workloads as W

    rng = np.random.default_rng(args.seed + 77)
    kernels = [(W.K_LOG, 0.0), (W.K_INV_R, 0.0), (W.K_MATERN32, 0.2), (W.K_GAUSS, 0.5)]
    specs = []
    for i in range(n_models):
        d = int(rng.integers(2, 5))
        N = int(round(np.exp(rng.uniform(np.log(4096), np.log(262144)))))
        k, p0 = kernels[i % len(kernels)]
        leaf = 64 if d <= 3 else 128
        tol = {W.K_LOG: 1e-8, W.K_INV_R: 1e-7, W.K_MATERN32: 1e-7, W.K_GAUSS: 1e-6}[k]
        specs.append(W.make(f"s{i}", d, N, k, (1.0 / N, 1.0, p0, 0.0), leaf, tol, nrhs=1, seed=2000 + i))
    srv = hd.Server(int(budget_gb * 1e9), workers=workers)
    ids = [srv.add(w.points, w.kernel, w.params, w.leaf, w.tol, precision=args.precision) for w in specs]
    xs32 = [np.ascontiguousarray(w.x, dtype=np.float32) for w in specs]
    t0 = time.perf_counter()
    warm = [srv.submit(ids[i], specs[i].x, kind=hd.REQ_SOLVE) for i in range(n_models)]
    warm += [srv.submit(ids[i], xs32[i]) for i in range(n_models)]
    for r in warm:
        srv.wait(r)
    t_warm = time.perf_counter() - t0
    def pct(v, q):
        v = sorted(v)
        return v[min(len(v) - 1, int(q * len(v)))] if v else None

    out = {"workload": f"{n_models} second-kind systems (I + K/N): d in 2..4, N log-uniform in [4096, 262144] "
                       f"(N = {[w.N for w in specs]}), log r / 1/r / Matern-3/2 / Gaussian; Poisson arrivals for "
                       f"{seconds:g} s, 70% products / 30% solves (GMRES + FP64 refinement to 1e-10); {workers} "
                       f"workers; budget {budget_gb:g} GB; latency = submission to completion",
           "precision": args.precision, "warm_up_s": t_warm, "runs": []}
    for rate in rates:
        # arrivals: exponential gaps at `rate`, kind and model drawn per request
        n = int(rate * seconds)
        gaps = rng.exponential(1.0 / rate, n)
        kinds = rng.random(n) < 0.3
        models = rng.integers(0, n_models, n)
        reqs = []
        t_start = time.perf_counter()
        t_next = t_start
        for j in range(n):
            t_next += gaps[j]
            while time.perf_counter() < t_next:
                time.sleep(max(0.0, min(t_next - time.perf_counter(), 0.001)))
            m = int(models[j])
            if kinds[j]:
                reqs.append(("solve", srv.submit(ids[m], specs[m].x, kind=hd.REQ_SOLVE)))
            else:
                reqs.append(("matvec", srv.submit(ids[m], xs32[m])))
        lat = {"matvec": [], "solve": []}
        svc = {"matvec": [], "solve": []}
        for kind, r in reqs:
            _, ms, sv = srv.wait(r, service=True)
            lat[kind].append(ms)
            svc[kind].append(sv)
        t_all = time.perf_counter() - t_start
        out["runs"].append({
            "offered_rps": rate, "requests": n, "achieved_rps": n / t_all,
            "matvec": {"count": len(lat["matvec"]), "p50_ms": pct(lat["matvec"], 0.5),
                       "p99_ms": pct(lat["matvec"], 0.99), "service_p50_ms": pct(svc["matvec"], 0.5)},
            "solve": {"count": len(lat["solve"]), "p50_ms": pct(lat["solve"], 0.5), "p99_ms": pct(lat["solve"], 0.99),
                      "service_p50_ms": pct(svc["solve"], 0.5)}})
    # a burst: 64 single-column products per model submitted at once, with the
    # model's queued products batched into wide products, and with batching off
    burst = {}
    for cols in (64, 0):
        srv.set_batching(cols)
        b0 = srv.stats()
        t0 = time.perf_counter()
        rb = [srv.submit(ids[m], xs32[m]) for _ in range(64) for m in range(n_models)]
        for r in rb:
            srv.wait(r)
        dt = time.perf_counter() - t0
        b1 = srv.stats()
        burst["batched" if cols else "alone"] = {
            "requests": len(rb), "seconds": dt, "rps": len(rb) / dt,
            "n_rhs_per_s": sum(w.N for w in specs) * 64 / dt,
            "batches": b1["batches"] - b0["batches"], "batched_requests": b1["batched_requests"] - b0["batched_requests"]}
    burst["speedup_batched_vs_alone"] = burst["alone"]["seconds"] / burst["batched"]["seconds"]
    out["burst"] = burst
    srv.set_batching(64)
    out["server"] = srv.stats()
    srv.close()
    return out


def admissibility_line(args, torch, stream, hd, N=65536):
    """The paper's comparison of admissibility conditions on one workload:
    strong (far-field only, H-matrix), HODLRdD (far-field and vertex-sharing),
    weak (every sibling, HODLR). Build time, product time, stored bytes and
    error against the GPU direct sum, per condition. In two dimensions, where
    the weak condition's edge-sharing blocks still compress."""
    import workloads as W

    w = W.make("adm d=2 log r", 2, N, W.K_LOG, (1.0, 0.0, 0.0, 0.0), 64, 1e-8, nrhs=1, seed=args.seed)
    pts = torch.from_numpy(w.points).cuda()
    x = torch.from_numpy(np.ascontiguousarray(w.x[:, 0], dtype=np.float32)).cuda()
    # uniform FP32 factors: this tree's finest low-rank level has 16-point boxes, whose one-stage panels
    # the mixed storage would apply in two passes
    prec = "fp32"
    out = {"workload": f"d=2 N={N} uniform [-1,1]^2, F=log r, leaf {w.leaf}, tol {w.tol:g}, one right-hand side; "
                       "error against the GPU direct O(N^2) sum (FP32, compensated)",
           "precision": prec}
    yd = None
    for name, amax in (("strong_H", -1), ("hodlrdd", 0), ("weak_HODLR", 1)):
        t0 = time.perf_counter()
        h = hd.Handle(pts, w.kernel, w.params, w.leaf, w.tol, precision=prec, admissible_face_dim=amax)
        t_build = time.perf_counter() - t0
        if yd is None:
            yd = torch.empty_like(x)
            h.direct(x, yd)
        y = torch.empty_like(x)
        n = 10
        t = time_steps(lambda: h.matvec(x, y), n, 3, torch, stream)
        err = float((torch.linalg.norm(y.double() - yd.double()) / torch.linalg.norm(yd.double())).item())
        s = h.stats()
        out[name] = {"admissible_face_dim": amax, "build_s": t_build, "ms_per_step": 1e3 * t / n,
                     "factor_gb": (s["factor_bytes_u"] + s["factor_bytes_v"]) / 1e9, "n_lowrank": s["n_lowrank"],
                     "n_dense": s["n_dense"], "n_rank_capped": s["n_rank_capped"], "max_rank": s["max_rank"],
                     "dense_pairs": s["dense_pairs"], "rel_err_vs_direct": err}
        h.close()
    return out


def solve_line(args, torch, hd, N=262144):
    """(I + K/N) u = b on N points of the benchmark distribution, to a relative
    FP64 residual of 1e-10: GMRES on the headline-precision operator inside FP64
    refinement, against GMRES on the FP64 operator alone."""
    import workloads as W

    w = W.precision_3d(N=N, seed=args.seed, system=True)
    pts = torch.from_numpy(w.points).cuda()
    h64 = hd.Handle(pts, w.kernel, w.params, w.leaf, w.tol, precision="fp64")
    hff = hd.Handle(pts, w.kernel, w.params, w.leaf, w.tol, precision="fp64", fp64_near="ff")
    hlo = hd.Handle(pts, w.kernel, w.params, w.leaf, w.tol, precision=args.precision)
    b = torch.from_numpy(np.ascontiguousarray(w.x[:, 0])).cuda()
    out = {"workload": f"(I + K/N) u = b, d=3 N={N} uniform [-1,1]^3, F=1/r, leaf {w.leaf}, tol {w.tol:g}; "
                       "GMRES(50), x0 = 0, stop at ||b - K x|| <= 1e-10 ||b|| with the FP64 operator",
           "legs": {"mixed_ff": f"inner {args.precision}, refinement FP64 with the float-float near field",
                    "mixed": f"inner {args.precision}, refinement plain FP64",
                    "fp64": "FP64-only GMRES (inner and refinement plain FP64)"}}
    for name, inner, outer in (("mixed_ff", hlo, hff), ("mixed", hlo, h64), ("fp64", h64, h64)):
        hd.solve(inner, outer, b, tol=1e-10)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x, st = hd.solve(inner, outer, b, tol=1e-10)
        torch.cuda.synchronize()
        out[name] = {"ms": 1e3 * (time.perf_counter() - t0), **st}
        # the residual against the plain FP64 operator, whichever operator refined
        r = b - h64.matvec(x)
        out[name]["residual_plain_fp64"] = float((torch.linalg.norm(r) / torch.linalg.norm(b)).item())
    out["speedup_mixed_ff_vs_fp64"] = out["fp64"]["ms"] / out["mixed_ff"]["ms"]
    out["speedup_mixed_vs_fp64"] = out["fp64"]["ms"] / out["mixed"]["ms"]
    hlo.close()
    hff.close()
    h64.close()
    return out


def batch_line(args, torch, hd):
    """48 clustered d=3 sets (N log-uniform in [2048, 131072], Gaussian h=0.5 +
    1e-3 I, leaf 64, tol 1e-6, 1..16 right-hand sides each), resident at once:
    one batch run (inputs resident, one graph launch) against one product per
    handle in turn, and the per-run latency."""
    import workloads as W

    ws = W.uneven_instances()
    # up to 16 right-hand sides per set: uniform FP32 factors take them in one chunk
    prec = "fp32" if args.precision == "fp32+fp16" else args.precision
    t0 = time.perf_counter()
    hs = [hd.Handle(torch.from_numpy(w.points).cuda(), w.kernel, w.params, w.leaf, w.tol, precision=prec,
                    max_nrhs=16) for w in ws]
    t_build = time.perf_counter() - t0
    units = sum(w.N * w.nrhs for w in ws)
    xs = [torch.from_numpy(np.ascontiguousarray(w.x, dtype=np.float32)).cuda() for w in ws]
    ys = [torch.empty_like(x) for x in xs]
    b = hd.Batch(hs, [w.nrhs for w in ws])

    def seq():
        for h, x, y in zip(hs, xs, ys):
            h.matvec(x, y)

    out = {"workload": f"48 clustered d=3 sets, N log-uniform 2048..131072 (total {sum(w.N for w in ws)}), "
                       f"Gaussian h=0.5 + 1e-3 I, leaf 64, tol 1e-6, 1..16 right-hand sides",
           "build_s": t_build, "precision": prec}
    for name, fn in (("sequential", seq), ("batch_graph", lambda: b.run(xs, ys))):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        lat = []
        for _ in range(20):
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            lat.append(1e3 * (time.perf_counter() - t0))
        lat.sort()
        out[name] = {"value": units / (statistics.median(lat) / 1e3), "unit": UNIT, "p50_ms": lat[len(lat) // 2],
                     "p99_ms": lat[-1]}
    # the forest: the same 48 sets in the tensor-core form, merged into one
    # launch per stage (64 columns wide, so every set's 1..16 columns ride along)
    t0 = time.perf_counter()
    ht = [hd.Handle(torch.from_numpy(w.points).cuda(), w.kernel, w.params, w.leaf, w.tol, precision="fp16x2",
                    max_nrhs=64, dense_if_cheaper="leaf") for w in ws]
    f = hd.Forest(ht, [w.nrhs for w in ws])
    t_forest = time.perf_counter() - t0
    yf = [torch.empty_like(x) for x in xs]
    for _ in range(3):
        f.run(xs, yf)
    lat = []
    for _ in range(20):
        t0 = time.perf_counter()
        f.run(xs, yf)
        lat.append(1e3 * (time.perf_counter() - t0))
    lat.sort()
    # errors against plain FP64 on every eighth set
    errs = []
    for i in range(0, len(ws), 8):
        w = ws[i]
        h64 = hd.Handle(torch.from_numpy(w.points).cuda(), w.kernel, w.params, w.leaf, w.tol, precision="fp64")
        y64 = h64.matvec(torch.from_numpy(np.ascontiguousarray(w.x)).cuda())
        e = torch.linalg.norm(yf[i].double() - y64, dim=0) / torch.linalg.norm(y64, dim=0)
        errs.append(float(e.max().item()))
        h64.close()
    fs = f.stats()
    pr = f.profile()
    hst = [h.stats() for h in ht]
    hbm, _ = measured_peaks()
    # the V-apply stage: its factor planes as streamed (FP16 pairs, panels padded to 16 rows and 64
    # columns), t written and x_t read, 64 columns of 4 bytes
    vbytes = (sum(s_["factor_bytes_v"] for s_ in hst) + sum(s_["total_rank"] for s_ in hst) * 256
              + sum(w.N for w in ws) * 256)
    roof = {"kernel": "forest V-apply (k_tc_apply<V>, 152 persistent CTAs)", "bound": "hbm",
            "bytes": vbytes, "stage_ms": pr["vapply_ms"], "achieved": vbytes / (pr["vapply_ms"] / 1e3) / 1e9,
            "peak": hbm, "unit": "GB/s", "frac": vbytes / (pr["vapply_ms"] / 1e3) / 1e9 / hbm,
            "stage_ms_all": {k: round(v, 3) for k, v in pr.items()}}
    out["forest_fp16x2"] = {"value": units / (statistics.median(lat) / 1e3), "unit": UNIT,
                            "p50_ms": lat[len(lat) // 2], "p99_ms": lat[-1], "build_s": t_forest,
                            "launches_per_run": fs["launches_per_run"], "near_passes": fs["near_passes"],
                            "graph_launches_per_run": 1,
                            "autotuned_panel_cost_bytes": {"vapply": fs["tuned_fixed_v"], "uapply": fs["tuned_fixed_u"]},
                            "rel_err_vs_fp64_max": max(errs), "err_sets": len(errs),
                            "speedup_vs_batch_graph": out["batch_graph"]["p50_ms"] / lat[len(lat) // 2],
                            "roofline": roof}
    f.close()
    for h in ht:
        h.close()
    b.close()
    for h in hs:
        h.close()
    return out


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    import oracle
    import workloads as W

    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    w = workload(args, 0)
    ws = W.subsample(w, args.cpu_sample_n, seed=args.seed + 12345)
    T = oracle.Tree(ws.points, ws.kernel, ws.params, ws.leaf, ws.tol, dense_if_cheaper=True)
    for _ in range(args.warmup):
        T.matvec(ws.x)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        T.matvec(ws.x)
    dt = time.perf_counter() - t0
    value = ws.N * ws.nrhs * args.steps / dt
    sample = (f"oracle FP64 HODLRdD matvec on a {ws.N}-point draw of the same distribution (each step one matvec "
              f"of the sample)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": workload_name(w), "sample_n": ws.N},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                         "sample_n": ws.N},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def optional_line(fn, *a):
    """A secondary line of the report: its failure is recorded in the line and
    does not lose the headline measurement."""
    try:
        return fn(*a)
    except Exception as e:  # noqa: BLE001 - reported, not hidden
        return {"error": f"{type(e).__name__}: {e}"}


def many_rhs_only(args):
    """Products of the many-right-hand-side workload in the tensor-core form only
    (d=4, Matern-3/2, leaf 128, tol 1e-8, 64 columns; N = --many-n)."""
    import torch

    import paper_2209_05819_gb300 as hd
    import workloads as W
    from paper_2209_05819_gb300 import build as cbuild

    cbuild.build()
    w = W.many_rhs_4d(N=args.many_n, seed=args.seed)
    h = hd.Handle(torch.from_numpy(w.points).cuda(), w.kernel, w.params, w.leaf, w.tol, precision="fp16x2",
                  dense_if_cheaper="leaf")
    x = torch.from_numpy(np.ascontiguousarray(w.x, dtype=np.float32)).cuda()
    y = torch.empty_like(x)
    t = time_steps(lambda: h.matvec(x, y), max(args.steps, 1), args.warmup, torch, torch.cuda.current_stream())
    h.sync()
    s = h.stats()
    print(json.dumps({"workload": f"d=4 N={w.N} Matern-3/2 leaf {w.leaf} tol {w.tol:g} nrhs {w.nrhs} fp16x2",
                      "ms_per_matvec": 1e3 * t / max(args.steps, 1), "factor_gb": (s["factor_bytes_u"] +
                      s["factor_bytes_v"]) / 1e9, "dense_pairs": s["dense_pairs"], "kappa": s["kappa"]}))


def batch_only(args):
    """The uneven-instances line alone (48 clustered d=3 sets: one graph-replayed
    batch, one forest run), for profiling."""
    import torch

    import paper_2209_05819_gb300 as hd
    from paper_2209_05819_gb300 import build as cbuild

    cbuild.build()
    print(json.dumps(batch_line(args, torch, hd)))


def solve_only(args):
    """The integral-equation solve line alone (d=3, N=262144), for profiling."""
    import torch

    import paper_2209_05819_gb300 as hd
    from paper_2209_05819_gb300 import build as cbuild

    cbuild.build()
    print(json.dumps(solve_line(args, torch, hd, N=args.solve_n)))


def serve_only(args):
    """The request-loop line alone, for profiling."""
    import torch

    import paper_2209_05819_gb300 as hd
    from paper_2209_05819_gb300 import build as cbuild

    cbuild.build()
    print(json.dumps(serving_line(args, torch, hd)))


def admissibility_only(args):
    """The admissibility comparison alone (d=2, N=65536, log r), for profiling."""
    import torch

    import paper_2209_05819_gb300 as hd
    from paper_2209_05819_gb300 import build as cbuild

    cbuild.build()
    print(json.dumps(admissibility_line(args, torch, torch.cuda.current_stream(), hd)))


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.only == "many_rhs":
        return many_rhs_only(args)
    if args.only == "batch":
        return batch_only(args)
    if args.only == "solve":
        return solve_only(args)
    if args.only == "serve":
        return serve_only(args)
    if args.only == "admissibility":
        return admissibility_only(args)
    import torch

    import paper_2209_05819_gb300 as hd
    from paper_2209_05819_gb300 import build as cbuild

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = init_group(world, "nccl")
    cbuild.build()
    stream = torch.cuda.current_stream()
    w = workload(args, rank)
    pts = torch.from_numpy(w.points).cuda()
    nrhs = w.nrhs
    units = w.N * nrhs

    h = hd.Handle(pts, w.kernel, w.params, w.leaf, w.tol, precision=args.precision, near_coords=args.near_coords,
                  near_sms=args.near_sms if args.near_sms == "auto" else int(args.near_sms))
    s = h.stats()
    io = torch.float64 if args.precision == "fp64" else torch.float32
    x = torch.from_numpy(np.ascontiguousarray(w.x.reshape(w.N, nrhs))).to(io).cuda()
    y = torch.empty_like(x)

    def step():
        h.matvec(x, y)

    # headline timing (with stage events recorded on the same stream)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    h.set_profiling(True)
    launches0 = h.profile()["launches"]
    with ClockSampler(torch.cuda.current_device()) as clk:
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    seconds = e0.elapsed_time(e1) / 1e3
    if dist is not None:
        dist.barrier()
    prof = h.profile()
    h.set_profiling(False)
    h.sync()  # raises if a bounded device-side wait expired during the timed steps
    launches = prof["launches"] - launches0
    total_units, max_seconds = aggregate(units * args.steps, seconds, dist, device="cuda")
    # measured FP32 / FP64 / MUFU throughput of this GPU at its current clocks:
    # the denominators of the near-field and FP64 rooflines
    peaks = hd.probe_peaks(stream)
    value = total_units / max_seconds
    ms_per_step = 1e3 * max_seconds / args.steps

    # plain FP64 form, and the headline form's error against it
    fp64 = None
    err = None
    y64 = None
    if not args.no_fp64:
        if args.precision == "fp64":
            h64, x64 = h, x
        else:
            h64 = hd.Handle(pts, w.kernel, w.params, w.leaf, w.tol, precision="fp64")
            x64 = x.to(torch.float64)
        y64 = torch.empty_like(x64)
        t64 = time_steps(lambda: h64.matvec(x64, y64), max(3, args.steps // 4), args.warmup, torch, stream)
        n64 = max(3, args.steps // 4)
        h.matvec(x, y)
        torch.cuda.synchronize()
        num = torch.linalg.norm((y.to(torch.float64) - y64), dim=0)
        den = torch.linalg.norm(y64, dim=0)
        err = float((num / den).max().item())
        s64 = h64.stats()
        fp64 = {"value": units * n64 / t64, "ms_per_step": 1e3 * t64 / n64, "build_ms": s64["t_build_ms"],
                "device_gb": s64["device_bytes"] / 1e9,
                "roofline": fp64_roofline(s64, w.d, nrhs, t64 / n64, peaks)}
        if h64 is not h:
            h64.close()

    # the direct O(N^2) product on the GPU (FP32, on the fly): comparator
    direct = None
    if args.precision != "fp64" and w.d <= 3 and nrhs == 1:
        xd = x.reshape(-1)
        yd = torch.empty_like(xd)
        n_d = 3
        t_d = time_steps(lambda: h.direct(xd, yd), n_d, 1, torch, stream)
        h.matvec(x, y)
        torch.cuda.synchronize()
        e_d = float((torch.linalg.norm(y.reshape(-1).double() - yd.double()) / torch.linalg.norm(yd.double())).item())
        direct = {"ms_per_step": 1e3 * t_d / n_d, "value": units * n_d / t_d,
                  "pair_evals_per_s": float(w.N) * w.N * n_d / t_d, "rel_err_hodlrdd_vs_direct": e_d}

    # end to end through the C ABI with host (pinned) buffers
    xh = x.cpu().pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    n_e2e = max(3, args.steps // 2)
    t_e2e = time_steps(lambda: h.matvec(xh, yh), n_e2e, 1, torch, stream)
    e2e_units, e2e_sec = aggregate(units * n_e2e, t_e2e, dist, device="cuda")
    io_bytes = x.element_size() * x.numel()
    # serving latency: one request = one synchronous call with host x and y
    lat = []
    for _ in range(max(20, min(args.steps, 200))):
        t0 = time.perf_counter()
        h.matvec(xh, yh)
        lat.append(1e3 * (time.perf_counter() - t0))
    lat.sort()
    serving = {"p50_ms": lat[len(lat) // 2], "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
               "requests": len(lat), "request": "one matvec through hodlrdd_matvec with pinned host x and y"}

    # roofline of the dominant kernel (bytes it must move per launch / its mean duration)
    ub, vb, tr, scales = factor_bytes(h, args.precision)
    acc = 8 if args.precision == "fp64" else 4
    n_chunks = max(prof["chunks"], 1)
    stage = {"vapply": prof["vapply_ms"] / n_chunks, "uapply": prof["uapply_ms"] / n_chunks,
             "near": prof["near_ms"] / n_chunks, "gather": prof["gather_ms"] / n_chunks}
    nr = min(nrhs, 8)
    slices = s["kappa"] * (2 if args.precision == "fp32+fp16" else 1)  # y_l slices the U-applies write
    algo = {"vapply": vb + scales + tr * nr * acc + w.N * nr * acc,
            "uapply": ub + tr * nr * acc + slices * w.N * nr * acc}
    dom = max(("vapply", "uapply"), key=lambda k: stage[k])
    peak, peak_kind = measured_peaks()
    achieved = algo[dom] / (stage[dom] / 1e3) / 1e9
    roof = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": scaled_traffic(dom, algo[dom], args.precision, nrhs, s["near_sms"]),
            "peak_source": peak_kind, "algorithmic_bytes": algo[dom],
            "algorithmic_bytes_per_kernel": algo,
            "stage_ms": {k: round(v, 4) for k, v in stage.items()},
            "stage_share": {k: round(v / sum(stage.values()), 4) for k, v in stage.items()}}

    roof["near"] = near_roofline(s, w.d, nrhs, stage["near"] / 1e3, peaks, s["near_sms"],
                                 torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)
    roof["fp64"] = fp64["roofline"] if fp64 else None

    # the plain FP64 configuration (d=2, N=4096, log r)
    c1 = None
    if rank == 0 and world == 1:
        c1 = optional_line(plain_fp64_line, args, torch, stream, hd, peaks)

    # many right-hand sides (d=4, N=65536, Matern-3/2, leaf 128, tol 1e-8, nrhs 64)
    many = None
    if rank == 0 and world == 1 and not args.no_many_rhs and args.precision != "fp64":
        many = optional_line(many_rhs_line, args, torch, stream, hd, peaks)

    # the paper's admissibility comparison (H-matrix / HODLRdD / HODLR)
    adm = None
    if rank == 0 and world == 1 and not args.no_admissibility and args.precision != "fp64":
        adm = optional_line(admissibility_line, args, torch, stream, hd)

    # the memory-efficient skeleton form of the low-rank blocks
    skel = None
    if rank == 0 and world == 1 and not args.no_skeleton and args.precision in ("fp32", "fp32+fp16") and nrhs == 1:
        skel = optional_line(skeleton_line, args, torch, stream, hd, w, pts, x, y64)

    # second-kind system (I + K/N) u = b: mixed-precision GMRES with FP64 refinement
    solve = None
    if rank == 0 and world == 1 and not args.no_solve and args.precision != "fp64":
        solve = optional_line(solve_line, args, torch, hd)

    # requests over resident models under an HBM budget
    serve = None
    if rank == 0 and world == 1 and not args.no_serve and args.precision != "fp64":
        serve = optional_line(serving_line, args, torch, hd)

    # 48 uneven trees served as one replayed CUDA graph
    batch = None
    if rank == 0 and world == 1 and not args.no_batch and args.precision != "fp64":
        batch = optional_line(batch_line, args, torch, hd)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args, w)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32", "fp16": "f16+f32", "bf16": "bf16+f32",
                                           "fp32+fp16": "f32 (factors f32 + f16)"}[
                args.precision], "data": "synthetic",
            "config": {"workload": workload_name(w), "precision": args.precision, "near_coords": args.near_coords,
                       "near_sms": s["near_sms"],
                       "factors": ("leading ACA terms FP32, trailing terms FP16 with FP32 column scales, FP32 "
                                   "arithmetic" if args.precision == "fp32+fp16" else
                                   f"{args.precision} U,V with FP32 accumulation" if args.precision != "fp64"
                                   else "fp64"), "parallelism": f"replicas x{world}",
                       "l2": f"inputs larger than L2: {(ub + vb) / 1e9:.2f} GB of factors streamed per step"},
            "rel_err_vs_fp64": err, "meets_err_bar": (err is not None and err <= ERR_BAR),
            "fp64": fp64, "speedup_vs_fp64": (value / (fp64["value"] * world)) if fp64 else None,
            "direct_gpu": direct,
            "plain_fp64_c1": c1,
            "many_rhs": many,
            "skeleton": skel,
            "admissibility": adm,
            "solve": solve,
            "batch": batch,
            "serving_loop": serve,
            "build": {k: round(s[k], 1) for k in ("t_build_ms", "t_tree_ms", "t_classify_ms", "t_aca_ms",
                                                   "t_pack_ms")},
            "structure": {"kappa": s["kappa"], "n_blocks": s["n_blocks"], "n_lowrank": s["n_lowrank"],
                          "n_dense": s["n_dense"], "max_rank": s["max_rank"], "factor_gb": (ub + vb) / 1e9,
                          "dense_pairs": s["dense_pairs"], "mean_rank_per_level":
                              [round(v, 1) for v in s["mean_rank_per_level"]]},
            "roofline": roof,
            "cpu_baseline": cpu,
            "peaks_probe": peaks,
            "e2e": {"value": e2e_units / e2e_sec, "unit": UNIT, "h2d_bytes_per_step": io_bytes,
                    "d2h_bytes_per_step": io_bytes},
            "serving": serving,
            "gpu_launches": launches,
            "clocks": clk.summary(),
        }
        print(json.dumps(line))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
