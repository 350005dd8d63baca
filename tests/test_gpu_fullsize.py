"""Parity at the full benchmark sizes, in the configurations bench.py times.

The oracle cannot run a whole HODLRdD build at these sizes within a test, so
the checks are (i) sampled output rows against the oracle's direct FP64 sum,
computed row by row, and (ii) properties that hold at any size: the FP32 forms
against the GPU FP64 form over every row, and bitwise determinism.
"""
import numpy as np
import pytest

import workloads as W
from gpu_util import relerr, require_cuda

pytestmark = pytest.mark.gpu

FP32_BOUND = 2e-6       # stored FP32 factors, one or two right-hand sides
FP32_WIDE_BOUND = 5e-6  # chunks of 4-16 right-hand sides (uncompensated applies)
SKELETON_FP32_BOUND = 5e-6
TC_BOUND = 5e-6          # the tensor-core form (FP16 high / scaled-low pairs, FP32 accumulation)
NEAR_HI_BOUND = 1e-6     # hi-only near-field coordinates at the benchmark size (the metric's bar)


@pytest.fixture(scope="module")
def env():
    torch = require_cuda()
    import oracle
    import paper_2209_05819_gb300 as hd

    oracle.build()
    return torch, oracle, hd


def sample_rows(N, n_ranges=4, width=64, seed=7):
    rng = np.random.default_rng(seed)
    starts = np.sort(rng.choice(N // width, n_ranges, replace=False)) * width
    return [(int(s), int(s) + width) for s in starts]


def direct_rows(oracle, w, ranges):
    return np.concatenate([oracle.direct(w.points, w.kernel, w.params, w.x, r) for r in ranges])


def pick(y, ranges):
    return np.concatenate([y[r0:r1] for r0, r1 in ranges])


def test_benchmark_workload_d3_n262144(env):
    """d=3, N=262144 uniform [-1,1]^3, 1/r, leaf 64, tol 1e-7, one right-hand side: FP64, FP32,
    the mixed FP32 / FP16 storage (the benchmark's) and the FP32 skeleton form."""
    torch, oracle, hd = env
    w = W.precision_3d()
    pts = torch.from_numpy(w.points).cuda()
    ranges = sample_rows(w.N)
    yd = direct_rows(oracle, w, ranges)
    x64 = torch.from_numpy(np.ascontiguousarray(w.x)).cuda()
    x32 = x64.float()
    h64 = hd.Handle(pts, w.kernel, w.params, w.leaf, w.tol, precision="fp64")
    y64 = h64.matvec(x64)
    torch.cuda.synchronize()
    y64n = y64.cpu().numpy()
    assert relerr(pick(y64n, ranges), yd) <= 10 * w.tol
    h64.close()
    # the benchmarked form: stored FP32 factors, packed near field on the second stream
    h32 = hd.Handle(pts, w.kernel, w.params, w.leaf, w.tol, precision="fp32")
    y1 = h32.matvec(x32)
    y2 = h32.matvec(x32)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)
    y32n = y1.cpu().numpy()
    assert relerr(y32n, y64n) <= 1e-6  # the benchmark's error bar, every row
    assert relerr(pick(y32n, ranges), yd) <= 10 * w.tol + FP32_BOUND
    # the same product through host buffers (the end-to-end leg)
    yh = h32.matvec(np.ascontiguousarray(w.x, dtype=np.float32))
    assert np.array_equal(np.asarray(yh), y32n)
    h32.close()
    # the storage bench.py times by default: leading terms FP32, trailing terms FP16
    hm = hd.Handle(pts, w.kernel, w.params, w.leaf, w.tol, precision="fp32+fp16")
    m1 = hm.matvec(x32)
    m2 = hm.matvec(x32)
    torch.cuda.synchronize()
    assert torch.equal(m1, m2)
    ymn = m1.cpu().numpy()
    # measured 2.6e-7: a defect in the FP16 tail adding 5e-7 of error fails here
    assert relerr(ymn, y64n) <= 5e-7
    assert relerr(pick(ymn, ranges), yd) <= 10 * w.tol + FP32_BOUND
    hm.close()
    # the same storage with hi-only tile coordinates (near_coords "hi", the
    # benchmark's setting): distances carry 2^-24 h absolute error; measured
    # 4.0e-7 against FP64, held to the metric's bar of 1e-6
    hh = hd.Handle(pts, w.kernel, w.params, w.leaf, w.tol, precision="fp32+fp16", near_coords="hi")
    q1 = hh.matvec(x32)
    q2 = hh.matvec(x32)
    torch.cuda.synchronize()
    assert torch.equal(q1, q2)
    yqn = q1.cpu().numpy()
    assert relerr(yqn, y64n) <= NEAR_HI_BOUND
    assert relerr(pick(yqn, ranges), yd) <= 10 * w.tol + NEAR_HI_BOUND
    hh.close()
    # the skeleton form on the same workload
    hs = hd.Handle(pts, w.kernel, w.params, w.leaf, w.tol, precision="fp32", lowrank_form="skeleton")
    ys = hs.matvec(x32)
    torch.cuda.synchronize()
    ysn = ys.cpu().numpy()
    assert relerr(ysn, y64n) <= SKELETON_FP32_BOUND
    assert relerr(pick(ysn, ranges), yd) <= 10 * w.tol + SKELETON_FP32_BOUND
    hs.close()


def test_many_rhs_workload_d4_n65536(env):
    """d=4, N=65536 uniform [0,1]^4, Matern-3/2 l=0.2, leaf 128, tol 1e-8, 64 right-hand sides."""
    torch, oracle, hd = env
    w = W.many_rhs_4d()
    pts = torch.from_numpy(w.points).cuda()
    ranges = sample_rows(w.N, n_ranges=2, width=32, seed=11)
    yd = direct_rows(oracle, w, ranges)
    h = hd.Handle(pts, w.kernel, w.params, w.leaf, w.tol, precision="fp32", max_nrhs=w.nrhs)
    x = torch.from_numpy(np.ascontiguousarray(w.x, dtype=np.float32)).cuda()
    y = h.matvec(x)
    torch.cuda.synchronize()
    yn = y.cpu().numpy()
    assert relerr(pick(yn, ranges), yd) <= 10 * w.tol + FP32_WIDE_BOUND
    # columns applied in the 16-wide chunks equal single-column products to the FP32 bound
    for c in (0, 37, 63):
        yc = h.matvec(x[:, c : c + 1].contiguous())
        torch.cuda.synchronize()
        assert relerr(yn[:, c : c + 1], yc.cpu().numpy()) <= 2 * FP32_WIDE_BOUND
    h.close()


def test_many_rhs_workload_tensor_cores(env):
    """The same workload in the tensor-core form the benchmark times: sampled rows
    against the oracle's direct FP64 sum, every row against the FP32 CUDA-core
    form, and bitwise determinism."""
    torch, oracle, hd = env
    w = W.many_rhs_4d()
    pts = torch.from_numpy(w.points).cuda()
    ranges = sample_rows(w.N, n_ranges=2, width=32, seed=12)
    yd = direct_rows(oracle, w, ranges)
    x = torch.from_numpy(np.ascontiguousarray(w.x, dtype=np.float32)).cuda()
    ht = hd.Handle(pts, w.kernel, w.params, w.leaf, w.tol, precision="fp16x2", dense_if_cheaper="leaf")
    y1 = ht.matvec(x)
    y2 = ht.matvec(x)
    torch.cuda.synchronize()
    ht.sync()
    assert torch.equal(y1, y2)
    yt = y1.cpu().numpy()
    ht.close()
    assert relerr(pick(yt, ranges), yd) <= 10 * w.tol + TC_BOUND
    h32 = hd.Handle(pts, w.kernel, w.params, w.leaf, w.tol, precision="fp32", max_nrhs=w.nrhs)
    y32 = h32.matvec(x)
    torch.cuda.synchronize()
    assert relerr(yt, y32.cpu().numpy()) <= TC_BOUND + FP32_WIDE_BOUND
    h32.close()
