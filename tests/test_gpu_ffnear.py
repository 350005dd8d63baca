"""The FP64 form's float-float near field (fp64_near "ff"): kernel values from
48-bit arithmetic on the FP32 pipes, then whole products.

Pins, independent of the GPU's FP64 path:
* every kernel function against its closed form evaluated by numpy in FP64,
  over distances from 1e-6 to 5 box sizes, at several box sizes: the
  float-float evaluation keeps a relative error of about 2^-44 (bound 2e-13;
  log r, which crosses zero, against max(|F|, |log r| + 1); the exponential
  kernels, bounded by 1, against max(|F|, 0.01), since exp(-a) inherits a times
  the relative error of its argument);
* products against the oracle's HODLRdD product on the oracle's own factors
  (imported), so the near field is the only part computed differently from the
  plain FP64 form: bound 1e-12 (the FP64 form's parity bar is 1e-10);
* a second-kind solve whose FP64 refinement operator uses the float-float near
  field reaches 1e-10 against the plain FP64 operator.
"""
import numpy as np
import pytest

import workloads as W
from gpu_util import gpu_handle, gpu_matvec, oracle_factors, relerr, require_cuda

pytestmark = pytest.mark.gpu

FF_KERNEL_BOUND = 2e-13
FF_PRODUCT_BOUND = 1e-12


@pytest.fixture(scope="module")
def env():
    torch = require_cuda()
    import oracle
    import paper_2209_05819_gb300 as hd

    oracle.build()
    return torch, oracle, hd


def closed_form(kernel, p, s):
    r = np.sqrt(s)
    if kernel == W.K_LOG:
        return np.where(s > 0, 0.5 * np.log(np.where(s > 0, s, 1.0)), 0.0)
    if kernel == W.K_INV_R:
        return np.where(s > 0, 1.0 / np.where(s > 0, r, 1.0), 0.0)
    if kernel == W.K_MATERN32:
        a = np.sqrt(3.0) * r / p[2]
        return (1.0 + a) * np.exp(-a)
    if kernel == W.K_GAUSS:
        return np.exp(-s / (2.0 * p[2] ** 2))
    if kernel == W.K_EXP:
        return np.exp(-r / p[2])
    if kernel == W.K_INV_R2_4D:
        return np.where(s > 0, -1.0 / (4.0 * np.pi ** 2 * np.where(s > 0, s, 1.0)), 0.0)
    if kernel == W.K_R:
        return r
    if kernel == W.K_INV_SQRT1P:
        return 1.0 / np.sqrt(1.0 + r)
    raise ValueError(kernel)


KERNELS = [(W.K_LOG, (1, 0, 0, 0)), (W.K_INV_R, (1, 0, 0, 0)), (W.K_MATERN32, (1, 0, 0.2, 0)),
           (W.K_GAUSS, (1, 0, 0.5, 0)), (W.K_EXP, (1, 0, 1.0, 0)), (W.K_INV_R2_4D, (1, 0, 0, 0)),
           (W.K_R, (1, 0, 0, 0)), (W.K_INV_SQRT1P, (1, 0, 0, 0))]
KIDS = ["log", "invr", "matern", "gauss", "exp", "invr2", "r", "invsqrt1p"]


@pytest.mark.parametrize("kernel,params", KERNELS, ids=KIDS)
@pytest.mark.parametrize("h", [0.125, 2.0 / 3.0, 1.7])
def test_kernel_values_against_closed_forms(env, kernel, params, h):
    torch, oracle, hd = env
    from paper_2209_05819_gb300 import _binding as B

    rng = np.random.default_rng(kernel + int(100 * h))
    r = h * np.exp(rng.uniform(np.log(1e-6), np.log(5.0), 4000))
    s = np.concatenate([[0.0], r * r])
    got = B.debug_ff_eval(kernel, params, h, s)
    ref = closed_form(kernel, params, s)
    if kernel == W.K_LOG:
        scale = np.maximum(np.abs(ref), np.abs(np.log(np.maximum(np.sqrt(s), 1e-300))) + 1.0)
    elif kernel in (W.K_MATERN32, W.K_GAUSS, W.K_EXP):
        # exp(-a) carries a times the relative error of its argument a (in any
        # arithmetic); these kernels are at most 1, so the error is taken
        # against max(|F|, 0.01)
        scale = np.maximum(np.abs(ref), 1e-2)
    else:
        scale = np.abs(ref)
    err = np.abs(got - ref) / np.where(scale > 0, scale, 1.0)
    print(f"{KIDS[[k for k, _ in KERNELS].index(kernel)]} h={h:.3f}: max rel err {err.max():.2e}")
    assert got[0] == ref[0] or kernel not in (W.K_LOG, W.K_INV_R, W.K_INV_R2_4D)
    assert err.max() <= FF_KERNEL_BOUND


CASES = [
    (1, 3000, W.K_EXP, (1, 0, 1.0, 0), 32, "uniform", 0),
    (2, 6000, W.K_LOG, (1, 0, 0, 0), 64, "uniform", 0),
    (3, 9000, W.K_INV_R, (1, 0, 0, 0), 64, "uniform", 0),
    (3, 7000, W.K_INV_R, (1.0 / 7000, 1.0, 0, 0), 32, "clustered", 0),
    (3, 8000, W.K_GAUSS, (1, 1e-3, 0.5, 0), 64, "clustered", 2),
    (4, 5000, W.K_MATERN32, (1, 0, 0.3, 0), 64, "uniform", 0),
    (4, 4000, W.K_INV_R2_4D, (1, 0, 0, 0), 32, "uniform", 1),
    (2, 5000, W.K_R, (1, 0, 0, 0), 32, "uniform", 0),
    (3, 5000, W.K_INV_SQRT1P, (0.5, 0.25, 0, 0), 32, "uniform", 0),
]
IDS = ["exp_d1", "log_d2", "invr_d3", "invr_d3_system_clustered", "gauss_d3_clustered_lists", "matern_d4",
       "invr2_d4_tiles", "r_d2", "invsqrt1p_d3"]


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_products_against_oracle(env, case):
    torch, oracle, hd = env
    d, N, kernel, params, leaf, dist, near_mode = case
    w = W.make("t", d, N, kernel, params, leaf, 1e-10, nrhs=1, seed=N + 7 * d, dist=dist)
    T = oracle.Tree(w.points, w.kernel, w.params, leaf, w.tol, dense_if_cheaper=True)
    yo = T.matvec(w.x)
    fac = oracle_factors(T)
    hf = gpu_handle(hd, w, fp64_near="ff", near_mode=near_mode)
    hf.import_factors(*fac)
    y1 = gpu_matvec(hf, w.x)
    y2 = gpu_matvec(hf, w.x)
    assert np.array_equal(y1, y2)
    err = relerr(y1, yo)
    h64 = gpu_handle(hd, w, near_mode=near_mode)
    h64.import_factors(*fac)
    e64 = relerr(gpu_matvec(h64, w.x), yo)
    print(f"{IDS[CASES.index(case)]}: ff {err:.2e}  fp64 {e64:.2e}")
    assert err <= FF_PRODUCT_BOUND
    # several right-hand sides go through the FP64 path column chunks; one column through the float-float one
    x3 = np.ascontiguousarray(np.stack([w.x[:, 0], 2 * w.x[:, 0], -w.x[:, 0]], axis=1))
    y3 = gpu_matvec(hf, x3)
    assert relerr(y3[:, :1], y1) <= FF_PRODUCT_BOUND
    hf.close()
    h64.close()


def test_solve_with_ff_refinement_operator(env):
    torch, oracle, hd = env
    N = 20000
    w = W.make("t", 3, N, W.K_INV_R, (1.0 / N, 1.0, 0, 0), 64, 1e-9, nrhs=1, seed=5)
    outer = gpu_handle(hd, w, fp64_near="ff")
    plain = gpu_handle(hd, w)
    inner = gpu_handle(hd, w, precision="fp32+fp16")
    b = torch.from_numpy(np.ascontiguousarray(w.x[:, 0])).cuda()
    x, st = hd.solve(inner, outer, b, tol=1e-10)
    torch.cuda.synchronize()
    assert st["residual"] <= 1e-10
    y = plain.matvec(x)
    torch.cuda.synchronize()
    assert relerr(y.cpu().numpy()[:, None], w.x) <= 1.1e-10


def test_ff_rejects_sin(env):
    torch, oracle, hd = env
    w = W.make("t", 2, 800, W.K_SIN, (1, 0, 0, 0), 32, 1e-8, seed=3)
    with pytest.raises(hd.HodlrddError) as e:
        gpu_handle(hd, w, fp64_near="ff")
    assert e.value.status == hd.ERR_UNSUPPORTED
    from paper_2209_05819_gb300 import _binding as B

    with pytest.raises(hd.HodlrddError) as e:
        B.debug_ff_eval(W.K_SIN, (1, 0, 0, 0), 1.0, np.ones(3))
    assert e.value.status == hd.ERR_UNSUPPORTED


def test_ff_stage_timing(env):
    """Stage events with the float-float near field on the second stream."""
    torch, oracle, hd = env
    w = W.make("t", 3, 6000, W.K_INV_R, (1, 0, 0, 0), 64, 1e-8, nrhs=1, seed=8)
    hf = gpu_handle(hd, w, fp64_near="ff")
    hf.set_profiling(True)
    gpu_matvec(hf, w.x)
    pr = hf.profile()
    hf.set_profiling(False)
    assert pr["chunks"] == 1 and pr["near_ms"] > 0 and pr["vapply_ms"] > 0
    hf.close()
