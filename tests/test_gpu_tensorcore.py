"""The tensor-core form (precision "fp16x2"): low-rank applies as tcgen05 MMAs
on FP16 high / scaled-low factor pairs, the near field's 64-wide accumulation on
the tensor cores for the bounded kernels (FP32 tiles for 1/r and 1/r^2).

Bound: the pair hi + 2^-11 lo carries about 22 significant bits of every
factor entry, kernel value and vector entry, and the MMAs accumulate in FP32,
so the product's error is of FP32 size, like the FP32 form's (2e-6 for one or
two right-hand sides there, 5e-6 for uncompensated wide chunks): TC_BOUND =
5e-6 against the FP64 product. Against the oracle's HODLRdD product on the
oracle's own factors the same bound holds.
"""
import numpy as np
import pytest

import workloads as W
from gpu_util import gpu_handle, gpu_matvec, oracle_factors, relerr, require_cuda

pytestmark = pytest.mark.gpu

TC_BOUND = 5e-6


@pytest.fixture(scope="module")
def env():
    torch = require_cuda()
    import oracle
    import paper_2209_05819_gb300 as hd

    oracle.build()
    return torch, oracle, hd


CASES = [
    (3, 9000, W.K_INV_R, None, 32, 1e-8),               # 1/r: near field on FP32 tiles
    (4, 6000, W.K_MATERN32, (1, 0, 0.3, 0), 64, 1e-7),  # near field on the tensor cores
    (2, 4096, W.K_LOG, None, 64, 1e-8),
    (3, 8000, W.K_GAUSS, (1, 1e-3, 0.5, 0), 64, 1e-6),
    (1, 3001, W.K_EXP, (1, 0, 1.0, 0), 16, 1e-10),
    (2, 3000, W.K_SIN, None, 25, 1e-9),
    (3, 3000, W.K_INV_SQRT1P, (0.5, 0.25, 0, 0), 25, 1e-9),
    (4, 3000, W.K_INV_R2_4D, None, 30, 1e-8),
]
IDS = ["invr_d3", "matern_d4", "log_d2", "gauss_d3", "exp_d1", "sin_d2", "invsqrt_d3", "invr2_d4"]


@pytest.mark.parametrize("case", CASES, ids=IDS)
@pytest.mark.parametrize("nrhs", [1, 17, 64, 70])
def test_matches_fp64(env, case, nrhs):
    torch, oracle, hd = env
    d, N, kernel, params, leaf, tol = case
    w = W.make("t", d, N, kernel, params or (1, 0, 0, 0), leaf, tol, nrhs=nrhs, seed=N + 31 * d + nrhs)
    h64 = gpu_handle(hd, w)
    ht = gpu_handle(hd, w, precision="fp16x2")
    assert np.array_equal(h64.blocks(), ht.blocks())
    y64 = gpu_matvec(h64, w.x)
    yt = gpu_matvec(ht, w.x)
    ht.sync()
    err = relerr(yt, y64)
    print(f"fp16x2 {IDS[CASES.index(case)]} nrhs={nrhs}: {err:.2e}")
    assert err <= TC_BOUND, err


@pytest.mark.parametrize("case", CASES[:4], ids=IDS[:4])
def test_on_oracle_factors(env, case):
    """The oracle's factors imported: the product equals the oracle's Algorithm 2
    within the FP32-size bound (no ACA difference remains)."""
    torch, oracle, hd = env
    d, N, kernel, params, leaf, tol = case
    w = W.make("t", d, N, kernel, params or (1, 0, 0, 0), leaf, tol, nrhs=64, seed=N + 5)
    T = oracle.Tree(w.points, w.kernel, w.params, leaf, tol, dense_if_cheaper=True)
    ht = gpu_handle(hd, w, precision="fp16x2")
    ht.import_factors(*oracle_factors(T))
    yt = gpu_matvec(ht, w.x)
    ht.sync()
    err = relerr(yt, T.matvec(w.x))
    print(f"fp16x2 on oracle factors {IDS[CASES.index(case)]}: {err:.2e}")
    assert err <= TC_BOUND, err


def test_against_direct_sum_and_determinism(env):
    torch, oracle, hd = env
    w = W.make("t", 4, 8000, W.K_MATERN32, (1, 0, 0.2, 0), 64, 1e-8, nrhs=64, seed=41)
    ht = gpu_handle(hd, w, precision="fp16x2")
    x = torch.from_numpy(np.ascontiguousarray(w.x, dtype=np.float32)).cuda()
    y1 = ht.matvec(x)
    y2 = ht.matvec(x)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)  # one writer per output, fixed order
    yh = ht.matvec(np.ascontiguousarray(w.x, dtype=np.float32))
    assert np.array_equal(np.asarray(yh), y1.cpu().numpy())
    yd = oracle.direct(w.points, w.kernel, w.params, w.x)
    assert relerr(y1.cpu().numpy(), yd) <= 10 * w.tol + TC_BOUND
    # columns of a chunk against the same columns alone
    y5 = gpu_matvec(ht, w.x[:, 5:6])
    assert relerr(y1.cpu().numpy()[:, 5:6], y5) <= 2 * TC_BOUND
    s = ht.stats()
    assert s["factor_bytes_u"] > 0 and s["factor_bytes_v"] > 0


def test_second_kind_and_uneven_clusters(env):
    """(I + K/N) with clustered points: diag and scale reach the tensor-core near
    field, boxes of uneven size give 64-row panels and cut U panels."""
    torch, oracle, hd = env
    N = 30000
    w = W.make("t", 3, N, W.K_GAUSS, (1.0 / N, 1.0, 0.5, 0), 64, 1e-6, nrhs=33, seed=77, dist="clustered")
    h64 = gpu_handle(hd, w)
    ht = gpu_handle(hd, w, precision="fp16x2")
    err = relerr(gpu_matvec(ht, w.x), gpu_matvec(h64, w.x))
    ht.sync()
    assert err <= TC_BOUND, err


@pytest.mark.parametrize("nrhs", [1, 64])
def test_dense_rule_leaf_only(env, nrhs):
    """The tensor-core form with dense_if_cheaper="leaf" (coarse admissible
    blocks streamed as factors, the leaf level evaluated on the fly) against
    the FP64 form built with the same rule."""
    torch, oracle, hd = env
    w = W.make("t", 3, 8000, W.K_MATERN32, (1, 0, 0.3, 0), 32, 1e-8, nrhs=nrhs, seed=90 + nrhs)
    h64 = gpu_handle(hd, w, dense_if_cheaper="leaf")
    ht = gpu_handle(hd, w, precision="fp16x2", dense_if_cheaper="leaf")
    assert np.array_equal(h64.blocks(), ht.blocks())
    err = relerr(gpu_matvec(ht, w.x), gpu_matvec(h64, w.x))
    ht.sync()
    assert err <= TC_BOUND, err


def test_rejected_configurations(env):
    torch, oracle, hd = env
    w5 = W.make("t", 5, 1500, W.K_GAUSS, (1, 0, 0.5, 0), 32, 1e-6, nrhs=1, seed=2)
    with pytest.raises(hd.HodlrddError) as e:
        gpu_handle(hd, w5, precision="fp16x2")
    assert e.value.status == hd.ERR_UNSUPPORTED
    w = W.make("t", 3, 2000, W.K_INV_R, (1, 0, 0, 0), 32, 1e-8, nrhs=1, seed=2)
    with pytest.raises(hd.HodlrddError) as e:
        gpu_handle(hd, w, precision="fp16x2", lowrank_form="skeleton")
    assert e.value.status == hd.ERR_UNSUPPORTED
    ht = gpu_handle(hd, w, precision="fp16x2")
    rec = ht.blocks()
    b = int(np.flatnonzero(rec[:, 7] > 0)[0])
    with pytest.raises(hd.HodlrddError) as e:
        ht.factors(b, int(rec[b, 4]), int(rec[b, 6]), int(rec[b, 7]))
    assert e.value.status == hd.ERR_UNSUPPORTED
