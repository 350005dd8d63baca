"""Forests: the products of many FP16X2 trees merged into one launch per stage.

Every tree's result is compared with that tree's FP64 product (the bound of
the tensor-core form, TC_BOUND = 5e-6, derived beside the tensor-core tests)
and with its own FP16X2 product (the same arithmetic; only the power-of-two
scale of each right-hand-side column, now the maximum over the forest, can move
an FP16 rounding, so twice the bound). Trees differ in size, point layout,
leaf size, dense rule, scale and diagonal, and right-hand-side count.
"""
import numpy as np
import pytest

import workloads as W
from gpu_util import gpu_handle, gpu_matvec, relerr, require_cuda

pytestmark = pytest.mark.gpu

TC_BOUND = 5e-6


@pytest.fixture(scope="module")
def env():
    torch = require_cuda()
    import oracle
    import paper_2209_05819_gb300 as hd

    oracle.build()
    return torch, oracle, hd


def _trees(kernel, d, shape, n, seed, nrhs_choice=(1, 5, 17, 33, 64)):
    out = []
    for s in range(n):
        rng = np.random.default_rng(seed + s)
        N = int(rng.integers(1500, 16000))
        nrhs = int(nrhs_choice[s % len(nrhs_choice)])
        second = s % 3 == 2
        scale, diag = (1.0 / N, 1.0) if second else (1.0, 0.0)
        w = W.make(f"f{s}", d, N, kernel, (scale, diag) + tuple(shape), 32 if s % 2 else 64, 1e-7, nrhs=nrhs,
                   seed=seed + s, dist="clustered" if s % 2 else "uniform")
        out.append((w, "leaf" if s % 2 else True))
    return out


def _check_forest(torch, hd, trees):
    hs = [gpu_handle(hd, w, precision="fp16x2", dense_if_cheaper=dr) for w, dr in trees]
    h64 = [gpu_handle(hd, w, dense_if_cheaper=dr) for w, dr in trees]
    xs = [torch.from_numpy(np.ascontiguousarray(w.x, dtype=np.float32)).cuda() for w, _ in trees]
    f = hd.Forest(hs, [w.nrhs for w, _ in trees])
    ys = f.run(xs)
    torch.cuda.synchronize()
    worst = 0.0
    for (w, _), y, ht, hr in zip(trees, ys, hs, h64):
        yf = y.cpu().numpy()
        e64 = relerr(yf, gpu_matvec(hr, w.x))
        etc = relerr(yf, gpu_matvec(ht, w.x))
        worst = max(worst, e64)
        assert e64 <= TC_BOUND, (w.name, w.N, w.nrhs, e64)
        assert etc <= 2 * TC_BOUND, (w.name, w.N, w.nrhs, etc)
    for h in hs:
        h.sync()
    return f, hs, xs, ys, worst


def test_forest_matches_trees(env):
    torch, oracle, hd = env
    trees = _trees(W.K_MATERN32, 4, (0.3, 0), 6, 500)
    f, hs, xs, ys, worst = _check_forest(torch, hd, trees)
    print(f"forest of {len(trees)} Matern d=4 trees: worst {worst:.2e}; {f.stats()}")
    # one writer per output, fixed order: runs repeat bitwise
    ys2 = f.run(xs)
    torch.cuda.synchronize()
    for a, b in zip(ys, ys2):
        assert torch.equal(a, b)
    # host buffers give the same results
    yh = f.run([x.cpu().numpy() for x in xs])
    for a, b in zip(ys, yh):
        assert np.array_equal(a.cpu().numpy(), b)
    s = f.stats()
    assert s["points"] == sum(w.N for w, _ in trees)
    assert s["launches_per_run"] >= 4 + s["near_passes"]
    f.close()


@pytest.mark.parametrize(
    "kernel,d,shape",
    [(W.K_LOG, 2, (0, 0)), (W.K_GAUSS, 3, (0.5, 0)), (W.K_EXP, 1, (1.0, 0)), (W.K_SIN, 2, (0, 0)),
     (W.K_INV_SQRT1P, 3, (0, 0))],
    ids=["log_d2", "gauss_d3", "exp_d1", "sin_d2", "invsqrt_d3"])
def test_forest_kernels(env, kernel, d, shape):
    torch, oracle, hd = env
    trees = _trees(kernel, d, shape, 4, 700 + 10 * kernel + d)
    f, *_ = _check_forest(torch, hd, trees)
    f.close()


def test_forest_against_direct_sum(env):
    """One tree of a forest against the oracle's dense product."""
    torch, oracle, hd = env
    trees = _trees(W.K_MATERN32, 3, (0.2, 0), 3, 900)
    hs = [gpu_handle(hd, w, precision="fp16x2", dense_if_cheaper=dr) for w, dr in trees]
    f = hd.Forest(hs, [w.nrhs for w, _ in trees])
    ys = f.run([np.ascontiguousarray(w.x, dtype=np.float32) for w, _ in trees])
    for (w, _), y in zip(trees, ys):
        yd = oracle.direct(w.points, w.kernel, w.params, w.x)
        assert relerr(y, yd) <= 10 * w.tol + TC_BOUND
    f.close()


def test_single_tree_forest(env):
    torch, oracle, hd = env
    w = W.make("one", 4, 9000, W.K_MATERN32, (1, 0, 0.3, 0), 64, 1e-7, nrhs=64, seed=5)
    ht = gpu_handle(hd, w, precision="fp16x2")
    f = hd.Forest([ht], [64])
    y = f.run([np.ascontiguousarray(w.x, dtype=np.float32)])[0]
    assert relerr(y, gpu_matvec(ht, w.x)) <= 2 * TC_BOUND
    f.close()


def test_forest_rejections(env):
    torch, oracle, hd = env
    wa = W.make("a", 3, 3000, W.K_GAUSS, (1, 0, 0.5, 0), 32, 1e-6, nrhs=1, seed=1)
    wb = W.make("b", 3, 2500, W.K_GAUSS, (1, 0, 0.7, 0), 32, 1e-6, nrhs=1, seed=2)
    wc = W.make("c", 2, 2500, W.K_GAUSS, (1, 0, 0.5, 0), 32, 1e-6, nrhs=1, seed=3)
    ha = gpu_handle(hd, wa, precision="fp16x2")
    with pytest.raises(hd.HodlrddError) as e:
        hd.Forest([ha, ha], [1, 1])
    assert e.value.status == hd.ERR_INVALID
    with pytest.raises(hd.HodlrddError) as e:
        hd.Forest([ha], [65])
    assert e.value.status == hd.ERR_INVALID
    for other in (gpu_handle(hd, wa, precision="fp32"), gpu_handle(hd, wb, precision="fp16x2"),
                  gpu_handle(hd, wc, precision="fp16x2")):
        with pytest.raises(hd.HodlrddError) as e:
            hd.Forest([ha, other], [1, 1])
        assert e.value.status == hd.ERR_UNSUPPORTED
    f = hd.Forest([ha], [1])
    with pytest.raises(ValueError):
        f.run([np.zeros((wa.N, 2), np.float32)])
    f.close()
