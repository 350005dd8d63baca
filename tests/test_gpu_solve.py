"""hodlrdd_solve: GMRES on a fast operator inside FP64 refinement, for the
second-kind integral-equation system (I + K/N) u = b of the paper's numerical
experiments. The solution is checked against the oracle's exact (direct-sum)
operator, so the pin is the system itself, not the GPU's own residual."""
import numpy as np
import pytest

import workloads as W
from gpu_util import gpu_handle, relerr, require_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = require_cuda()
    import oracle
    import paper_2209_05819_gb300 as hd

    oracle.build()
    return torch, oracle, hd


@pytest.mark.parametrize("inner_prec", ["fp32", "fp16", "fp64"])
def test_second_kind_system(env, inner_prec):
    torch, oracle, hd = env
    N = 6000
    w = W.make("t", 3, N, W.K_INV_R, (1.0 / N, 1.0, 0, 0), 32, 1e-10, nrhs=1, seed=21)
    outer = gpu_handle(hd, w)
    inner = outer if inner_prec == "fp64" else gpu_handle(hd, w, precision=inner_prec)
    b = torch.from_numpy(np.ascontiguousarray(w.x[:, 0])).cuda()
    x, st = hd.solve(inner, outer, b, tol=1e-10)
    torch.cuda.synchronize()
    assert st["residual"] <= 1e-10
    assert 1 <= st["refinements"] <= 20 and st["inner_iterations"] >= 1
    xs = x.cpu().numpy()
    # the exact operator: (I + K/N) x against b, direct sum in FP64
    kx = oracle.direct(w.points, w.kernel, w.params, xs[:, None])[:, 0]
    assert relerr(kx[:, None], w.x) <= 1e-8  # HODLRdD approximation at ACA tol 1e-10
    # the GPU's FP64 HODLRdD operator on x reproduces b to the solve tolerance
    y = outer.matvec(x)
    torch.cuda.synchronize()
    assert relerr(y.cpu().numpy()[:, None], w.x) <= 1.1e-10


def test_solve_rejects_bad_arguments(env):
    torch, oracle, hd = env
    w = W.make("t", 2, 800, W.K_LOG, (1.0 / 800, 1.0, 0, 0), 32, 1e-8, seed=3)
    h64 = gpu_handle(hd, w)
    h32 = gpu_handle(hd, w, precision="fp32")
    b = torch.from_numpy(np.ascontiguousarray(w.x[:, 0])).cuda()
    with pytest.raises(hd.HodlrddError) as e:
        hd.solve(h64, h32, b)  # outer must be FP64
    assert e.value.status == hd.ERR_INVALID
    with pytest.raises(hd.HodlrddError) as e:
        hd.solve(h32, h64, b, restart=0)
    assert e.value.status == hd.ERR_INVALID
    w2 = W.make("t", 2, 900, W.K_LOG, (1.0 / 900, 1.0, 0, 0), 32, 1e-8, seed=4)
    h2 = gpu_handle(hd, w2)
    with pytest.raises(hd.HodlrddError) as e:
        hd.solve(h32, h2, b)  # different point sets
    assert e.value.status == hd.ERR_INVALID
