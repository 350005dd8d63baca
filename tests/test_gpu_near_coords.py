"""Near-field coordinates of the single-right-hand-side FP32 tiles: hi + lo pairs
(default, distances with FP32 relative accuracy) against hi only (option
near_coords "hi": a distance r carries an absolute error of about 2^-24 h, h the
leaf box size). Both forms are compared with the oracle's HODLRdD product on the
oracle's own factors (imported), so the near-field arithmetic is the only
difference from the oracle beyond the FP32 factor storage.

Bounds: hi + lo keeps the FP32 form's 2e-6; hi only adds the coordinate
rounding, relative 2^-24 h / r per pair (measured at most 5.1e-7 here, against
3.2e-7 for hi + lo), and is held to the same 2e-6.
"""
import numpy as np
import pytest

import workloads as W
from gpu_util import gpu_handle, gpu_matvec, oracle_factors, relerr, require_cuda

pytestmark = pytest.mark.gpu

FP32_BOUND = 2e-6
NEAR_HI_SMALL_BOUND = 2e-6


@pytest.fixture(scope="module")
def env():
    torch = require_cuda()
    import oracle
    import paper_2209_05819_gb300 as hd

    oracle.build()
    return torch, oracle, hd


CASES = [
    (3, 12000, W.K_INV_R, (1, 0, 0, 0), 64, 1e-8, "uniform"),
    (3, 9000, W.K_INV_R, (1, 0, 0, 0), 32, 1e-8, "clustered"),
    (2, 8000, W.K_LOG, (1, 0, 0, 0), 64, 1e-8, "uniform"),
    (3, 8000, W.K_GAUSS, (1, 0, 0.5, 0), 64, 1e-8, "uniform"),
    (1, 6000, W.K_EXP, (1, 0, 1.0, 0), 32, 1e-10, "uniform"),
]
IDS = ["invr_d3", "invr_d3_clustered", "log_d2", "gauss_d3", "exp_d1"]


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_near_coords_against_oracle(env, case):
    torch, oracle, hd = env
    d, N, kernel, params, leaf, tol, dist = case
    w = W.make("t", d, N, kernel, params, leaf, tol, nrhs=1, seed=N + d, dist=dist)
    T = oracle.Tree(w.points, w.kernel, w.params, leaf, tol, dense_if_cheaper=True)
    yo = T.matvec(w.x)
    fac = oracle_factors(T)
    errs = {}
    for mode in ("hilo", "hi"):
        h = gpu_handle(hd, w, precision="fp32", near_coords=mode)
        h.import_factors(*fac)
        y1 = gpu_matvec(h, w.x)
        y2 = gpu_matvec(h, w.x)
        assert np.array_equal(y1, y2)
        errs[mode] = relerr(y1, yo)
        h.close()
    print(f"{IDS[CASES.index(case)]}: hilo {errs['hilo']:.2e}  hi {errs['hi']:.2e}")
    assert errs["hilo"] <= FP32_BOUND
    assert errs["hi"] <= NEAR_HI_SMALL_BOUND


def test_near_coords_rejects_bad_value(env):
    torch, oracle, hd = env
    w = W.make("t", 2, 500, W.K_LOG, (1, 0, 0, 0), 32, 1e-8, seed=1)
    with pytest.raises(KeyError):
        gpu_handle(hd, w, near_coords="exact")
