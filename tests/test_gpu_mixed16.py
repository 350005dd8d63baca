"""Mixed FP32 / FP16 factor storage (precision "fp32+fp16"): each block's
leading ACA terms in FP32, its trailing terms (every term after the last one
above 2^-13 of the block's Frobenius norm estimate) in FP16 with power-of-two
column scales, all arithmetic in FP32.

Bound against the FP64 product: a tail term has ||u_k|| ||v_k|| <= 2^-13 ||A_b||
and FP16 keeps 2^-11 of each scaled entry, so its rounding is about 2^-24 of the
block, the size of the FP32 rounding of the leading terms; the stated FP32
bounds (2e-6 for one or two right-hand sides, 5e-6 for wider chunks) apply."""
import numpy as np
import pytest

import workloads as W
from gpu_util import gpu_handle, gpu_matvec, relerr, require_cuda

pytestmark = pytest.mark.gpu

BOUND = 2e-6
WIDE_BOUND = 5e-6

CASES = [
    (3, 9000, W.K_INV_R, None, 32, 1e-8),
    (2, 4096, W.K_LOG, None, 64, 1e-8),
    (4, 5000, W.K_MATERN32, (1, 0, 0.2, 0), 40, 1e-7),
    (3, 5000, W.K_GAUSS, (1, 1e-3, 0.5, 0), 32, 1e-6),
    (1, 3001, W.K_EXP, (1, 0, 1.0, 0), 16, 1e-10),
    (2, 3000, W.K_SIN, None, 25, 1e-9),
]


@pytest.fixture(scope="module")
def env():
    torch = require_cuda()
    import oracle
    import paper_2209_05819_gb300 as hd

    oracle.build()
    return torch, oracle, hd


@pytest.mark.parametrize("d,N,kernel,params,leaf,tol", CASES)
@pytest.mark.parametrize("nrhs", [1, 2, 6])
def test_bound_against_fp64(env, d, N, kernel, params, leaf, tol, nrhs):
    torch, oracle, hd = env
    w = W.make("t", d, N, kernel, params or (1, 0, 0, 0), leaf, tol, nrhs=nrhs, seed=N + 13 * d + nrhs)
    h64 = gpu_handle(hd, w)
    hm = gpu_handle(hd, w, precision="fp32+fp16")
    assert np.array_equal(h64.blocks(), hm.blocks())
    err = relerr(gpu_matvec(hm, w.x), gpu_matvec(h64, w.x))
    assert err <= (BOUND if nrhs < 4 else WIDE_BOUND), err
    hm.sync()


def test_storage_and_structure(env):
    torch, oracle, hd = env
    w = W.make("t", 3, 40000, W.K_INV_R, (1, 0, 0, 0), 64, 1e-7, nrhs=1, seed=3)
    hm = gpu_handle(hd, w, precision="fp32+fp16")
    hf = gpu_handle(hd, w, precision="fp32")
    sm, sf = hm.stats(), hf.stats()
    assert sm["total_rank"] == sf["total_rank"]
    assert 0 < sm["tail_cols"] < sm["total_rank"]
    fm = sm["factor_bytes_u"] + sm["factor_bytes_v"]
    ff = sf["factor_bytes_u"] + sf["factor_bytes_v"]
    assert fm < 0.85 * ff  # a share of the terms moved to two-byte storage
    x = torch.from_numpy(np.ascontiguousarray(w.x, dtype=np.float32)).cuda()
    y1 = hm.matvec(x)
    y2 = hm.matvec(x)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)
    yh = hm.matvec(np.ascontiguousarray(w.x, dtype=np.float32))
    assert np.array_equal(np.asarray(yh), y1.cpu().numpy())
    rec = hm.blocks()
    b = int(np.flatnonzero(rec[:, 7] > 0)[0])
    with pytest.raises(hd.HodlrddError) as e:
        hm.factors(b, int(rec[b, 4]), int(rec[b, 6]), int(rec[b, 7]))
    assert e.value.status == hd.ERR_UNSUPPORTED


def test_against_direct_sum_and_general_path(env):
    """The product against the oracle's direct sum (10 tol + the bound), and the
    packed near field against the general path (lists instead of tiles)."""
    torch, oracle, hd = env
    w = W.make("t", 3, 6000, W.K_INV_R, (1, 0, 0, 0), 32, 1e-8, nrhs=1, seed=77)
    yd = oracle.direct(w.points, w.kernel, w.params, w.x)
    for mode in (1, 2):
        hm = gpu_handle(hd, w, precision="fp32+fp16", near_mode=mode)
        assert relerr(gpu_matvec(hm, w.x), yd) <= 10 * w.tol + BOUND
