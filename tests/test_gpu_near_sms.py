"""The single-right-hand-side FP32 near field on SMs of its own (option near_sms).

With R > 0 the persistent apply kernels run on SMs - R CTAs and the near field
on R CTAs, each reserving a whole SM's shared memory, and all near-field passes
are one launch whose groups take tasks from a counter. The apply schedule cuts
panels at the same places whatever the CTA count, and each near-field pass sums
into a buffer of its own that the final sum adds in pass order, the order in
which the shared setting accumulates them: products are bitwise equal to those
of the shared setting (near_sms 0) built from the same points. One case is also
held to the FP32 form's bound against the oracle's product on the oracle's own
factors.
"""
import numpy as np
import pytest

import workloads as W
from gpu_util import gpu_handle, gpu_matvec, oracle_factors, relerr, require_cuda

pytestmark = pytest.mark.gpu

FP32_BOUND = 2e-6


@pytest.fixture(scope="module")
def env():
    torch = require_cuda()
    import oracle
    import paper_2209_05819_gb300 as hd

    oracle.build()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    return torch, oracle, hd, sms


CASES = [
    # d, N, kernel, params, leaf, tol, points, precision, coordinates, near_mode
    (3, 30000, W.K_INV_R, (1, 0, 0, 0), 64, 1e-7, "uniform", "fp32+fp16", "hi", 0),
    (3, 12000, W.K_INV_R, (1.0 / 12000, 1.0, 0, 0), 32, 1e-7, "clustered", "fp32", "hilo", 1),
    (2, 20000, W.K_LOG, (1, 0, 0, 0), 64, 1e-8, "uniform", "fp32", "hilo", 2),
    (1, 8000, W.K_EXP, (1, 0, 1.0, 0), 32, 1e-8, "uniform", "fp16", "hi", 0),
    (3, 9000, W.K_GAUSS, (1, 1e-3, 0.5, 0), 64, 1e-8, "clustered", "bf16", "hilo", 0),
]
IDS = ["invr_d3_mixed_hi", "invr_d3_system_tiles", "log_d2_lists", "exp_d1_fp16", "gauss_d3_bf16"]


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_split_equals_shared(env, case):
    torch, oracle, hd, sms = env
    d, N, kernel, params, leaf, tol, dist, prec, coords, mode = case
    w = W.make("t", d, N, kernel, params, leaf, tol, nrhs=1, seed=N + 3 * d, dist=dist)
    kw = dict(precision=prec, near_coords=coords, near_mode=mode)
    h0 = gpu_handle(hd, w, **kw)
    y0 = gpu_matvec(h0, w.x)
    x3 = np.ascontiguousarray(np.stack([w.x[:, 0], -2 * w.x[:, 0], 0.5 * w.x[:, 0]], axis=1))
    y03 = gpu_matvec(h0, x3)
    for R in (1, 37, sms - 1):
        h = gpu_handle(hd, w, near_sms=R, **kw)
        y1 = gpu_matvec(h, w.x)
        y2 = gpu_matvec(h, w.x)
        assert np.array_equal(y1, y2), R
        assert np.array_equal(y1, y0), (R, relerr(y1, y0))
        # several right-hand sides: chunks without the split near field, applies on SMs - R CTAs
        assert np.array_equal(gpu_matvec(h, x3), y03), R
        h.close()
    h0.close()


def test_split_against_oracle(env):
    torch, oracle, hd, sms = env
    w = W.make("t", 3, 15000, W.K_INV_R, (1, 0, 0, 0), 64, 1e-8, nrhs=1, seed=41)
    T = oracle.Tree(w.points, w.kernel, w.params, w.leaf, w.tol, dense_if_cheaper=True)
    yo = T.matvec(w.x)
    h = gpu_handle(hd, w, precision="fp32", near_sms=40)
    h.import_factors(*oracle_factors(T))
    err = relerr(gpu_matvec(h, w.x), yo)
    print(f"near_sms 40 vs oracle: {err:.2e}")
    assert err <= FP32_BOUND
    h.close()


def test_split_rejects_all_sms(env):
    torch, oracle, hd, sms = env
    w = W.make("t", 2, 2000, W.K_LOG, (1, 0, 0, 0), 32, 1e-8, nrhs=1, seed=2)
    with pytest.raises(hd.HodlrddError) as e:
        gpu_handle(hd, w, precision="fp32", near_sms=sms)
    assert e.value.status == hd.ERR_INVALID


def test_split_stage_timing(env):
    """Profiling events around the near field on SMs of its own."""
    torch, oracle, hd, sms = env
    w = W.make("t", 3, 20000, W.K_INV_R, (1, 0, 0, 0), 64, 1e-7, nrhs=1, seed=9)
    h = gpu_handle(hd, w, precision="fp32+fp16", near_coords="hi", near_sms=32)
    h.set_profiling(True)
    gpu_matvec(h, w.x)
    pr = h.profile()
    h.set_profiling(False)
    assert pr["chunks"] == 1 and pr["near_ms"] > 0 and pr["vapply_ms"] > 0 and pr["uapply_ms"] > 0
    h.close()


def test_auto_choice(env):
    """near_sms = -1: the build times the settings and keeps one; the product is the same."""
    torch, oracle, hd, sms = env
    w = W.make("t", 3, 60000, W.K_INV_R, (1, 0, 0, 0), 64, 1e-7, nrhs=1, seed=12)
    kw = dict(precision="fp32+fp16", near_coords="hi")
    h0 = gpu_handle(hd, w, **kw)
    ha = gpu_handle(hd, w, near_sms="auto", **kw)
    R = ha.stats()["near_sms"]
    print(f"auto near_sms: {R}")
    assert h0.stats()["near_sms"] == 0
    assert R == 0 or 1 <= R <= sms // 3
    assert np.array_equal(gpu_matvec(ha, w.x), gpu_matvec(h0, w.x))
    # forms without the single-right-hand-side FP32 tiles resolve to 0
    h64 = gpu_handle(hd, W.make("t", 2, 3000, W.K_LOG, (1, 0, 0, 0), 32, 1e-8, seed=3), near_sms="auto")
    assert h64.stats()["near_sms"] == 0
    for h in (h0, ha, h64):
        h.close()
