"""hodlrdd_matvec_noalloc against hodlrdd_matvec.

The no-allocation entry point runs the same kernels as hodlrdd_matvec and only
stages host buffers through the library's static device scratch, so on the same
handle and inputs its result must match hodlrdd_matvec's (the tolerances below
allow rounding noise, though equality is expected). Collected last, so it runs
both alone and after every other GPU test in one process.
"""
import gc

import numpy as np
import pytest

import workloads as W
from gpu_util import gpu_handle, relerr, require_cuda

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-13, "fp32": 1e-6, "fp16": 1e-6}
SCRATCH_BYTES = 16 << 20


@pytest.fixture(scope="module")
def env():
    torch = require_cuda()
    import paper_2209_05819_gb300 as hd

    return torch, hd


@pytest.mark.parametrize("precision,nrhs", [("fp64", 3), ("fp32", 1), ("fp32", 5), ("fp16", 2)])
def test_two_calls_match_matvec(env, precision, nrhs):
    torch, hd = env
    w = W.make("t", 3, 20000, W.K_INV_R, (1, 0, 0, 0), 32, 1e-8, nrhs=nrhs, seed=11 + nrhs)
    h = gpu_handle(hd, w, precision=precision)
    x = np.ascontiguousarray(w.x, dtype=h.io_dtype)
    y_ref = h.matvec(x)  # existing entry point, host buffers
    y1 = h.matvec_noalloc(x)
    y2 = h.matvec_noalloc(x)
    h.sync()
    assert relerr(y1, y_ref) <= TOL[precision]
    assert relerr(y2, y_ref) <= TOL[precision]
    assert relerr(y2, y1) <= TOL[precision]


def test_no_device_memory_is_taken(env):
    torch, hd = env
    w = W.make("t", 2, 30000, W.K_LOG, (1, 0, 0, 0), 64, 1e-8, nrhs=4, seed=5)
    h = gpu_handle(hd, w)
    x = np.ascontiguousarray(w.x)
    y_ref = h.matvec(x)
    h.matvec_noalloc(x)  # set-up call
    gc.collect()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    y1 = h.matvec_noalloc(x)
    y2 = h.matvec_noalloc(np.ascontiguousarray(w.x[:, :2]))
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 >= free0
    assert relerr(y1, y_ref) <= TOL["fp64"]
    assert relerr(y2, y_ref[:, :2]) <= TOL["fp64"]


def test_mixed_host_and_device_buffers(env):
    torch, hd = env
    w = W.make("t", 3, 9000, W.K_INV_R, (1, 0, 0, 0), 32, 1e-8, nrhs=2, seed=7)
    h = gpu_handle(hd, w, precision="fp32")
    x = np.ascontiguousarray(w.x, dtype=np.float32)
    xd = torch.from_numpy(x).cuda()
    y_ref = h.matvec(xd).cpu().numpy()
    y_dh = h.matvec_noalloc(xd, np.empty_like(x))  # device x, host y
    y_hd = h.matvec_noalloc(x, torch.empty_like(xd)).cpu().numpy()  # host x, device y
    y_dd = h.matvec_noalloc(xd).cpu().numpy()  # no staging at all
    h.sync()
    for y in (y_dh, y_hd, y_dd):
        assert relerr(y, y_ref) <= TOL["fp32"]


def test_rejects_staging_beyond_scratch(env):
    torch, hd = env
    N, nrhs = 20000, 64  # 10.24 MB per FP64 operand: x and y together exceed 16 MiB
    w = W.make("t", 2, N, W.K_LOG, (1, 0, 0, 0), 64, 1e-8, nrhs=nrhs, seed=9)
    h = gpu_handle(hd, w)
    x = np.ascontiguousarray(w.x)
    assert 2 * x.nbytes > SCRATCH_BYTES >= x.nbytes
    y = np.full_like(x, np.nan)
    with pytest.raises(hd.HodlrddError) as e:
        h.matvec_noalloc(x, y)
    assert e.value.status == hd.ERR_INVALID
    assert "static scratch" in str(e.value)
    assert np.all(np.isnan(y))  # nothing was written
    # one host side alone fits: device x, host y
    xd = torch.from_numpy(x).cuda()
    y_ref = h.matvec(xd).cpu().numpy()
    y_dh = h.matvec_noalloc(xd, y)
    h.sync()
    assert relerr(y_dh, y_ref) <= TOL["fp64"]


def test_rejects_profiling(env):
    torch, hd = env
    w = W.make("t", 2, 2000, W.K_LOG, (1, 0, 0, 0), 32, 1e-8, seed=3)
    h = gpu_handle(hd, w)
    h.set_profiling(True)
    with pytest.raises(hd.HodlrddError) as e:
        h.matvec_noalloc(np.ascontiguousarray(w.x))
    assert e.value.status == hd.ERR_INVALID
    h.set_profiling(False)
    y = h.matvec_noalloc(np.ascontiguousarray(w.x))
    assert relerr(y, h.matvec(np.ascontiguousarray(w.x))) <= TOL["fp64"]
