"""Batched products over uneven trees (one CUDA graph replayed): every result
equals the single-handle product bitwise, run after run, with host or device
buffers."""
import numpy as np
import pytest

import workloads as W
from gpu_util import gpu_handle, require_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = require_cuda()
    import paper_2209_05819_gb300 as hd

    return torch, hd


def _sets(n=7):
    out = []
    for s in range(n):
        rng = np.random.default_rng(300 + s)
        N = int(rng.integers(1500, 12000))
        nrhs = int(rng.integers(1, 11))
        d = 3 if s % 3 else 2
        w = W.make(f"b{s}", d, N, W.K_GAUSS if s % 2 else W.K_INV_R, (1.0, 1e-3, 0.5, 0) if s % 2 else (1, 0, 0, 0),
                   48, 1e-7, nrhs=nrhs, seed=300 + s, dist="clustered" if s % 2 else "uniform")
        out.append(w)
    return out


def test_batch_equals_single_products(env):
    torch, hd = env
    ws = _sets()
    precs = ["fp32", "fp32", "fp16", "fp64", "fp32", "bf16", "fp32"]
    hs = [gpu_handle(hd, w, precision=p) for w, p in zip(ws, precs)]
    xs = [torch.from_numpy(np.ascontiguousarray(w.x, dtype=h.io_dtype)).cuda() for w, h in zip(ws, hs)]
    singles = [h.matvec(x).cpu().numpy() for h, x in zip(hs, xs)]
    b = hd.Batch(hs, [w.nrhs for w in ws])
    for _ in range(2):
        ys = b.run(xs)
        torch.cuda.synchronize()
        for y, ref in zip(ys, singles):
            assert np.array_equal(y.cpu().numpy(), ref)
    # host buffers
    xh = [x.cpu().numpy() for x in xs]
    yh = b.run(xh)
    for y, ref in zip(yh, singles):
        assert np.array_equal(y, ref)
    b.close()


def test_batch_rejects_duplicates_and_profiling(env):
    torch, hd = env
    ws = _sets(2)
    hs = [gpu_handle(hd, w, precision="fp32") for w in ws]
    with pytest.raises(hd.HodlrddError) as e:
        hd.Batch([hs[0], hs[0]], [1, 1])
    assert e.value.status == hd.ERR_INVALID
    hs[1].set_profiling(True)
    with pytest.raises(hd.HodlrddError) as e:
        hd.Batch(hs, [1, 1])
    assert e.value.status == hd.ERR_INVALID
    hs[1].set_profiling(False)
