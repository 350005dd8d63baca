"""hodlrdd_server: requests over models kept resident under a device-memory
budget. Every result equals the model's handle alone (bitwise for products);
a budget below the models' total size evicts and rebuilds without changing a
result; solves reach the FP64 system's tolerance."""
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


def models():
    """Five uneven second-kind systems (I + K/N): d = 2..4, four kernels."""
    specs = [(2, 3000, W.K_LOG, 32, 1e-8), (3, 9000, W.K_INV_R, 32, 1e-8), (4, 5000, W.K_MATERN32, 40, 1e-7),
             (3, 6000, W.K_GAUSS, 32, 1e-6), (2, 12000, W.K_INV_R, 64, 1e-8)]
    out = []
    for i, (d, N, k, leaf, tol) in enumerate(specs):
        p0 = {W.K_MATERN32: 0.2, W.K_GAUSS: 0.5}.get(k, 0.0)
        out.append(W.make(f"m{i}", d, N, k, (1.0 / N, 1.0, p0, 0), leaf, tol, nrhs=2, seed=500 + i))
    return out


def alone(hd, ws, prec):
    ys, sizes = [], []
    for w in ws:
        h = gpu_handle(hd, w, precision=prec)
        ys.append(np.asarray(h.matvec(np.ascontiguousarray(w.x, dtype=h.io_dtype))))
        sizes.append(h.stats()["device_bytes"])
        h.close()
    return ys, sizes


@pytest.mark.parametrize("tight", [False, True])
def test_products_equal_alone_and_in_the_mix(env, tight):
    torch, oracle, hd = env
    ws = models()
    prec = "fp32+fp16"
    ref, sizes = alone(hd, ws, prec)
    # tight: room for the largest model and a bit more, far below all of them together
    budget = int(1.5 * max(sizes)) if tight else int(64e9)
    srv = hd.Server(budget, workers=3)
    ids = [srv.add(w.points, w.kernel, w.params, w.leaf, w.tol, precision=prec) for w in ws]
    rng = np.random.default_rng(0)
    order = rng.integers(0, len(ws), 40)
    reqs = [(m, srv.submit(ids[m], np.ascontiguousarray(ws[m].x, dtype=np.float32))) for m in order]
    for m, r in reqs:
        y, lat = srv.wait(r)
        assert np.array_equal(y, ref[m])
        assert lat > 0.0
    st = srv.stats()
    assert st["resident_bytes"] <= budget
    if tight:  # smaller than the models together: evictions and rebuilds
        assert st["evictions"] > 0 and st["builds"] > len(ws)
        assert st["resident_models"] >= 1
    else:
        assert st["evictions"] == 0 and st["builds"] == len(ws)
    srv.close()


def test_solves_and_mixed_kinds(env):
    torch, oracle, hd = env
    ws = models()[:3]
    srv = hd.Server(int(64e9), workers=2)
    ids = [srv.add(w.points, w.kernel, w.params, w.leaf, w.tol, precision="fp32") for w in ws]
    reqs = []
    for m, w in enumerate(ws):
        reqs.append(("solve", m, srv.submit(ids[m], w.x, kind=hd.REQ_SOLVE)))
        reqs.append(("matvec", m, srv.submit(ids[m], np.ascontiguousarray(w.x, dtype=np.float32))))
    for kind, m, r in reqs:
        y, _ = srv.wait(r)
        w = ws[m]
        if kind == "solve":
            # the FP64 HODLRdD operator applied to u reproduces b
            h64 = gpu_handle(hd, w)
            b = np.asarray(h64.matvec(np.ascontiguousarray(y)))
            assert relerr(b, w.x) <= 1.1e-10
            h64.close()
    assert srv.stats()["builds"] == 2 * len(ws)  # each model and its FP64 twin
    srv.close()


def test_rejections(env):
    torch, oracle, hd = env
    with pytest.raises(hd.HodlrddError):
        hd.Server(0)
    srv = hd.Server(int(1e9), workers=1)
    w = models()[0]
    mid = srv.add(w.points, w.kernel, w.params, w.leaf, w.tol)
    with pytest.raises(hd.HodlrddError):
        srv.submit(mid + 5, np.zeros((w.N, 1), np.float32))
    # a model larger than the budget fails its request, the server keeps going
    tiny = hd.Server(1000, workers=1)
    t = tiny.add(w.points, w.kernel, w.params, w.leaf, w.tol)
    r = tiny.submit(t, np.ascontiguousarray(w.x, dtype=np.float32))
    with pytest.raises(hd.HodlrddError) as e:
        tiny.wait(r)
    assert e.value.status == hd.ERR_OOM
    tiny.close()
    srv.close()


def test_bounded_wait_expiry_is_reported_and_recoverable(env):
    """A bounded device wait that nothing completes (about a second) records its
    error code; hodlrdd_sync reports ERR_TIMEOUT, clears it, and the handle's
    next product is correct."""
    torch, oracle, hd = env
    w = models()[1]
    h = gpu_handle(hd, w, precision="fp32")
    x = np.ascontiguousarray(w.x, dtype=np.float32)
    y0 = np.asarray(h.matvec(x))
    h.debug_expire_wait(2_000_000_000)
    with pytest.raises(hd.HodlrddError) as e:
        h.sync()
    assert e.value.status == hd.ERR_TIMEOUT
    h.sync()  # cleared
    assert np.array_equal(np.asarray(h.matvec(x)), y0)
    h.close()
